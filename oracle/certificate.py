"""Test infrastructure (oracle): a duality certificate for an iterate known only on E.

For the paper's pair (Sec. 1), weak duality gives  b^T z <= opt <= A_0 . X  for every dual
feasible z (Y = A_0 - sum_k z_k A_k positive semidefinite) and every primal feasible X.  An
MC-PDIPM iterate holds X̄ only on the extended pattern E; by the theorem of Grone et al. quoted in
Sec. 2.1, X̄ has a positive definite completion exactly when every clique block X̄_{C_r C_r} is
positive definite, and both A_0 . X and A(X) read only the aggregate pattern, which lies in E.
So (b^T z, A_0 . X̄) brackets the optimum once Y(z) and every clique block are positive definite
and A(X̄) = b; with A(X̄) = b only to a residual, the upper end holds to that residual.  This
certifies a solve too large for the dense PDIPM.  Plain dense FP64, slow.
"""
import numpy as np

from .sdp import dual_slack


def _is_pd(M):
    try:
        np.linalg.cholesky(M)
        return True
    except np.linalg.LinAlgError:
        return False


def certify(A, b, perm, cliques, Xbar, z):
    """Xbar: dense n x n in the caller's order, read only on E; cliques: (rows, |S_r|) in the
    elimination order perm (new -> caller index).  Returns lower = b^T z, upper = A_0 . X̄, the
    relative primal residual max|A(X̄) - b| / max(1, max|b|), whether Y(z) is positive definite,
    whether every clique block of X̄ is, and the smallest eigenvalue over the clique blocks."""
    p = np.asarray(perm)
    Xn = Xbar[np.ix_(p, p)]
    lam = np.inf
    for rows, _ in cliques:
        lam = min(lam, float(np.linalg.eigvalsh(Xn[np.ix_(rows, rows)])[0]))
    Y = dual_slack(A, np.asarray(z, dtype=np.float64))
    Xsym = 0.5 * (Xbar + Xbar.T)
    pinf = float(np.max(np.abs(A.op(Xsym) - b))) / max(1.0, float(np.max(np.abs(b))))
    return dict(lower=float(np.dot(b, z)), upper=float(np.sum(A.dense(0) * Xsym)), pinf=pinf,
                y_pd=_is_pd(Y), cliques_pd=bool(lam > 0.0), min_clique_eig=lam)
