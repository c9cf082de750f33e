"""Max-determinant positive definite completion and the factor L̂ of its inverse (Sec. 2.1, 3.1).

All matrices are dense and indexed in the elimination (new) order; cliques are (rows, |S_r|)
pairs as returned by oracle.chordal.cliques_from_supernodes: rows = C_r sorted, first |S_r| rows
are the clique's own columns S_r, the rest is U_r.
"""
import numpy as np
import scipy.linalg as sla


def max_det_completion(Xbar, cliques):
    """X̂ from the entries of X̄ on E = union C_r x C_r, by Lemma 2.6 (Sec. 3.1) applied clique by
    clique from the root of the clique tree downwards.

    When clique r is added, every later column is already completed; with S = S_r, U = U_r and
    T = (later columns) minus U, the unknown block is X̂_ST = X̄_SU X̄_UU^{-1} X̂_UT and the known
    blocks X̄_SS, X̄_SU are copied.  Pins: X̂ = X̄ on E, (X̂^{-1})_ij = 0 off E (the max-det
    optimality condition of Grone et al.), X̂ positive definite, log det X̂ above any perturbed
    completion, the two-clique closed form; see tests/test_oracle_completion.py.
    """
    n = Xbar.shape[0]
    Xh = np.zeros((n, n))
    for rows, ns in reversed(cliques):
        S = rows[:ns]
        U = rows[ns:]
        last = S[-1]
        later = np.arange(last + 1, n)
        T = np.setdiff1d(later, U)
        Xh[np.ix_(S, S)] = Xbar[np.ix_(S, S)]
        if len(U):
            XSU = Xbar[np.ix_(S, U)]
            Xh[np.ix_(S, U)] = XSU
            Xh[np.ix_(U, S)] = XSU.T
            if len(T):
                XUU = Xbar[np.ix_(U, U)]
                XST = XSU @ np.linalg.solve(XUU, Xh[np.ix_(U, T)])
                Xh[np.ix_(S, T)] = XST
                Xh[np.ix_(T, S)] = XST.T
        elif len(T):
            # disconnected component: U empty, the max-det completion puts zeros in X̂_ST
            Xh[np.ix_(S, T)] = 0.0
            Xh[np.ix_(T, S)] = 0.0
    return 0.5 * (Xh + Xh.T)


def algorithm1(Xbar, cliques):
    """Algorithm 1 (Sec. 3.1): L̂ with X̂^{-1} = L̂ L̂^T, clique by clique, never forming X̂.

    For each clique r: P_r reverses the order of C_r; P_r X̄_CC P_r^T = M_r M_r^T (Cholesky);
    L_r = P_r M_r^{-T} P_r^T; the first |S_r| columns of L_r go to L̂_{C_r S_r}.
    Pin: equals chol(X̂^{-1}) (lower, positive diagonal, unique) and vanishes off lower(E).
    """
    n = Xbar.shape[0]
    Lh = np.zeros((n, n))
    for rows, ns in cliques:
        XCC = Xbar[np.ix_(rows, rows)]
        k = len(rows)
        P = np.eye(k)[::-1]
        M = np.linalg.cholesky(P @ XCC @ P.T)
        Lr = P @ np.linalg.inv(M).T @ P.T
        Lh[np.ix_(rows, rows[:ns])] = Lr[:, :ns]
    return Lh


def inverse_cholesky_definition(Xh):
    """The unique lower-triangular L̂ with positive diagonal and L̂ L̂^T = X̂^{-1} (Sec. 3.1)."""
    return np.linalg.cholesky(np.linalg.inv(Xh))


def dense_cholesky_on_pattern(Y):
    """N with Y = N N^T (Sec. 2.1 / type (v) of Sec. 3.1), dense."""
    return sla.cholesky(Y, lower=True)
