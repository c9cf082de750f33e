"""Primal-dual interior-point method with the HKM direction (Sec. 2.2), dense FP64.

Basic framework (Sec. 2.2, Steps 0-4): from (X, Y, z) with X, Y positive definite, compute
(dX, dY, dz) from B dz = g, dY = G - sum_k A_k dz_k, dX̂ = beta mu Y^{-1} - X - X dY Y^{-1},
dX = (dX̂ + dX̂^T)/2, take alpha_p, alpha_d = max{alpha in (0,1] : . + alpha d. psd} and update
with gamma alpha.  Parameters not printed in the paper (it says "default parameters", Sec. 4)
are beta = 0.1, gamma = 0.9, relative gap / feasibility tolerance 1e-7, at most 60 iterations.

`solve_dense` keeps the full dense X (the plain PDIPM).  `mc_newton_step` computes the same
direction at the completed matrix X̂ of an iterate X̄ known only on E, and `solve_mc` iterates it
with the clique-wise primal step length of eq. (primal_length2): this is what MC-PDIPM computes.
"""
import numpy as np
import scipy.linalg as sla

from .completion import max_det_completion
from .scm import scm_sparse_rows, scm_dense, hkm_rhs
from .sdp import dual_slack

BETA, GAMMA, TOL, MAX_ITER = 0.1, 0.9, 1e-7, 60


def max_step(M, D):
    """max{alpha in (0, 1] : M + alpha D psd} for M positive definite (eq. primal_length):
    with M = L L^T, the bound is -1/lambda_min(L^{-1} D L^{-T}) when that eigenvalue is negative."""
    L = np.linalg.cholesky(M)
    W = sla.solve_triangular(L, D, lower=True)
    W = sla.solve_triangular(L, W.T, lower=True)
    lam = np.linalg.eigvalsh(0.5 * (W + W.T))[0]
    if lam >= -1.0:
        return 1.0
    return -1.0 / lam


def measures(A, b, X, Y, z):
    A0 = A.dense(0)
    pobj = float(np.sum(A0 * X))
    dobj = float(np.dot(b, z))
    gap = abs(pobj - dobj) / max(1.0, (abs(pobj) + abs(dobj)) / 2)
    pinf = float(np.max(np.abs(A.op(X) - b))) / max(1.0, float(np.max(np.abs(b))))
    dres = A0 - A.adjoint(z) - Y
    dinf = float(np.max(np.abs(dres))) / max(1.0, float(np.max(np.abs(A0))))
    return pobj, dobj, gap, pinf, dinf


def solve_dense(A, b, z0, X0=None, beta=BETA, gamma=GAMMA, tol=TOL, max_iter=MAX_ITER,
                dense_scm=False, log=None):
    """Plain dense HKM PDIPM with full X.  Pins: closed-form max-cut optima (bipartite graphs,
    odd cycles, complete graphs), weak duality at every iterate, brute-force max-cut bounds."""
    n = A.n
    X = np.eye(n) if X0 is None else X0.copy()
    z = np.asarray(z0, dtype=np.float64).copy()
    Y = dual_slack(A, z)
    A0 = A.dense(0)
    hist = []
    status = "maxiter"
    for it in range(max_iter + 1):
        pobj, dobj, gap, pinf, dinf = measures(A, b, X, Y, z)
        hist.append(dict(it=it, pobj=pobj, dobj=dobj, gap=gap, pinf=pinf, dinf=dinf))
        if log:
            log(hist[-1])
        if gap <= tol and pinf <= tol and dinf <= tol:
            status = "optimal"
            break
        if it == max_iter:
            break
        mu = float(np.sum(X * Y)) / n
        Yinv = np.linalg.inv(Y)
        Yinv = 0.5 * (Yinv + Yinv.T)
        G = A0 - A.adjoint(z) - Y
        B = scm_dense(A, X, Yinv) if dense_scm else scm_sparse_rows(A, X, Yinv)
        g = hkm_rhs(A, b, X, Yinv, G, beta, mu)
        dz = sla.cho_solve(sla.cho_factor(B, lower=True), g)
        dY = G - A.adjoint(dz)
        dXh = beta * mu * Yinv - X - X @ dY @ Yinv
        dX = 0.5 * (dXh + dXh.T)
        ap = max_step(X, dX)
        ad = max_step(Y, dY)
        hist[-1].update(mu=mu, alpha_p=ap, alpha_d=ad)
        X = X + gamma * ap * dX
        Y = Y + gamma * ad * dY
        z = z + gamma * ad * dz
    return dict(status=status, X=X, Y=Y, z=z, pobj=pobj, dobj=dobj, gap=gap, pinf=pinf,
                dinf=dinf, iters=it, history=hist)


def _perm_mats(perm):
    perm = np.asarray(perm)
    return perm


def mc_newton_step(A, b, perm, cliques, Xbar, z, beta=BETA):
    """HKM direction of MC-PDIPM at the iterate (X̄ on E, z), Sec. 2.2 eqs. (SCE), (dX) with X
    replaced by the max-det completion X̂ (eqs. newSCM2 / newdX2 evaluate exactly this).

    Xbar: dense n x n in the ORIGINAL order, read only on E.  Y = A_0 - sum z_k A_k (dual
    feasible, so G = 0).  Returns the direction restricted to E plus every intermediate.
    """
    n = A.n
    p = np.asarray(perm)
    Xn = Xbar[np.ix_(p, p)]
    Xh_n = max_det_completion(Xn, cliques)
    inv = np.empty_like(p)
    inv[p] = np.arange(n)
    Xh = Xh_n[np.ix_(inv, inv)]
    Y = dual_slack(A, z)
    Yinv = np.linalg.inv(Y)
    Yinv = 0.5 * (Yinv + Yinv.T)
    mu = float(np.sum(Xh * Y)) / n
    B = scm_sparse_rows(A, Xh, Yinv)
    g = hkm_rhs(A, b, Xh, Yinv, None, beta, mu)
    dz = sla.cho_solve(sla.cho_factor(B, lower=True), g)
    dY = -A.adjoint(dz)
    dXh = beta * mu * Yinv - Xh - Xh @ dY @ Yinv
    dX = 0.5 * (dXh + dXh.T)
    # clique-wise primal step, eq. (primal_length2), cliques in the new order
    dXn = dX[np.ix_(p, p)]
    ap = 1.0
    for rows, ns in cliques:
        ap = min(ap, max_step(Xn[np.ix_(rows, rows)], dXn[np.ix_(rows, rows)]))
    ad = max_step(Y, dY)
    return dict(Xh=Xh, Y=Y, Yinv=Yinv, mu=mu, B=B, g=g, dz=dz, dY=dY, dX=dX,
                alpha_p=ap, alpha_d=ad)


def solve_mc(A, b, z0, perm, cliques, Emask_orig, beta=BETA, gamma=GAMMA, tol=TOL,
             max_iter=MAX_ITER, log=None):
    """MC-PDIPM iterated with the oracle's dense algebra: X̄ lives on E only (Emask_orig, original
    order), X̄0 = I.  Pins: same optimal value as solve_dense, closed forms."""
    n = A.n
    Xbar = np.eye(n)
    z = np.asarray(z0, dtype=np.float64).copy()
    hist = []
    status = "maxiter"
    for it in range(max_iter + 1):
        Y = dual_slack(A, z)
        pobj, dobj, gap, pinf, dinf = measures(A, b, Xbar, Y, z)
        hist.append(dict(it=it, pobj=pobj, dobj=dobj, gap=gap, pinf=pinf))
        if log:
            log(hist[-1])
        if gap <= tol and pinf <= tol:
            status = "optimal"
            break
        if it == max_iter:
            break
        st = mc_newton_step(A, b, perm, cliques, Xbar, z, beta)
        hist[-1].update(mu=st["mu"], alpha_p=st["alpha_p"], alpha_d=st["alpha_d"])
        Xbar = Xbar + gamma * st["alpha_p"] * np.where(Emask_orig, st["dX"], 0.0)
        z = z + gamma * st["alpha_d"] * st["dz"]
    return dict(status=status, Xbar=Xbar, z=z, pobj=pobj, dobj=dobj, gap=gap, pinf=pinf,
                iters=it, history=hist)
