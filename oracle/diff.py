"""Test infrastructure (oracle): implicit differentiation of the central-path point.

An extension beyond the paper (derivatives of the solution).  The point differentiated is the
central-path point for a fixed mu > 0 of (P)/(D) (Sec. 1, Sec. 2.2):

    A(X) = b,   Y = A_0 - sum_k z_k A_k,   X Y = mu I,

i.e. X = mu Y^{-1} with z the root of F(z) = A(mu Y(z)^{-1}) - b.  F'(z) is the Schur complement
matrix at X = mu Y^{-1} (B_pq = A_p . (X A_q Y^{-1}), eq. newSCM), so Newton's method on z is the
centring step of the method.  For a loss  l = <G, X> + g_z^T z  (G symmetric) the adjoint is

    R   = sym(X G Y^{-1}),   v = B^{-1} (A(R) + g_z),
    g_b = v,   g_{A_0} = sym(X (A^*(v) - G) Y^{-1}),   g_{A_k} = -z_k g_{A_0} - v_k X,

(sym(M) = (M + M^T)/2, A^*(v) = sum_k v_k A_k), obtained by differentiating F(z; b, A_0, A_k) = 0
and X = mu Y^{-1}.  Plain dense FP64; B is formed row by row from the nonzeros of the A_k
(oracle.scm.scm_sparse_rows, pinned against the definition scm_dense), so instances up to
n = m = 1000 or so take seconds per Newton step.
"""
import numpy as np

from .scm import scm_sparse_rows
from .sdp import dual_slack


def _sym(M):
    return 0.5 * (M + M.T)


def central_point(A, b, mu, z0, tol=1e-13, max_newton=60):
    """Newton on F(z) = A(mu Y(z)^{-1}) - b from a dual-feasible z0, halving the step until
    Y stays positive definite, until max|F| <= tol max(1, max|b|).  If Newton stops gaining
    (three full steps in a row that do not halve the residual) the point is accepted only when the
    residual is at the rounding level of evaluating F, rho = 64 eps cond(Y) max_k |A_k|.|X| /
    max(1, max|b|) (Y^{-1} is formed with relative error about eps cond(Y)); above it Newton goes
    on, and it raises after max_newton steps.
    Returns z, Y, X = mu Y^{-1} and the relative residual reached."""
    z = np.array(z0, dtype=np.float64)
    scale = max(1.0, float(np.max(np.abs(b))))
    eps = np.finfo(np.float64).eps
    best = None
    stalled = 0
    full = False
    for _ in range(max_newton):
        Y = dual_slack(A, z)
        Yinv = np.linalg.inv(Y)
        Yinv = _sym(Yinv)
        X = mu * Yinv
        AX = A.op(X)
        F = AX - b
        res = np.max(np.abs(F)) / scale
        if res <= tol:
            return z, Y, X, res
        # a full Newton step (t = 1) that does not halve the residual: rounding, not the
        # damping that keeps Y positive definite far from the point, limits the progress
        stalled = stalled + 1 if best is not None and full and res > 0.5 * best else 0
        best = res if best is None else min(best, res)
        if stalled >= 3:
            # |A|(|X|): the magnitudes the residual's rounding scales with
            absAX = np.bincount(A.k, weights=np.abs(A.v) * np.abs(X[A.r, A.c]),
                                minlength=A.m + 1)[1:]
            rho = 64.0 * eps * np.linalg.cond(Y) * max(1.0, float(np.max(absAX))) / scale
            if res <= rho:
                return z, Y, X, res
            # above the rounding level slow full steps are Newton's global phase (a start far
            # from the central point), not a floor: keep iterating
            stalled = 0
        Bm = scm_sparse_rows(A, X, Yinv)
        dz = np.linalg.solve(Bm, -F)
        t = 1.0
        while True:
            try:
                np.linalg.cholesky(dual_slack(A, z + t * dz))
                break
            except np.linalg.LinAlgError:
                t *= 0.5
                if t < 1e-12:
                    raise RuntimeError("centring step collapsed")
        z = z + t * dz
        full = t == 1.0
    raise RuntimeError("centring did not converge")


def backward(A, z, Y, X, G, gz, with_gA=True):
    """Gradients of l = <G, X> + gz^T z at the central point (z, Y, X): returns (g_b, g_{A_0},
    g_A) with g_A[k-1] the dense gradient with respect to A_k (symmetric matrices; the gradient
    with respect to a stored off-diagonal entry that also sets its mirror is twice the entry).
    with_gA=False returns None for g_A (m dense n x n matrices; entry_gradients needs only
    g_b, g_{A_0} and X)."""
    Yinv = _sym(np.linalg.inv(Y))
    R = _sym(X @ G @ Yinv)
    Bm = scm_sparse_rows(A, X, Yinv)
    v = np.linalg.solve(Bm, A.op(R) + gz)
    gA0 = _sym(X @ (A.adjoint(v) - G) @ Yinv)
    gA = [-z[k] * gA0 - v[k] * X for k in range(A.m)] if with_gA else None
    return v, gA0, gA


def entry_gradients(A_inst, z, v, gA0, X):
    """Per stored entry (mat, row, col) of the input (row <= col): d l / d val."""
    out = np.empty(len(A_inst.val))
    for e, (k, i, j) in enumerate(zip(A_inst.mat, A_inst.row, A_inst.col)):
        f = 1.0 if i == j else 2.0
        g = gA0[i, j] if k == 0 else (-z[k - 1] * gA0[i, j] - v[k - 1] * X[i, j])
        out[e] = f * g
    return out


def loss(A, b, mu, z0, G, gz):
    """l at the central point for (A, b, mu), started from z0."""
    z, Y, X, res = central_point(A, b, mu, z0)
    if res > 1e-12:
        raise RuntimeError(f"central point residual {res:.1e} too large for a finite difference")
    return float(np.sum(G * X) + gz @ z)
