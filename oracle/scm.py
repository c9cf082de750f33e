"""Schur complement matrix of the HKM direction, eq. (SCM) of Sec. 2.2:

    B_ij = (X A_i Y^{-1}) . A_j      (i, j = 1..m)

and the right-hand side of B dz = g.  With X the dense completed matrix X̂ this is the value
that eq. (newSCM2) reaches through the sparse factors (the reformulation is exact, Sec. 2.2).
"""
import numpy as np


def scm_dense(A, X, Yinv):
    """B by the definition with dense matrices: for each i form X A_i Y^{-1}, dot with every A_j.
    For small n only.  Pins: symmetric, positive definite, max-cut Hadamard form X ∘ Y^{-1},
    LP normal matrix for diagonal data (tests/test_oracle_scm.py)."""
    m = A.m
    B = np.zeros((m, m))
    for i in range(1, m + 1):
        T = X @ A.dense(i) @ Yinv
        B[i - 1, :] = A.op(T)
    return B


def scm_sparse_rows(A, X, Yinv, rows=None):
    """Rows of B by the same definition, using only the nonzeros of the A's:
    (X A_i Y^{-1})[c, d] = sum over nonzeros (a, b) of A_i of X[c, a] [A_i]_ab Y^{-1}[b, d],
    evaluated at the nonzero positions (c, d) of every A_j, then B_ij = sum A_j[c,d] (.)[c,d].
    Pinned against scm_dense on small cases."""
    m = A.m
    rows = range(1, m + 1) if rows is None else [r + 1 for r in rows]
    sel = A.k >= 1
    pc, pd, pv, pk = A.r[sel], A.c[sel], A.v[sel], A.k[sel]
    out = []
    for i in rows:
        a, b, v = A.entries(i)
        Xg = X[np.ix_(pc, a)]            # (P, t)
        Yg = Yinv[np.ix_(b, pd)].T       # (P, t)
        T = (Xg * Yg) @ v                # (X A_i Y^{-1}) at every position
        out.append(np.bincount(pk - 1, weights=pv * T, minlength=m))
    return np.array(out)


def scm_entry(A, X, Yinv, i, j):
    """One entry B_ij (0-based constraint indices) by the definition."""
    a, b, v = A.entries(i + 1)
    c, d, w = A.entries(j + 1)
    # (X A_i Y^{-1})[c, d] at the nonzeros of A_j
    T = (X[np.ix_(c, a)] * Yinv[np.ix_(b, d)].T) @ v
    return float(np.dot(w, T))


def hkm_rhs(A, b, X, Yinv, G, beta, mu):
    """g with B dz = g for the HKM direction.

    From A(X + dX) = b, sum_k A_k dz_k + dY = G (G = A_0 - sum A_k z_k - Y) and
    dX̂ = beta mu Y^{-1} - X - X dY Y^{-1} (eq. dX), eliminating dY and dX gives
    g_i = b_i - A_i . (beta mu Y^{-1} - X G Y^{-1}).  (Sec. 2.2 prints g with another sign
    convention and without b; this is the reading the derivation fixes, pinned by the test that a
    unit step zeroes the linear residuals.)
    """
    M = beta * mu * Yinv
    if G is not None and np.any(G):
        M = M - X @ G @ Yinv
    return b - A.op(M)
