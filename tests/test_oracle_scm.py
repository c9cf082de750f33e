"""Pins of the oracle SCM (eq. SCM) and HKM direction (Sec. 2.2)."""
import numpy as np
import pytest
import scipy.linalg as sla

from instances import lattice_maxcut, small_random_sdp, diagonal_lp_sdp, block_arrow
from oracle.sdp import SparseSym, dual_slack
from oracle.scm import scm_dense, scm_sparse_rows, scm_entry, hkm_rhs


def _pd(n, seed):
    rng = np.random.default_rng(seed)
    G = rng.standard_normal((n, 2 * n))
    return G @ G.T / (2 * n) + 0.3 * np.eye(n)


def test_maxcut_scm_is_hadamard():
    inst = lattice_maxcut(4, 3, seed=5)
    A = SparseSym.from_instance(inst)
    X = _pd(inst.n, 1)
    Yinv = np.linalg.inv(_pd(inst.n, 2))
    Yinv = 0.5 * (Yinv + Yinv.T)
    B = scm_dense(A, X, Yinv)
    assert np.allclose(B, X * Yinv, atol=1e-14)
    assert np.allclose(scm_sparse_rows(A, X, Yinv), X * Yinv, atol=1e-14)


def test_diagonal_lp_scm_is_normal_matrix():
    inst = diagonal_lp_sdp(9, 6, seed=3)
    A = SparseSym.from_instance(inst)
    x = np.random.default_rng(0).uniform(0.5, 2, 9)
    y = np.random.default_rng(1).uniform(0.5, 2, 9)
    Amat = np.array([[A.dense(k)[i, i] for i in range(9)] for k in range(1, 7)])
    B = scm_dense(A, np.diag(x), np.diag(1 / y))
    assert np.allclose(B, Amat @ np.diag(x / y) @ Amat.T, atol=1e-13)


@pytest.mark.parametrize("seed", [1, 2])
def test_scm_symmetric_pd_and_forms_agree(seed):
    inst = small_random_sdp(7, 10, seed)
    A = SparseSym.from_instance(inst)
    X = _pd(7, seed + 10)
    Yinv = np.linalg.inv(_pd(7, seed + 20))
    Yinv = 0.5 * (Yinv + Yinv.T)
    B = scm_dense(A, X, Yinv)
    assert np.allclose(B, B.T, atol=1e-12 * np.abs(B).max())
    assert np.linalg.eigvalsh(B)[0] > 0
    Bs = scm_sparse_rows(A, X, Yinv)
    assert np.allclose(Bs, B, atol=1e-12 * np.abs(B).max())
    assert abs(scm_entry(A, X, Yinv, 3, 5) - B[3, 5]) < 1e-12 * np.abs(B).max()


def test_hkm_direction_zeroes_linear_residuals():
    inst = small_random_sdp(6, 8, 4)
    A = SparseSym.from_instance(inst)
    rng = np.random.default_rng(2)
    X = _pd(6, 3)                               # primal infeasible on purpose
    z = inst.z0 + 0.05 * rng.standard_normal(8)
    Y = _pd(6, 4)                               # dual infeasible on purpose: G != 0
    G = A.dense(0) - A.adjoint(z) - Y
    Yinv = np.linalg.inv(Y)
    mu = np.sum(X * Y) / 6
    beta = 0.1
    B = scm_dense(A, X, Yinv)
    g = hkm_rhs(A, inst.b, X, Yinv, G, beta, mu)
    dz = sla.solve(B, g)
    dY = G - A.adjoint(dz)
    dXh = beta * mu * Yinv - X - X @ dY @ Yinv
    dX = 0.5 * (dXh + dXh.T)
    assert np.allclose(A.op(X + dX), inst.b, atol=1e-10)
    assert np.allclose(A.adjoint(z + dz) + Y + dY, A.dense(0), atol=1e-10)
    # linearised complementarity X dY + dX̂ Y = beta mu I - X Y
    assert np.allclose(X @ dY + dXh @ Y, beta * mu * np.eye(6) - X @ Y, atol=1e-10)
