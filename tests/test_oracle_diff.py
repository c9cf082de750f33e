"""Pins of oracle.diff (implicit differentiation of the central-path point at fixed mu).

* the centring reaches A(X) = b with X = mu Y^{-1}, Y = A_0 - sum z_k A_k positive definite;
* scalar closed form (n = m = 1): X = b/a, z = (c - mu a / b)/a, so for l = X: dl/db = 1/a,
  dl/dc = 0, dl/da = -b/a^2;
* central finite differences (h = 1e-6) of the map (b, A) -> l(X(b, A), z(b, A)) for every b_p
  and every stored entry, on small random instances (LP-like diagonal and dense)."""
import numpy as np
import pytest

from instances import small_random_sdp, diagonal_lp_sdp, SDPInstance
from oracle import diff
from oracle.sdp import SparseSym, dual_slack


def _loss_setup(inst, seed):
    A = SparseSym.from_instance(inst)
    rng = np.random.default_rng(seed)
    n = inst.n
    G = rng.standard_normal((n, n))
    G = 0.5 * (G + G.T)
    gz = rng.standard_normal(inst.m)
    return A, G, gz


def _perturbed(inst, e=None, db=None):
    val = inst.val.copy()
    b = inst.b.copy()
    if e is not None:
        val[e[0]] += e[1]
    if db is not None:
        b[db[0]] += db[1]
    return SparseSym(inst.n, inst.m, inst.mat, inst.row, inst.col, val), b


@pytest.mark.parametrize("mk", [lambda: small_random_sdp(4, 3, 11), lambda: diagonal_lp_sdp(5, 3, 4)],
                         ids=["dense4", "lp5"])
def test_centring_reaches_the_central_point(mk):
    inst = mk()
    A = SparseSym.from_instance(inst)
    mu = 0.3
    z, Y, X, res = diff.central_point(A, inst.b, mu, inst.z0)
    assert res <= 1e-13
    assert np.max(np.abs(A.op(X) - inst.b)) <= 1e-12 * max(1, np.max(np.abs(inst.b)))
    assert np.linalg.eigvalsh(Y)[0] > 0
    assert np.allclose(X @ Y, mu * np.eye(inst.n), atol=1e-10)
    assert np.allclose(Y, dual_slack(A, z))


def test_scalar_closed_form():
    # min c x  s.t.  a x = b, x >= 0, with c = 2, a = 1.5, b = 3, mu = 0.1
    a, b, c, mu = 1.5, 3.0, 2.0, 0.1
    inst = SDPInstance("scalar", 1, 1, np.array([b]), np.array([0, 1], np.int32),
                       np.array([0, 0], np.int32), np.array([0, 0], np.int32),
                       np.array([c, a]), z0=np.array([0.0]), meta={})
    A = SparseSym.from_instance(inst)
    z, Y, X, res = diff.central_point(A, inst.b, mu, inst.z0)
    assert res <= 1e-13
    assert abs(X[0, 0] - b / a) < 1e-13
    assert abs(z[0] - (c - mu * a / b) / a) < 1e-12
    G = np.array([[1.0]])
    gb, gA0, gA = diff.backward(A, z, Y, X, G, np.zeros(1))
    g = diff.entry_gradients(inst, z, gb, gA0, X)
    assert abs(gb[0] - 1.0 / a) < 1e-12
    assert abs(g[0]) < 1e-12                  # dl/dc
    assert abs(g[1] + b / a ** 2) < 1e-12     # dl/da


@pytest.mark.parametrize("mk", [lambda: small_random_sdp(4, 3, 11), lambda: diagonal_lp_sdp(5, 3, 4)],
                         ids=["dense4", "lp5"])
def test_gradients_match_central_differences(mk):
    inst = mk()
    A, G, gz = _loss_setup(inst, 3)
    mu = 0.3
    z, Y, X, res = diff.central_point(A, inst.b, mu, inst.z0)
    # the finite differences below re-centre every perturbed problem; oracle.diff.loss raises
    # unless each of those points also reaches a residual of 1e-12 or less
    assert res <= 1e-12
    gb, gA0, gA = diff.backward(A, z, Y, X, G, gz)
    g_entries = diff.entry_gradients(inst, z, gb, gA0, X)
    h = 1e-6
    scale = max(1.0, np.max(np.abs(g_entries)), np.max(np.abs(gb)))
    for p in range(inst.m):
        Ap, bp = _perturbed(inst, db=(p, h))
        Am, bm = _perturbed(inst, db=(p, -h))
        fd = (diff.loss(Ap, bp, mu, z, G, gz) - diff.loss(Am, bm, mu, z, G, gz)) / (2 * h)
        assert abs(fd - gb[p]) <= 1e-6 * scale
    for e in range(len(inst.val)):
        Ap, bp = _perturbed(inst, e=(e, h))
        Am, bm = _perturbed(inst, e=(e, -h))
        fd = (diff.loss(Ap, bp, mu, z, G, gz) - diff.loss(Am, bm, mu, z, G, gz)) / (2 * h)
        assert abs(fd - g_entries[e]) <= 1e-6 * scale
