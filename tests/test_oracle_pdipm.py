"""Pins of the oracle's building blocks that the end-to-end pins only reach indirectly: the
step length of eq. (primal_length), the residual and gap measures of the stopping test, the
constraint map A and its adjoint (Sec. 1), and the Cholesky factor of Y on a chordal pattern
(type (v) of Sec. 3.1)."""
import numpy as np
import pytest

from instances import block_arrow, lattice_maxcut, small_random_sdp
from oracle import maxcut
from oracle.completion import dense_cholesky_on_pattern
from oracle.pdipm import max_step, measures
from oracle.sdp import SparseSym, dual_slack


def _spd(rng, n, shift=0.5):
    G = rng.standard_normal((n, n))
    return G @ G.T / n + shift * np.eye(n)


def test_max_step_diagonal_closed_form():
    # M = diag(m), D = diag(d): M + a D stays psd up to a = min over d_i < 0 of m_i / -d_i
    m = np.array([2.0, 1.0, 4.0, 0.5])
    d = np.array([-1.0, 3.0, -10.0, 0.0])
    assert max_step(np.diag(m), np.diag(d)) == pytest.approx(0.4, rel=1e-14)
    # no direction of decrease, or a bound beyond 1: the step is capped at 1
    assert max_step(np.diag(m), np.diag(np.abs(d))) == 1.0
    assert max_step(np.diag(m), np.diag([-1.0, -0.5, -2.0, -0.25])) == 1.0


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_max_step_is_the_psd_boundary(seed):
    # bisection on lambda_min(M + a D) by dense eigenvalues, a route independent of the
    # Cholesky-whitened eigenvalue problem that max_step solves
    rng = np.random.default_rng(seed)
    n = 7
    M = _spd(rng, n)
    D = rng.standard_normal((n, n))
    D = 4.0 * (D + D.T)
    a = max_step(M, D)
    assert 0.0 < a < 1.0
    lo, hi = 0.0, 1.0
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if np.linalg.eigvalsh(M + mid * D)[0] >= 0.0:
            lo = mid
        else:
            hi = mid
    assert a == pytest.approx(lo, rel=1e-10)
    assert np.linalg.eigvalsh(M + a * D)[0] == pytest.approx(0.0, abs=1e-10)


def test_measures_vanish_at_the_lattice_optimum():
    # the bipartite closed form: X* = x x^T for the 2-colouring x, z*_i = -deg_w(i)/2 and
    # Y* = A_0 - diag(z*) (the signless Laplacian / 4); both objectives equal -sum w
    inst = lattice_maxcut(4, 3, seed=11)
    A = SparseSym.from_instance(inst)
    n = inst.n
    x = np.array([1.0 if (i % 4 + i // 4) % 2 == 0 else -1.0 for i in range(n)])
    X, z = maxcut.bipartite_certificates(n, inst.meta["edges"], inst.meta["weights"],
                                         (x < 0).astype(int))
    assert np.array_equal(X, np.outer(x, x))
    Y = dual_slack(A, z)
    assert np.linalg.eigvalsh(Y)[0] > -1e-12 and np.allclose(Y @ x, 0.0, atol=1e-12)
    pobj, dobj, gap, pinf, dinf = measures(A, inst.b, X, Y, z)
    W = float(sum(inst.meta["weights"]))
    assert pobj == pytest.approx(-W, rel=1e-14) and dobj == pytest.approx(-W, rel=1e-14)
    assert gap < 1e-15 and pinf == 0.0 and dinf < 1e-15


def test_measures_on_a_perturbed_point():
    # moving X off A(X) = b and Y off the dual constraint shows up in pinf and dinf as the
    # infinity norms the stopping test defines
    inst = small_random_sdp(5, 4, seed=3)
    A = SparseSym.from_instance(inst)
    X = np.eye(5)
    z = inst.z0.copy()
    Y = dual_slack(A, z)
    _, _, _, pinf0, dinf0 = measures(A, inst.b, X, Y, z)
    assert pinf0 < 1e-14 and dinf0 < 1e-14
    E = np.zeros((5, 5))
    E[1, 1] = 1e-3
    Y2 = Y + E
    pobj, dobj, gap, pinf, dinf = measures(A, inst.b, X + E, Y2, z)
    r = A.op(X + E) - inst.b
    assert pinf == pytest.approx(np.max(np.abs(r)) / max(1.0, np.max(np.abs(inst.b))))
    A0 = A.dense(0)
    assert dinf == pytest.approx(1e-3 / max(1.0, np.max(np.abs(A0))))
    assert gap == pytest.approx(abs(pobj - dobj) / max(1.0, (abs(pobj) + abs(dobj)) / 2))


@pytest.mark.parametrize("seed", [0, 4])
def test_constraint_map_and_adjoint(seed):
    inst = small_random_sdp(6, 5, seed=seed)
    A = SparseSym.from_instance(inst)
    rng = np.random.default_rng(seed)
    M = rng.standard_normal((6, 6))
    M = M + M.T
    y = rng.standard_normal(5)
    # <A(M), y> = <M, A*(y)> (the adjoint identity)
    assert np.dot(A.op(M), y) == pytest.approx(float(np.sum(M * A.adjoint(y))), rel=1e-13)
    # A_k . M from the stored upper-triangle entries: diagonal once, off-diagonal twice
    for k in range(1, 6):
        r, c, v = inst.matrix_entries(k)
        ref = sum(val * M[i, j] * (1.0 if i == j else 2.0) for i, j, val in zip(r, c, v))
        assert A.op(M)[k - 1] == pytest.approx(ref, rel=1e-13)
    P = A.aggregate_pattern()
    assert np.array_equal(P, P.T) and np.all(np.diag(P))


def test_cholesky_of_y_has_no_fill_on_a_chordal_pattern():
    # block-arrow: the natural order (blocks, then the border) is a perfect elimination ordering
    # of the block + border pattern, so the factor N of Y stays inside that pattern
    inst = block_arrow(4, 6, 3, 20, per_matrix=8, seed=2)
    A = SparseSym.from_instance(inst)
    rng = np.random.default_rng(5)
    Y = dual_slack(A, inst.z0 + 0.01 * rng.standard_normal(inst.m))
    N = dense_cholesky_on_pattern(Y)
    assert np.allclose(N @ N.T, Y, atol=1e-13)
    assert np.array_equal(N, np.tril(N)) and np.all(np.diag(N) > 0)
    n = inst.n
    blk = np.minimum(np.arange(n) // 6, 4)
    inside = (blk[:, None] == blk[None, :]) | (blk[:, None] == 4) | (blk[None, :] == 4)
    assert np.all(N[~inside] == 0.0)
