"""Pins of the oracle's max-det completion and Algorithm 1 (Sec. 2.1, 3.1)."""
import numpy as np
import pytest

from oracle.completion import (max_det_completion, algorithm1, inverse_cholesky_definition)
from oracle.chordal import (check_structure, pattern_from_cliques, is_perfect_elimination)
from tests.chordal_helper import (eliminate, supernodes, column_cliques, random_pattern,
                                  pd_on_pattern)


def _case(n, density, seed):
    rng = np.random.default_rng(seed)
    P = random_pattern(n, density, rng)
    F = eliminate(P)
    cl = supernodes(F)
    X = pd_on_pattern(F, rng, cl)
    return F, cl, X


@pytest.mark.parametrize("n,density,seed", [(8, 0.2, 1), (15, 0.15, 2), (30, 0.08, 3),
                                            (40, 0.05, 4), (25, 0.3, 5)])
def test_completion_invariants(n, density, seed):
    F, cl, X = _case(n, density, seed)
    check_structure(n, cl)
    assert is_perfect_elimination(F)
    assert np.array_equal(pattern_from_cliques(n, cl), F)
    Xh = max_det_completion(X, cl)
    # agrees with X̄ on E
    assert np.allclose(Xh[F], X[F], rtol=0, atol=1e-13)
    # positive definite
    assert np.linalg.eigvalsh(Xh)[0] > 0
    # max-det stationarity: the inverse vanishes off E (Sec. 3.1)
    Xi = np.linalg.inv(Xh)
    assert np.max(np.abs(Xi[~F])) <= 1e-10 * np.max(np.abs(Xi))
    # the clique partition does not matter: column cliques give the same completion
    Xh2 = max_det_completion(X, column_cliques(F))
    assert np.allclose(Xh, Xh2, atol=1e-12)


def test_completion_is_max_determinant():
    F, cl, X = _case(20, 0.15, 11)
    Xh = max_det_completion(X, cl)
    ld0 = np.linalg.slogdet(Xh)[1]
    rng = np.random.default_rng(0)
    off = np.argwhere(~F)
    assert len(off) > 0
    for _ in range(20):
        H = np.zeros_like(Xh)
        for (i, j) in off[rng.choice(len(off), size=min(5, len(off)), replace=False)]:
            t = 1e-2 * rng.standard_normal()
            H[i, j] += t
            H[j, i] += t
        sgn, ld = np.linalg.slogdet(Xh + H)
        if sgn > 0:
            assert ld < ld0


def test_two_clique_closed_form():
    # cliques {0,1} and {1,2}: the lemma's formula gives X̂_02 = X_01 X_12 / X_11
    X = np.array([[2.0, 0.5, 0.0], [0.5, 1.5, -0.3], [0.0, -0.3, 1.0]])
    cl = [(np.array([0, 1]), 1), (np.array([1, 2]), 2)]
    Xh = max_det_completion(X, cl)
    assert abs(Xh[0, 2] - 0.5 * -0.3 / 1.5) < 1e-15
    # scalar check of max det over the free entry t
    ts = np.linspace(-0.6, 0.6, 24001)
    dets = [np.linalg.det(np.array([[2.0, 0.5, t], [0.5, 1.5, -0.3], [t, -0.3, 1.0]])) for t in ts]
    assert abs(ts[int(np.argmax(dets))] - Xh[0, 2]) < 1e-4


@pytest.mark.parametrize("n,density,seed", [(12, 0.2, 1), (30, 0.1, 2), (45, 0.06, 3)])
def test_algorithm1_equals_definition(n, density, seed):
    F, cl, X = _case(n, density, seed)
    Lh = algorithm1(X, cl)
    Xh = max_det_completion(X, cl)
    Ld = inverse_cholesky_definition(Xh)
    assert np.allclose(Lh, Ld, atol=1e-10 * np.max(np.abs(Ld)))
    # L̂ lives on lower(E) only
    low = np.tril(np.ones((n, n), dtype=bool))
    assert np.all(Ld[low & ~F] == 0) or np.max(np.abs(Ld[low & ~F])) < 1e-10
    assert np.all(Lh[~(low & F)] == 0)
    # X̂ = L̂^{-T} L̂^{-1} (validity of Algorithm 1)
    Li = np.linalg.inv(Lh)
    assert np.allclose(Li.T @ Li, Xh, atol=1e-10 * np.max(np.abs(Xh)))


def test_algorithm1_block_identities_two_cliques():
    # C_1 = S ∪ U, C_2' = U ∪ T with S = {0,1}, U = {2,3}, T = {4,5}
    rng = np.random.default_rng(5)
    G = rng.standard_normal((6, 12))
    X = G @ G.T / 12 + np.eye(6)
    F = np.ones((6, 6), dtype=bool)
    F[np.ix_([0, 1], [4, 5])] = False
    F[np.ix_([4, 5], [0, 1])] = False
    Xb = np.where(F, X, 0.0)
    cl = [(np.array([0, 1, 2, 3]), 2), (np.array([2, 3, 4, 5]), 4)]
    Lh = algorithm1(Xb, cl)
    S, U, T = [0, 1], [2, 3], [4, 5]
    C1, C2 = S + U, U + T
    M = np.linalg.cholesky(np.linalg.inv(Xb[np.ix_(C1, C1)]))
    N = np.linalg.cholesky(np.linalg.inv(Xb[np.ix_(C2, C2)]))
    # eq. (widehatL): L̂ = [[M_SS], [M_US, N_UU], [0, N_TU, N_TT]]
    assert np.allclose(Lh[np.ix_(S, S)], M[:2, :2])
    assert np.allclose(Lh[np.ix_(U, S)], M[2:, :2])
    assert np.allclose(Lh[np.ix_(U, U)], N[:2, :2])
    assert np.allclose(Lh[np.ix_(T, U)], N[2:, :2])
    assert np.allclose(Lh[np.ix_(T, T)], N[2:, 2:])
    # eq. (elements-wise): X̄_SU = -M_SS^{-T} M_US^T M_UU^{-T} M_UU^{-1}
    Mi = np.linalg.inv
    lhs = -Mi(M[:2, :2]).T @ M[2:, :2].T @ Mi(M[2:, 2:]).T @ Mi(M[2:, 2:])
    assert np.allclose(lhs, Xb[np.ix_(S, U)])
