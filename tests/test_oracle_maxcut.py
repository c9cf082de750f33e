"""Pins of the dense oracle PDIPM (Sec. 2.2) against max-cut closed forms and brute force."""
import numpy as np
import pytest

from instances import lattice_maxcut, cycle_maxcut, complete_maxcut, random_gnm_maxcut
from oracle.sdp import SparseSym
from oracle import pdipm, maxcut


def _solve(inst):
    A = SparseSym.from_instance(inst)
    return A, pdipm.solve_dense(A, inst.b, inst.z0)


def _two_coloring(n, edges):
    adj = [[] for _ in range(n)]
    for u, v in edges:
        adj[u].append(v)
        adj[v].append(u)
    side = [-1] * n
    for s in range(n):
        if side[s] >= 0:
            continue
        side[s] = 0
        stack = [s]
        while stack:
            u = stack.pop()
            for w in adj[u]:
                if side[w] < 0:
                    side[w] = 1 - side[u]
                    stack.append(w)
    return side


def test_bipartite_lattice_closed_form():
    inst = lattice_maxcut(5, 4, seed=7)
    A, res = _solve(inst)
    W = sum(inst.meta["weights"])
    assert res["status"] == "optimal"
    assert abs(res["pobj"] - (-W)) <= 1e-6 * W
    assert abs(res["dobj"] - (-W)) <= 1e-6 * W
    # the closed-form certificates are feasible and tight (independent of the solver)
    side = _two_coloring(inst.n, inst.meta["edges"])
    X, z = maxcut.bipartite_certificates(inst.n, inst.meta["edges"], inst.meta["weights"], side)
    Y = A.dense(0) - A.adjoint(z)
    assert np.allclose(np.diag(X), 1.0)
    assert np.linalg.eigvalsh(Y)[0] > -1e-12
    assert abs(np.sum(A.dense(0) * X) + W) < 1e-9 * W
    assert abs(np.dot(inst.b, z) + W) < 1e-9 * W


@pytest.mark.parametrize("n", [5, 7, 9])
def test_odd_cycle_closed_form(n):
    inst = cycle_maxcut(n)
    A, res = _solve(inst)
    opt = maxcut.odd_cycle_optimum(n)
    assert res["status"] == "optimal"
    assert abs(res["pobj"] - opt) <= 2e-7 * abs(opt)
    X, z = maxcut.odd_cycle_certificates(n)
    assert np.allclose(np.diag(X), 1.0) and np.linalg.eigvalsh(X)[0] > -1e-12
    Y = A.dense(0) - A.adjoint(z)
    assert np.linalg.eigvalsh(Y)[0] > -1e-12
    assert abs(np.sum(A.dense(0) * X) - opt) < 1e-10 * abs(opt)
    assert abs(np.dot(inst.b, z) - opt) < 1e-10 * abs(opt)


@pytest.mark.parametrize("n", [4, 6])
def test_complete_graph_closed_form(n):
    inst = complete_maxcut(n)
    A, res = _solve(inst)
    opt = maxcut.complete_graph_optimum(n)
    assert abs(res["pobj"] - opt) <= 2e-7 * abs(opt)
    X, z = maxcut.complete_graph_certificates(n)
    assert np.linalg.eigvalsh(X)[0] > -1e-12 and np.allclose(np.diag(X), 1.0)
    assert abs(np.sum(A.dense(0) * X) - opt) < 1e-10 * abs(opt)


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_sdp_bound_vs_brute_force(seed):
    n = 11
    inst = random_gnm_maxcut(n, 22, seed)
    A, res = _solve(inst)
    mc = maxcut.brute_force_maxcut(n, inst.meta["edges"], inst.meta["weights"])
    sdp = -res["pobj"]
    assert sdp >= mc - 1e-6 * mc
    assert mc >= 0.878 * sdp


def test_weak_duality_and_convergence():
    inst = lattice_maxcut(4, 4, seed=3)
    A, res = _solve(inst)
    for h in res["history"]:
        assert h["dobj"] <= h["pobj"] + 1e-9 * max(1.0, abs(h["pobj"]))
    assert res["gap"] <= 1e-7 and res["pinf"] <= 1e-7 and res["dinf"] <= 1e-7
