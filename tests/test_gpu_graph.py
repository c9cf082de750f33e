"""The graph forms of the iteration against the ordinary host-driven loop.  options.graph = 1:
from the second iteration on, each iteration's direction, update and new factors are captured
once into a CUDA graph and replayed, with the step lengths chosen on the device; graph = 2: the
same iteration as the body of a WHILE conditional node whose loop test runs on the device (the
host loop's convergence and failure tests on the new iterate), so the rest of the solve is one
graph launch.  Both give the same iterates bit for bit (the device keeps the dual step's
candidate bracket by the host loop's own rule, and decides the loop's end from the same FP64
scalars), hence the same optimum and iteration count, on problems of the batched
configuration's kinds, and at an iteration limit."""
import numpy as np
import pytest
import torch

from instances import lattice_maxcut, block_arrow, random_gnm_maxcut, batch_mix

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1310_6919_gb300 import build_library
    build_library()
    assert torch.cuda.is_available()


def _solve(inst, **opts):
    from paper_1310_6919_gb300 import Problem
    P = Problem.from_instance(inst, device=0, **opts)
    if inst.meta.get("kind") != "maxcut":
        P.set_iterate(None, torch.tensor(inst.z0, device="cuda:0"))
    r = P.solve()
    X, z, _ = P.get_iterate()
    return P, r, X.cpu().numpy(), z.cpu().numpy()


CASES = [lambda: lattice_maxcut(10, 10), lambda: block_arrow(6, 12, 4, 60, per_matrix=8, seed=5),
         lambda: random_gnm_maxcut(90, 200, 4), lambda: batch_mix(2, 2)[1],
         lambda: batch_mix(2, 2)[3]]
IDS = ["grid100", "arrow6x12", "gnm90", "mix_maxcut", "mix_arrow"]


@pytest.mark.parametrize("graph", [1, 2], ids=["per_iteration", "solve_graph"])
@pytest.mark.parametrize("mk", CASES, ids=IDS)
def test_graph_iterates_equal_host_loop(mk, graph):
    inst = mk()
    P0, r0, X0, z0 = _solve(inst)
    P1, r1, X1, z1 = _solve(inst, graph=graph)
    assert r0["status"] == 0 and r1["status"] == 0
    assert r1["iters"] == r0["iters"]
    assert r1["pobj"] == r0["pobj"] and r1["dobj"] == r0["dobj"]
    assert np.array_equal(X1, X0) and np.array_equal(z1, z0)
    # the replayed graph's launches are counted; the host loop issues more synchronisations,
    # not fewer kernels
    assert P1.stats()["launches"] > 0


@pytest.mark.parametrize("max_iter", [3, 9])
def test_solve_graph_stops_at_the_iteration_limit(max_iter):
    from paper_1310_6919_gb300 import Problem
    inst = lattice_maxcut(10, 10)
    z0 = torch.tensor(inst.z0, device="cuda:0")
    out = []
    for g in (0, 2, 2):
        P = out[-1][0] if len(out) == 2 else Problem.from_instance(inst, device=0, graph=g,
                                                                     max_iter=max_iter)
        P.set_iterate(P.identity_layout(), z0)
        r = P.solve()
        X, z, _ = P.get_iterate()
        out.append((P, r, X.cpu().numpy(), z.cpu().numpy()))
    # host loop, solve graph, and the solve graph again on the same context (graph reused)
    for P, r, X, z in out:
        assert r["status"] == 3 and r["iters"] == max_iter  # MCSDP_ERR_MAXITER
        assert np.array_equal(X, out[0][2]) and np.array_equal(z, out[0][3])


@pytest.mark.parametrize("graph", [1, 2], ids=["per_iteration", "solve_graph"])
def test_graph_batch(graph):
    from paper_1310_6919_gb300 import Problem, solve_batch
    mix = batch_mix(12, 4)
    plain, graphed = [], []
    for q in mix:
        for lst, g in ((plain, 0), (graphed, graph)):
            P = Problem.from_instance(q, device=0, stream=torch.cuda.Stream(0), graph=g)
            if q.meta.get("kind") != "maxcut":
                P.set_iterate(None, torch.tensor(q.z0, device="cuda:0"))
            lst.append(P)
    ra = solve_batch(plain, nthreads=8)
    rb = solve_batch(graphed, nthreads=8)
    assert all(r["status"] == 0 for r in rb)
    assert [r["pobj"] for r in ra] == [r["pobj"] for r in rb]
