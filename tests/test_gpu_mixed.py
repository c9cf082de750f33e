"""Mixed form (precision = 1).  The SCM solves and contraction (K3) and the P-MATRIX solves (K6)
run in FP32 from FP32 copies of L̂ and N; the SCE B dz = g is solved with an FP32 Cholesky factor
of the stored B and FP64 iterative refinement against it; everything else is FP64; the solve
promotes to FP64 throughout near the optimum (relative gap below 1e-5) or when the refinement
cannot reach FP64 accuracy.

Tolerances: B entries 1e-5 relative to the largest entry (FP32 operands and sums over the
nonzero pairs of two constraints); dz solves the SCE with the same (FP32-assembled) B to a
backward error of 1e-10 (the refinement target when B carries FP32 assembly error: far below that
error); optimal values 1e-7 relative at relative gap 1e-7 (the last iterations run in FP64)."""
import json
import os

import numpy as np
import pytest
import torch

from instances import (lattice_maxcut, block_arrow, small_random_sdp, random_gnm_maxcut,
                       cycle_maxcut, workload, SDPInstance)
from oracle import maxcut

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")

SMALL = [
    lambda: lattice_maxcut(10, 10),
    lambda: block_arrow(6, 12, 4, 60, per_matrix=8, seed=5),
    lambda: small_random_sdp(9, 14, 2),
    lambda: random_gnm_maxcut(90, 200, 4),
]
IDS = ["grid100", "arrow6x12", "dense9", "gnm90"]


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1310_6919_gb300 import build_library
    build_library()
    assert torch.cuda.is_available()


def _solve(inst, **opts):
    from paper_1310_6919_gb300 import Problem
    P = Problem.from_instance(inst, device=0, **opts)
    if inst.meta.get("kind") != "maxcut":
        P.set_iterate(None, inst.z0)
    return P, P.solve()


@pytest.mark.parametrize("mk", SMALL, ids=IDS)
def test_mixed_scm_matches_oracle(mk):
    from tests.gpu_helpers import Case
    c = Case(mk(), precision=1)
    Xbar, z = c.random_iterate(5)
    B, h = c.P.scm_assemble(c.to_layout(Xbar), torch.tensor(z, device="cuda:0"), precision=1)
    Bg = B.cpu().numpy()
    Bref, Xh, Yinv = c.oracle_scm(Xbar, z)
    low = np.tril(np.ones_like(Bref, dtype=bool))
    assert np.max(np.abs(Bg[low] - Bref[low])) <= 1e-5 * np.max(np.abs(Bref))
    href = c.A.op(Yinv)
    assert np.max(np.abs(h.cpu().numpy() - href)) <= 1e-5 * np.max(np.abs(href))


@pytest.mark.parametrize("mk", SMALL + [lambda: lattice_maxcut(70, 70)], ids=IDS + ["grid4900"])
def test_mixed_newton_step_solves_its_sce(mk):
    """grid4900: m = 4900 takes the refinement's wide substitutions (all SMs, ticket-ordered
    row blocks) and the tensor-core FP32 factor."""
    from tests.gpu_helpers import Case, rel_err
    inst = mk()
    c = Case(inst, precision=1)
    Xbar, z = c.random_iterate(7)
    Xl, zt = c.to_layout(Xbar), torch.tensor(z, device="cuda:0")
    st = c.P.newton_step(Xl, zt)
    Bt, h = c.P.scm_assemble(Xl, zt, precision=1)
    Bl = np.tril(Bt.cpu().numpy())
    Bs = Bl + np.tril(Bl, -1).T
    g = inst.b - 0.1 * st["mu"] * h.cpu().numpy()
    dz = st["dz"].cpu().numpy()
    # backward error of the refined solve (the refinement target for an FP32-assembled B is
    # 1e-10), and the forward error it implies
    omega = np.max(np.abs(g - Bs @ dz)) / np.max(np.abs(Bs) @ np.abs(dz) + np.abs(g))
    assert omega <= 1e-10
    dz_exact = np.linalg.solve(Bs, g)
    assert rel_err(dz, dz_exact) < 1e-10 * np.linalg.cond(Bs) * 10
    if inst.m >= 4096:
        # the FP32 factor and its refinement solved it: no FP64 SCM factorisation ran
        cnt = c.P.stats()["count"]
        assert cnt["scm_chol32"] > 0 and cnt["scm_chol"] == 0


def test_mixed_scm_full_size_sampled_entries():
    from tests.gpu_helpers import Case
    from oracle.scm import scm_entry
    c = Case(workload("block_arrow_2020"), precision=1)
    Xbar, z = c.random_iterate(11, zscale=0.002)
    B, h = c.P.scm_assemble(c.to_layout(Xbar), torch.tensor(z, device="cuda:0"), precision=1)
    Bg = B.cpu().numpy()
    Xh, _ = c.oracle_completion(Xbar)
    Yinv = np.linalg.inv(c.A.dense(0) - c.A.adjoint(z))
    rng = np.random.default_rng(1)
    m = c.inst.m
    pairs = [(i, j) for i, j in rng.integers(0, m, size=(200, 2))] + [(m - 1, 0), (0, 0)]
    ref = np.array([scm_entry(c.A, Xh, Yinv, max(i, j), min(i, j)) for i, j in pairs])
    got = np.array([Bg[max(i, j), min(i, j)] for i, j in pairs])
    assert np.max(np.abs(got - ref)) <= 1e-5 * np.max(np.abs(np.diag(Bg)))


@pytest.mark.parametrize("name", ["block_arrow_1020", "block_arrow_2020"])
def test_mixed_solve_matches_golden(name):
    with open(os.path.join(GOLDEN, name + ".json")) as f:
        g = json.load(f)
    P, r = _solve(workload(name), precision=1)
    assert r["status"] == 0, r
    assert r["precision"] == 1 and r["refine_steps"] >= 1
    assert 0 < r["promoted_iter"] <= r["iters"]
    scale = max(1.0, abs(g["pobj"]))
    assert abs(r["pobj"] - g["pobj"]) <= 1e-7 * scale
    assert abs(r["dobj"] - g["dobj"]) <= 1e-7 * scale


def test_mixed_closed_forms():
    inst = lattice_maxcut(10, 10)
    P, r = _solve(inst, precision=1)
    W = sum(inst.meta["weights"])
    assert r["status"] == 0 and abs(r["pobj"] + W) <= 1e-7 * W
    inst = cycle_maxcut(9)
    P, r = _solve(inst, precision=1)
    assert r["status"] == 0
    assert abs(r["pobj"] - maxcut.odd_cycle_optimum(9)) <= 1e-7 * abs(maxcut.odd_cycle_optimum(9))


def _near_dependent(delta):
    """min diag(1,2,3,4) . X  s.t.  X11 = 1, X11 + delta X22 = 1 + delta, X33 = 1, X44 = 1.
    The diagonal of X is fixed, so the optimum is 1 + 2 + 3 + 4 = 10.  At X = I, Y = A_0 the SCM
    is [[1, 1], [1, 1 + delta^2 / 2]] in its leading block: exactly singular once formed or
    rounded in FP32 for delta = 1e-4, well conditioned enough (~1e9) for FP64."""
    mat = [0, 0, 0, 0, 1, 2, 2, 3, 4]
    row = [0, 1, 2, 3, 0, 0, 1, 2, 3]
    val = [1.0, 2.0, 3.0, 4.0, 1.0, 1.0, delta, 1.0, 1.0]
    b = np.array([1.0, 1.0 + delta, 1.0, 1.0])
    return SDPInstance("near_dependent", 4, 4, b, np.array(mat, np.int32), np.array(row, np.int32),
                       np.array(row, np.int32), np.array(val), z0=np.zeros(4), meta={"kind": "lp"})


def test_mixed_promotes_when_fp32_factor_breaks_down():
    inst = _near_dependent(1e-4)
    _, r64 = _solve(inst)
    _, rmx = _solve(inst, precision=1)
    assert r64["status"] == 0 and rmx["status"] == 0
    assert abs(r64["pobj"] - 10.0) <= 1e-7 * 10
    assert rmx["promoted_iter"] == 0
    # promotion at the first iteration recomputes that iteration's SCM in FP64, so the mixed
    # solve runs the FP64 path throughout
    assert rmx["iters"] == r64["iters"]
    assert rmx["pobj"] == r64["pobj"] and rmx["dobj"] == r64["dobj"]
