"""Mixed form (precision = 1): FP32 Cholesky factor of the FP64 SCM, FP64 iterative refinement of
the SCE B dz = g (eq. SCE), promotion to the FP64 factor when the refinement cannot reach FP64
accuracy.  The refinement stops at a backward error of sqrt(m) * 2^-53, so the direction carries
the FP64 tolerances of the FP64 form: 1e-8 against the oracle, 1e-9 against the FP64 form at
full size; optimal values 1e-7 relative at relative gap 1e-7."""
import json
import os

import numpy as np
import pytest
import torch

from instances import (lattice_maxcut, block_arrow, small_random_sdp, random_gnm_maxcut,
                       cycle_maxcut, workload, SDPInstance)
from oracle import pdipm, maxcut

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
def test_mixed_newton_step_matches_oracle(mk):
    from tests.gpu_helpers import Case, rel_err
    c = Case(mk(), precision=1)
    Xbar, z = c.random_iterate(7)
    st = c.P.newton_step(c.to_layout(Xbar), torch.tensor(z, device="cuda:0"))
    ref = pdipm.mc_newton_step(c.A, c.inst.b, c.perm, c.cliques, Xbar, z)
    assert rel_err(st["dz"].cpu().numpy(), ref["dz"]) < 1e-8
    dX = c.from_layout(st["dX"])
    assert rel_err(dX[c.E], ref["dX"][c.E]) < 1e-8
    assert abs(st["alpha_p"] - ref["alpha_p"]) <= 1e-7 * ref["alpha_p"]


def test_mixed_direction_matches_fp64_full_size():
    from tests.gpu_helpers import Case, rel_err
    inst = workload("block_arrow_1020")
    c64 = Case(inst)
    c32 = Case(inst, precision=1)
    Xbar, z = c64.random_iterate(11, zscale=0.002)
    zt = torch.tensor(z, device="cuda:0")
    a = c64.P.newton_step(c64.to_layout(Xbar), zt)
    b = c32.P.newton_step(c32.to_layout(Xbar), zt)
    assert rel_err(b["dz"].cpu().numpy(), a["dz"].cpu().numpy()) < 1e-9
    assert rel_err(b["dX"].cpu().numpy(), a["dX"].cpu().numpy()) < 1e-9
    assert abs(b["alpha_p"] - a["alpha_p"]) <= 1e-8 * a["alpha_p"]


@pytest.mark.parametrize("name", ["block_arrow_1020", "block_arrow_2020"])
def test_mixed_solve_matches_golden(name):
    with open(os.path.join(GOLDEN, name + ".json")) as f:
        g = json.load(f)
    P, r = _solve(workload(name), precision=1)
    assert r["status"] == 0, r
    assert r["precision"] == 1 and r["refine_steps"] >= 1
    assert r["promoted_iter"] == -1 or 0 <= r["promoted_iter"] <= r["iters"]
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
    is [[1, 1], [1, 1 + delta^2 / 2]] in its leading block: exactly singular once rounded to FP32
    for delta = 1e-4, well conditioned enough (~1e9) for FP64."""
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
    # after promotion at the first iteration the mixed solve runs the FP64 path throughout
    assert rmx["iters"] == r64["iters"]
    assert rmx["pobj"] == r64["pobj"] and rmx["dobj"] == r64["dobj"]
