"""Batched form (mcsdp_solve_batch): independent problems solved concurrently, each context on
its own stream, give exactly the results of solving them one at a time (every kernel is
deterministic), and the optima match the oracle's dense PDIPM."""
import numpy as np
import pytest
import torch

from instances import random_gnm_maxcut, block_arrow, lattice_maxcut
from oracle import pdipm
from oracle.sdp import SparseSym

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1310_6919_gb300 import build_library
    build_library()
    assert torch.cuda.is_available()


def _instances():
    return [random_gnm_maxcut(60, 150, 1), random_gnm_maxcut(90, 225, 2),
            random_gnm_maxcut(120, 300, 3), lattice_maxcut(6, 7),
            block_arrow(3, 30, 20, 110, per_matrix=8, seed=9),
            block_arrow(4, 25, 20, 120, per_matrix=8, seed=10),
            random_gnm_maxcut(75, 187, 4), block_arrow(2, 40, 20, 100, per_matrix=8, seed=11)]


def _problem(inst, stream=None):
    from paper_1310_6919_gb300 import Problem
    P = Problem.from_instance(inst, device=0, stream=stream)
    if inst.meta.get("kind") != "maxcut":
        P.set_iterate(None, inst.z0)
    return P


def test_batch_equals_one_at_a_time():
    from paper_1310_6919_gb300 import solve_batch
    insts = _instances()
    ref = []
    for inst in insts:
        r = _problem(inst).solve()
        assert r["status"] == 0, r
        ref.append(r)
    probs = [_problem(inst, torch.cuda.Stream()) for inst in insts]
    torch.cuda.synchronize()
    out = solve_batch(probs, nthreads=4)
    for r, q in zip(ref, out):
        assert q["status"] == 0, q
        assert q["iters"] == r["iters"]
        assert q["pobj"] == r["pobj"] and q["dobj"] == r["dobj"]


def test_batch_optima_match_oracle():
    from paper_1310_6919_gb300 import solve_batch
    insts = _instances()[:3] + _instances()[4:5]
    probs = [_problem(inst, torch.cuda.Stream()) for inst in insts]
    out = solve_batch(probs)
    for inst, q in zip(insts, out):
        A = SparseSym.from_instance(inst)
        z0 = inst.z0
        ref = pdipm.solve_dense(A, inst.b, z0)
        assert q["status"] == 0 and ref["status"] == "optimal"
        scale = max(1.0, abs(ref["pobj"]))
        assert abs(q["pobj"] - ref["pobj"]) <= 1e-7 * scale
