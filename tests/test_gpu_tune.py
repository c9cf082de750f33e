"""The tile-shape tuner on the device (mcsdp_tune): it times the candidate SCM groupings, keeps
the fastest, caches it per (n, m, largest clique) rounded up to powers of two, and the tuned
options solve to the oracle's optimum."""
import numpy as np
import pytest
import torch

from instances import SDPInstance, batch_mix, random_gnm_maxcut
from oracle import pdipm
from oracle.sdp import SparseSym

pytestmark = pytest.mark.gpu

CAND = [(64, 80), (32, 80), (16, 80), (64, 96), (32, 48)]


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1310_6919_gb300 import build_library
    build_library()
    assert torch.cuda.is_available()


def test_tune_picks_fastest_and_caches():
    from paper_1310_6919_gb300 import tune, tune_cache_clear, Problem
    tune_cache_clear()
    inst = random_gnm_maxcut(180, 450, 11)
    opts, info = tune(inst, iters=3)
    assert not info["cached"] and info["ncand"] == 5
    ms = np.array(info["ms_per_iter"])
    assert np.all(ms > 0)
    pick = (opts["group_max"], opts["panel_max"])
    assert pick == CAND[int(np.argmin(ms))]
    assert info["key"] == [256, 256, info["key"][2]] and info["key"][2] >= 1
    # a problem of the same key takes the cached choice without timing
    inst2 = random_gnm_maxcut(200, 500, 12)
    opts2, info2 = tune(inst2, iters=3)
    if info2["key"] == info["key"]:
        assert info2["cached"] and (opts2["group_max"], opts2["panel_max"]) == pick
    # the tuned grouping solves to the oracle's optimum
    P = Problem.from_instance(inst, device=0, **opts)
    r = P.solve()
    ref = pdipm.solve_dense(SparseSym.from_instance(inst), inst.b, inst.z0)
    assert r["status"] == 0
    assert abs(r["pobj"] - ref["pobj"]) <= 1e-7 * max(1.0, abs(ref["pobj"]))


def test_tune_with_start():
    from paper_1310_6919_gb300 import tune, tune_cache_clear
    tune_cache_clear()
    # a block-arrow SDP of the batch mix (its z0 is required: A_0 is not the max-cut form)
    inst = batch_mix(0, 1)[0]
    opts, info = tune(inst, z0=inst.z0, iters=3)
    ms = np.array(info["ms_per_iter"])
    assert info["ncand"] == 5 and np.all(ms > 0)
    assert (opts["group_max"], opts["panel_max"]) == CAND[int(np.argmin(ms))]


def test_tune_skips_a_candidate_the_constraint_does_not_fit():
    from paper_1310_6919_gb300 import tune, tune_cache_clear, Problem
    tune_cache_clear()
    # min tr(X) s.t. X_00 + .. + X_59,59 = 1 (n = 64): optimum 1; one constraint on 60 rows, more
    # than the (32, 48) candidate's panel
    n = 64
    mat = np.array([0] * n + [1] * 60, np.int32)
    row = np.array(list(range(n)) + list(range(60)), np.int32)
    inst = SDPInstance("wide", n, 1, np.array([1.0]), mat, row, row.copy(), np.ones(len(mat)),
                       z0=np.zeros(1), meta={})
    opts, info = tune(inst, z0=inst.z0, iters=2)
    ms = np.array(info["ms_per_iter"])
    assert ms[4] < 0 and np.all(ms[:4] > 0) and info["ncand"] == 4
    assert (opts["group_max"], opts["panel_max"]) != (32, 48)
    P = Problem.from_instance(inst, device=0, **opts)
    P.set_iterate(None, torch.tensor(inst.z0, device="cuda:0"))
    r = P.solve()
    assert r["status"] == 0 and abs(r["pobj"] - 1.0) <= 1e-7
