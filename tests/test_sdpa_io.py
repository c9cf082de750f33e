"""SDPA sparse text format: round trips, the SDPA -> paper sign map (Sec. 1), several blocks on
one diagonal, and the content hashes of the named workloads.

The map is pinned through the oracle: a max-cut relaxation written in SDPA's convention
(maximise F_0 . Y, F_0 = L/4) must come back as the paper's minimisation with A_0 = -L/4, whose
optimum on a bipartite graph is minus the total weight; a problem of two independent blocks must
have the sum of the two blocks' optima.
"""
import os

import numpy as np
import pytest

from instances import block_arrow, lattice_maxcut, small_random_sdp, workload, sdpa
from oracle import pdipm
from oracle.sdp import SparseSym

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# 4-cycle, unit weights, in SDPA's convention: max (L/4) . Y  s.t.  Y_ii = 1
CYCLE4 = """"4-cycle max-cut relaxation
* SDPA dual: max F0.Y s.t. Fk.Y = ck
4 =mdim
1 =nblock
{4}
{1.0, 1.0, 1.0, 1.0}
0 1 1 1 0.5
0 1 2 2 0.5
0 1 3 3 0.5
0 1 4 4 0.5
0 1 1 2 -0.25
0 1 2 3 -0.25
0 1 3 4 -0.25
0 1 1 4 -0.25
1 1 1 1 1
2 1 2 2 1
3 1 3 3 1
4 1 4 4 1
"""

# the same cycle plus a diagonal (LP) block: y_1 = 1, y_2 = 2, objective 3 y_1 - y_2 = 1
TWO_BLOCKS = """6
2
4 -2
1 1 1 1 1 2
0 1 1 1 0.5
0 1 2 2 0.5
0 1 3 3 0.5
0 1 4 4 0.5
0 1 1 2 -0.25
0 1 2 3 -0.25
0 1 3 4 -0.25
0 1 1 4 -0.25
0 2 1 1 3
0 2 2 2 -1
1 1 1 1 1
2 1 2 2 1
3 1 3 3 1
4 1 4 4 1
5 2 1 1 1
6 2 2 2 1
"""


def _same(a, b):
    assert (a.n, a.m) == (b.n, b.m)
    assert np.array_equal(a.b, b.b)
    for f in ("mat", "row", "col", "val"):
        assert np.array_equal(getattr(a, f), getattr(b, f)), f


@pytest.mark.parametrize("inst", [lattice_maxcut(4, 3, seed=2), small_random_sdp(6, 5, 1),
                                  block_arrow(3, 5, 2, 12, per_matrix=4, seed=9)],
                         ids=lambda i: i.name)
def test_round_trip_is_exact(inst, tmp_path):
    h = sdpa.write(inst, tmp_path / "p.dat-s")
    back, h2 = sdpa.read(tmp_path / "p.dat-s")
    assert h == h2 == sdpa.content_hash(sdpa.to_text(inst))
    _same(back, inst)
    # the text carries F_0 = -A_0 and c = b
    body = sdpa.to_text(inst).splitlines()
    assert body[1:4] == [str(inst.m), "1", str(inst.n)]


def _diag_dominant_start(inst):
    """z0_k = -(sum_j |[A_0]_ij|) - 1 for constraints A_k = e_i e_i^T: A_0 - sum z_k A_k is
    strictly diagonally dominant."""
    A = SparseSym.from_instance(inst)
    A0 = A.dense(0)
    z0 = np.empty(inst.m)
    for k in range(1, inst.m + 1):
        r, c, v = inst.matrix_entries(k)
        assert len(v) == 1 and r[0] == c[0] and v[0] == 1.0
        z0[k - 1] = -np.abs(A0[r[0]]).sum() - 1.0
    return A, z0


def test_sdpa_sign_map_through_the_oracle():
    inst = sdpa.parse(CYCLE4, "cycle4")
    assert (inst.n, inst.m) == (4, 4) and np.all(inst.b == 1.0)
    A, z0 = _diag_dominant_start(inst)
    A0 = A.dense(0)
    assert A0[0, 0] == -0.5 and A0[0, 1] == 0.25      # A_0 = -F_0 = -L/4
    res = pdipm.solve_dense(A, inst.b, z0)
    assert res["status"] == "optimal"
    # paper optimum -4 (all four edges cut); SDPA's dual optimum is +4
    assert res["pobj"] == pytest.approx(-4.0, rel=1e-7)


def test_two_blocks_on_one_diagonal():
    inst = sdpa.parse(TWO_BLOCKS, "cycle4+lp2")
    assert (inst.n, inst.m) == (6, 6)
    assert inst.meta["block_offsets"] == [0, 4, 6]
    A, z0 = _diag_dominant_start(inst)
    A0 = A.dense(0)
    assert np.all(A0[:4, 4:] == 0.0) and A0[4, 4] == -3.0 and A0[5, 5] == 1.0
    X0 = np.diag([1.0, 1.0, 1.0, 1.0, 1.0, 2.0])       # primal feasible: A(X0) = b
    res = pdipm.solve_dense(A, inst.b, z0, X0=X0)
    assert res["status"] == "optimal"
    # independent blocks: -(4 + (3 * 1 - 1 * 2)) = -5
    assert res["pobj"] == pytest.approx(-5.0, rel=1e-7)


@pytest.mark.parametrize("bad,msg", [
    (TWO_BLOCKS.replace("0 2 2 2 -1", "0 2 1 2 -1"), "off-diagonal entry in diagonal block"),
    (CYCLE4.replace("4 1 4 4 1", "4 1 4 5 1"), "outside block"),
    (CYCLE4.replace("4 1 4 4 1", "4 1 4 4 1\n4 1 4 4 2"), "duplicate"),
    (CYCLE4.replace("{1.0, 1.0, 1.0, 1.0}", "{1.0, 1.0, 1.0}"), "more than m entries"),
    (CYCLE4.replace("0 1 1 1 0.5", "0 1 1 1"), "5 fields"),
])
def test_malformed_text_is_rejected(bad, msg):
    with pytest.raises(ValueError, match=msg):
        sdpa.parse(bad)


def test_library_accepts_both_input_forms():
    # the library's form 0 takes the SDPA data as written (F_0, c); form 1 the paper's (A_0, b):
    # both describe the same problem, so the host analysis must agree
    from paper_1310_6919_gb300 import Problem
    inst = sdpa.parse(TWO_BLOCKS, "cycle4+lp2")
    F = np.where(inst.mat == 0, -inst.val, inst.val)
    P0 = Problem(inst.n, inst.m, inst.b, inst.mat, inst.row, inst.col, F, form=0, device=-1)
    P1 = Problem.from_instance(inst, device=-1)
    s0, s1 = P0.sym_export(), P1.sym_export()
    for k in s1:
        assert np.array_equal(s0[k], s1[k]), k
    assert P0.info == P1.info


def test_named_workload_hashes():
    # the seeded generators still write the same bytes (inputs never change silently)
    want = {}
    with open(os.path.join(ROOT, "instances", "workloads.sha256")) as f:
        for line in f:
            h, name = line.split()
            want[name[:-len(".dat-s")]] = h
    assert set(want) == set(sdpa.NAMED)
    for name in sdpa.NAMED:
        assert sdpa.content_hash(sdpa.to_text(workload(name))) == want[name], name


def test_golden_values_belong_to_the_current_inputs():
    # the stored oracle optima were computed on exactly the instances the generators write now
    import json
    gdir = os.path.join(ROOT, "tests", "golden")
    names = sorted(f[:-5] for f in os.listdir(gdir) if f.endswith(".json"))
    assert names
    for name in names:
        with open(os.path.join(gdir, name + ".json")) as f:
            g = json.load(f)
        inst = workload(g["workload"])
        assert (g["n"], g["m"]) == (inst.n, inst.m)
        assert g["instance_sha256"] == sdpa.content_hash(sdpa.to_text(inst)), name
