"""Block-diagonal SCM (the sparse-SCM case of Sec. 3.1), host side: the symbolic analysis finds
the connected components of the SCM's structure (aggregate pattern joined through each
constraint's support), keeps each one contiguous in the internal constraint order, and the work
model counts the diagonal blocks only.  The oracle pins: the optimum of a direct sum is the sum of
the parts' closed-form optima, and the oracle's SCM of a direct sum is zero between parts and
equal to each part's own SCM on the diagonal blocks."""
import numpy as np
import pytest

from instances import (SDPInstance, block_arrow, complete_maxcut, cycle_maxcut, diagonal_lp_sdp,
                       direct_sum, lattice_maxcut, random_gnm_maxcut, small_random_sdp)
from oracle import maxcut, pdipm
from oracle.scm import scm_sparse_rows
from oracle.sdp import SparseSym


def scalar_sdp():
    # n = m = 1: min 2x s.t. x = 3
    return SDPInstance("scalar", 1, 1, np.array([3.0]), np.array([0, 1], np.int32),
                       np.array([0, 0], np.int32), np.array([0, 0], np.int32),
                       np.array([2.0, 1.0]), z0=np.array([0.0]), meta={"kind": "scalar"})


def parts():
    return [lattice_maxcut(4, 8, seed=3), block_arrow(3, 12, 4, 40, per_matrix=8, seed=9),
            diagonal_lp_sdp(12, 7, 3), small_random_sdp(9, 14, 2), scalar_sdp()]


def _problem(inst, **kw):
    from paper_1310_6919_gb300 import Problem
    return Problem.from_instance(inst, device=-1, **kw)


def _part_of(ps, con_order):
    bounds = np.cumsum([0] + [p.m for p in ps])
    return np.searchsorted(bounds, con_order, side="right") - 1


def test_direct_sum_components_are_contiguous():
    ps = parts()
    P = _problem(direct_sum(ps))
    # diagonal_lp_sdp's pattern is diagonal (12 components of one vertex); its constraints'
    # supports join them into one
    assert P.info["ncomp"] == len(ps)
    assert P.info["scm_blocks"] == 1
    part = _part_of(ps, P.sym_export()["con_order"])
    changes = np.flatnonzero(np.diff(part)) + 1
    assert len(changes) == len(ps) - 1
    assert sorted(part[np.r_[0, changes]].tolist()) == list(range(len(ps)))


def test_components_joined_through_supports():
    # A_0 = I (pattern: four isolated vertices); A_1 = e0 e0^T + e2 e2^T, A_2 = e1 e1^T,
    # A_3 = e3 e3^T + e1 e1^T: B is block-diagonal over {A_1} and {A_2, A_3}
    mat = np.array([0, 0, 0, 0, 1, 1, 2, 3, 3], np.int32)
    row = np.array([0, 1, 2, 3, 0, 2, 1, 1, 3], np.int32)
    inst = SDPInstance("supports", 4, 3, np.ones(3), mat, row, row.copy(),
                       np.ones(9), z0=np.zeros(3), meta={})
    P = _problem(inst)
    assert P.info["ncomp"] == 2
    order = P.sym_export()["con_order"].tolist()
    assert order in ([0, 1, 2], [0, 2, 1], [1, 2, 0], [2, 1, 0])


def test_connected_pattern_has_one_component():
    for inst in (lattice_maxcut(10, 10), block_arrow(6, 12, 4, 60, seed=5), cycle_maxcut(17)):
        info = _problem(inst).info
        assert info["ncomp"] == 1 and info["scm_blocks"] == 0


def test_isolated_vertex_is_a_component():
    # G(40, 90) of this seed leaves vertices outside the giant component
    inst = random_gnm_maxcut(40, 90, 6)
    A = SparseSym.from_instance(inst)
    E = A.aggregate_pattern()
    # components of the pattern by breadth-first search
    seen = np.full(inst.n, -1)
    nc = 0
    for s in range(inst.n):
        if seen[s] >= 0:
            continue
        stack = [s]
        seen[s] = nc
        while stack:
            u = stack.pop()
            for v in np.flatnonzero(E[u]):
                if seen[v] < 0:
                    seen[v] = nc
                    stack.append(v)
        nc += 1
    assert nc > 1
    assert _problem(inst).info["ncomp"] == nc


def test_whole_matrix_option():
    info = _problem(direct_sum(parts()), scm_blocks=1).info
    assert info["ncomp"] == len(parts()) and info["scm_blocks"] == 0


def test_work_model_counts_diagonal_blocks():
    ps = parts()
    d = direct_sum(ps)
    wb = _problem(d).work_model()
    ww = _problem(d, scm_blocks=1).work_model()
    ms = np.array([p.m for p in ps], dtype=float)
    assert wb["flops"]["scm_chol"] == pytest.approx(np.sum(ms ** 3 / 3 + ms ** 2), rel=1e-12)
    assert wb["bytes"]["scm_chol"] == pytest.approx(np.sum(16 * ms * (ms + 1) / 2), rel=1e-12)
    assert wb["flops"]["sce_backsolve"] == pytest.approx(np.sum(ms ** 2), rel=1e-12)
    m = d.m
    assert ww["flops"]["scm_chol"] == pytest.approx(m ** 3 / 3 + m ** 2, rel=1e-12)
    # tile contraction: pairs of nonzeros within each part
    tiles = 0.0
    for p in ps:
        cnt = np.zeros(p.m)
        for k, i, j in zip(p.mat, p.row, p.col):
            if k > 0:
                cnt[k - 1] += 1 if i == j else 2
        tiles += 2 * (cnt.sum() ** 2 + (cnt ** 2).sum()) / 2
    assert wb["flops"]["scm_tile"] == pytest.approx(tiles, rel=1e-12)


def test_oracle_direct_sum_optimum_is_sum_of_closed_forms():
    # odd cycle C_5 and complete graph K_4 (closed-form max-cut SDP optima) as one SDP
    ps = [cycle_maxcut(5), complete_maxcut(4), cycle_maxcut(7)]
    d = direct_sum(ps)
    ref = pdipm.solve_dense(SparseSym.from_instance(d), d.b, d.z0)
    assert ref["status"] == "optimal"
    opt = (maxcut.odd_cycle_optimum(5) + maxcut.complete_graph_optimum(4) +
           maxcut.odd_cycle_optimum(7))
    assert abs(ref["pobj"] - opt) <= 1e-6 * abs(opt)


def test_oracle_scm_of_direct_sum_is_block_diagonal():
    rng = np.random.default_rng(3)
    ps = [block_arrow(2, 6, 3, 12, per_matrix=4, seed=4), small_random_sdp(5, 6, 1),
          lattice_maxcut(3, 3, seed=2)]
    d = direct_sum(ps)
    A = SparseSym.from_instance(d)
    # block-diagonal X̂ and Y^{-1} (any symmetric positive definite blocks)
    Xh = np.zeros((d.n, d.n))
    Yi = np.zeros((d.n, d.n))
    Bparts = []
    o = 0
    for p in ps:
        G = rng.standard_normal((p.n, p.n + 2))
        H = rng.standard_normal((p.n, p.n + 2))
        Xp, Yp = G @ G.T + np.eye(p.n), H @ H.T + np.eye(p.n)
        Xh[o:o + p.n, o:o + p.n] = Xp
        Yi[o:o + p.n, o:o + p.n] = Yp
        Bparts.append(scm_sparse_rows(SparseSym.from_instance(p), Xp, Yp))
        o += p.n
    B = scm_sparse_rows(A, Xh, Yi)
    mo = np.cumsum([0] + [p.m for p in ps])
    for a in range(len(ps)):
        for c in range(len(ps)):
            blk = B[mo[a]:mo[a + 1], mo[c]:mo[c + 1]]
            if a == c:
                assert np.allclose(blk, Bparts[a], rtol=1e-13, atol=1e-13 * np.abs(blk).max())
            else:
                assert not blk.any()


def _components_reference(inst):
    """Connected components of the SCM structure, by breadth-first search over a graph on the
    vertices: an edge for every input entry (i, j) and between all vertices one constraint
    touches; a constraint's component is that of its vertices."""
    n = inst.n
    adj = [set() for _ in range(n)]
    supp = [set() for _ in range(inst.m)]
    for k, i, j in zip(inst.mat, inst.row, inst.col):
        adj[i].add(j)
        adj[j].add(i)
        if k > 0:
            supp[k - 1].update((int(i), int(j)))
    for s in supp:
        s = sorted(s)
        for a in s[1:]:
            adj[s[0]].add(a)
            adj[a].add(s[0])
    comp = [-1] * n
    nc = 0
    for v in range(n):
        if comp[v] >= 0:
            continue
        stack = [v]
        comp[v] = nc
        while stack:
            u = stack.pop()
            for w in adj[u]:
                if comp[w] < 0:
                    comp[w] = nc
                    stack.append(w)
        nc += 1
    return [comp[min(s)] for s in supp]


@pytest.mark.parametrize("seed", range(6))
def test_components_match_a_graph_search(seed):
    # random direct sums of small SDPs, plus random diagonal-only constraints that may bridge
    # parts (joining their components through the constraint's support alone)
    rng = np.random.default_rng(seed)
    ps = []
    for q in range(int(rng.integers(2, 6))):
        kind = int(rng.integers(0, 3))
        if kind == 0:
            ps.append(lattice_maxcut(int(rng.integers(2, 5)), int(rng.integers(2, 5)), seed=seed + q))
        elif kind == 1:
            ps.append(random_gnm_maxcut(int(rng.integers(8, 30)), int(rng.integers(4, 20)), seed + q))
        else:
            ps.append(small_random_sdp(int(rng.integers(3, 7)), int(rng.integers(2, 6)), seed + q))
    d = direct_sum(ps)
    extra = int(rng.integers(0, 3))
    mat, row, col, val = list(d.mat), list(d.row), list(d.col), list(d.val)
    for e in range(extra):
        for v in rng.choice(d.n, size=2, replace=False):
            mat.append(d.m + e + 1)
            row.append(int(v))
            col.append(int(v))
            val.append(1.0)
    inst = SDPInstance("bridged", d.n, d.m + extra, np.ones(d.m + extra),
                       np.array(mat, np.int32), np.array(row, np.int32), np.array(col, np.int32),
                       np.array(val), z0=None, meta={})
    ref = _components_reference(inst)
    P = _problem(inst)
    assert P.info["ncomp"] == len(set(ref))
    order = P.sym_export()["con_order"]
    labels = [ref[k] for k in order]
    # each component's constraints are contiguous in the internal order
    runs = [labels[0]] + [b for a, b in zip(labels, labels[1:]) if a != b]
    assert len(runs) == len(set(runs))
