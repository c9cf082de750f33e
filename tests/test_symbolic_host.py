"""Host-side tests of libmcsdp (no GPU): the library loads, exports every symbol of
include/mcsdp.h, validates input, and its symbolic analysis yields a clique tree that the oracle's
checks accept (PEO, E ⊇ aggregate pattern, running intersection property)."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from instances import (lattice_maxcut, block_arrow, random_gnm_maxcut, small_random_sdp,
                       cycle_maxcut, workload)
from oracle.chordal import (cliques_from_supernodes, check_structure, pattern_from_cliques,
                            is_perfect_elimination, covers)
from oracle.sdp import SparseSym

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1310_6919_gb300 import build_library, _lib
    build_library()
    return _lib.load()


def test_exports_every_declared_symbol(lib):
    hdr = open(os.path.join(ROOT, "include", "mcsdp.h")).read()
    declared = set(re.findall(r"\b(mcsdp_[a-z_]+)\s*\(", hdr))
    assert len(declared) >= 14
    for name in declared:
        assert hasattr(lib, name), name


def _problem(inst, **kw):
    from paper_1310_6919_gb300 import Problem
    return Problem.from_instance(inst, device=-1, **kw)


@pytest.mark.parametrize("inst", [lattice_maxcut(10, 10), lattice_maxcut(6, 5, seed=3),
                                  block_arrow(6, 12, 4, 60, seed=5), random_gnm_maxcut(60, 150, 4),
                                  small_random_sdp(9, 12, 2), cycle_maxcut(17),
                                  # n = 8400: above 8192 vertices (the ordering's larger-n range)
                                  lattice_maxcut(4, 2100, seed=9)],
                         ids=lambda i: i.name)
def test_symbolic_structure_is_valid(inst):
    P = _problem(inst)
    s = P.sym_export()
    n = inst.n
    cl = cliques_from_supernodes(s["sn_col"], s["sn_rowptr"], s["sn_rows"])
    check_structure(n, cl)
    E = pattern_from_cliques(n, cl)
    assert is_perfect_elimination(E)
    A = SparseSym.from_instance(inst)
    assert covers(E, s["perm"], A.aggregate_pattern())
    assert sorted(s["perm"].tolist()) == list(range(n))
    assert sorted(s["con_order"].tolist()) == list(range(inst.m))
    info = P.info
    assert info["nnz_layout"] == int(s["sn_valptr"][-1])
    assert info["nnz_lower_E"] == int(np.tril(E).sum())


def _min_degree_fill(P):
    """Filled pattern (original indices) of exact minimum-degree elimination on the elimination
    graph, ties broken by the smallest index: at each step the vertex of least current degree is
    eliminated and its neighbours become a clique."""
    n = P.shape[0]
    adj = [set(np.nonzero(P[v])[0].tolist()) - {v} for v in range(n)]
    alive = set(range(n))
    F = P | P.T | np.eye(n, dtype=bool)
    while alive:
        v = min(alive, key=lambda u: (len(adj[u]), u))
        N = adj[v]
        for u in N:
            adj[u] |= N
            adj[u].discard(u)
            adj[u].discard(v)
        K = sorted(N | {v})
        F[np.ix_(K, K)] = True
        alive.remove(v)
        adj[v] = set()
    return F


@pytest.mark.parametrize("inst", [lattice_maxcut(6, 5, seed=3), random_gnm_maxcut(60, 150, 4),
                                  random_gnm_maxcut(150, 400, 7), block_arrow(6, 12, 4, 60, seed=5),
                                  small_random_sdp(9, 12, 2), cycle_maxcut(17)],
                         ids=lambda i: i.name)
def test_pattern_is_the_minimum_degree_fill(inst):
    # without amalgamation the cliques are the fundamental supernodes, so E is exactly the
    # filled graph of the ordering: it must be that of exact minimum degree with smallest-index
    # ties (the etree postorder the library applies afterwards does not change the filled graph)
    P = _problem(inst, relax=0)
    s = P.sym_export()
    cl = cliques_from_supernodes(s["sn_col"], s["sn_rowptr"], s["sn_rows"])
    E_new = pattern_from_cliques(inst.n, cl)
    iperm = np.empty(inst.n, dtype=np.int64)
    iperm[s["perm"]] = np.arange(inst.n)
    E_orig = E_new[np.ix_(iperm, iperm)]
    A = SparseSym.from_instance(inst)
    assert np.array_equal(E_orig, _min_degree_fill(A.aggregate_pattern()))


def test_block_arrow_pattern_stays_block_arrow():
    # the n = 2020 block-arrow SDP (40 blocks of 50, border 20): its aggregate pattern is chordal
    # in any order that eliminates each block before the border, and minimum degree does so
    # (block vertices have degree < 70, border vertices about 2000), so E adds no entry between
    # two blocks, no clique exceeds block + border (70), and nnz(lower E) stays under the
    # block-arrow bound 40 (50 * 20 + 50 * 51 / 2) + 20 * 21 / 2 = 91210
    inst = workload("block_arrow_2020")
    P = _problem(inst)
    s = P.sym_export()
    cl = cliques_from_supernodes(s["sn_col"], s["sn_rowptr"], s["sn_rows"])
    assert max(len(r) for r, _ in cl) <= 70
    E_new = pattern_from_cliques(inst.n, cl)
    iperm = np.empty(inst.n, dtype=np.int64)
    iperm[s["perm"]] = np.arange(inst.n)
    E = E_new[np.ix_(iperm, iperm)]
    blk = np.minimum(np.arange(inst.n) // 50, 40)      # border vertices -> 40
    I, J = np.nonzero(E)
    assert np.all((blk[I] == blk[J]) | (blk[I] == 40) | (blk[J] == 40))
    assert P.info["nnz_lower_E"] <= 40 * (50 * 20 + 50 * 51 // 2) + 20 * 21 // 2


def test_sorted_list_ordering_range():
    # n = 34000 > 32768: the ordering keeps its elimination graph as sorted lists instead of
    # bitsets.  Dense E would not fit a test, so the checks are sparse: the cliques form a clique
    # tree with the running intersection property, and every aggregate entry lies in the clique
    # of its smaller (elimination-order) index.
    inst = lattice_maxcut(4, 8500, seed=3)
    P = _problem(inst)
    s = P.sym_export()
    n = inst.n
    cl = cliques_from_supernodes(s["sn_col"], s["sn_rowptr"], s["sn_rows"])
    check_structure(n, cl)
    assert sorted(s["perm"].tolist()) == list(range(n))
    iperm = np.empty(n, dtype=np.int64)
    iperm[s["perm"]] = np.arange(n)
    col2c = np.empty(n, dtype=np.int64)
    for r, (rows, ns) in enumerate(cl):
        col2c[rows[:ns]] = r
    rowsets = [set(rows.tolist()) for rows, _ in cl]
    for i, j in zip(inst.row, inst.col):
        p, q = sorted((int(iperm[i]), int(iperm[j])))
        assert q in rowsets[col2c[p]]


def test_host_only_context_refuses_device_work():
    from paper_1310_6919_gb300 import MCSDPError
    P = _problem(lattice_maxcut(4, 4))
    with pytest.raises(MCSDPError) as e:
        P.solve()
    assert "ERR_STATE" in str(e.value)


def _raw_create(lib, n, m, b, mat, row, col, val):
    from paper_1310_6919_gb300 import _lib
    b = np.asarray(b, np.float64)
    arrs = [np.asarray(a, np.int32) for a in (mat, row, col)]
    v = np.asarray(val, np.float64)
    prob = _lib.Problem_t(n, m, 1, b.ctypes.data_as(C.POINTER(C.c_double)), len(v),
                          *[a.ctypes.data_as(C.POINTER(C.c_int32)) for a in arrs],
                          v.ctypes.data_as(C.POINTER(C.c_double)))
    opt = _lib.Options_t()
    lib.mcsdp_default_options(C.byref(opt))
    opt.device = -1
    ctx = C.c_void_p()
    st = lib.mcsdp_create(C.byref(prob), C.byref(opt), None, C.byref(ctx))
    msg = lib.mcsdp_last_error(ctx).decode()
    lib.mcsdp_destroy(ctx)
    return st, msg


def test_input_validation(lib):
    ok = ([0, 1, 1], [0, 0, 1], [1, 0, 1], [1.0, 1.0, 1.0])
    assert _raw_create(lib, 2, 1, [1.0], *ok)[0] == 0
    st, msg = _raw_create(lib, 2, 1, [1.0], [0, 1, 1], [1, 0, 0], [0, 0, 0], [1.0, 1.0, 1.0])
    assert st == 1 and "row > col" in msg
    st, msg = _raw_create(lib, 2, 1, [1.0], [0, 1, 1], [0, 0, 0], [0, 0, 0], [1.0, 1.0, 2.0])
    assert st == 1 and "duplicate" in msg
    st, msg = _raw_create(lib, 2, 1, [1.0], [0, 3], [0, 0], [0, 0], [1.0, 1.0])
    assert st == 1 and "out of range" in msg
    st, msg = _raw_create(lib, 0, 1, [1.0], [0], [0], [0], [1.0])
    assert st == 1
    st, msg = _raw_create(lib, 2, 1, [np.nan], *ok)
    assert st == 1


@pytest.mark.parametrize("inst", [lattice_maxcut(6, 5, seed=3), block_arrow(6, 12, 4, 60, seed=5),
                                  small_random_sdp(9, 12, 2)], ids=lambda i: i.name)
def test_layout_index_covers_lower_E_once(inst):
    # the binding's map from layout positions to (row, col) in the caller's indices, which the
    # GPU parity tests use to compare layouts with dense oracle matrices: its valid positions are
    # the entries of lower(E), each exactly once, rows >= columns in the elimination order
    P = _problem(inst)
    ro, co, valid, s = P.layout_index()
    assert len(ro) == P.info["nnz_layout"]
    cl = cliques_from_supernodes(s["sn_col"], s["sn_rowptr"], s["sn_rows"])
    E_new = np.tril(pattern_from_cliques(inst.n, cl))
    perm = s["perm"].astype(np.int64)
    want = {(int(perm[i]), int(perm[j])) for i, j in zip(*np.nonzero(E_new))}
    got = list(zip(ro[valid].tolist(), co[valid].tolist()))
    assert len(got) == len(set(got)) == len(want) == P.info["nnz_lower_E"]
    assert set(got) == want
