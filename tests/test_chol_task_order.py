"""The ticket order of the FP64 SCM factorisation's task queue (no GPU).

The persistent factorisation hands out tasks of a right-looking blocked Cholesky on 32 x 32 tiles
(Sec. 3.1, type (i)) in ticket order; a CTA waits for a task's inputs before it runs it.  The queue
cannot deadlock if every task's inputs come from tasks with smaller tickets: the CTA holding the
smallest unfinished ticket then never waits on anything unfinished.  The library's host copy of
the ticket decode (mcsdp_chol_task_order) is the same function the kernel calls, so these checks
cover the order the kernel uses.

The dependencies are those of the blocked algorithm, written here from its definition:
  L(k, k)   = chol(B(k, k) - sum_{l<k} L(k, l) L(k, l)^T)
  L(i, k)   = (B(i, k) - sum_{l<k} L(i, l) L(k, l)^T) L(k, k)^-T       (i > k)
with the updates of one tile applied in the order l = 0, 1, ... (the kernel serialises them).
Tile (k+1, k) is solved in eight four-row pieces and the update of (k+1, k+1) by panel k in eight
pieces; each piece has the dependencies of the whole task it is part of."""
import ctypes as C
from collections import Counter

import numpy as np
import pytest

NB = 32
PIECES = NB // 4
POTRF0, TRSM, UPD, DIAG, TS, UD = range(6)


@pytest.fixture(scope="module")
def lib():
    from paper_1310_6919_gb300 import build_library, _lib
    build_library()
    return _lib.load()


def _order(lib, m, rows):
    n = C.c_int64(-1)
    assert lib.mcsdp_chol_task_order(m, rows, C.byref(n), None) == 0
    t = np.full((n.value, 4), -7, np.int32)
    assert lib.mcsdp_chol_task_order(m, rows, C.byref(n), C.c_void_p(t.ctypes.data)) == 0
    return [tuple(int(v) for v in r) for r in t]


def _expected_tasks(R, Cn):
    """every task of the blocked factorisation of an R x Cn tile matrix (lower part)"""
    out = [(POTRF0, 0, 0, 0)]
    for p in range(1, Cn):
        out.append((DIAG, p, p, p))
        out += [(TS, p, s, p) for s in range(PIECES)]
        out += [(UD, p, s, p) for s in range(PIECES)]
    for k in range(Cn):
        for i in range(k + 1, R):
            if not (i == k + 1 and i < Cn):  # tile (k+1, k) goes to the TS pieces
                out.append((TRSM, i, k, k))
        for j in range(k + 1, Cn):
            for i in range(j, R):
                if not (i == j == k + 1):    # update of (k+1, k+1) by panel k: the UD pieces
                    out.append((UPD, i, j, k))
    return out


def _key(task):
    """the (kind, tile, panel) a task completes: 'L' = L(i, k) final, 'U' = the update of tile
    (i, j) by panel k applied"""
    ty, i, j, k = task
    if ty == POTRF0:
        return ("L", 0, 0)
    if ty == DIAG:
        return ("L", k, k)
    if ty == TRSM:
        return ("L", i, k)
    if ty == TS:
        return ("L", k, k - 1)
    if ty == UPD:
        return ("U", i, j, k)
    return ("U", k, k, k - 1)  # UD


def _needs(task, Cn):
    """keys that must be complete (all pieces) before the task may start"""
    ty, i, j, k = task
    if ty == POTRF0:
        return []
    if ty == DIAG:      # L(k, k): every update of (k, k)
        return [("U", k, k, l) for l in range(k)]
    if ty == TRSM:      # L(i, k): L(k, k) and every update of (i, k)
        return [("L", k, k)] + [("U", i, k, l) for l in range(k)]
    if ty == TS:        # a piece of L(k, k-1)
        return [("L", k - 1, k - 1)] + [("U", k, k - 1, l) for l in range(k - 1)]
    if ty == UPD:       # (i, j) -= L(i, k) L(j, k)^T after the earlier updates of (i, j)
        return [("L", i, k), ("L", j, k)] + [("U", i, j, l) for l in range(k)]
    # UD: a piece of the update of (k, k) by panel k-1
    return [("L", k, k - 1)] + [("U", k, k, l) for l in range(k - 1)]


def _check(lib, m, rows):
    R, Cn = -(-rows // NB), -(-m // NB)
    order = _order(lib, m, rows)
    # every task exactly once
    got = Counter(order)
    assert max(got.values()) == 1, [t for t, c in got.items() if c > 1][:5]
    want = _expected_tasks(R, Cn)
    assert set(order) == set(want) and len(order) == len(want)
    # pieces per key: a key is complete once all its tasks have been handed out
    pieces = Counter(_key(t) for t in order)
    done = Counter()
    for ticket, task in enumerate(order):
        for need in _needs(task, Cn):
            assert done[need] == pieces[need], (m, rows, ticket, task, need)
        done[_key(task)] += 1
    return order


@pytest.mark.parametrize("m", [1, 2, 31, 32, 33, 60, 63, 64, 65, 95, 96, 97, 128, 200, 257, 400])
def test_every_task_once_and_inputs_earlier(lib, m):
    _check(lib, m, m + 1)
    _check(lib, m, m)


def test_order_at_the_bench_scale(lib):
    # the 2020-column SCM of the block-arrow workload (64 column tiles, about 45k tasks)
    order = _check(lib, 2020, 2021)
    # the chain runs ahead: the diagonal factor of tile p is handed out before the updates by
    # panel p - 1 of the columns right of p + 1 (lookahead), and the tiles' first panel solves
    # before any update
    pos = {t: n for n, t in enumerate(order)}
    for p in range(2, 62):
        first_late = min(pos[(UPD, i, p + 2, p - 1)] for i in range(p + 2, 64))
        assert pos[(DIAG, p, p, p)] < first_late


def test_bad_arguments(lib):
    n = C.c_int64(0)
    assert lib.mcsdp_chol_task_order(0, 1, C.byref(n), None) != 0
    assert lib.mcsdp_chol_task_order(5, 4, C.byref(n), None) != 0
    assert lib.mcsdp_chol_task_order(5, 6, None, None) != 0


def _block_order(lib, mb):
    arr = np.array(mb, np.int32)
    n = C.c_int64(-1)
    assert lib.mcsdp_chol_block_task_order(len(mb), C.c_void_p(arr.ctypes.data), C.byref(n),
                                           None) == 0
    t = np.full((n.value, 5), -7, np.int32)
    assert lib.mcsdp_chol_block_task_order(len(mb), C.c_void_p(arr.ctypes.data), C.byref(n),
                                           C.c_void_p(t.ctypes.data)) == 0
    return t


@pytest.mark.parametrize("mb", [[1], [1, 1, 1], [31, 32, 33], [64, 1, 100, 7, 400, 33],
                                [5] * 40 + [200], list(range(1, 70, 3))],
                         ids=["one", "ones", "tile_edges", "mixed", "many_small", "ramp"])
def test_block_queue_keeps_each_blocks_order(lib, mb):
    """The block-diagonal SCM's one-launch factorisation interleaves the blocks' tickets phase by
    phase.  Blocks share no data, so the queue is deadlock-free if each block's tasks appear in
    its own single-matrix order (checked above for every size): then the smallest unfinished
    ticket's inputs are earlier tasks of its block, all finished."""
    t = _block_order(lib, mb)
    assert (t[:, 0] >= 0).all() and (t[:, 0] < len(mb)).all()
    for b, m in enumerate(mb):
        own = [tuple(int(v) for v in r) for r in t[t[:, 0] == b, 1:]]
        assert own == _order(lib, m, m + 1), b
    # interleaved, not concatenated: every block starts before any block of three or more tile
    # columns (whose tickets span more than the first phase) has finished
    first = [int(np.flatnonzero(t[:, 0] == b)[0]) for b in range(len(mb))]
    last = [int(np.flatnonzero(t[:, 0] == b)[-1]) for b in range(len(mb))]
    for b, m in enumerate(mb):
        if m > 64:
            assert max(first) < last[b]


def test_block_queue_rejects_bad_sizes(lib):
    arr = np.array([3, 0], np.int32)
    n = C.c_int64(-1)
    assert lib.mcsdp_chol_block_task_order(2, C.c_void_p(arr.ctypes.data), C.byref(n), None) == 1
