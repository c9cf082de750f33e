"""Shared-memory layouts of the staged level solves (mcsdp_lsolve_layout, host only) for every
admissible clique size (|C_r| <= 160 rows, |S_r| <= 96 columns: a margin over the 112 / 96 that
create enforces for the cliques outside a dense root):
regions 16-byte aligned (cp.async destinations), in order and disjoint, each as large as the
kernel's accesses (acc[j * 32 + lane] and the diagonal block for j < nc, the update ring's
source values, factor rows and row indices, the backward solve's clique block and vectors), and
every FP32 level within the staged kernels' cap: the FP32 solves of the mixed form have no
unstaged fallback."""
import ctypes as C

import pytest

NC_MAX, NR_MAX, CW_MAX = 96, 160, 8


@pytest.fixture(scope="module")
def layout():
    from paper_1310_6919_gb300 import build_library, _lib
    build_library()
    L = _lib.load()
    f = L.mcsdp_lsolve_layout
    f.argtypes = [C.c_int32] * 6 + [C.POINTER(C.c_int32)] * 3
    f.restype = C.c_int

    def call(nc, nr, cw, np_, with_d, es):
        fw = (C.c_int32 * 7)()
        bw = (C.c_int32 * 6)()
        cap = C.c_int32()
        st = f(nc, nr, cw, np_, with_d, es, fw, bw, C.byref(cap))
        assert st == 0
        return list(fw), list(bw), cap.value
    return call


def _check_fwd(fw, nc, cw, np_, with_d, es):
    acc, ds, meta, hdr, buf, bufsz, total = fw
    assert all(x % 16 == 0 for x in (acc, ds, meta, hdr, buf, bufsz, total))
    assert 0 == acc <= ds <= meta <= hdr <= buf <= total
    assert ds - acc >= nc * 32 * es
    assert meta - ds >= (nc * nc * es if with_d else 0)
    if cw == 0:
        assert bufsz == 0 and total == buf
    else:
        assert bufsz >= cw * 32 * es + cw * np_ * es + np_ * 4
        assert (total - buf) % bufsz == 0 and (total - buf) // bufsz >= 2   # a ring of slots


def _check_bwd(bw, nr, nc, es):
    ls, ds, acc, wv, rws, total = bw
    assert all(x % 16 == 0 for x in bw)
    assert 0 == ls <= ds <= acc <= wv <= rws <= total
    assert ds - ls >= nr * nc * es and acc - ds >= nc * nc * es and wv - acc >= nc * 32 * es
    assert rws - wv >= nr * 32 * es and total - rws >= nr * 4


@pytest.mark.parametrize("es", [4, 8])
def test_layouts_for_every_clique_size(layout, es):
    cap = None
    worst_fwd = worst_bwd = 0
    for nc in range(1, NC_MAX + 1):
        for nr in range(nc, NR_MAX + 1):
            fw, bw, cap = layout(nc, nr, 0, 0, 1, es)
            _check_bwd(bw, nr, nc, es)
            worst_bwd = max(worst_bwd, bw[-1])
        for cw in range(0, CW_MAX + 1):
            for np_ in (0, 1, 7, 31, 32, 33, 96, 159, NR_MAX):
                for with_d in (0, 1):
                    fw, _, _ = layout(nc, nc, cw, np_, with_d, es)
                    _check_fwd(fw, nc, cw, np_, with_d, es)
                    worst_fwd = max(worst_fwd, fw[-1])
    if es == 4:
        assert worst_fwd <= cap and worst_bwd <= cap


def test_bad_arguments(layout):
    from paper_1310_6919_gb300 import _lib
    f = _lib.load().mcsdp_lsolve_layout
    fw = (C.c_int32 * 7)()
    bw = (C.c_int32 * 6)()
    assert f(0, 1, 0, 0, 1, 8, fw, bw, None) == 1
    assert f(4, 3, 0, 0, 1, 8, fw, bw, None) == 1
    assert f(4, 4, 0, 0, 1, 2, fw, bw, None) == 1
    assert f(4, 4, 0, 0, 1, 8, None, bw, None) == 1
