"""The tile-shape tuner's host side (no GPU): the workspace it asks for covers every candidate
grouping the problem fits, and a problem whose constraints are wider than a candidate's panel
still gets a size from the others."""
import ctypes as C

import numpy as np
import pytest

from instances import block_arrow, lattice_maxcut


@pytest.fixture(scope="module")
def lib():
    from paper_1310_6919_gb300 import build_library, _lib
    build_library()
    return _lib.load()


def _ws(lib, inst, **opts):
    from paper_1310_6919_gb300.binding import _problem_t
    from paper_1310_6919_gb300 import _lib
    arrs, prob = _problem_t(inst.n, inst.m, inst.b, inst.mat, inst.row, inst.col, inst.val, 1)
    opt = _lib.Options_t()
    lib.mcsdp_default_options(C.byref(opt))
    for k, v in opts.items():
        setattr(opt, k, v)
    nb = C.c_size_t()
    st = lib.mcsdp_tune_workspace_size(C.byref(prob), C.byref(opt), C.byref(nb))
    return st, int(nb.value)


@pytest.mark.parametrize("inst", [lattice_maxcut(10, 10), block_arrow(6, 12, 4, 60, seed=5)],
                         ids=lambda i: i.name)
def test_tune_workspace_covers_every_candidate(lib, inst):
    from paper_1310_6919_gb300 import Problem
    st, need = _ws(lib, inst)
    assert st == 0
    for gm, pm in [(64, 80), (32, 80), (16, 80), (64, 96), (32, 48)]:
        P = Problem.from_instance(inst, device=-1, group_max=gm, panel_max=pm)
        nb = C.c_size_t()
        assert lib.mcsdp_workspace_size(P._ctx, C.byref(nb)) == 0
        assert need >= nb.value


def test_tune_skips_candidates_a_constraint_does_not_fit(lib):
    # one constraint touching 60 rows: the panel_max 48 candidate cannot hold it
    n = 64
    mat = [0] * n + [1] * 60
    row = list(range(n)) + list(range(60))
    inst = type("I", (), {})()
    inst.n, inst.m = n, 1
    inst.b = np.array([1.0])
    inst.mat, inst.row = np.array(mat, np.int32), np.array(row, np.int32)
    inst.col, inst.val = inst.row.copy(), np.ones(len(mat))
    st, need = _ws(lib, inst)
    assert st == 0 and need > 0
    st, _ = _ws(lib, inst, panel_max=48)  # the given panel_max is not what is tuned
    assert st == 0


def test_tune_needs_a_device(lib):
    from paper_1310_6919_gb300.binding import _problem_t
    from paper_1310_6919_gb300 import _lib
    inst = lattice_maxcut(4, 4)
    arrs, prob = _problem_t(inst.n, inst.m, inst.b, inst.mat, inst.row, inst.col, inst.val, 1)
    opt = _lib.Options_t()
    lib.mcsdp_default_options(C.byref(opt))
    opt.device = -1
    info = _lib.TuneInfo_t()
    buf = C.create_string_buffer(256)
    assert lib.mcsdp_tune(C.byref(prob), C.byref(opt), None, None, buf, 256, 3,
                          C.byref(info)) == 1  # MCSDP_ERR_ARG


def test_tune_workspace_when_no_candidate_fits(lib):
    # one constraint touching 97 rows: wider than every candidate's panel (and the limit, 96)
    n = 100
    inst = type("I", (), {})()
    inst.n, inst.m = n, 1
    inst.b = np.array([1.0])
    inst.mat = np.array([0] * n + [1] * 97, np.int32)
    inst.row = np.array(list(range(n)) + list(range(97)), np.int32)
    inst.col, inst.val = inst.row.copy(), np.ones(n + 97)
    st, _ = _ws(lib, inst)
    assert st == 1  # MCSDP_ERR_ARG
