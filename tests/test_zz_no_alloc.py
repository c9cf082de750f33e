"""The allocation-free Schur complement solve (mcsdp_sce_solve_noalloc) against the existing
path.  Some callers cannot allocate device memory on their code path (their device memory is
owned by another framework's caching allocator, or the loop must not pay for a synchronising
allocation); this entry point keeps its working storage in a fixed device array of the library.

Reference: mcsdp_newton_step's dz solves B dz = g with B from mcsdp_scm_assemble and
g = b - beta mu h at the same iterate, so the new entry point must return that dz when given
that B and g.  Two calls in a row (the shared array keeps the previous call's contents), and two
problem sizes.  This file is collected last on purpose."""
import ctypes as C

import numpy as np
import pytest
import torch

from instances import block_arrow, lattice_maxcut

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    from paper_1310_6919_gb300 import build_library, _lib
    build_library()
    assert torch.cuda.is_available()
    return _lib.load()


def _reference(inst, seed):
    from tests.gpu_helpers import Case
    c = Case(inst)
    Xbar, z = c.random_iterate(seed)
    Xl = c.to_layout(Xbar)
    zt = torch.tensor(z, device="cuda:0")
    st = c.P.newton_step(Xl, zt)
    Bt, h = c.P.scm_assemble(Xl, zt)
    B = Bt.t().contiguous().t()  # column-major storage, lower triangle valid
    g = torch.tensor(inst.b, device="cuda:0") - 0.1 * st["mu"] * h
    return B, g.contiguous(), st["dz"]


def _call(lib, B, g, m):
    x = torch.full((m,), float("nan"), dtype=torch.float64, device="cuda:0")
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    st = lib.mcsdp_sce_solve_noalloc(C.c_void_p(B.data_ptr()), m, C.c_void_p(g.data_ptr()),
                                     C.c_void_p(x.data_ptr()), m, stream)
    return st, x


@pytest.mark.parametrize("mk", [lambda: block_arrow(6, 12, 4, 60, per_matrix=8, seed=5),
                                lambda: lattice_maxcut(10, 10)], ids=["arrow60", "grid100"])
def test_noalloc_solve_matches_newton_step(lib, mk):
    inst = mk()
    B, g, dz_ref = _reference(inst, 7)
    m = inst.m
    assert B.stride(0) == 1 and B.stride(1) == m
    ref = dz_ref.cpu().numpy()
    for _ in range(2):
        st, x = _call(lib, B, g, m)
        assert st == 0
        got = x.cpu().numpy()
        assert np.max(np.abs(got - ref)) / np.max(np.abs(ref)) < 1e-8


def test_noalloc_rejects_oversize_and_indefinite(lib):
    m = 1025
    B = torch.eye(m, dtype=torch.float64, device="cuda:0")
    g = torch.ones(m, dtype=torch.float64, device="cuda:0")
    st, _ = _call(lib, B, g, m)
    assert st == 1  # MCSDP_ERR_ARG: beyond MCSDP_SCE_NOALLOC_MAX_M
    m = 70
    B = -torch.eye(m, dtype=torch.float64, device="cuda:0")
    g = torch.ones(m, dtype=torch.float64, device="cuda:0")
    st, _ = _call(lib, B, g, m)
    assert st == 2  # MCSDP_ERR_NOT_PD
    # the next call after a failed one starts clean
    B = 2.0 * torch.eye(m, dtype=torch.float64, device="cuda:0")
    st, x = _call(lib, B, g, m)
    assert st == 0 and torch.allclose(x, 0.5 * g)


def test_noalloc_at_the_maximum_size(lib):
    """m = MCSDP_SCE_NOALLOC_MAX_M fills the bordered copy ((m+1) x m) and the diagonal-block
    inverses of the fixed array exactly: a random SPD B = Q Q^T / m + I with a known x, checked
    against torch.linalg.solve in FP64, twice in a row."""
    m = 1024
    gen = torch.Generator(device="cpu").manual_seed(11)
    Q = torch.randn(m, m, generator=gen, dtype=torch.float64)
    B = (Q @ Q.t() / m + torch.eye(m, dtype=torch.float64)).to("cuda:0")
    xt = torch.randn(m, generator=gen, dtype=torch.float64).to("cuda:0")
    g = (B @ xt).contiguous()
    ref = torch.linalg.solve(B, g)
    Bc = B.t().contiguous().t()
    for _ in range(2):
        st, x = _call(lib, Bc, g, m)
        assert st == 0
        assert torch.max(torch.abs(x - ref)) / torch.max(torch.abs(ref)) < 1e-10
