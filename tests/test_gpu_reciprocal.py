"""The pivot reciprocal of the serial Cholesky loops (mcsdp_pivot_reciprocal) against IEEE
division.  The factorisations of Sec. 3.1 (types (i) and (ii)) take one reciprocal per pivot; the
library forms it from an FP32 seed and one third-order series step in FP64 (relative error of
the step below 2^-59), so the result must be faithfully rounded: equal to numpy's correctly
rounded 1/d or one ulp away, and equal in all but a small fraction of cases.  Outside the seed's
exponent range, for zero, negative and non-finite d, the library divides, so those must match
division exactly."""
import ctypes as C

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    from paper_1310_6919_gb300 import build_library, _lib
    build_library()
    assert torch.cuda.is_available()
    return _lib.load()


def _rcp(lib, d):
    dt = torch.tensor(d, dtype=torch.float64, device="cuda:0")
    r = torch.full_like(dt, float("nan"))
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    st = lib.mcsdp_pivot_reciprocal(C.c_void_p(dt.data_ptr()), C.c_void_p(r.data_ptr()),
                                    dt.numel(), stream)
    assert st == 0
    torch.cuda.synchronize()
    return r.cpu().numpy()


def _ulps(a, b):
    """distance in units in the last place between two positive finite doubles"""
    ia = a.view(np.int64)
    ib = b.view(np.int64)
    return np.abs(ia - ib)


def test_reciprocal_faithful_over_the_seed_range(lib):
    rng = np.random.default_rng(20131103)
    # log-uniform over the range where the FP32 seed is used, plus mantissas near 1 and 2
    d = np.exp2(rng.uniform(-119.5, 120.5, size=200000))
    d = np.concatenate([d, 1.0 + rng.random(20000) * 2.0 ** -20, 2.0 - rng.random(20000) * 2.0 ** -20,
                        np.exp2(np.arange(-120, 121, dtype=np.float64)),
                        np.nextafter(np.exp2(np.arange(-120, 121, dtype=np.float64)), np.inf)])
    r = _rcp(lib, d)
    ref = 1.0 / d
    u = _ulps(r, ref)
    assert u.max() <= 1
    assert np.mean(u == 0) >= 0.99


def test_reciprocal_divides_outside_the_seed_range(lib):
    tiny = np.finfo(np.float64).tiny
    d = np.array([0.0, -0.0, -1.5, -3e200, np.inf, -np.inf, np.nan, tiny, tiny / 8.0, 1e-300,
                  2.0 ** -121, 2.0 ** 122, 1e300, np.finfo(np.float64).max])
    r = _rcp(lib, d)
    with np.errstate(divide="ignore", over="ignore"):
        ref = 1.0 / d
    same = (r == ref) | (np.isnan(r) & np.isnan(ref))
    assert same.all(), (d[~same], r[~same], ref[~same])
    assert np.signbit(r[1]) and not np.signbit(r[0])


def test_reciprocal_empty_and_bad_arguments(lib):
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert lib.mcsdp_pivot_reciprocal(None, None, 0, stream) == 0
    assert lib.mcsdp_pivot_reciprocal(None, None, 5, stream) != 0
    assert lib.mcsdp_pivot_reciprocal(None, None, -1, stream) != 0
