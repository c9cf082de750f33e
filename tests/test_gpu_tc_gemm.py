"""The tensor-core FP32 product (mcsdp_gemm_tc: tcgen05 kind::tf32 MMAs on TMA-loaded tiles,
three TF32 products per FP32 product) against an FP64 product of the same FP32 inputs.

Bound: a three-term TF32 split represents each operand to about 2^-21 relative, so each product
term is within a few 2^-21 of the FP32 inputs' exact product and the sum of K terms within
K 2^-21 max|a| max|b| (FP32 accumulation adds K 2^-24 of the partial sums): the test asks for
4 K 2^-21 max|a| max|b| on every entry.  Sizes: single tiles, ragged edges in M, N and K (the
TMA zero fill), several K blocks through the three-stage ring, alpha/beta combinations."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1310_6919_gb300 import build_library
    build_library()
    assert torch.cuda.is_available()


@pytest.mark.parametrize("M,N,K", [(128, 128, 32), (128, 128, 96), (200, 130, 45), (512, 384, 256),
                                   (1000, 999, 1001), (33, 257, 7)],
                         ids=["one_tile", "three_kblocks", "ragged", "multi_tile", "odd", "thin"])
def test_gemm_tc_matches_fp64(M, N, K):
    from paper_1310_6919_gb300 import gemm_tc
    g = torch.Generator(device="cpu").manual_seed(M * 7 + N * 3 + K)
    A = torch.randn(M, K, generator=g, dtype=torch.float32).cuda()   # row i = K values
    B = torch.randn(N, K, generator=g, dtype=torch.float32).cuda()
    C = gemm_tc(A.t(), B.t())
    ref = A.double() @ B.double().t()
    bound = 4 * K * 2.0 ** -21 * A.abs().max().item() * B.abs().max().item()
    err = (C.double() - ref).abs().max().item()
    assert err <= bound, (err, bound)
    # a one-term TF32 product would miss this bound by orders of magnitude: the split is used
    assert err <= 1e-3 * ref.abs().max().item()


def test_gemm_tc_alpha_beta():
    from paper_1310_6919_gb300 import gemm_tc
    g = torch.Generator(device="cpu").manual_seed(5)
    M, N, K = 300, 260, 140
    A = torch.randn(M, K, generator=g).cuda()
    B = torch.randn(N, K, generator=g).cuda()
    C0 = torch.randn(N, M, generator=g).cuda().t()
    C = C0.clone()
    gemm_tc(A.t(), B.t(), C, alpha=-0.5, beta=2.0)
    ref = -0.5 * (A.double() @ B.double().t()) + 2.0 * C0.double()
    bound = 4 * K * 2.0 ** -21 * A.abs().max().item() * B.abs().max().item() * 0.5 + 1e-5
    assert (C.double() - ref).abs().max().item() <= bound
