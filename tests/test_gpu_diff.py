"""Differentiation (mcsdp_backward) against the oracle: the re-centred central-path point for
the iterate's mu and the gradients of l = gX . X̄ + gz . z with respect to b and every input
entry, after a solve stopped early (mu around 1e-2, where B is well conditioned).  Tolerance
1e-8 relative to the largest gradient (both sides FP64; B^{-1} and two completed products in
between)."""
import numpy as np
import pytest
import torch

from instances import block_arrow, small_random_sdp, diagonal_lp_sdp, lattice_maxcut
from oracle import diff
from oracle.sdp import SparseSym, dual_slack

pytestmark = pytest.mark.gpu

CASES = [lambda: small_random_sdp(9, 14, 2), lambda: block_arrow(6, 12, 4, 60, per_matrix=8, seed=5),
         lambda: diagonal_lp_sdp(12, 7, 3), lambda: lattice_maxcut(6, 6)]
IDS = ["dense9", "arrow6x12", "lp12", "grid36"]


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1310_6919_gb300 import build_library
    build_library()
    assert torch.cuda.is_available()


def _layout_to_sym(c, g):
    """The symmetric matrix G with <G, X> = sum over layout entries g . X̄."""
    n = c.inst.n
    G = np.zeros((n, n))
    r, q, v = c.ro[c.valid], c.co[c.valid], g[c.valid]
    diag = r == q
    G[r[diag], q[diag]] = v[diag]
    G[r[~diag], q[~diag]] = 0.5 * v[~diag]
    G[q[~diag], r[~diag]] = 0.5 * v[~diag]
    return G


@pytest.mark.parametrize("mk", CASES, ids=IDS)
def test_backward_matches_oracle(mk):
    from tests.gpu_helpers import Case
    inst = mk()
    c = Case(inst, max_iter=6)
    if inst.meta.get("kind") != "maxcut":
        c.P.set_iterate(None, inst.z0)
    r = c.P.solve()
    assert r["status"] in (0, 3)
    X, z, _ = c.P.get_iterate()
    A = SparseSym.from_instance(inst)
    Xd = c.from_layout(X)
    zn = z.cpu().numpy()
    mu = float(np.sum(Xd * dual_slack(A, zn))) / inst.n
    rng = np.random.default_rng(4)
    gX = np.where(c.valid, rng.standard_normal(c.valid.shape[0]), 0.0)
    gz = rng.standard_normal(inst.m)
    out = c.P.backward(torch.tensor(gX, device="cuda:0"), torch.tensor(gz, device="cuda:0"))
    zc, Yc, Xc, res = diff.central_point(A, inst.b, mu, zn)
    # no finite difference here: the comparison below (1e-8 of the largest gradient) only needs
    # both central points far closer than that; at this mu (about 1e-3) the residual's rounding
    # floor in FP64 is near 1e-12
    assert res <= 1e-11
    gb, gA0, gA = diff.backward(A, zc, Yc, Xc, _layout_to_sym(c, gX), gz)
    ge = diff.entry_gradients(inst, zc, gb, gA0, Xc)
    scale = max(np.max(np.abs(ge)), np.max(np.abs(gb)))
    assert np.max(np.abs(out["gb"].cpu().numpy() - gb)) <= 1e-8 * scale
    assert np.max(np.abs(out["g_entries"].cpu().numpy() - ge)) <= 1e-8 * scale
    # the context's iterate is now the central point
    X2, z2, _ = c.P.get_iterate()
    # the library's own central point: its residual, evaluated here in FP64 on the CPU
    z2n = z2.cpu().numpy()
    F = A.op(mu * np.linalg.inv(dual_slack(A, z2n))) - inst.b
    assert np.max(np.abs(F)) / max(1.0, np.max(np.abs(inst.b))) <= 1e-10
    assert np.max(np.abs(z2.cpu().numpy() - zc)) <= 1e-9 * max(1.0, np.max(np.abs(zc)))
    E = c.E
    assert np.max(np.abs(c.from_layout(X2)[E] - Xc[E])) <= 1e-9 * np.max(np.abs(Xc))


def test_autograd_layer():
    """solve_layer's gradients (through torch.autograd) against the oracle's adjoint at the same
    central point: loss = sum of W . X̄ over the layout entries + g . z, W and g seeded."""
    from paper_1310_6919_gb300.autograd import solve_layer
    from tests.gpu_helpers import Case
    inst = small_random_sdp(9, 14, 2)
    c = Case(inst, max_iter=6)  # the layout map (same symbolic analysis as the layer's)
    b = torch.tensor(inst.b, requires_grad=True)
    val = torch.tensor(inst.val, requires_grad=True)
    X, z = solve_layer(b, val, inst.n, inst.m, inst.mat, inst.row, inst.col,
                       z0=torch.tensor(inst.z0, device="cuda:0"), device=0, max_iter=6)
    rng = np.random.default_rng(8)
    W = torch.tensor(np.where(c.valid, rng.standard_normal(c.valid.shape[0]), 0.0), device=X.device)
    g = torch.tensor(rng.standard_normal(inst.m), device=z.device)
    loss = (W * X).sum() + (g * z).sum()
    loss.backward()
    assert b.grad.shape == b.shape and val.grad.shape == val.shape
    # the oracle at the central point for the forward iterate's mu
    A = SparseSym.from_instance(inst)
    Xd = c.from_layout(X.detach())
    zn = z.detach().cpu().numpy()
    mu = float(np.sum(Xd * dual_slack(A, zn))) / inst.n
    zc, Yc, Xc, res = diff.central_point(A, inst.b, mu, zn)
    assert res <= 1e-11
    gb, gA0, _ = diff.backward(A, zc, Yc, Xc, _layout_to_sym(c, W.cpu().numpy()), g.cpu().numpy(),
                               with_gA=False)
    ge = diff.entry_gradients(inst, zc, gb, gA0, Xc)
    scale = max(np.max(np.abs(ge)), np.max(np.abs(gb)))
    assert np.max(np.abs(b.grad.numpy() - gb)) <= 1e-8 * scale
    assert np.max(np.abs(val.grad.numpy() - ge)) <= 1e-8 * scale
