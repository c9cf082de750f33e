"""Config 5: derivatives of the solution of block_arrow_1020 (n = 1020, m = 1000) on the device,
for the loss l = sum over the stored entries of E of W_ij X̄_ij with W ~ N(0, 1) (seeded).

The point differentiated is the central-path point for the iterate's mu (mcsdp_backward, through
autograd.solve_layer).  Two solves of the same problem:

* stopped after 16 iterations (relative gap about 0.07, mu about 3e-3, cond(Y) about 5e4): there
  both centrings reach their rounding level (about 1e-10 relative on the device, whose Y^{-1}
  comes from sparse triangular solves, below that on the host), so (a) central finite
  differences of the device path itself at h = 1e-6 (each perturbed problem re-centred on the
  device at the same mu) match the gradients within 1e-5 of the largest gradient, for 4 entries
  of b and 4 input entries (diagonal and off-diagonal, of A_0 and of the A_k), and (b) the
  gradients match the oracle's adjoint (oracle.diff, dense FP64) element by element at 1e-8 of
  the largest;
* converged (relative gap 1e-7): mu is about 1e-9 and cond(Y) about 1e10, so the central point is
  determined only to the rounding level eps cond(Y) of evaluating its residual (about 1e-6 on
  both sides; a finite difference at h = 1e-6 has no significant digit there).  The gradients
  are nevertheless well determined: the oracle's own gradients move by 1.9e-7 of the largest when
  its centring starts from another feasible point (measured on the host at this iterate), so the
  device's gradients are compared with the oracle's at the same mu within 1e-5 of the largest.
"""
import dataclasses

import numpy as np
import pytest
import torch

from instances import workload
from oracle import diff
from oracle.sdp import SparseSym, dual_slack

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1310_6919_gb300 import build_library
    build_library()
    assert torch.cuda.is_available()


def _layout_to_sym(c, g):
    n = c.inst.n
    G = np.zeros((n, n))
    r, q, v = c.ro[c.valid], c.co[c.valid], g[c.valid]
    diag = r == q
    G[r[diag], q[diag]] = v[diag]
    G[r[~diag], q[~diag]] = 0.5 * v[~diag]
    G[q[~diag], r[~diag]] = 0.5 * v[~diag]
    return G


def _layer(inst, W, max_iter):
    """solve_layer forward + backward; returns (b.grad, val.grad, X̄ layout, z)."""
    from paper_1310_6919_gb300.autograd import solve_layer
    b = torch.tensor(inst.b, requires_grad=True)
    val = torch.tensor(inst.val, requires_grad=True)
    X, z = solve_layer(b, val, inst.n, inst.m, inst.mat, inst.row, inst.col,
                       z0=torch.tensor(inst.z0, device="cuda:0"), device=0, max_iter=max_iter)
    loss = (torch.tensor(W, device=X.device) * X).sum()
    loss.backward()
    return b.grad.numpy(), val.grad.numpy(), X.detach(), z.detach()


def _oracle_grads(c, inst, W, X, z):
    A = SparseSym.from_instance(inst)
    Xd = c.from_layout(X)
    zn = z.cpu().numpy()
    mu = float(np.sum(Xd * dual_slack(A, zn))) / inst.n
    zc, Yc, Xc, res = diff.central_point(A, inst.b, mu, zn)
    gb, gA0, _ = diff.backward(A, zc, Yc, Xc, _layout_to_sym(c, W), np.zeros(inst.m), with_gA=False)
    return gb, diff.entry_gradients(inst, zc, gb, gA0, Xc), mu, res


@pytest.fixture(scope="module")
def case():
    from tests.gpu_helpers import Case
    inst = workload("block_arrow_1020")
    c = Case(inst)
    rng = np.random.default_rng(1020)
    W = np.where(c.valid, rng.standard_normal(c.valid.shape[0]), 0.0)
    return inst, c, W


def test_config5_early_finite_differences(case):
    from paper_1310_6919_gb300 import Problem
    inst, c, W = case
    gb, ge, X, z = _layer(inst, W, max_iter=16)
    # the central point the layer differentiated, from a solve with the same options
    P = Problem.from_instance(inst, device=0, max_iter=16)
    P.set_iterate(None, inst.z0)
    P.solve()
    P.backward(torch.tensor(W, device="cuda:0"), None)
    Xc_l, zc_t, _ = P.get_iterate()
    Xc = c.from_layout(Xc_l)
    zc = zc_t.cpu().numpy()
    A = SparseSym.from_instance(inst)
    n = inst.n
    mu = float(np.sum(Xc * dual_slack(A, zc))) / n
    # the residual of that point, evaluated here in FP64 (the device's centring stops at its own
    # rounding level, about 1e-10 here: eps cond(Y) |A||X| / |b| with cond(Y) about 5e4)
    F = A.op(mu * np.linalg.inv(dual_slack(A, zc))) - inst.b
    res = np.max(np.abs(F)) / max(1.0, np.max(np.abs(inst.b)))
    assert res <= 1e-9

    def central_loss(inst2):
        A2 = SparseSym.from_instance(inst2)
        s = mu * n / float(np.sum(Xc * dual_slack(A2, zc)))  # the same mu at the start
        P2 = Problem.from_instance(inst2, device=0)
        P2.set_iterate(c.to_layout(s * Xc), torch.tensor(zc, device="cuda:0"))
        P2.backward(None, None)
        X2, _, _ = P2.get_iterate()
        return float(np.sum(W * X2.cpu().numpy()))

    h = 1e-6
    scale = max(np.max(np.abs(gb)), np.max(np.abs(ge)))
    rng = np.random.default_rng(5)
    for p in rng.choice(inst.m, 4, replace=False):
        bp, bm = inst.b.copy(), inst.b.copy()
        bp[p] += h
        bm[p] -= h
        fd = (central_loss(dataclasses.replace(inst, b=bp)) -
              central_loss(dataclasses.replace(inst, b=bm))) / (2 * h)
        assert abs(fd - gb[p]) <= 1e-5 * scale, (p, fd, gb[p], scale, res)
    mats, rows, cols = inst.mat, inst.row, inst.col
    picks = [int(np.flatnonzero((mats == 0) & (rows == cols))[3]),
             int(np.flatnonzero((mats == 0) & (rows != cols))[5]),
             int(np.flatnonzero((mats > 0) & (rows == cols))[7]),
             int(np.flatnonzero((mats > 0) & (rows != cols))[11])]
    for e in picks:
        vp, vm = inst.val.copy(), inst.val.copy()
        vp[e] += h
        vm[e] -= h
        fd = (central_loss(dataclasses.replace(inst, val=vp)) -
              central_loss(dataclasses.replace(inst, val=vm))) / (2 * h)
        assert abs(fd - ge[e]) <= 1e-5 * scale, (e, fd, ge[e], scale, res)
    # the oracle's adjoint at the same mu
    gb_o, ge_o, mu_o, res = _oracle_grads(c, inst, W, X, z)
    assert res <= 1e-9
    assert np.max(np.abs(gb - gb_o)) <= 1e-8 * scale, np.max(np.abs(gb - gb_o)) / scale
    assert np.max(np.abs(ge - ge_o)) <= 1e-8 * scale, np.max(np.abs(ge - ge_o)) / scale


def test_config5_converged_gradients(case):
    inst, c, W = case
    gb, ge, X, z = _layer(inst, W, max_iter=100)
    gb_o, ge_o, mu, res = _oracle_grads(c, inst, W, X, z)
    assert mu < 1e-6  # converged: the ill-conditioned end of the central path
    g = np.concatenate([gb, ge])
    go = np.concatenate([gb_o, ge_o])
    scale = np.max(np.abs(go))
    assert np.all(np.isfinite(g))
    assert np.max(np.abs(g - go)) <= 1e-5 * scale
