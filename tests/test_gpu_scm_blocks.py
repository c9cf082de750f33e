"""Block-diagonal SCM on the device (the sparse-SCM case of Sec. 3.1: constraints in different
connected components give B_pq = 0): cross-component tiles are not assembled, and each diagonal
block gets its own bordered Cholesky and backward substitution, its right-hand side in the row
after the block.  Parity with the oracle as for a connected pattern (SCM entries 1e-10 of the
largest, Newton direction 1e-8, optimal values 1e-7), on a direct sum whose blocks have 32, 40,
7, 14 and 1 constraints (a block that is a whole tile, ragged ones, a one-constraint block) and a
max-cut part of several components; the whole-matrix form (options.scm_blocks = 1) reaches the
same optimum, the graph form the same iterates bit for bit."""
import numpy as np
import pytest
import torch

from instances import (SDPInstance, block_arrow, diagonal_lp_sdp, direct_sum, lattice_maxcut,
                       random_gnm_maxcut, small_random_sdp, workload)
from oracle import diff, pdipm
from oracle.sdp import SparseSym, dual_slack

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1310_6919_gb300 import build_library
    build_library()
    assert torch.cuda.is_available()


def _scalar():
    return SDPInstance("scalar", 1, 1, np.array([3.0]), np.array([0, 1], np.int32),
                       np.array([0, 0], np.int32), np.array([0, 0], np.int32),
                       np.array([2.0, 1.0]), z0=np.array([0.0]), meta={"kind": "scalar"})


def _sum():
    return direct_sum([lattice_maxcut(4, 8, seed=3), block_arrow(3, 12, 4, 40, per_matrix=8, seed=9),
                       diagonal_lp_sdp(12, 7, 3), small_random_sdp(9, 14, 2), _scalar(),
                       random_gnm_maxcut(40, 90, 6)])


def _solve(inst, **opts):
    from paper_1310_6919_gb300 import Problem
    P = Problem.from_instance(inst, device=0, **opts)
    P.set_iterate(None, inst.z0)
    return P, P.solve()


def test_scm_matches_oracle():
    from tests.gpu_helpers import Case, rel_err
    c = Case(_sum())
    assert c.P.info["scm_blocks"] == 1 and c.P.info["ncomp"] == 7
    for seed in (2, 3):
        Xbar, z = c.random_iterate(seed)
        B, h = c.P.scm_assemble(c.to_layout(Xbar), torch.tensor(z, device="cuda:0"))
        Bg = B.cpu().numpy()
        Bref, Xh, Yinv = c.oracle_scm(Xbar, z)
        low = np.tril(np.ones_like(Bref, dtype=bool))
        assert rel_err(Bg[low], Bref[low]) < 1e-10
        assert not Bg[low & (Bref == 0.0)].any()  # nothing between components
        assert rel_err(h.cpu().numpy(), c.A.op(Yinv)) < 1e-10


@pytest.mark.parametrize("blocks", [0, 1], ids=["blocks", "whole"])
def test_newton_step_matches_oracle(blocks):
    from tests.gpu_helpers import Case, rel_err
    c = Case(_sum(), scm_blocks=blocks)
    Xbar, z = c.random_iterate(7)
    st = c.P.newton_step(c.to_layout(Xbar), torch.tensor(z, device="cuda:0"))
    ref = pdipm.mc_newton_step(c.A, c.inst.b, c.perm, c.cliques, Xbar, z)
    assert rel_err(st["dz"].cpu().numpy(), ref["dz"]) < 1e-8
    dX = c.from_layout(st["dX"])
    assert rel_err(dX[c.E], ref["dX"][c.E]) < 1e-8
    dY = c.from_layout(st["dY"])
    assert rel_err(dY[c.E], ref["dY"][c.E]) < 1e-8
    assert abs(st["alpha_p"] - ref["alpha_p"]) <= 1e-7 * ref["alpha_p"]


def test_solve_matches_oracle_optimum():
    inst = _sum()
    P, r = _solve(inst)
    ref = pdipm.solve_dense(SparseSym.from_instance(inst), inst.b, inst.z0)
    assert r["status"] == 0 and ref["status"] == "optimal"
    scale = max(1.0, abs(ref["pobj"]))
    assert abs(r["pobj"] - ref["pobj"]) <= 1e-7 * scale
    assert abs(r["dobj"] - ref["dobj"]) <= 1e-7 * scale
    # the whole-matrix factorisation of the same B: the same optimum
    _, r1 = _solve(inst, scm_blocks=1)
    assert r1["status"] == 0
    assert abs(r1["pobj"] - r["pobj"]) <= 1e-9 * scale


def test_mixed_form_keeps_fp64_block_factor():
    inst = _sum()
    P, r = _solve(inst, precision=1, profile=1)
    ref = pdipm.solve_dense(SparseSym.from_instance(inst), inst.b, inst.z0)
    assert r["status"] == 0
    assert abs(r["pobj"] - ref["pobj"]) <= 1e-7 * max(1.0, abs(ref["pobj"]))
    cnt = P.stats()["count"]
    assert cnt["scm_chol"] > 0 and cnt["scm_chol32"] == 0


def test_graph_form_same_iterates():
    inst = _sum()
    P0, r0 = _solve(inst)
    P1, r1 = _solve(inst, graph=1)
    assert r0["iters"] == r1["iters"] and r0["status"] == r1["status"] == 0
    z0 = P0.get_iterate()[1].cpu().numpy()
    z1 = P1.get_iterate()[1].cpu().numpy()
    assert np.array_equal(z0, z1)


def _layout_to_sym(c, g):
    n = c.inst.n
    G = np.zeros((n, n))
    r, q, v = c.ro[c.valid], c.co[c.valid], g[c.valid]
    diag = r == q
    G[r[diag], q[diag]] = v[diag]
    G[r[~diag], q[~diag]] = 0.5 * v[~diag]
    G[q[~diag], r[~diag]] = 0.5 * v[~diag]
    return G


def test_backward_matches_oracle():
    from tests.gpu_helpers import Case
    inst = _sum()
    c = Case(inst, max_iter=6)
    c.P.set_iterate(None, inst.z0)
    r = c.P.solve()
    assert r["status"] in (0, 3)
    X, z, _ = c.P.get_iterate()
    A = SparseSym.from_instance(inst)
    zn = z.cpu().numpy()
    mu = float(np.sum(c.from_layout(X) * dual_slack(A, zn))) / inst.n
    rng = np.random.default_rng(4)
    gX = np.where(c.valid, rng.standard_normal(c.valid.shape[0]), 0.0)
    gz = rng.standard_normal(inst.m)
    out = c.P.backward(torch.tensor(gX, device="cuda:0"), torch.tensor(gz, device="cuda:0"))
    zc, Yc, Xc, res = diff.central_point(A, inst.b, mu, zn)
    assert res <= 1e-11
    gb, gA0, gA = diff.backward(A, zc, Yc, Xc, _layout_to_sym(c, gX), gz)
    ge = diff.entry_gradients(inst, zc, gb, gA0, Xc)
    scale = max(np.max(np.abs(ge)), np.max(np.abs(gb)))
    assert np.max(np.abs(out["gb"].cpu().numpy() - gb)) <= 1e-8 * scale
    assert np.max(np.abs(out["g_entries"].cpu().numpy() - ge)) <= 1e-8 * scale


def test_maxcut_sum_64_per_part_dual_objectives():
    """64 random max-cut SDPs as one (n = m = 13367, block sizes 50..400): solved block by block.
    A property that holds at any size: Y = A_0 - diag(z) is block-diagonal and positive definite,
    so z_p is dual feasible for part p and b_p^T z_p <= opt_p (weak duality); and since every
    part's shortfall opt_p - b_p^T z_p is non-negative, each is at most the whole problem's,
    opt - b^T z, about the final duality gap.  The oracle solves three sampled parts."""
    from instances.problems import Xoshiro256ss, SEED_BASE
    inst = workload("maxcut_sum_64")
    P, r = _solve(inst)
    assert P.info["ncomp"] >= 64 and P.info["scm_blocks"] == 1
    assert r["status"] == 0 and r["gap"] <= 1e-7 and r["pinf"] <= 1e-7
    gap_abs = abs(r["pobj"] - r["dobj"])
    z = P.get_iterate()[1].cpu().numpy()
    # regenerate the parts (same draws as maxcut_direct_sum)
    rng = Xoshiro256ss(SEED_BASE + 7)
    sizes = [50 + rng.below(351) for _ in range(64)]
    offs = np.cumsum([0] + sizes)
    for p in (0, 17, 63):
        part = random_gnm_maxcut(sizes[p], (5 * sizes[p]) // 2, SEED_BASE + 7 + 1000 + p)
        ref = pdipm.solve_dense(SparseSym.from_instance(part), part.b, part.z0)
        assert ref["status"] == "optimal"
        zp = z[offs[p]:offs[p + 1]]
        dp = float(part.b @ zp)
        slack = 1e-7 * max(1.0, abs(ref["dobj"]))  # the oracle's own stopping bracket
        assert dp <= ref["pobj"] + slack
        # opt - b^T z <= the final gap plus the primal residual's share (pinf <= 1e-7)
        assert dp >= ref["dobj"] - gap_abs - 1e-6 * abs(r["dobj"]) - slack
