"""GPU parity of libmcsdp (through the C ABI) against the oracle, element by element.

Tolerances: SCM entries and factors 1e-10 relative to the largest entry (the FP64 gate of the
SCM); Newton direction 1e-8 (it passes through B^{-1}); optimal values 1e-7 relative at relative
gap 1e-7 (both runs stop inside the same 1e-7 duality bracket)."""
import json
import os

import numpy as np
import pytest
import torch

from instances import (lattice_maxcut, block_arrow, small_random_sdp, diagonal_lp_sdp,
                       complete_maxcut, cycle_maxcut, random_gnm_maxcut, workload, SDPInstance)
from oracle import pdipm, maxcut
from oracle.sdp import SparseSym

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")

SMALL = [
    lambda: lattice_maxcut(10, 10),                    # grid, n = m = 100, two groups (64 + 36)
    lambda: block_arrow(6, 12, 4, 60, per_matrix=8, seed=5),   # several tiles, ragged groups
    lambda: block_arrow(3, 25, 6, 75, per_matrix=8, seed=8),
    lambda: small_random_sdp(9, 14, 2),                # dense pattern, one clique
    lambda: diagonal_lp_sdp(12, 7, 3),                 # LP special case: E = diagonal
    lambda: random_gnm_maxcut(90, 200, 4),             # random sparse graph with fill
]
IDS = ["grid100", "arrow6x12", "arrow3x25", "dense9", "lp12", "gnm90"]


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1310_6919_gb300 import build_library
    build_library()
    assert torch.cuda.is_available()


@pytest.mark.parametrize("mk", SMALL, ids=IDS)
def test_factors_match_oracle(mk):
    from tests.gpu_helpers import Case, rel_err
    c = Case(mk())
    Xbar, z = c.random_iterate(1)
    Lh, N = c.P.factors(c.to_layout(Xbar), torch.tensor(z, device="cuda:0"))
    Lref, Nref = c.oracle_factors(Xbar, z)
    r, q, v = c.layout_values_new(Lh)
    assert rel_err(v, Lref[r, q]) < 1e-10
    r, q, v = c.layout_values_new(N)
    assert rel_err(v, Nref[r, q]) < 1e-10


@pytest.mark.parametrize("mk", SMALL, ids=IDS)
def test_scm_matches_oracle(mk):
    from tests.gpu_helpers import Case, rel_err
    c = Case(mk())
    for seed in (2, 3):
        Xbar, z = c.random_iterate(seed)
        B, h = c.P.scm_assemble(c.to_layout(Xbar), torch.tensor(z, device="cuda:0"))
        Bg = B.cpu().numpy()
        Bref, Xh, Yinv = c.oracle_scm(Xbar, z)
        low = np.tril(np.ones_like(Bref, dtype=bool))
        assert rel_err(Bg[low], Bref[low]) < 1e-10
        # h_i = A_i . Y^{-1}
        assert rel_err(h.cpu().numpy(), c.A.op(Yinv)) < 1e-10


def test_scm_maxcut_is_hadamard():
    from tests.gpu_helpers import Case, rel_err
    c = Case(lattice_maxcut(8, 7, seed=4))
    Xbar, z = c.random_iterate(5)
    B, _ = c.P.scm_assemble(c.to_layout(Xbar), torch.tensor(z, device="cuda:0"))
    Xh, _ = c.oracle_completion(Xbar)
    Yinv = np.linalg.inv(c.A.dense(0) - c.A.adjoint(z))
    low = np.tril(np.ones((c.inst.n, c.inst.n), dtype=bool))
    assert rel_err(B.cpu().numpy()[low], (Xh * Yinv)[low]) < 1e-10


@pytest.mark.parametrize("mk", SMALL[:4] + [SMALL[5]], ids=IDS[:4] + [IDS[5]])
def test_newton_step_matches_oracle(mk):
    from tests.gpu_helpers import Case, rel_err
    c = Case(mk())
    Xbar, z = c.random_iterate(7)
    st = c.P.newton_step(c.to_layout(Xbar), torch.tensor(z, device="cuda:0"))
    ref = pdipm.mc_newton_step(c.A, c.inst.b, c.perm, c.cliques, Xbar, z)
    assert abs(st["mu"] - ref["mu"]) <= 1e-12 * abs(ref["mu"])
    assert rel_err(st["dz"].cpu().numpy(), ref["dz"]) < 1e-8
    dX = c.from_layout(st["dX"])
    assert rel_err(dX[c.E], ref["dX"][c.E]) < 1e-8
    dY = c.from_layout(st["dY"])
    assert rel_err(dY[c.E], ref["dY"][c.E]) < 1e-8
    assert abs(st["alpha_p"] - ref["alpha_p"]) <= 1e-7 * ref["alpha_p"]
    # dual step: bisection lower bound within 1e-3 of the exact eigenvalue bound
    assert st["alpha_d"] <= ref["alpha_d"] * (1 + 1e-9)
    assert st["alpha_d"] >= ref["alpha_d"] * (1 - 2e-3)


@pytest.mark.parametrize("shape", [(8, 8), (16, 16), (11, 9), (7, 5)],
                         ids=["m64", "m256", "m99", "m35"])
def test_newton_step_scm_factor_tile_edges(shape):
    """The SCM factorisation runs on 32 x 32 tiles of the (m + 1) x m bordered matrix: m a
    multiple of 32 puts the right-hand-side row in a tile row of its own (m = 64, 256; eight
    column tiles for 256), m = 99 and 35 leave ragged last tiles."""
    from tests.gpu_helpers import Case, rel_err
    c = Case(lattice_maxcut(*shape, seed=2))
    Xbar, z = c.random_iterate(3)
    st = c.P.newton_step(c.to_layout(Xbar), torch.tensor(z, device="cuda:0"))
    ref = pdipm.mc_newton_step(c.A, c.inst.b, c.perm, c.cliques, Xbar, z)
    assert rel_err(st["dz"].cpu().numpy(), ref["dz"]) < 1e-8


def _solve(inst, **opts):
    from paper_1310_6919_gb300 import Problem
    P = Problem.from_instance(inst, device=0, **opts)
    if inst.meta.get("kind") != "maxcut":
        P.set_iterate(None, inst.z0)
    return P, P.solve()


def test_solve_grid_closed_form():
    inst = lattice_maxcut(10, 10)
    P, r = _solve(inst)
    W = sum(inst.meta["weights"])
    assert r["status"] == 0, r
    assert r["gap"] <= 1e-7 and r["pinf"] <= 1e-7
    assert abs(r["pobj"] + W) <= 1e-7 * W
    assert r["dobj"] <= -W * (1 - 1e-12) + 1e-9 and r["pobj"] >= -W * (1 + 1e-12) - 1e-9


@pytest.mark.parametrize("n", [7, 9])
def test_solve_odd_cycle_closed_form(n):
    inst = cycle_maxcut(n)
    P, r = _solve(inst)
    opt = maxcut.odd_cycle_optimum(n)
    assert r["status"] == 0
    assert abs(r["pobj"] - opt) <= 1e-7 * abs(opt)


def test_solve_complete_graph_closed_form():
    inst = complete_maxcut(8)
    P, r = _solve(inst)
    assert r["status"] == 0
    assert abs(r["pobj"] + 16.0) <= 1e-7 * 16


@pytest.mark.parametrize("mk", [SMALL[1], SMALL[2], SMALL[3], SMALL[5]],
                         ids=[IDS[1], IDS[2], IDS[3], IDS[5]])
def test_solve_matches_oracle_optimum(mk):
    inst = mk()
    P, r = _solve(inst)
    A = SparseSym.from_instance(inst)
    ref = pdipm.solve_dense(A, inst.b, inst.z0)
    assert r["status"] == 0 and ref["status"] == "optimal"
    scale = max(1.0, abs(ref["pobj"]))
    assert abs(r["pobj"] - ref["pobj"]) <= 1e-7 * scale
    assert abs(r["dobj"] - ref["dobj"]) <= 1e-7 * scale


def test_tiny_scalar_sdp():
    # n = m = 1: min 2x s.t. x = 3, x >= 0  ->  6
    inst = SDPInstance("scalar", 1, 1, np.array([3.0]), np.array([0, 1], np.int32),
                       np.array([0, 0], np.int32), np.array([0, 0], np.int32),
                       np.array([2.0, 1.0]), z0=np.array([0.0]), meta={"kind": "scalar"})
    P, r = _solve(inst)
    assert r["status"] == 0
    assert abs(r["pobj"] - 6.0) <= 1e-7 * 6


# ---------------- full-size workloads ----------------

def _golden(name):
    with open(os.path.join(GOLDEN, name + ".json")) as f:
        return json.load(f)


@pytest.fixture(scope="module")
def full_scm_2020():
    """The oracle's whole SCM (eq. newSCM, row by row from the A_k's nonzeros) of block_arrow_2020
    at one seeded interior iterate: about a minute on the host, shared by both precisions."""
    from tests.gpu_helpers import Case
    c = Case(workload("block_arrow_2020"), precision=1)  # precision 1 admits both forms
    Xbar, z = c.random_iterate(11, zscale=0.002)
    Bref, Xh, Yinv = c.oracle_scm(Xbar, z)
    return c, Xbar, z, Bref, c.A.op(Yinv)


@pytest.mark.parametrize("precision,tol", [(0, 1e-10), (1, 1e-5)], ids=["fp64", "mixed"])
def test_full_size_scm_whole_triangle(full_scm_2020, precision, tol):
    """Every entry of the lower triangle of B (2.0e6 entries at m = 2000) and h = A(Y^{-1})
    against the oracle, in the launch configuration the solves use."""
    from tests.gpu_helpers import rel_err
    c, Xbar, z, Bref, href = full_scm_2020
    B, h = c.P.scm_assemble(c.to_layout(Xbar), torch.tensor(z, device="cuda:0"),
                            precision=precision)
    Bg = B.cpu().numpy()
    low = np.tril(np.ones_like(Bref, dtype=bool))
    assert rel_err(Bg[low], Bref[low]) < tol
    assert rel_err(h.cpu().numpy(), href) < tol
    if precision == 0:
        # symmetric positive definite (linearly independent A_p)
        Bs = np.tril(Bg) + np.tril(Bg, -1).T
        assert np.linalg.eigvalsh(Bs)[0] > 0


@pytest.mark.parametrize("name", ["block_arrow_1020", "block_arrow_2020"])
def test_full_size_solve_matches_golden(name):
    g = _golden(name)
    inst = workload(name)
    P, r = _solve(inst)
    assert r["status"] == 0, r
    scale = max(1.0, abs(g["pobj"]))
    assert abs(r["pobj"] - g["pobj"]) <= 1e-7 * scale
    assert abs(r["dobj"] - g["dobj"]) <= 1e-7 * scale


def test_full_size_grid_solve():
    inst = workload("grid_maxcut_100")
    P, r = _solve(inst)
    W = sum(inst.meta["weights"])
    assert r["status"] == 0 and abs(r["pobj"] + W) <= 1e-7 * W
