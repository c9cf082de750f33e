"""GPU parity of the dense-root path against the oracle.

When the chordal extension has cliques beyond the small-clique kernels (more than 160 rows or 96
columns; the random-graph max-cut of n = 20000 has a separator clique of thousands), those cliques
and their ancestors become one dense root clique R, handled by dense kernels (Cholesky, triangular
inverse, X^T X, GEMM, Lanczos step-length bounds); the forest below keeps the small-clique
kernels.  The option root_rows lowers the threshold so that small problems, which the oracle
solves in seconds, take the same path: root_rows = 6 or 10 here puts most of each problem into
the root while leaving a forest of several levels.

Tolerances as in test_gpu_parity: factors and SCM entries 1e-10 relative to the largest entry
(FP64); Newton direction 1e-8; the mixed form's FP32 SCM 1e-5; optimal values 1e-7 at relative
gap 1e-7.  The step lengths are Lanczos bounds (reading: the paper gives no dual step rule for
sparse Y; the root clique's primal step is its eq. primal_length2 bound estimated without a dense
eigendecomposition): each may not exceed the exact bound and must reach 99% of it."""
import os
import json

import numpy as np
import pytest
import torch

from instances import (lattice_maxcut, block_arrow, small_random_sdp, random_gnm_maxcut,
                       random_ring_maxcut, cycle_maxcut, workload)
from oracle import pdipm, maxcut
from oracle.sdp import SparseSym

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")

CASES = [
    (lambda: lattice_maxcut(10, 10), 6),
    (lambda: block_arrow(6, 12, 4, 60, per_matrix=8, seed=5), 10),
    (lambda: random_gnm_maxcut(90, 200, 4), 10),
    (lambda: random_ring_maxcut(150, seed=9), 10),
    (lambda: small_random_sdp(9, 14, 2), 4),
]
IDS = ["grid100", "arrow6x12", "gnm90", "ring150", "dense9"]


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1310_6919_gb300 import build_library
    build_library()
    assert torch.cuda.is_available()


def _case(mk, rr, **opts):
    from tests.gpu_helpers import Case
    c = Case(mk(), root_rows=rr, **opts)
    info = c.P.info
    # the path under test: a dense root (the last supernode) and a forest below it
    assert info["max_nrow"] > rr or info["nsuper"] == 1
    return c


@pytest.mark.parametrize("mk,rr", CASES, ids=IDS)
def test_dense_root_factors_match_oracle(mk, rr):
    from tests.gpu_helpers import rel_err
    c = _case(mk, rr)
    Xbar, z = c.random_iterate(1)
    Lh, N = c.P.factors(c.to_layout(Xbar), torch.tensor(z, device="cuda:0"))
    Lref, Nref = c.oracle_factors(Xbar, z)
    r, q, v = c.layout_values_new(Lh)
    assert rel_err(v, Lref[r, q]) < 1e-10
    r, q, v = c.layout_values_new(N)
    assert rel_err(v, Nref[r, q]) < 1e-10


@pytest.mark.parametrize("mk,rr", CASES, ids=IDS)
def test_dense_root_scm_matches_oracle(mk, rr):
    from tests.gpu_helpers import rel_err
    c = _case(mk, rr)
    for seed in (2, 3):
        Xbar, z = c.random_iterate(seed)
        B, h = c.P.scm_assemble(c.to_layout(Xbar), torch.tensor(z, device="cuda:0"))
        Bg = B.cpu().numpy()
        Bref, Xh, Yinv = c.oracle_scm(Xbar, z)
        low = np.tril(np.ones_like(Bref, dtype=bool))
        assert rel_err(Bg[low], Bref[low]) < 1e-10
        assert rel_err(h.cpu().numpy(), c.A.op(Yinv)) < 1e-10


@pytest.mark.parametrize("mk,rr", CASES[:4], ids=IDS[:4])
def test_dense_root_mixed_scm(mk, rr):
    """The mixed form's FP32 solves, triangular inverse and contraction at the root."""
    from tests.gpu_helpers import rel_err
    c = _case(mk, rr, precision=1)
    Xbar, z = c.random_iterate(4)
    B, h = c.P.scm_assemble(c.to_layout(Xbar), torch.tensor(z, device="cuda:0"), precision=1)
    Bref, Xh, Yinv = c.oracle_scm(Xbar, z)
    low = np.tril(np.ones_like(Bref, dtype=bool))
    assert rel_err(B.cpu().numpy()[low], Bref[low]) < 1e-5
    assert rel_err(h.cpu().numpy(), c.A.op(Yinv)) < 1e-5


@pytest.mark.parametrize("mk,rr", CASES, ids=IDS)
def test_dense_root_newton_step(mk, rr):
    from tests.gpu_helpers import rel_err
    c = _case(mk, rr)
    Xbar, z = c.random_iterate(7)
    st = c.P.newton_step(c.to_layout(Xbar), torch.tensor(z, device="cuda:0"))
    ref = pdipm.mc_newton_step(c.A, c.inst.b, c.perm, c.cliques, Xbar, z)
    assert abs(st["mu"] - ref["mu"]) <= 1e-12 * abs(ref["mu"])
    assert rel_err(st["dz"].cpu().numpy(), ref["dz"]) < 1e-8
    dX = c.from_layout(st["dX"])
    assert rel_err(dX[c.E], ref["dX"][c.E]) < 1e-8
    dY = c.from_layout(st["dY"])
    assert rel_err(dY[c.E], ref["dY"][c.E]) < 1e-8
    for key in ("alpha_p", "alpha_d"):
        assert st[key] <= ref[key] * (1 + 1e-9)
        assert st[key] >= ref[key] * 0.99


def _solve(inst, **opts):
    from paper_1310_6919_gb300 import Problem
    P = Problem.from_instance(inst, device=0, **opts)
    if inst.meta.get("kind") != "maxcut":
        P.set_iterate(None, inst.z0)
    return P, P.solve()


@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "mixed"])
def test_dense_root_solve_grid_closed_form(precision):
    inst = lattice_maxcut(10, 10)
    _, r = _solve(inst, root_rows=6, precision=precision)
    assert r["status"] == 0
    W = float(np.sum(inst.meta["weights"]))
    assert abs(r["pobj"] - (-W)) <= 1e-7 * W


@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "mixed"])
def test_dense_root_solve_odd_cycle(precision):
    n = 21
    _, r = _solve(cycle_maxcut(n), root_rows=2, precision=precision)
    assert r["status"] == 0
    opt = maxcut.odd_cycle_optimum(n)
    assert abs(r["pobj"] - opt) <= 1e-7 * abs(opt)


@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "mixed"])
def test_dense_root_solve_block_arrow_golden(precision):
    with open(os.path.join(GOLDEN, "block_arrow_1020.json")) as f:
        g = json.load(f)
    inst = workload("block_arrow_1020")
    _, r = _solve(inst, root_rows=40, precision=precision)
    assert r["status"] == 0
    assert abs(r["pobj"] - g["pobj"]) <= 1e-7 * abs(g["pobj"])


def test_dense_root_solve_matches_dense_oracle():
    """A random sparse max-cut whose separator goes into the root: the optimum against the
    oracle's dense PDIPM."""
    inst = random_ring_maxcut(150, seed=9)
    _, r = _solve(inst, root_rows=10)
    assert r["status"] == 0
    A = SparseSym.from_instance(inst)
    ref = pdipm.solve_dense(A, inst.b, inst.z0)
    assert abs(r["pobj"] - ref["pobj"]) <= 1e-7 * abs(ref["pobj"])
