"""Pins of the oracle's MC-PDIPM step and iteration (Sec. 2.2 with the completion of Sec. 2.1)."""
import numpy as np

from instances import block_arrow, complete_maxcut, lattice_maxcut
from oracle.sdp import SparseSym
from oracle import pdipm
from oracle.chordal import check_structure
from tests.chordal_helper import eliminate, supernodes


def _struct(inst, order=None):
    A = SparseSym.from_instance(inst)
    P = A.aggregate_pattern()
    perm = np.arange(inst.n) if order is None else np.asarray(order)
    F = eliminate(P[np.ix_(perm, perm)])
    cl = supernodes(F)
    check_structure(inst.n, cl)
    inv = np.empty_like(perm)
    inv[perm] = np.arange(inst.n)
    Eorig = F[np.ix_(inv, inv)]
    return A, perm, cl, Eorig


def test_dense_pattern_step_equals_dense_pdipm_step():
    # K_n max-cut: one clique, X̂ = X̄, so MC-PDIPM and the dense PDIPM take identical steps
    inst = complete_maxcut(6)
    A, perm, cl, E = _struct(inst)
    assert len(cl) == 1
    mc = pdipm.solve_mc(A, inst.b, inst.z0, perm, cl, E)
    de = pdipm.solve_dense(A, inst.b, inst.z0)
    assert mc["iters"] == de["iters"]
    for hm, hd in zip(mc["history"], de["history"]):
        assert abs(hm["pobj"] - hd["pobj"]) < 1e-9 * max(1, abs(hd["pobj"]))
        assert abs(hm["dobj"] - hd["dobj"]) < 1e-9 * max(1, abs(hd["dobj"]))


def test_mc_pdipm_matches_dense_optimum_block_arrow():
    inst = block_arrow(nblocks=3, bsize=5, border=2, m=12, per_matrix=4, seed=9)
    A, perm, cl, E = _struct(inst)
    mc = pdipm.solve_mc(A, inst.b, inst.z0, perm, cl, E)
    de = pdipm.solve_dense(A, inst.b, inst.z0)
    assert mc["status"] == "optimal" and de["status"] == "optimal"
    assert abs(mc["pobj"] - de["pobj"]) <= 1e-7 * max(1, abs(de["pobj"]))


def test_mc_pdipm_lattice_closed_form():
    inst = lattice_maxcut(4, 3, seed=2)
    A, perm, cl, E = _struct(inst)
    mc = pdipm.solve_mc(A, inst.b, inst.z0, perm, cl, E)
    W = sum(inst.meta["weights"])
    assert mc["status"] == "optimal"
    assert abs(mc["pobj"] + W) <= 1e-6 * W


def test_mc_step_unit_step_residuals():
    inst = block_arrow(nblocks=2, bsize=4, border=2, m=8, per_matrix=4, seed=3)
    A, perm, cl, E = _struct(inst)
    X = np.eye(inst.n)
    st = pdipm.mc_newton_step(A, inst.b, perm, cl, X, inst.z0)
    # A(X̂ + dX) = b and sum A (z + dz) + Y + dY = A_0
    assert np.allclose(A.op(st["Xh"] + st["dX"]), inst.b, atol=1e-10)
    assert np.allclose(A.adjoint(inst.z0 + st["dz"]) + st["Y"] + st["dY"], A.dense(0), atol=1e-10)
    assert 0 < st["alpha_p"] <= 1 and 0 < st["alpha_d"] <= 1
