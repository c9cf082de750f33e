"""Pins of oracle.certificate (weak duality plus Grone's completion theorem, Sec. 1 and 2.1)."""
import numpy as np
import pytest

from instances import block_arrow, lattice_maxcut
from oracle import pdipm
from oracle.certificate import certify
from oracle.sdp import SparseSym
from tests.chordal_helper import eliminate, supernodes


def _solved(inst):
    A = SparseSym.from_instance(inst)
    perm = np.arange(inst.n)
    F = eliminate(A.aggregate_pattern())
    cl = supernodes(F)
    mc = pdipm.solve_mc(A, inst.b, inst.z0, perm, cl, F)
    assert mc["status"] == "optimal"
    return A, perm, cl, F, mc


def test_certificate_brackets_the_lattice_closed_form():
    inst = lattice_maxcut(4, 3, seed=2)
    A, perm, cl, F, mc = _solved(inst)
    c = certify(A, inst.b, perm, cl, mc["Xbar"], mc["z"])
    W = float(sum(inst.meta["weights"]))
    assert c["y_pd"] and c["cliques_pd"] and c["pinf"] <= 1e-7
    assert c["lower"] <= -W + 1e-9 * W and -W <= c["upper"] + 1e-7 * W
    assert c["upper"] - c["lower"] <= 2e-7 * W


def test_certificate_brackets_the_dense_optimum():
    inst = block_arrow(nblocks=3, bsize=5, border=2, m=12, per_matrix=4, seed=9)
    A, perm, cl, F, mc = _solved(inst)
    de = pdipm.solve_dense(A, inst.b, inst.z0)
    c = certify(A, inst.b, perm, cl, mc["Xbar"], mc["z"])
    assert c["y_pd"] and c["cliques_pd"]
    s = max(1.0, abs(de["pobj"]))
    assert c["lower"] - 1e-7 * s <= de["pobj"] <= c["upper"] + 1e-7 * s


def test_certificate_rejects_infeasible_points():
    inst = lattice_maxcut(4, 3, seed=2)
    A, perm, cl, F, mc = _solved(inst)
    # z raised until Y(z) has a negative eigenvalue: not dual feasible
    z = mc["z"].copy()
    z[0] += 10.0
    assert not certify(A, inst.b, perm, cl, mc["Xbar"], z)["y_pd"]
    # one clique block made indefinite (an off-diagonal entry beyond the diagonal's product):
    # no positive definite completion exists
    rows, _ = max(cl, key=lambda c: len(c[0]))
    i, j = int(rows[0]), int(rows[1])
    X = mc["Xbar"].copy()
    X[i, j] = X[j, i] = 2.0 * np.sqrt(X[i, i] * X[j, j])
    c = certify(A, inst.b, perm, cl, X, mc["z"])
    assert not c["cliques_pd"] and c["min_clique_eig"] < 0
    # a diagonal entry moved off A(X) = b shows as the primal residual
    X = mc["Xbar"].copy()
    X[3, 3] += 1e-3
    assert certify(A, inst.b, perm, cl, X, mc["z"])["pinf"] == pytest.approx(1e-3, rel=1e-3)
