"""Planted mistakes in the oracle are caught by its pins.

Each case takes the source of one oracle module, changes one expression into a plausible
mistake (a dropped term, a wrong sign, a wrong index, a transposed operand, a wrong
permutation), executes the changed module in a fresh namespace and runs the pins of the changed
function against it: at least one pin must fail.  The unchanged source passes the same pins, so
the failure belongs to the planted mistake.  Everything runs on the CPU.
"""
import inspect

import numpy as np
import pytest
import scipy.linalg as sla

import oracle.certificate
import oracle.completion
import oracle.diff
import oracle.pdipm
import oracle.scm
import oracle.sdp
from instances import (block_arrow, complete_maxcut, diagonal_lp_sdp, lattice_maxcut,
                       small_random_sdp)
from oracle import maxcut
from oracle.sdp import SparseSym
from tests.chordal_helper import eliminate, pd_on_pattern, random_pattern, supernodes

CAUGHT = (AssertionError, np.linalg.LinAlgError, sla.LinAlgError, RuntimeError)


def load(module, old=None, new=None):
    """The module's namespace, executed from its source with `old` replaced by `new`."""
    src = inspect.getsource(module)
    if old is not None:
        assert src.count(old) == 1, f"mutation site not found exactly once: {old!r}"
        src = src.replace(old, new)
    ns = {"__name__": module.__name__ + "_planted", "__package__": "oracle",
          "__file__": module.__file__}
    exec(compile(src, module.__file__, "exec"), ns)
    return ns


def _pd(n, seed):
    rng = np.random.default_rng(seed)
    G = rng.standard_normal((n, 2 * n))
    return G @ G.T / (2 * n) + 0.3 * np.eye(n)


def _sym_inv(M):
    Mi = np.linalg.inv(M)
    return 0.5 * (Mi + Mi.T)


# ---- pins, each a function of a module namespace ----

def pins_scm(ns):
    for f in (ns["scm_dense"], ns["scm_sparse_rows"]):
        # max-cut: B = X ∘ Y^{-1}
        A = SparseSym.from_instance(lattice_maxcut(4, 3, seed=5))
        X, Yinv = _pd(12, 1), _sym_inv(_pd(12, 2))
        assert np.allclose(f(A, X, Yinv), X * Yinv, atol=1e-14)
        # diagonal data: the LP normal matrix
        inst = diagonal_lp_sdp(9, 6, seed=3)
        A = SparseSym.from_instance(inst)
        x = np.random.default_rng(0).uniform(0.5, 2, 9)
        y = np.random.default_rng(1).uniform(0.5, 2, 9)
        Am = np.array([[A.dense(k)[i, i] for i in range(9)] for k in range(1, 7)])
        assert np.allclose(f(A, np.diag(x), np.diag(1 / y)), Am @ np.diag(x / y) @ Am.T,
                           atol=1e-13)
    # general data: symmetric positive definite, both forms agree
    A = SparseSym.from_instance(small_random_sdp(7, 10, 1))
    X, Yinv = _pd(7, 11), _sym_inv(_pd(7, 21))
    B = ns["scm_dense"](A, X, Yinv)
    assert np.allclose(B, B.T, atol=1e-12 * np.abs(B).max())
    assert np.linalg.eigvalsh(B)[0] > 0
    assert np.allclose(ns["scm_sparse_rows"](A, X, Yinv), B, atol=1e-12 * np.abs(B).max())


def pins_rhs(ns):
    # a unit step of the direction built on g zeroes both linear residuals
    inst = small_random_sdp(6, 8, 4)
    A = SparseSym.from_instance(inst)
    X, Y = _pd(6, 3), _pd(6, 4)
    z = inst.z0 + 0.05 * np.random.default_rng(2).standard_normal(8)
    G = A.dense(0) - A.adjoint(z) - Y
    Yinv = np.linalg.inv(Y)
    mu, beta = np.sum(X * Y) / 6, 0.1
    B = oracle.scm.scm_dense(A, X, Yinv)
    dz = sla.solve(B, ns["hkm_rhs"](A, inst.b, X, Yinv, G, beta, mu))
    dY = G - A.adjoint(dz)
    dXh = beta * mu * Yinv - X - X @ dY @ Yinv
    assert np.allclose(A.op(X + 0.5 * (dXh + dXh.T)), inst.b, atol=1e-10)
    assert np.allclose(A.adjoint(z + dz) + Y + dY, A.dense(0), atol=1e-10)


def _chordal_case(seed=2):
    rng = np.random.default_rng(seed)
    F = eliminate(random_pattern(15, 0.15, rng))
    cl = supernodes(F)
    return F, cl, pd_on_pattern(F, rng, cl)


def pins_completion(ns):
    F, cl, X = _chordal_case()
    Xh = ns["max_det_completion"](X, cl)
    assert np.allclose(Xh[F], X[F], rtol=0, atol=1e-13)
    assert np.linalg.eigvalsh(Xh)[0] > 0
    Xi = np.linalg.inv(Xh)
    assert np.max(np.abs(Xi[~F])) <= 1e-10 * np.max(np.abs(Xi))


def pins_algorithm1(ns):
    F, cl, X = _chordal_case()
    Lh = ns["algorithm1"](X, cl)
    Xh = oracle.completion.max_det_completion(X, cl)
    assert np.allclose(Lh, oracle.completion.inverse_cholesky_definition(Xh), atol=1e-10)
    assert np.all(Lh[~np.tril(F)] == 0.0)


def pins_max_step(ns):
    f = ns["max_step"]
    m, d = np.array([2.0, 1.0, 4.0, 0.5]), np.array([-1.0, 3.0, -10.0, 0.0])
    assert f(np.diag(m), np.diag(d)) == pytest.approx(0.4, rel=1e-14)
    assert f(np.diag(m), np.diag([-1.0, -0.5, -2.0, -0.25])) == 1.0
    rng = np.random.default_rng(0)
    M = _pd(7, 5)
    D = rng.standard_normal((7, 7))
    D = 4.0 * (D + D.T)
    a = f(M, D)
    assert 0.0 < a <= 1.0
    assert np.linalg.eigvalsh(M + a * D)[0] == pytest.approx(0.0, abs=1e-10)


def pins_measures(ns):
    inst = lattice_maxcut(4, 3, seed=11)
    A = SparseSym.from_instance(inst)
    side = [(i % 4 + i // 4) % 2 for i in range(12)]
    X, z = maxcut.bipartite_certificates(12, inst.meta["edges"], inst.meta["weights"], side)
    Y = A.dense(0) - A.adjoint(z)
    pobj, dobj, gap, pinf, dinf = ns["measures"](A, inst.b, X, Y, z)
    W = float(sum(inst.meta["weights"]))
    assert pobj == pytest.approx(-W, rel=1e-14) and dobj == pytest.approx(-W, rel=1e-14)
    assert gap < 1e-15 and pinf == 0.0 and dinf < 1e-15


def pins_sdp(ns):
    S = ns["SparseSym"]
    inst = small_random_sdp(6, 5, seed=0)
    A = S.from_instance(inst)
    rng = np.random.default_rng(0)
    M = rng.standard_normal((6, 6))
    M = M + M.T
    y = rng.standard_normal(5)
    assert np.dot(A.op(M), y) == pytest.approx(float(np.sum(M * A.adjoint(y))), rel=1e-13)
    for k in range(1, 6):
        r, c, v = inst.matrix_entries(k)
        ref = sum(val * M[i, j] * (1.0 if i == j else 2.0) for i, j, val in zip(r, c, v))
        assert A.op(M)[k - 1] == pytest.approx(ref, rel=1e-13)
    # the dual slack at the bipartite optimum annihilates the cut vector
    inst = lattice_maxcut(4, 3, seed=11)
    A = S.from_instance(inst)
    x = np.array([1.0 if (i % 4 + i // 4) % 2 == 0 else -1.0 for i in range(12)])
    _, z = maxcut.bipartite_certificates(12, inst.meta["edges"], inst.meta["weights"],
                                         (x < 0).astype(int))
    Y = ns["dual_slack"](A, z)
    assert np.allclose(Y @ x, 0.0, atol=1e-12) and np.linalg.eigvalsh(Y)[0] > -1e-12


def pins_solve_dense(ns):
    inst = lattice_maxcut(4, 3, seed=7)
    A = SparseSym.from_instance(inst)
    res = ns["solve_dense"](A, inst.b, inst.z0)
    W = sum(inst.meta["weights"])
    assert res["status"] == "optimal"
    assert abs(res["pobj"] + W) <= 1e-6 * W


def pins_mc_step(ns):
    # a non-identity elimination order and an X̄ that is not the identity, so a wrong
    # permutation or a wrong completion shows
    inst = block_arrow(nblocks=2, bsize=4, border=2, m=8, per_matrix=4, seed=3)
    A = SparseSym.from_instance(inst)
    n = inst.n
    perm = np.random.default_rng(1).permutation(n)
    F = eliminate(A.aggregate_pattern()[np.ix_(perm, perm)])
    cl = supernodes(F)
    inv = np.empty_like(perm)
    inv[perm] = np.arange(n)
    E = F[np.ix_(inv, inv)]
    Xn = pd_on_pattern(F, np.random.default_rng(4), cl)
    Xbar = np.where(E, Xn[np.ix_(inv, inv)], 0.0)
    st = ns["mc_newton_step"](A, inst.b, perm, cl, Xbar, inst.z0)
    assert np.allclose(st["Xh"][E], Xbar[E], atol=1e-13)
    Xi = np.linalg.inv(st["Xh"])
    assert np.max(np.abs(Xi[~E])) <= 1e-10 * np.max(np.abs(Xi))
    assert np.allclose(A.op(st["Xh"] + st["dX"]), inst.b, atol=1e-10)
    assert np.allclose(A.adjoint(inst.z0 + st["dz"]) + st["Y"] + st["dY"], A.dense(0),
                       atol=1e-10)
    # one clique (K_n): the step is the dense PDIPM's
    inst = complete_maxcut(5)
    A = SparseSym.from_instance(inst)
    full = np.ones((5, 5), bool)
    cl1 = supernodes(full)
    assert len(cl1) == 1
    X = _pd(5, 9)
    X = X / np.sqrt(np.outer(np.diag(X), np.diag(X)))      # diag 1: primal feasible
    st = ns["mc_newton_step"](A, inst.b, np.arange(5), cl1, X, inst.z0)
    Y = A.dense(0) - A.adjoint(inst.z0)
    Yinv = np.linalg.inv(Y)
    mu = np.sum(X * Y) / 5
    B = oracle.scm.scm_dense(A, X, Yinv)
    dz = sla.solve(B, inst.b - 0.1 * mu * A.op(Yinv))
    assert np.allclose(st["dz"], dz, rtol=1e-9, atol=1e-12)


def pins_diff(ns):
    inst = small_random_sdp(4, 3, 11)
    A = SparseSym.from_instance(inst)
    rng = np.random.default_rng(3)
    G = rng.standard_normal((4, 4))
    G = 0.5 * (G + G.T)
    gz = rng.standard_normal(3)
    mu, h = 0.3, 1e-6
    z, Y, X, res = ns["central_point"](A, inst.b, mu, inst.z0)
    assert res <= 1e-12
    assert np.max(np.abs(A.op(X) - inst.b)) <= 1e-12 * max(1, np.max(np.abs(inst.b)))
    assert np.allclose(X @ Y, mu * np.eye(4), atol=1e-10)
    gb, gA0, _ = ns["backward"](A, z, Y, X, G, gz)
    ge = ns["entry_gradients"](inst, z, gb, gA0, X)
    scale = max(1.0, np.max(np.abs(ge)), np.max(np.abs(gb)))

    def l_at(val, b):
        Ap = SparseSym(inst.n, inst.m, inst.mat, inst.row, inst.col, val)
        return oracle.diff.loss(Ap, b, mu, z, G, gz)

    for p in range(inst.m):
        e = np.zeros(inst.m)
        e[p] = h
        fd = (l_at(inst.val, inst.b + e) - l_at(inst.val, inst.b - e)) / (2 * h)
        assert abs(fd - gb[p]) <= 1e-6 * scale
    for t in range(len(inst.val)):
        e = np.zeros(len(inst.val))
        e[t] = h
        fd = (l_at(inst.val + e, inst.b) - l_at(inst.val - e, inst.b)) / (2 * h)
        assert abs(fd - ge[t]) <= 1e-6 * scale


def pins_certificate(ns):
    inst = lattice_maxcut(4, 3, seed=2)
    A = SparseSym.from_instance(inst)
    perm = np.arange(12)
    F = eliminate(A.aggregate_pattern())
    cl = supernodes(F)
    mc = oracle.pdipm.solve_mc(A, inst.b, inst.z0, perm, cl, F)
    c = ns["certify"](A, inst.b, perm, cl, mc["Xbar"], mc["z"])
    W = float(sum(inst.meta["weights"]))
    assert c["y_pd"] and c["cliques_pd"]
    assert c["lower"] <= -W + 1e-9 * W and -W <= c["upper"] + 1e-7 * W
    rows, _ = max(cl, key=lambda q: len(q[0]))
    X = mc["Xbar"].copy()
    i, j = int(rows[0]), int(rows[1])
    X[i, j] = X[j, i] = 2.0 * np.sqrt(X[i, i] * X[j, j])
    assert not ns["certify"](A, inst.b, perm, cl, X, mc["z"])["cliques_pd"]


# (module, pin set, planted mistake: original text -> changed text)
MUTANTS = [
    # eq. (SCM): dropped Y^{-1}, wrong operand, wrong sign
    (oracle.scm, pins_scm, "T = X @ A.dense(i) @ Yinv", "T = X @ A.dense(i)"),
    (oracle.scm, pins_scm, "T = X @ A.dense(i) @ Yinv", "T = Yinv @ A.dense(i) @ Yinv"),
    (oracle.scm, pins_scm, "B[i - 1, :] = A.op(T)", "B[i - 1, :] = -A.op(T)"),
    # nonzero-wise rows: wrong index into Y^{-1}, dropped value of A_j, dropped value of A_i
    (oracle.scm, pins_scm, "Yg = Yinv[np.ix_(b, pd)].T", "Yg = Yinv[np.ix_(a, pd)].T"),
    (oracle.scm, pins_scm, "weights=pv * T", "weights=T"),
    (oracle.scm, pins_scm, "T = (Xg * Yg) @ v ", "T = (Xg * Yg) @ np.abs(v) "),
    # right-hand side: wrong sign of the centring term, of the G term, dropped b
    (oracle.scm, pins_rhs, "M = beta * mu * Yinv", "M = -beta * mu * Yinv"),
    (oracle.scm, pins_rhs, "M = M - X @ G @ Yinv", "M = M + X @ G @ Yinv"),
    (oracle.scm, pins_rhs, "return b - A.op(M)", "return -A.op(M)"),
    # Lemma 2.6: dropped X_UU^{-1}, zero fill instead of the completion
    (oracle.completion, pins_completion, "XSU @ np.linalg.solve(XUU, Xh[np.ix_(U, T)])",
     "XSU @ Xh[np.ix_(U, T)]"),
    (oracle.completion, pins_completion, "XST = XSU @ np.linalg.solve(",
     "XST = 0.0 * XSU @ np.linalg.solve("),
    # Algorithm 1: no reversal, transposed inverse, last instead of first |S_r| columns
    (oracle.completion, pins_algorithm1, "P = np.eye(k)[::-1]", "P = np.eye(k)"),
    (oracle.completion, pins_algorithm1, "Lr = P @ np.linalg.inv(M).T @ P.T",
     "Lr = P @ np.linalg.inv(M) @ P.T"),
    (oracle.completion, pins_algorithm1, "= Lr[:, :ns]", "= Lr[:, len(rows) - ns:]"),
    # step length: largest instead of smallest eigenvalue, no cap at 1
    (oracle.pdipm, pins_max_step, "(0.5 * (W + W.T))[0]", "(0.5 * (W + W.T))[-1]"),
    (oracle.pdipm, pins_max_step, "if lam >= -1.0:", "if lam >= 0.0:"),
    # stopping test: sum instead of difference of the objectives, dual residual without Y
    (oracle.pdipm, pins_measures, "gap = abs(pobj - dobj)", "gap = abs(pobj + dobj)"),
    (oracle.pdipm, pins_measures, "dres = A0 - A.adjoint(z) - Y", "dres = A0 - A.adjoint(z)"),
    # dense PDIPM: wrong sign of the dY update, dropped Y^{-1} in dX
    (oracle.pdipm, pins_solve_dense, "dY = G - A.adjoint(dz)", "dY = G + A.adjoint(dz)"),
    (oracle.pdipm, pins_solve_dense, "dXh = beta * mu * Yinv - X - X @ dY @ Yinv",
     "dXh = beta * mu * Yinv - X - X @ dY"),
    # MC step: completion mapped back with the wrong permutation, wrong sign of dY
    (oracle.pdipm, pins_mc_step, "Xh = Xh_n[np.ix_(inv, inv)]", "Xh = Xh_n[np.ix_(p, p)]"),
    (oracle.pdipm, pins_mc_step, "dY = -A.adjoint(dz)", "dY = A.adjoint(dz)"),
    # problem data: transposed index in A(M), wrong sign in Y(z)
    (oracle.sdp, pins_sdp, "w = self.v * M[self.r, self.c]", "w = self.v * M[self.r, self.r]"),
    (oracle.sdp, pins_sdp, "return A.dense(0) - A.adjoint(z)", "return A.dense(0) + A.adjoint(z)"),
    # implicit derivatives: wrong sign of G in g_{A_0}, of v_k X in g_{A_k}, dropped X in R,
    # dropped mirror factor of off-diagonal entries
    (oracle.diff, pins_diff, "(A.adjoint(v) - G)", "(A.adjoint(v) + G)"),
    (oracle.diff, pins_diff, "else (-z[k - 1] * gA0[i, j] - v[k - 1] * X[i, j])",
     "else (-z[k - 1] * gA0[i, j] + v[k - 1] * X[i, j])"),
    (oracle.diff, pins_diff, "R = _sym(X @ G @ Yinv)", "R = _sym(G @ Yinv)"),
    (oracle.diff, pins_diff, "f = 1.0 if i == j else 2.0", "f = 1.0"),
    # certificate: largest instead of smallest clique eigenvalue, wrong sign of the lower end
    (oracle.certificate, pins_certificate, "(Xn[np.ix_(rows, rows)])[0]",
     "(Xn[np.ix_(rows, rows)])[-1]"),
    (oracle.certificate, pins_certificate, "lower=float(np.dot(b, z))",
     "lower=-float(np.dot(b, z))"),
]

UNCHANGED = [(oracle.scm, pins_scm), (oracle.scm, pins_rhs),
             (oracle.completion, pins_completion), (oracle.completion, pins_algorithm1),
             (oracle.pdipm, pins_max_step), (oracle.pdipm, pins_measures),
             (oracle.pdipm, pins_solve_dense), (oracle.pdipm, pins_mc_step),
             (oracle.sdp, pins_sdp), (oracle.diff, pins_diff),
             (oracle.certificate, pins_certificate)]


@pytest.mark.parametrize("module,pins", UNCHANGED,
                         ids=[f"{m.__name__}-{p.__name__}" for m, p in UNCHANGED])
def test_unchanged_source_passes(module, pins):
    pins(load(module))


@pytest.mark.parametrize("module,pins,old,new", MUTANTS,
                         ids=[f"{m.__name__}-{i}" for i, (m, _, _, _) in enumerate(MUTANTS)])
def test_planted_mistake_is_caught(module, pins, old, new):
    ns = load(module, old, new)
    with pytest.raises(CAUGHT):
        pins(ns)
