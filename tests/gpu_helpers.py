"""Glue for the GPU parity tests: runs libmcsdp on a seeded instance and the oracle on the same
data, and converts between the library's supernodal layout and dense matrices (index mapping
only; no arithmetic of the method lives here)."""
import numpy as np
import torch

from oracle.sdp import SparseSym, dual_slack
from oracle.chordal import cliques_from_supernodes, pattern_from_cliques
from oracle.completion import max_det_completion, algorithm1
from oracle.scm import scm_sparse_rows, scm_entry


class Case:
    def __init__(self, inst, **opts):
        from paper_1310_6919_gb300 import Problem
        self.inst = inst
        self.P = Problem.from_instance(inst, device=0, **opts)
        self.A = SparseSym.from_instance(inst)
        ro, co, valid, s = self.P.layout_index()
        self.ro, self.co, self.valid, self.sym = ro, co, valid, s
        self.perm = s["perm"].astype(np.int64)
        self.cliques = cliques_from_supernodes(s["sn_col"], s["sn_rowptr"], s["sn_rows"])
        n = inst.n
        En = pattern_from_cliques(n, self.cliques)
        inv = np.empty_like(self.perm)
        inv[self.perm] = np.arange(n)
        self.E = En[np.ix_(inv, inv)]          # original order
        # layout position (new indices) for comparisons in the elimination order
        self.rn = inv[ro]
        self.cn = inv[co]

    # ---- conversions ----
    def to_layout(self, Xd):
        v = np.where(self.valid, Xd[self.ro, self.co], 0.0)
        return torch.tensor(v, dtype=torch.float64, device="cuda:0")

    def from_layout(self, t):
        v = t.detach().cpu().numpy()
        n = self.inst.n
        X = np.zeros((n, n))
        X[self.ro[self.valid], self.co[self.valid]] = v[self.valid]
        X[self.co[self.valid], self.ro[self.valid]] = v[self.valid]
        return X

    def layout_values_new(self, t):
        """(rows_new, cols_new, values) of the stored lower entries."""
        v = t.detach().cpu().numpy()
        return self.rn[self.valid], self.cn[self.valid], v[self.valid]

    # ---- iterates ----
    def random_iterate(self, seed, zscale=0.01):
        rng = np.random.default_rng(seed)
        n = self.inst.n
        G = rng.standard_normal((n, n + 5))
        Xd = G @ G.T / (n + 5) + 0.5 * np.eye(n)
        Xbar = np.where(self.E, Xd, 0.0)
        z = self.inst.z0 + zscale * rng.standard_normal(self.inst.m)
        return Xbar, z

    # ---- oracle quantities at (Xbar, z) ----
    def oracle_completion(self, Xbar):
        p = self.perm
        Xn = Xbar[np.ix_(p, p)]
        Xhn = max_det_completion(Xn, self.cliques)
        inv = np.empty_like(p)
        inv[p] = np.arange(len(p))
        return Xhn[np.ix_(inv, inv)], Xn

    def oracle_scm(self, Xbar, z, rows=None):
        Xh, _ = self.oracle_completion(Xbar)
        Y = dual_slack(self.A, z)
        Yinv = np.linalg.inv(Y)
        Yinv = 0.5 * (Yinv + Yinv.T)
        return scm_sparse_rows(self.A, Xh, Yinv, rows), Xh, Yinv

    def oracle_factors(self, Xbar, z):
        p = self.perm
        Xn = Xbar[np.ix_(p, p)]
        Lh = algorithm1(Xn, self.cliques)
        Y = dual_slack(self.A, z)
        N = np.linalg.cholesky(Y[np.ix_(p, p)])
        return Lh, N


def rel_err(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))
