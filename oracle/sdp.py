"""Problem data helpers for the oracle (Sec. 1: (P) min A_0.X s.t. A_k.X = b_k, X psd;
(D) max b^T z s.t. sum_k A_k z_k + Y = A_0, Y psd).  U.V = sum_ij U_ij V_ij."""
import numpy as np


class SparseSym:
    """Symmetric matrices A_0..A_m as full (both triangles) coordinate lists."""

    def __init__(self, n, m, mat, row, col, val):
        self.n, self.m = int(n), int(m)
        mat = np.asarray(mat, dtype=np.int64)
        row = np.asarray(row, dtype=np.int64)
        col = np.asarray(col, dtype=np.int64)
        val = np.asarray(val, dtype=np.float64)
        off = row != col
        self.k = np.concatenate([mat, mat[off]])
        self.r = np.concatenate([row, col[off]])
        self.c = np.concatenate([col, row[off]])
        self.v = np.concatenate([val, val[off]])
        order = np.argsort(self.k, kind="stable")
        self.k, self.r, self.c, self.v = self.k[order], self.r[order], self.c[order], self.v[order]
        self.ptr = np.searchsorted(self.k, np.arange(self.m + 2))

    @classmethod
    def from_instance(cls, inst):
        return cls(inst.n, inst.m, inst.mat, inst.row, inst.col, inst.val)

    def entries(self, k):
        s, e = self.ptr[k], self.ptr[k + 1]
        return self.r[s:e], self.c[s:e], self.v[s:e]

    def dense(self, k):
        A = np.zeros((self.n, self.n))
        r, c, v = self.entries(k)
        np.add.at(A, (r, c), v)
        return A

    def inner(self, k, M):
        """A_k . M for a dense M."""
        r, c, v = self.entries(k)
        return float(np.sum(v * M[r, c]))

    def op(self, M):
        """A(M) = (A_k . M)_{k=1..m}."""
        w = self.v * M[self.r, self.c]
        out = np.bincount(self.k, weights=w, minlength=self.m + 1)
        return out[1:self.m + 1]

    def adjoint(self, y):
        """sum_k y_k A_k as a dense matrix (k = 1..m)."""
        S = np.zeros((self.n, self.n))
        sel = self.k >= 1
        np.add.at(S, (self.r[sel], self.c[sel]), self.v[sel] * y[self.k[sel] - 1])
        return S

    def aggregate_pattern(self):
        """Aggregate sparsity pattern: (i, j) with [A_k]_ij != 0 for some k = 0..m, plus the
        diagonal (Sec. 1)."""
        P = np.zeros((self.n, self.n), dtype=bool)
        P[self.r, self.c] = True
        P[np.arange(self.n), np.arange(self.n)] = True
        return P


def dual_slack(A, z):
    """Y = A_0 - sum_k A_k z_k (dual constraint of (D))."""
    return A.dense(0) - A.adjoint(z)
