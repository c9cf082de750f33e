"""Synthetic SDPs in the paper's standard form (Sec. 1):

    (P) min A_0 . X  s.t.  A_k . X = b_k (k = 1..m),  X psd
    (D) max b^T z    s.t.  sum_k A_k z_k + Y = A_0,    Y psd

Each instance stores the upper triangle (row <= col, 0-based) of A_0..A_m as one COO list
(mat = 0 for A_0, k for A_k).  Shapes follow the paper's workloads (Sec. 4): max-cut SDPs
(Goemans-Williamson relaxation, A_k = e_k e_k^T, b = 1) over lattice and random sparse graphs,
and chordal block-arrow SDPs.
"""
from dataclasses import dataclass, field
from typing import Optional

import numpy as np

from .rng import Xoshiro256ss

SEED_BASE = 20131101


@dataclass
class SDPInstance:
    name: str
    n: int
    m: int
    b: np.ndarray            # (m,) float64
    mat: np.ndarray          # (nnz,) int32, 0 = A_0
    row: np.ndarray          # (nnz,) int32, row <= col
    col: np.ndarray          # (nnz,) int32
    val: np.ndarray          # (nnz,) float64
    z0: Optional[np.ndarray] = None   # a point with A_0 - sum z0_k A_k positive definite
    meta: dict = field(default_factory=dict)

    @property
    def nnz(self):
        return int(self.val.shape[0])

    def matrix_entries(self, k):
        sel = self.mat == k
        return self.row[sel], self.col[sel], self.val[sel]


def _pack(name, n, m, b, entries, z0=None, meta=None):
    """entries: dict (mat, i, j) -> value with i <= j."""
    keys = sorted(entries.keys())
    mat = np.array([k[0] for k in keys], dtype=np.int32)
    row = np.array([k[1] for k in keys], dtype=np.int32)
    col = np.array([k[2] for k in keys], dtype=np.int32)
    val = np.array([entries[k] for k in keys], dtype=np.float64)
    return SDPInstance(name, n, m, np.asarray(b, dtype=np.float64), mat, row, col, val,
                       None if z0 is None else np.asarray(z0, dtype=np.float64), meta or {})


def graph_maxcut(n, edges, weights, name="maxcut", extra_meta=None):
    """Max-cut relaxation with A_0 = -L/4 (L the weighted Laplacian), A_k = e_k e_k^T, b = 1.

    z0_k = -(sum_j |[A_0]_kj|) - 1 makes Y0 = A_0 - diag(z0) strictly diagonally dominant.
    """
    ent = {}
    deg = np.zeros(n)
    for (u, v), w in zip(edges, weights):
        i, j = (u, v) if u < v else (v, u)
        assert i != j
        ent[(0, i, j)] = ent.get((0, i, j), 0.0) + w / 4.0
        deg[u] += w
        deg[v] += w
    for i in range(n):
        if deg[i] != 0.0:
            ent[(0, i, i)] = -deg[i] / 4.0
        ent[(i + 1, i, i)] = 1.0
    rowabs = np.zeros(n)
    for (k, i, j), v in ent.items():
        if k == 0:
            rowabs[i] += abs(v)
            if i != j:
                rowabs[j] += abs(v)
    meta = {"edges": list(edges), "weights": list(weights), "kind": "maxcut"}
    if extra_meta:
        meta.update(extra_meta)
    return _pack(name, n, n, np.ones(n), ent, z0=-(rowabs + 1.0), meta=meta)


def lattice_edges(p, q):
    """Lattice graph of Sec. 4 (vertices i + (j-1)p), converted to 0-based indices."""
    E = []
    for j in range(1, q + 1):
        for i in range(1, p):
            E.append((i + (j - 1) * p - 1, i + 1 + (j - 1) * p - 1))
    for j in range(1, q):
        for i in range(1, p + 1):
            E.append((i + (j - 1) * p - 1, i + j * p - 1))
    return E


def lattice_maxcut(p=10, q=10, seed=SEED_BASE + 1, wmin=1, wmax=10):
    """10x10 grid max-cut with integer weights uniform in [wmin, wmax]."""
    rng = Xoshiro256ss(seed)
    E = lattice_edges(p, q)
    W = [float(rng.randint(wmin, wmax)) for _ in E]
    return graph_maxcut(p * q, E, W, name=f"lattice_maxcut_{p}x{q}", extra_meta={"bipartite": True})


def cycle_maxcut(n):
    E = [(i, (i + 1) % n) for i in range(n)]
    return graph_maxcut(n, E, [1.0] * n, name=f"cycle_maxcut_{n}",
                        extra_meta={"bipartite": n % 2 == 0})


def complete_maxcut(n):
    E = [(i, j) for i in range(n) for j in range(i + 1, n)]
    return graph_maxcut(n, E, [1.0] * len(E), name=f"complete_maxcut_{n}",
                        extra_meta={"bipartite": n <= 2})


def random_ring_maxcut(n=20000, extra=None, seed=SEED_BASE + 3):
    """Hamiltonian ring over a seeded random permutation plus `extra` distinct non-ring edges
    (default 2n, average degree 6), weights uniform in [0, 1)."""
    rng = Xoshiro256ss(seed)
    extra = 2 * n if extra is None else extra
    perm = rng.permutation(n)
    es = set()
    E = []
    for t in range(n):
        u, v = perm[t], perm[(t + 1) % n]
        key = (min(u, v), max(u, v))
        es.add(key)
        E.append(key)
    while len(E) < n + extra:
        u, v = rng.below(n), rng.below(n)
        if u == v:
            continue
        key = (min(u, v), max(u, v))
        if key in es:
            continue
        es.add(key)
        E.append(key)
    W = [rng.uniform() for _ in E]
    return graph_maxcut(n, E, W, name=f"ring_maxcut_{n}")


def random_gnm_maxcut(n, M, seed):
    """G(n, M) random graph (M distinct edges), weights uniform in [0, 1)."""
    rng = Xoshiro256ss(seed)
    es = set()
    E = []
    while len(E) < M:
        u, v = rng.below(n), rng.below(n)
        if u == v:
            continue
        key = (min(u, v), max(u, v))
        if key in es:
            continue
        es.add(key)
        E.append(key)
    W = [rng.uniform() for _ in E]
    return graph_maxcut(n, E, W, name=f"gnm_maxcut_{n}_{M}")


def block_arrow(nblocks=40, bsize=50, border=20, m=2000, per_matrix=8, seed=SEED_BASE + 2,
                block_sizes=None):
    """Chordal block-arrow SDP: diagonal blocks plus a dense border.

    Constraint p lives in clique K_r = block r ∪ border with r = p mod nblocks and holds
    `per_matrix` distinct upper-triangle positions of K_r x K_r drawn without replacement with
    N(0,1) values.  b = A(I) so X0 = I is strictly primal feasible; A_0 = I + sum_p y0_p A_p with
    y0 ~ N(0,1) so z0 = y0 gives Y0 = I (strictly dual feasible).
    """
    rng = Xoshiro256ss(seed)
    if block_sizes is None:
        block_sizes = [bsize] * nblocks
    nblocks = len(block_sizes)
    starts = np.concatenate([[0], np.cumsum(block_sizes)]).astype(int)
    nb_total = int(starts[-1])
    n = nb_total + border
    border_idx = list(range(nb_total, n))
    ent = {}
    b = np.zeros(m)
    for p in range(m):
        r = p % nblocks
        K = list(range(starts[r], starts[r + 1])) + border_idx
        kk = len(K)
        npos = kk * (kk + 1) // 2
        chosen = set()
        picks = []
        while len(picks) < min(per_matrix, npos):
            t = rng.below(npos)
            if t in chosen:
                continue
            chosen.add(t)
            picks.append(t)
        for t in picks:
            # position t of the packed upper triangle of K x K (row-major over a <= c)
            a = 0
            while t >= kk - a:
                t -= kk - a
                a += 1
            c = a + t
            i, j = K[a], K[c]
            v = rng.normal()
            ent[(p + 1, i, j)] = v
            if i == j:
                b[p] += v
    y0 = np.array([rng.normal() for _ in range(m)])
    A0 = {(i, i): 1.0 for i in range(n)}
    for (k, i, j), v in ent.items():
        A0[(i, j)] = A0.get((i, j), 0.0) + y0[k - 1] * v
    for (i, j), v in A0.items():
        ent[(0, i, j)] = v
    return _pack(f"block_arrow_{nblocks}x{block_sizes[0]}+{border}_m{m}", n, m, b, ent, z0=y0,
                 meta={"kind": "block_arrow", "y0": y0, "X0_identity_feasible": True,
                       "block_sizes": list(block_sizes), "border": border})


def small_random_sdp(n, m, seed, density=0.3):
    """Dense-ish small random SDP with X0 = I primal feasible and Y0 = I dual feasible."""
    rng = Xoshiro256ss(seed)
    ent = {}
    b = np.zeros(m)
    for p in range(m):
        for i in range(n):
            for j in range(i, n):
                if rng.uniform() < density or (i == j and i == p % n):
                    v = rng.normal()
                    ent[(p + 1, i, j)] = v
                    if i == j:
                        b[p] += v
    y0 = np.array([rng.normal() for _ in range(m)])
    A0 = {(i, i): 1.0 for i in range(n)}
    for (k, i, j), v in ent.items():
        A0[(i, j)] = A0.get((i, j), 0.0) + y0[k - 1] * v
    for (i, j), v in A0.items():
        ent[(0, i, j)] = v
    return _pack(f"small_random_{n}_{m}", n, m, b, ent, z0=y0, meta={"kind": "random"})


def diagonal_lp_sdp(n, m, seed):
    """All A_k diagonal (an LP in SDP form): the SCM is the LP normal matrix."""
    rng = Xoshiro256ss(seed)
    ent = {}
    b = np.zeros(m)
    for p in range(m):
        for i in range(n):
            if rng.uniform() < 0.5 or i == p % n:
                v = rng.normal()
                ent[(p + 1, i, i)] = v
                b[p] += v
    y0 = np.array([rng.normal() for _ in range(m)])
    A0 = {(i, i): 1.0 for i in range(n)}
    for (k, i, j), v in ent.items():
        A0[(i, j)] = A0.get((i, j), 0.0) + y0[k - 1] * v
    for (i, j), v in A0.items():
        ent[(0, i, j)] = v
    return _pack(f"diag_lp_{n}_{m}", n, m, b, ent, z0=y0, meta={"kind": "lp"})


def batch_mix(n_maxcut, n_arrow, seed=SEED_BASE + 4):
    """Many small SDPs (the batched configuration): max-cut on G(n, floor(5n/2)) with
    n ~ U{50..400}, weights U[0,1); block-arrow with n ~ U{100..600}, border 20, ceil((n-20)/50)
    blocks of sizes split evenly, m = n.  Problem p draws from seed + p."""
    rng = Xoshiro256ss(seed)
    out = []
    for p in range(n_maxcut):
        n = 50 + rng.below(351)
        out.append(random_gnm_maxcut(n, (5 * n) // 2, seed + 1000 + p))
    for p in range(n_arrow):
        n = 100 + rng.below(501)
        nb = -(-(n - 20) // 50)
        base, extra = divmod(n - 20, nb)
        sizes = [base + (1 if q < extra else 0) for q in range(nb)]
        out.append(block_arrow(nb, sizes[0], 20, n, seed=seed + 5000 + p, block_sizes=sizes))
    return out


def direct_sum(parts, name=None):
    """Block-diagonal SDP from independent ones: part p's matrices on rows/columns offset by
    n_0 + .. + n_{p-1}, its constraints numbered after the earlier parts' (A_0 is the sum of the
    parts' A_0), b and z0 concatenated.  Its aggregate pattern, X̂, Y^{-1} and Schur complement
    matrix are block-diagonal over the parts, and its optimal value is the sum of theirs."""
    mats, rows, cols, vals, bs, z0s = [], [], [], [], [], []
    no = mo = 0
    for inst in parts:
        mats.append(np.where(inst.mat > 0, inst.mat + mo, 0).astype(np.int32))
        rows.append(inst.row + no)
        cols.append(inst.col + no)
        vals.append(inst.val)
        bs.append(inst.b)
        z0s.append(inst.z0)
        no += inst.n
        mo += inst.m
    mat, row, col = np.concatenate(mats), np.concatenate(rows), np.concatenate(cols)
    order = np.lexsort((col, row, mat))
    z0 = None if any(z is None for z in z0s) else np.concatenate(z0s)
    meta = {"kind": "direct_sum", "parts": [(p.name, p.n, p.m) for p in parts]}
    return SDPInstance(name or f"direct_sum_{len(parts)}", no, mo, np.concatenate(bs),
                       mat[order].astype(np.int32), row[order].astype(np.int32),
                       col[order].astype(np.int32), np.concatenate(vals)[order], z0, meta)


def maxcut_direct_sum(k, seed=SEED_BASE + 7):
    """Direct sum of k max-cut relaxations on G(n, floor(5n/2)) with n ~ U{50..400}, weights
    U[0,1) (the max-cut half of the batched configuration's mix, as one SDP): a problem whose
    Schur complement matrix is block-diagonal with k blocks.  Part p draws from seed + 1000 + p."""
    rng = Xoshiro256ss(seed)
    parts = []
    for p in range(k):
        n = 50 + rng.below(351)
        parts.append(random_gnm_maxcut(n, (5 * n) // 2, seed + 1000 + p))
    return direct_sum(parts, name=f"maxcut_sum_{k}")


def workload(name, seed=None):
    """Named workloads: 'grid_maxcut_100' (10x10 lattice), 'block_arrow_2020' (40 x 50 + 20,
    m = 2000), 'block_arrow_1020' (20 x 50 + 20, m = 1000), 'ring_maxcut_20000', and
    'ring_maxcut_8000' (the same family at n = 8000: a case small enough for profiler captures),
    and 'maxcut_sum_64' (64 random max-cut SDPs as one block-diagonal SDP)."""
    if name == "grid_maxcut_100":
        return lattice_maxcut(10, 10, seed=SEED_BASE + 1 if seed is None else seed)
    if name == "block_arrow_2020":
        return block_arrow(40, 50, 20, 2000, seed=SEED_BASE + 2 if seed is None else seed)
    if name == "block_arrow_1020":
        return block_arrow(20, 50, 20, 1000, seed=SEED_BASE + 5 if seed is None else seed)
    if name == "ring_maxcut_20000":
        return random_ring_maxcut(20000, seed=SEED_BASE + 3 if seed is None else seed)
    if name == "ring_maxcut_8000":
        return random_ring_maxcut(8000, seed=SEED_BASE + 6 if seed is None else seed)
    if name == "maxcut_sum_64":
        return maxcut_direct_sum(64, seed=SEED_BASE + 7 if seed is None else seed)
    raise KeyError(name)
