"""The seeded input generators produce the workloads they are documented to produce.

These checks pin the input recipe, not the method: the sizes and patterns of the max-cut lattice
of Sec. 4, the block-arrow SDPs with their strictly feasible start (X0 = I, Y0 = I), the ring
max-cut graph, the batched mix and the 64-part direct sum.  Dense matrices are built here with plain numpy from the
instance arrays (paper notation: Y(z) = A_0 - sum_k z_k A_k, A_k . X = b_k).
"""
import numpy as np
import pytest

from instances import batch_mix, random_ring_maxcut, workload


def dense(inst, k):
    """A_k of an instance as a dense symmetric matrix."""
    r, c, v = inst.matrix_entries(k)
    M = np.zeros((inst.n, inst.n))
    M[r, c] = v
    M[c, r] = v
    return M


def dual_slack_dense(inst, z):
    Y = dense(inst, 0)
    for k in range(1, inst.m + 1):
        r, c, v = inst.matrix_entries(k)
        Y[r, c] -= z[k - 1] * v
        Y[c, r] = Y[r, c]
    return Y


def test_grid_maxcut_recipe():
    inst = workload("grid_maxcut_100")
    assert (inst.n, inst.m) == (100, 100)
    edges, w = inst.meta["edges"], np.array(inst.meta["weights"])
    assert len(edges) == 180 == len(set(map(tuple, edges)))
    assert np.all(w == np.round(w)) and w.min() >= 1 and w.max() <= 10
    # the lattice of Sec. 4: horizontal neighbours i, i+1 within a row of 10, vertical i, i+10
    for u, v in edges:
        a, b = min(u, v), max(u, v)
        assert (b - a == 1 and a % 10 != 9) or b - a == 10
    # A_0 = -L/4: rows sum to zero, off-diagonal entries w/4
    A0 = dense(inst, 0)
    assert np.allclose(A0.sum(axis=1), 0.0, atol=1e-12)
    L = np.zeros((100, 100))
    for (u, v), wt in zip(edges, w):
        L[u, v] -= wt
        L[v, u] -= wt
        L[u, u] += wt
        L[v, v] += wt
    assert np.array_equal(A0, -L / 4)
    for k in range(1, 101):
        r, c, v = inst.matrix_entries(k)
        assert r.tolist() == [k - 1] and c.tolist() == [k - 1] and v.tolist() == [1.0]
    assert np.all(inst.b == 1.0)
    # aggregate pattern: the diagonal plus both triangles of the 180 edges = 460 entries
    pat = np.zeros((100, 100), bool)
    for k in range(101):
        r, c, _ = inst.matrix_entries(k)
        pat[r, c] = pat[c, r] = True
    assert int(pat.sum()) == 100 + 2 * 180
    # the default start Y(z0) is strictly diagonally dominant, hence positive definite
    Y = dual_slack_dense(inst, inst.z0)
    off = np.abs(Y).sum(axis=1) - np.abs(np.diag(Y))
    assert np.all(np.diag(Y) > off)


@pytest.mark.parametrize("name,nblocks,m", [("block_arrow_2020", 40, 2000),
                                            ("block_arrow_1020", 20, 1000)])
def test_block_arrow_recipe(name, nblocks, m):
    inst = workload(name)
    n = nblocks * 50 + 20
    assert (inst.n, inst.m) == (n, m)
    border = set(range(nblocks * 50, n))
    for p in range(m):
        r, c, v = inst.matrix_entries(p + 1)
        assert len(v) == 8, "8 distinct upper-triangle positions per constraint"
        assert np.all(r <= c)
        blk = p % nblocks
        allowed = set(range(blk * 50, blk * 50 + 50)) | border
        assert set(r.tolist()) | set(c.tolist()) <= allowed
        # b = A(I) = trace(A_p): X0 = I is primal feasible
        assert inst.b[p] == pytest.approx(float(np.sum(v[r == c])), abs=1e-14)
    # A_0 = I + sum y0_p A_p, so Y(y0) = I: Z0 = I is dual feasible
    Y = dual_slack_dense(inst, inst.z0)
    assert np.max(np.abs(Y - np.eye(n))) < 1e-12
    # the aggregate pattern is the block-arrow shape: no entry couples two diagonal blocks
    pat = np.zeros((n, n), bool)
    for k in range(m + 1):
        r, c, _ = inst.matrix_entries(k)
        pat[r, c] = pat[c, r] = True
    blk_of = np.minimum(np.arange(n) // 50, nblocks)   # border vertices -> nblocks
    I, J = np.nonzero(pat)
    bi, bj = blk_of[I], blk_of[J]
    assert np.all((bi == bj) | (bi == nblocks) | (bj == nblocks))


def test_ring_maxcut_recipe():
    n = 500
    inst = random_ring_maxcut(n, seed=7)
    edges = [tuple(e) for e in inst.meta["edges"]]
    w = np.array(inst.meta["weights"])
    assert (inst.n, inst.m) == (n, n)
    assert len(edges) == 3 * n == len(set(edges)), "ring plus 2n distinct edges: average degree 6"
    assert np.all((w >= 0) & (w < 1))
    # the first n edges form one Hamiltonian cycle
    nbr = {v: [] for v in range(n)}
    for u, v in edges[:n]:
        nbr[u].append(v)
        nbr[v].append(u)
    assert all(len(x) == 2 for x in nbr.values())
    prev, cur, seen = None, 0, {0}
    for _ in range(n - 1):
        nxt = nbr[cur][0] if nbr[cur][0] != prev else nbr[cur][1]
        prev, cur = cur, nxt
        seen.add(cur)
    assert len(seen) == n and 0 in nbr[cur]


def test_batch_mix_recipe():
    probs = batch_mix(12, 6)
    assert len(probs) == 18
    for inst in probs[:12]:
        assert 50 <= inst.n <= 400 and inst.m == inst.n
        assert len(inst.meta["edges"]) == (5 * inst.n) // 2
    for inst in probs[12:]:
        sizes, border = inst.meta["block_sizes"], inst.meta["border"]
        assert 100 <= inst.n <= 600 and inst.m == inst.n and border == 20
        assert sum(sizes) + border == inst.n
        assert len(sizes) == -(-(inst.n - 20) // 50) and max(sizes) - min(sizes) <= 1
        Y = dual_slack_dense(inst, inst.z0)
        assert np.max(np.abs(Y - np.eye(inst.n))) < 1e-12


def test_direct_sum_recipe():
    """maxcut_sum_64: 64 max-cut SDPs of the batch mix's max-cut kind, part p on rows offset by
    the earlier parts' sizes, its constraints after theirs; no entry crosses two parts, b = 1 and
    z0 is the parts' z0 (Y0 strictly diagonally dominant)."""
    from instances.problems import Xoshiro256ss, SEED_BASE, random_gnm_maxcut
    inst = workload("maxcut_sum_64")
    parts = inst.meta["parts"]
    assert len(parts) == 64 and inst.n == inst.m == sum(p[1] for p in parts)
    rng = Xoshiro256ss(SEED_BASE + 7)
    sizes = [50 + rng.below(351) for _ in range(64)]
    assert [p[1] for p in parts] == sizes and all(50 <= s <= 400 for s in sizes)
    offs = np.cumsum([0] + sizes)
    part_of = np.searchsorted(offs, np.arange(inst.n), side="right") - 1
    assert np.array_equal(part_of[inst.row], part_of[inst.col])  # block-diagonal data
    k = inst.mat > 0
    assert np.array_equal(inst.row[k], inst.mat[k] - 1) and np.array_equal(inst.col[k], inst.row[k])
    assert np.all(inst.b == 1.0)
    # part 5 as generated on its own, shifted into place
    p = 5
    one = random_gnm_maxcut(sizes[p], (5 * sizes[p]) // 2, SEED_BASE + 7 + 1000 + p)
    sel = (inst.mat == 0) & (part_of[inst.row] == p)
    got = sorted(zip(inst.row[sel] - offs[p], inst.col[sel] - offs[p], inst.val[sel]))
    want = sorted(zip(*one.matrix_entries(0)))
    assert got == want
    assert np.array_equal(inst.z0[offs[p]:offs[p + 1]], one.z0)
    # Y0 = A_0 - diag(z0) strictly diagonally dominant with positive diagonal
    diag = np.zeros(inst.n)
    off = np.zeros(inst.n)
    a0 = inst.mat == 0
    for r, c, v in zip(inst.row[a0], inst.col[a0], inst.val[a0]):
        if r == c:
            diag[r] += v
        else:
            off[r] += abs(v)
            off[c] += abs(v)
    assert np.all(diag - inst.z0 > off)
