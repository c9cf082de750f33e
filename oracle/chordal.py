"""Checks of an imported extended sparsity pattern E (Sec. 2.1).

The oracle never computes E itself: E depends on the ordering heuristic, so it is taken as data
(elimination order + clique list) and verified here:
  * the order is a perfect elimination ordering of E (E is chordal, no fill),
  * E covers the aggregate sparsity pattern,
  * cliques C_r list S_r (the clique's own columns) first, U_r = C_r minus S_r is contained in
    the clique holding its smallest element (running intersection property).
"""
import numpy as np


def cliques_from_supernodes(sn_ptr, sn_rowptr, sn_rows):
    """Clique r = rows of supernode r (new indices); S_r = columns sn_ptr[r]..sn_ptr[r+1]-1."""
    out = []
    for s in range(len(sn_ptr) - 1):
        rows = np.asarray(sn_rows[sn_rowptr[s]:sn_rowptr[s + 1]], dtype=np.int64)
        out.append((rows, int(sn_ptr[s + 1] - sn_ptr[s])))
    return out


def pattern_from_cliques(n, cliques):
    """E = union of C_r x C_r as a dense boolean matrix in the new (elimination) order."""
    E = np.zeros((n, n), dtype=bool)
    for rows, ns in cliques:
        E[np.ix_(rows, rows)] = True
    return E


def check_structure(n, cliques):
    """Raise AssertionError unless the cliques form a supernodal clique tree with S_r first."""
    covered = np.zeros(n, dtype=int)
    first_col = []
    for r, (rows, ns) in enumerate(cliques):
        assert len(rows) >= ns >= 1
        assert np.all(np.diff(rows) > 0), "clique rows not strictly increasing"
        S = rows[:ns]
        assert np.all(S == np.arange(S[0], S[0] + ns)), "S_r not a contiguous column range"
        covered[S] += 1
        first_col.append(int(S[0]))
    assert np.all(covered == 1), "columns not partitioned by the S_r"
    assert first_col == sorted(first_col), "cliques not in elimination order"
    col2clique = np.zeros(n, dtype=int)
    for r, (rows, ns) in enumerate(cliques):
        col2clique[rows[:ns]] = r
    for r, (rows, ns) in enumerate(cliques):
        U = rows[ns:]
        if len(U) == 0:
            continue
        parent = col2clique[U[0]]
        assert parent > r
        prow = set(cliques[parent][0].tolist())
        assert set(U.tolist()) <= prow, "running intersection property violated"


def is_perfect_elimination(E):
    """True if for every v the later neighbours of v are pairwise adjacent in E."""
    n = E.shape[0]
    for v in range(n):
        U = np.nonzero(E[v + 1:, v])[0] + v + 1
        if len(U) > 1 and not np.all(E[np.ix_(U, U)]):
            return False
    return True


def covers(E_new, perm, pattern_old):
    """E (new order) contains the aggregate pattern given in the original order."""
    inv = np.empty_like(perm)
    inv[perm] = np.arange(len(perm))
    I, J = np.nonzero(pattern_old)
    return bool(np.all(E_new[inv[I], inv[J]]))
