"""Small test-side symbolic analysis: elimination in a given order on a dense boolean pattern,
fundamental supernodes as cliques.  Used only to build patterns for oracle-only tests; the
library's own symbolic layer is tested separately against the oracle's structure checks."""
import numpy as np


def eliminate(P):
    """Filled pattern (dense bool, symmetric) of eliminating vertices 0..n-1 in order."""
    F = P.copy() | P.T
    n = F.shape[0]
    np.fill_diagonal(F, True)
    for v in range(n):
        U = np.nonzero(F[v + 1:, v])[0] + v + 1
        if len(U) > 1:
            F[np.ix_(U, U)] = True
    return F


def supernodes(F):
    """Fundamental supernodes of the filled pattern F: (rows, ns) cliques, S_r first."""
    n = F.shape[0]
    struct = [np.nonzero(F[v + 1:, v])[0] + v + 1 for v in range(n)]
    parent = [int(s[0]) if len(s) else -1 for s in struct]
    nchild = np.zeros(n, dtype=int)
    for v in range(n):
        if parent[v] >= 0:
            nchild[parent[v]] += 1
    cliques = []
    v = 0
    while v < n:
        start = v
        while (v + 1 < n and parent[v] == v + 1 and nchild[v + 1] == 1
               and len(struct[v]) == len(struct[v + 1]) + 1):
            v += 1
        rows = np.concatenate([np.arange(start, v + 1), struct[v]]).astype(np.int64)
        cliques.append((rows, v - start + 1))
        v += 1
    return cliques


def column_cliques(F):
    n = F.shape[0]
    return [(np.concatenate([[v], np.nonzero(F[v + 1:, v])[0] + v + 1]).astype(np.int64), 1)
            for v in range(n)]


def random_pattern(n, density, rng):
    P = rng.random((n, n)) < density
    P = P | P.T
    np.fill_diagonal(P, True)
    return P


def pd_on_pattern(F, rng, cliques):
    """Random X̄ with every clique block positive definite: a random dense PD matrix restricted
    to E (every principal submatrix of a PD matrix is PD)."""
    n = F.shape[0]
    G = rng.standard_normal((n, 3 * n))
    X = G @ G.T / (3 * n) + 0.5 * np.eye(n)
    return np.where(F, X, 0.0)
