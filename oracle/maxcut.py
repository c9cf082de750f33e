"""Closed forms and brute force for the max-cut SDP of Sec. 4 (A_0 = -L/4, A_k = e_k e_k^T,
b = 1), used to pin the oracle PDIPM.

For x in {-1, 1}^n, (-L/4) . x x^T = -cut(x); the SDP minimum is therefore <= -maxcut.
  * bipartite graph: optimum = -(sum of weights), attained by x x^T with x the bipartition;
    dual certificate z_i = -deg_w(i)/2 with Y = (D + W)/4 psd.
  * vertex-transitive graphs: optimum = -(n/4) lambda_max(L); odd cycle C_n (unit weights):
    -(n/2)(1 + cos(pi/n)); complete graph K_n: -n^2/4.
"""
import itertools

import numpy as np


def laplacian(n, edges, weights):
    L = np.zeros((n, n))
    for (u, v), w in zip(edges, weights):
        L[u, u] += w
        L[v, v] += w
        L[u, v] -= w
        L[v, u] -= w
    return L


def brute_force_maxcut(n, edges, weights):
    """Exact max-cut by enumerating the 2^(n-1) cuts (vertex 0 fixed on one side)."""
    best = 0.0
    E = np.array(edges)
    W = np.array(weights)
    for bits in itertools.product([0, 1], repeat=n - 1):
        side = np.array((0,) + bits)
        cut = float(np.sum(W[side[E[:, 0]] != side[E[:, 1]]]))
        best = max(best, cut)
    return best


def odd_cycle_optimum(n):
    return -(n / 2.0) * (1.0 + np.cos(np.pi / n))


def complete_graph_optimum(n):
    return -n * n / 4.0


def odd_cycle_certificates(n):
    """Primal X_ij = cos(2 pi k (i-j)/n), k = (n-1)/2, and dual z = -lambda_max(L)/4 * 1."""
    k = (n - 1) // 2
    idx = np.arange(n)
    X = np.cos(2 * np.pi * k * (idx[:, None] - idx[None, :]) / n)
    lam = 2.0 - 2.0 * np.cos(2 * np.pi * k / n)
    z = -lam / 4.0 * np.ones(n)
    return X, z


def complete_graph_certificates(n):
    X = (n / (n - 1.0)) * (np.eye(n) - np.ones((n, n)) / n)
    z = -n / 4.0 * np.ones(n)
    return X, z


def bipartite_certificates(n, edges, weights, side):
    x = np.where(np.asarray(side) == 0, 1.0, -1.0)
    X = np.outer(x, x)
    deg = np.zeros(n)
    for (u, v), w in zip(edges, weights):
        deg[u] += w
        deg[v] += w
    z = -deg / 2.0
    return X, z
