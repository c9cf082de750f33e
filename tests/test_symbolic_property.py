"""Property-based tests of the host symbolic analysis (Sec. 2.1: ordering, chordal extension,
cliques with the running intersection property) on random sparsity patterns, with shrinking to a
smallest failing pattern.  Needs `hypothesis` (skipped where it is not installed)."""
import numpy as np
import pytest

hypothesis = pytest.importorskip("hypothesis")
from hypothesis import given, settings, strategies as st  # noqa: E402

from instances import graph_maxcut  # noqa: E402
from oracle.chordal import (check_structure, cliques_from_supernodes, covers,  # noqa: E402
                            is_perfect_elimination, pattern_from_cliques)
from oracle.sdp import SparseSym  # noqa: E402
from tests.test_symbolic_host import _min_degree_fill  # noqa: E402


@st.composite
def graphs(draw):
    n = draw(st.integers(min_value=1, max_value=40))
    pairs = [(i, j) for i in range(n) for j in range(i + 1, n)]
    chosen = draw(st.lists(st.sampled_from(pairs), unique=True, max_size=min(len(pairs), 3 * n))
                  if pairs else st.just([]))
    return n, sorted(chosen)


def _export(inst, relax):
    from paper_1310_6919_gb300 import Problem
    P = Problem.from_instance(inst, device=-1, relax=relax)
    s = P.sym_export()
    cl = cliques_from_supernodes(s["sn_col"], s["sn_rowptr"], s["sn_rows"])
    iperm = np.empty(inst.n, dtype=np.int64)
    iperm[s["perm"]] = np.arange(inst.n)
    return P, s, cl, iperm


@settings(max_examples=60, deadline=None)
@given(graphs(), st.sampled_from([0, 1]))
def test_structure_on_random_patterns(g, relax):
    n, edges = g
    inst = graph_maxcut(n, edges, [1.0] * len(edges), name="random")
    P, s, cl, iperm = _export(inst, relax)
    check_structure(n, cl)
    E_new = pattern_from_cliques(n, cl)
    assert is_perfect_elimination(E_new)
    A = SparseSym.from_instance(inst)
    agg = A.aggregate_pattern()
    assert covers(E_new, s["perm"], agg)
    E = E_new[np.ix_(iperm, iperm)]
    fill = _min_degree_fill(agg)
    if relax == 0:
        # fundamental supernodes: E is exactly the minimum-degree filled graph
        assert np.array_equal(E, fill)
    else:
        # amalgamation only adds explicit zeros to the filled graph
        assert np.all(E[fill])
    assert P.info["nnz_lower_E"] == int(np.tril(E_new).sum())
