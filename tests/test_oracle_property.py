"""Property-based pins of the oracle's completion and Algorithm 1 (Sec. 2.1, 3.1) on random
chordal patterns and random data, with shrinking to a smallest failing case.  Needs
`hypothesis` (skipped where it is not installed)."""
import numpy as np
import pytest

hypothesis = pytest.importorskip("hypothesis")
from hypothesis import given, settings, strategies as st  # noqa: E402

from oracle.completion import (algorithm1, inverse_cholesky_definition,  # noqa: E402
                               max_det_completion)
from tests.chordal_helper import (eliminate, pd_on_pattern, random_pattern,  # noqa: E402
                                  supernodes)


@st.composite
def chordal_cases(draw):
    n = draw(st.integers(min_value=1, max_value=24))
    density = draw(st.floats(min_value=0.0, max_value=0.5))
    seed = draw(st.integers(min_value=0, max_value=2 ** 31 - 1))
    rng = np.random.default_rng(seed)
    F = eliminate(random_pattern(n, density, rng))
    cl = supernodes(F)
    return F, cl, pd_on_pattern(F, rng, cl)


@settings(max_examples=80, deadline=None)
@given(chordal_cases())
def test_completion_properties(case):
    F, cl, X = case
    Xh = max_det_completion(X, cl)
    assert np.allclose(Xh[F], X[F], rtol=0, atol=1e-12)
    assert np.linalg.eigvalsh(Xh)[0] > 0
    Xi = np.linalg.inv(Xh)
    assert np.max(np.abs(Xi[~F]), initial=0.0) <= 1e-9 * np.max(np.abs(Xi))


@settings(max_examples=80, deadline=None)
@given(chordal_cases())
def test_algorithm1_properties(case):
    F, cl, X = case
    Lh = algorithm1(X, cl)
    ref = inverse_cholesky_definition(max_det_completion(X, cl))
    assert np.allclose(Lh, ref, atol=1e-9 * np.max(np.abs(ref)))
    assert np.all(Lh[~np.tril(F)] == 0.0)
