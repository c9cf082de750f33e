"""Config 3 end to end: the max-cut SDP of a random sparse graph with n = m = 20000 (Hamiltonian ring
plus 2n random edges, average degree 6; the instance the mixed-vs-FP64 metric is quoted on)
solved on the device in the mixed form, its result certified on the CPU by the oracle's duality
sandwich (oracle/certificate.py): Y(z) positive definite (dense FP64 Cholesky), every clique
block of X̄ positive definite (Grone's theorem, Sec. 2.1: X̄ then has a positive definite
completion), A(X̄) = b to 1e-7, so b^T z <= opt <= A_0 . X̄, and the two ends agree to the
relative gap 1e-7: the reported optimum is within 1e-7 of the true one.  The dense FP64 oracle
PDIPM cannot run at this size (its iterations are O(n^3) with n = 20000), so the sandwich stands
in for it.  About two minutes of device time and a few minutes of host time."""
import numpy as np
import pytest
import torch

from instances import workload
from oracle.certificate import certify

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1310_6919_gb300 import build_library
    build_library()
    assert torch.cuda.is_available()


def test_config3_mixed_solve_certified():
    from tests.gpu_helpers import Case
    inst = workload("ring_maxcut_20000")
    c = Case(inst, precision=1)
    info = c.P.info
    assert info["max_nrow"] > 112  # the dense root carries the separator cliques
    r = c.P.solve()
    assert r["status"] == 0, r
    assert r["gap"] <= 1e-7 and r["pinf"] <= 1e-7
    X, z, _ = c.P.get_iterate()
    Xd = c.from_layout(X)
    zn = z.cpu().numpy()
    del X
    cert = certify(c.A, inst.b, c.perm, c.cliques, Xd, zn)
    assert cert["y_pd"], "Y(z) is not positive definite"
    assert cert["cliques_pd"], cert["min_clique_eig"]
    assert cert["pinf"] <= 1e-7
    lo, up = cert["lower"], cert["upper"]
    scale = max(1.0, (abs(lo) + abs(up)) / 2)
    assert lo <= up + 1e-9 * scale  # weak duality at the certified pair
    assert (up - lo) / scale <= 1e-7
    # the library's objectives are the ends of the certified bracket
    assert abs(r["pobj"] - up) <= 1e-9 * scale
    assert abs(r["dobj"] - lo) <= 1e-9 * scale
