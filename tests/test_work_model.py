"""The algorithmic work figures behind the bench line's roofline (mcsdp_work_model, host-only
context) against counts made here from the problem data: the SCM Cholesky with its bordered
right-hand side (m^3/3 + m^2 flops, each lower-triangle entry of B read and written once), the
back substitution (m^2), and the tile contraction of eq. (newSCM2): one multiply-add per pair of
nonzeros (both triangles) of A_i and A_j, i >= j."""
import numpy as np
import pytest

from instances import block_arrow, lattice_maxcut, workload


@pytest.mark.parametrize("inst", [lattice_maxcut(10, 10), block_arrow(6, 12, 4, 60, seed=5),
                                  workload("block_arrow_2020")], ids=lambda i: i.name)
def test_work_model_against_direct_counts(inst):
    from paper_1310_6919_gb300 import Problem
    P = Problem.from_instance(inst, device=-1)
    w = P.work_model()
    m = inst.m
    assert w["flops"]["scm_chol"] == pytest.approx(m ** 3 / 3 + m ** 2, rel=1e-12)
    assert w["bytes"]["scm_chol"] == pytest.approx(16 * m * (m + 1) / 2, rel=1e-12)
    assert w["flops"]["sce_backsolve"] == pytest.approx(m ** 2, rel=1e-12)
    # nonzeros of each A_k counting both triangles
    cnt = np.zeros(m)
    for k, i, j in zip(inst.mat, inst.row, inst.col):
        if k > 0:
            cnt[k - 1] += 1 if i == j else 2
    pairs = (cnt.sum() ** 2 + (cnt ** 2).sum()) / 2      # sum over i >= j of cnt_i cnt_j
    assert w["flops"]["scm_tile"] == pytest.approx(2 * pairs, rel=1e-12)


@pytest.mark.parametrize("inst", [lattice_maxcut(10, 10), workload("block_arrow_2020")],
                         ids=lambda i: i.name)
def test_clique_factor_work(inst):
    # Algorithm 1 per clique: Cholesky of the reversed block plus a triangular inverse,
    # 2 |C_r|^3 / 3 flops; the clique factors are read and written once: 16 bytes per stored
    # lower entry of the supernodal layout (|S_r| (|S_r| + 1) / 2 + (|C_r| - |S_r|) |S_r|)
    from paper_1310_6919_gb300 import Problem
    P = Problem.from_instance(inst, device=-1)
    s = P.sym_export()
    w = P.work_model()
    r = np.diff(s["sn_rowptr"]).astype(float)
    k = np.diff(s["sn_col"]).astype(float)
    assert w["flops"]["alg1"] == pytest.approx(float(np.sum(2 * r ** 3 / 3)), rel=1e-12)
    ent = float(np.sum(k * (k + 1) / 2 + (r - k) * k))
    assert w["bytes"]["alg1"] == pytest.approx(16 * ent, rel=1e-12)
    assert w["bytes"]["ychol"] == pytest.approx(16 * ent, rel=1e-12)
