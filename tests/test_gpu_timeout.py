"""Failure detection without a GPU fault: the SCM factorisation's task dependencies are bounded
device waits (options.timeout_cycles, SM clock cycles).  With a budget of one cycle the first
wait that is not already satisfied gives up: the kernel raises its abort word, every CTA leaves,
the host reads the timeout status and the call returns MCSDP_ERR_TIMEOUT.  Nothing hangs and the
device stays usable: a context with the default budget then solves the same problem."""
import pytest
import torch

from instances import block_arrow

pytestmark = pytest.mark.gpu

MCSDP_ERR_TIMEOUT = 8


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1310_6919_gb300 import build_library
    build_library()
    assert torch.cuda.is_available()


def _problem(inst, **opts):
    from paper_1310_6919_gb300 import Problem
    P = Problem.from_instance(inst, device=0, **opts)
    P.set_iterate(None, inst.z0)
    return P


def test_factorisation_wait_budget_times_out_and_device_recovers():
    from paper_1310_6919_gb300 import MCSDPError
    # m = 60: two column tiles, so the panel-solve tasks of the second tile wait on the first
    # diagonal factor (about 18 us) and cannot be ready at their first poll
    inst = block_arrow(6, 12, 4, 60, per_matrix=8, seed=5)
    P = _problem(inst, timeout_cycles=1)
    with pytest.raises(MCSDPError) as ei:
        P.solve()
    assert ei.value.status == MCSDP_ERR_TIMEOUT
    # the same context times out again (the abort word is reset by every launch, not sticky)
    with pytest.raises(MCSDPError) as ei:
        P.solve()
    assert ei.value.status == MCSDP_ERR_TIMEOUT
    torch.cuda.synchronize()
    Q = _problem(inst)
    r = Q.solve()
    assert r["status"] == 0 and r["gap"] <= 1e-7
