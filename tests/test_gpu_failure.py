"""Failure detection without a GPU fault: a bounded device wait that has nothing
to wait for runs out, the kernel records ERR_TIMEOUT in the plan's error word
and returns; etd_sync reports ETD_ERR_TIMEOUT, and the plan keeps working."""
import pytest

from gpu_util import need_gpu, rel_err
from oracle import oracle as O
from paper_2601_06849_gb300 import etd, inputs


@pytest.mark.gpu
def test_bounded_wait_reports_timeout_and_plan_recovers():
    torch = need_gpu()
    n = 64
    plan = etd.Plan(2, n, 0.01, 0.0, 1e-3, precision="tf32x3", reaction="allen_cahn")
    etd.etd_selftest_wait_timeout(plan.handle, 20.0)
    with pytest.raises(etd.EtdError) as ei:
        plan.sync()
    assert ei.value.status == etd.ETD_ERR_TIMEOUT
    plan.sync()  # the flag was cleared
    u0 = inputs.allen_cahn_2d(n, workload=0)
    u = torch.tensor(u0, dtype=torch.float32, device="cuda")
    plan.step(u, 10)
    plan.sync()
    ref = O.run(O.Problem(d=2, n=n, kappa=(0.01,), q=0.0, tau=1e-3, reaction="allen_cahn"), u0, 10)
    assert rel_err(u.double().cpu().numpy(), ref) < 1e-6
    plan.close()


def test_selftest_rejects_bad_limits():
    import __graft_entry__

    __graft_entry__.build()
    with pytest.raises(etd.EtdError):
        etd.etd_selftest_wait_timeout(0, 10.0)
