"""In-step field check (step a8): the plan reduces max |u| and the number of
non-finite values on the device every diag_every steps and reports a failed
check at the next etd_sync as ETD_ERR_DIVERGED. The stability theorem of
Section 4 bounds max |U^n|; a NaN or a field beyond the caller's bound is a
failed run. Nothing here faults the GPU: NaN and Inf are ordinary IEEE values
for every kernel of the step."""
import numpy as np
import pytest

from gpu_util import need_gpu, rel_err
from oracle import oracle as O
from paper_2601_06849_gb300 import etd, inputs

FHN = (1.0, 0.01, 0.5, 0.1)


def fhn_plan(n, **kw):
    return etd.Plan(2, n, 1e-3, 0.0, 1e-2, precision=kw.pop("precision", "bf16x6"), reaction="fhn", rx_params=FHN,
                    n_comp=2, kappa_comp=(1e-3, 5e-3), **kw)


@pytest.mark.gpu
@pytest.mark.parametrize("precision", ["bf16x6", "fp64", "fp64split", "fp64split32"])
def test_nan_field_reports_diverged_and_plan_recovers(precision):
    """A NaN in the field: the in-step check reports ETD_ERR_DIVERGED from etd_sync
    (the FP64-split slicer gives a row with NaN or Inf a code that makes its products
    NaN), the flag clears, and the plan then steps a finite field correctly."""
    torch = need_gpu()
    n = 96
    plan = fhn_plan(n, precision=precision, diag_every=1)
    u0 = inputs.fhn_uniform(n, 2, workload=20)
    bad = torch.tensor(u0, dtype=plan.dtype, device="cuda")
    bad[0, 40, 17] = float("nan")
    plan.step(bad, 3)
    with pytest.raises(etd.EtdError) as ei:
        plan.sync()
    assert ei.value.status == etd.ETD_ERR_DIVERGED
    assert "after step 1" in str(ei.value) and "non-finite" in str(ei.value)
    plan.sync()  # the flag was cleared
    # the plan keeps working on a finite field
    good = torch.tensor(u0, dtype=plan.dtype, device="cuda")
    plan.step(good, 4)
    plan.sync()
    ref = O.run(O.Problem(d=2, n=n, kappa=(1e-3, 5e-3), q=0.0, tau=1e-2, reaction="fhn", rp=FHN), u0, 4)
    assert rel_err(good.double().cpu().numpy(), ref) < (1e-10 if precision in ("fp64", "fp64split") else 1e-6)
    plan.close()


@pytest.mark.gpu
def test_bound_on_max_abs_and_no_effect_on_results():
    torch = need_gpu()
    n = 128
    u0 = inputs.allen_cahn_2d(n, workload=21)  # max |u0| about 0.5
    kw = dict(precision="bf16x6", reaction="allen_cahn")
    ref = torch.tensor(u0, dtype=torch.float32, device="cuda")
    p0 = etd.Plan(2, n, 0.01, 0.0, 1e-3, **kw)
    p0.step(ref, 10)
    p0.sync()
    # a bound the run respects: no error, and the checks change nothing
    p1 = etd.Plan(2, n, 0.01, 0.0, 1e-3, diag_every=2, diag_max_abs=2.0, **kw)
    u = torch.tensor(u0, dtype=torch.float32, device="cuda")
    p1.step(u, 10)
    p1.sync()
    assert torch.equal(u, ref)
    # a bound it does not respect
    p2 = etd.Plan(2, n, 0.01, 0.0, 1e-3, diag_every=5, diag_max_abs=0.1, **kw)
    v = torch.tensor(u0, dtype=torch.float32, device="cuda")
    p2.step(v, 10)
    with pytest.raises(etd.EtdError) as ei:
        p2.sync()
    assert ei.value.status == etd.ETD_ERR_DIVERGED and "after step 5" in str(ei.value)
    for p in (p0, p1, p2):
        p.close()


@pytest.mark.gpu
def test_host_entry_point_reports_diverged():
    torch = need_gpu()
    n = 64
    plan = fhn_plan(n, diag_every=2)
    host = torch.tensor(inputs.fhn_uniform(n, 2, workload=22), dtype=torch.float32).pin_memory()
    host[1, 5, 6] = float("inf")
    with pytest.raises(etd.EtdError) as ei:
        plan.step_host(host, 2)
    assert ei.value.status == etd.ETD_ERR_DIVERGED
    plan.close()


@pytest.mark.gpu
def test_ensemble_checks_every_group():
    torch = need_gpu()
    ns = [64, 96, 64]
    b = etd.Batch(2, ns, [1e-3] * 3, [0.0] * 3, [1e-2] * 3, precision="bf16x6", reaction="fhn", rx_params=FHN, n_comp=2,
                  kappa_v=5e-3, diag_every=1)
    fields = [torch.tensor(inputs.fhn_uniform(n, 2, workload=23 + i), dtype=torch.float32, device="cuda")
              for i, n in enumerate(ns)]
    b.step(fields, 3)
    b.sync()  # all finite
    fields[1][0, 3, 3] = float("nan")
    b.invalidate()
    b.step(fields, 3)
    with pytest.raises(etd.EtdError) as ei:
        b.sync()
    assert ei.value.status == etd.ETD_ERR_DIVERGED
    b.close()
