"""Parity at the workload sizes, in the launch configuration bench.py times.

- 2D FitzHugh-Nagumo n = 4096 (two fields) in the FP64-split precision bench.py
  times by default (FP64 bar), its four-slice variant, split BF16 x6 and split
  TF32, and 3D Allen-Cahn n = 256 and n = 384: two steps against the full FP64
  oracle field.
- Maximum sizes (2D n = 16384, the largest K the FP64-split level sums hold
  exactly in int32; 3D n = 512): no oracle run at that size; the
  f = 0 closed form holds at any size: a sine mode prod sin(k pi x) is
  multiplied per step by prod E_1(tau lambda_k) (Section 3.1 with the
  eigenpairs of Section 3.3.2).
"""
import numpy as np
import pytest

from gpu_util import need_gpu, rel_err
from oracle import oracle as O
from paper_2601_06849_gb300 import etd, inputs

FHN = (1.0, 0.01, 0.5, 0.1)


BAR = {"fp64split": 1e-10, "fp64split32": 1e-6, "bf16x6": 1e-6, "tf32x3": 1e-6}


@pytest.mark.gpu
@pytest.mark.parametrize("precision", ["fp64split", "fp64split32", "bf16x6", "tf32x3"])
def test_fhn_2d_n4096_bench_configuration(precision):
    torch = need_gpu()
    n, steps, tau = 4096, 2, 1e-2
    u0 = inputs.fhn_uniform(n, 2, workload=1)
    stream = torch.cuda.Stream()
    plan = etd.Plan(2, n, 1e-3, 0.0, tau, pade=2, precision=precision, reaction="fhn", rx_params=FHN, n_comp=2,
                    kappa_comp=(1e-3, 5e-3), stream=stream)
    with torch.cuda.stream(stream):
        u = torch.tensor(u0, dtype=plan.dtype, device="cuda")
        plan.step(u, steps)
        plan.sync()
    got = u.double().cpu().numpy()
    plan.close()
    ref = O.run(O.Problem(d=2, n=n, kappa=(1e-3, 5e-3), q=0.0, tau=tau, reaction="fhn", rp=FHN), u0, steps)
    for c in range(2):
        assert rel_err(got[c], ref[c]) < BAR[precision]


@pytest.mark.gpu
@pytest.mark.parametrize("precision,n", [("bf16x6", 256), ("tf32x3", 256), ("bf16x6", 384)])
def test_allen_cahn_3d_workload_sizes(precision, n):
    torch = need_gpu()
    steps, tau = 2, 5e-3
    u0 = inputs.gaussian_bump(n, 3)
    plan = etd.Plan(3, n, 1e-3, 0.1, tau, pade=2, precision=precision, reaction="allen_cahn")
    u = torch.tensor(u0, dtype=torch.float32, device="cuda")
    plan.step(u, steps)
    plan.sync()
    got = u.double().cpu().numpy()
    plan.close()
    ref = O.run(O.Problem(d=3, n=n, kappa=(1e-3,), q=0.1, tau=tau, reaction="allen_cahn"), u0, steps)
    assert rel_err(got, ref) < 1e-6


def pade02_e1(x):
    return 2.0 / (x * x + 2 * x + 2)


@pytest.mark.gpu
@pytest.mark.parametrize("precision", ["tf32x3", "fp64split"])
@pytest.mark.parametrize("d,n,modes", [(2, 16384, (3, 11)), (3, 512, (2, 5, 1))])
def test_maximum_sizes_sine_mode(d, n, modes, precision):
    torch = need_gpu()
    kappa, q, tau, steps = 1e-3, 0.2, 1e-2, 3
    plan = etd.Plan(d, n, kappa, q, tau, pade=2, precision=precision, reaction="none")
    shape = inputs.sine_mode(n, d, modes)
    if precision != "fp64split":
        shape = shape.astype(np.float32)
    u = torch.tensor(shape[None], device="cuda", dtype=plan.dtype)
    plan.step(u, steps)
    plan.sync()
    h = 1.0 / (n + 1)
    amp = 1.0
    for k in modes:
        lam = 4 * kappa / h ** 2 * np.sin(k * np.pi * h / 2) ** 2 + q / d
        amp *= pade02_e1(tau * lam)
    got = u[0].double().cpu().numpy()
    plan.close()
    assert rel_err(got, amp ** steps * shape.astype(np.float64)) < (1e-10 if precision == "fp64split" else 1e-6)


@pytest.mark.gpu
def test_zero_steps_is_identity():
    torch = need_gpu()
    plan = etd.Plan(2, 70, 0.01, 0.0, 1e-3)  # the default precision (FP64-split: double fields)
    u = torch.rand((1, 70, 70), device="cuda", dtype=plan.dtype)
    before = u.clone()
    plan.step(u, 0)
    plan.sync()
    assert torch.equal(u, before)
    plan.close()
