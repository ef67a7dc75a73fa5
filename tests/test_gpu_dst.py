"""The fast sine transform path (ETD_PREC_DST32): every transform pass as
FFT-based DST-I transforms in FP32 instead of the dense product with P.

Checked against the FP64 transform P X P (2D) / the three mode products (3D)
and against the FP64 oracle over full steps. Bounds: an FP32 radix-2 FFT of
length N = 2(n+1) rounds each of its log2 N butterfly stages to 2^-24, so a
transform's error relative to max|T(x)| stays within a few times
log2(N) 2^-24 (2e-6 covers N <= 8192 with margin); a step adds the per-pass
errors of its reactions' transforms scaled by tau, and the returned field
carries one such transform error.
"""
import numpy as np
import pytest

from gpu_util import need_gpu, rel_err, sine_basis
from oracle import oracle as O
from paper_2601_06849_gb300 import etd, inputs

FHN = (1.0, 0.01, 0.5, 0.1)


@pytest.mark.gpu
@pytest.mark.parametrize("d,n", [(2, 63), (2, 255), (2, 1023), (3, 31), (3, 63)])
def test_dst_transform_matches_fp64(d, n):
    torch = need_gpu()
    x = inputs.random_field((2,) + (n,) * d, workload=40 + n)
    P = sine_basis(n)
    if d == 2:
        ref = np.stack([P @ x[c] @ P.T for c in range(2)])
    else:
        ref = np.einsum("ip,jq,kr,cpqr->cijk", P, P, P, x, optimize=True)
    plan = etd.Plan(d, n, 1e-3, 0.0, 1e-2, precision="dst32", reaction="fhn", rx_params=FHN, n_comp=2,
                    kappa_comp=(1e-3, 5e-3))
    got = plan.transform(torch.tensor(x, dtype=torch.float32, device="cuda")).double().cpu().numpy()
    plan.close()
    assert rel_err(got, ref) < 2e-6, (d, n)


@pytest.mark.gpu
def test_dst_fhn_2d_matches_oracle():
    torch = need_gpu()
    n = 255
    u0 = inputs.fhn_uniform(n, 2, workload=41)
    ref = O.run(O.Problem(d=2, n=n, kappa=(1e-3, 5e-3), q=0.0, tau=1e-2, reaction="fhn", rp=FHN), u0, 20)
    plan = etd.Plan(2, n, 1e-3, 0.0, 1e-2, precision="dst32", reaction="fhn", rx_params=FHN, n_comp=2,
                    kappa_comp=(1e-3, 5e-3))
    u = torch.tensor(u0, dtype=torch.float32, device="cuda")
    plan.step(u, 20)
    plan.sync()
    got = u.double().cpu().numpy()
    plan.close()
    for c in range(2):
        assert rel_err(got[c], ref[c]) < 3e-6, c


@pytest.mark.gpu
def test_dst_allen_cahn_3d_matches_oracle():
    torch = need_gpu()
    n = 63
    u0 = inputs.gaussian_bump(n, d=3)
    ref = O.run(O.Problem(d=3, n=n, kappa=(1e-3,), q=0.1, tau=5e-3, reaction="allen_cahn"), u0, 10)
    plan = etd.Plan(3, n, 1e-3, 0.1, 5e-3, precision="dst32", reaction="allen_cahn")
    u = torch.tensor(u0, dtype=torch.float32, device="cuda")
    plan.step(u, 10)
    plan.sync()
    assert rel_err(u.double().cpu().numpy(), ref) < 3e-6
    plan.close()


@pytest.mark.gpu
def test_dst_needs_power_of_two_grid():
    need_gpu()
    with pytest.raises(etd.EtdError) as ei:
        etd.Plan(2, 100, 1e-3, 0.0, 1e-2, precision="dst32", reaction="allen_cahn")
    assert ei.value.status == etd.ETD_ERR_UNSUPPORTED
