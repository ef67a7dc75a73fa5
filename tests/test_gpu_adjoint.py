"""GPU adjoint (etd_step_adjoint) against the FP64 adjoint oracle and against
central finite differences of the GPU forward run."""
import numpy as np
import pytest

from gpu_util import need_gpu, rel_err
from oracle import adjoint as A
from oracle import oracle as O
from paper_2601_06849_gb300 import etd, inputs

FHN = (1.0, 0.3, 0.5, 0.1)


def setup(d, n, kind, precision, pade=2):
    kap = (0.02, 0.05) if kind == "fhn" else (0.03,)
    rp = FHN if kind == "fhn" else ((0.7,) if kind == "linear" else ())
    P = O.Problem(d=d, n=n, kappa=kap, q=0.2, tau=0.03, pade=pade, reaction=kind, rp=rp)
    plan = etd.Plan(d, n, kap[0], 0.2, 0.03, pade=pade, precision=precision, reaction=kind, rx_params=rp,
                    n_comp=len(kap), kappa_comp=kap)
    return P, plan


@pytest.mark.gpu
@pytest.mark.parametrize("precision,bar", [("fp64", 1e-9), ("fp64split", 1e-9), ("tf32x3", 1e-5), ("bf16x6", 1e-5)])
@pytest.mark.parametrize("d,n,kind,pade", [(2, 20, "fhn", 2), (3, 10, "allen_cahn", 2), (2, 33, "linear", 4),
                                           (3, 12, "fhn", 4)])
def test_adjoint_matches_fp64_oracle(precision, bar, d, n, kind, pade):
    torch = need_gpu()
    P, plan = setup(d, n, kind, precision, pade)
    N = 6
    u0 = inputs.random_field((P.ncomp,) + (n,) * d, workload=110, scale=0.4)
    lamN = inputs.random_field(u0.shape, workload=111)
    ref_u, ref_k, ref_r = A.adjoint_run(P, u0, N, lamN)
    u = torch.tensor(u0, dtype=plan.dtype, device="cuda")
    lam = torch.tensor(lamN, dtype=plan.dtype, device="cuda")
    gk, gr = plan.adjoint(u, lam, N)
    assert rel_err(lam.double().cpu().numpy(), ref_u) < bar
    for c in range(P.ncomp):
        assert gk[c] == pytest.approx(ref_k[c], rel=bar, abs=bar * np.abs(ref_k).max())
    for i in range(len(ref_r)):
        assert gr[i] == pytest.approx(ref_r[i], rel=bar, abs=bar * np.abs(ref_r).max())
    plan.close()


@pytest.mark.gpu
def test_adjoint_matches_gpu_finite_differences_3d_fhn():
    """Loss 0.5 ||u(T) - target||^2 of a 3D FitzHugh-Nagumo run: adjoint
    gradients w.r.t. kappa_u, eps and u0 agree with central differences of the
    GPU's own forward run (FP64 path, 2 checkpoint segments)."""
    torch = need_gpu()
    from paper_2601_06849_gb300 import autograd as AG

    n, steps, tau = 16, 40, 1e-2
    rp = torch.tensor([1.0, 0.01, 0.5, 0.1], dtype=torch.float64)
    kap = torch.tensor([1e-3, 5e-3], dtype=torch.float64)
    u0 = torch.tensor(inputs.fhn_uniform(n, 3, workload=112), dtype=torch.float64, device="cuda")
    target = torch.tensor(inputs.fhn_uniform(n, 3, workload=113), dtype=torch.float64, device="cuda")

    def loss(u0_, kap_, rp_):
        u = AG.solve(u0_, kap_, rp_, d=3, n=n, q=0.0, dt=tau, n_steps=steps, precision="fp64", reaction="fhn",
                     checkpoint_every=20)
        return 0.5 * ((u - target) ** 2).sum()

    u0r = u0.clone().requires_grad_(True)
    kr = kap.clone().requires_grad_(True)
    rr = rp.clone().requires_grad_(True)
    L = loss(u0r, kr, rr)
    L.backward()
    h = 1e-5
    with torch.no_grad():
        for c in range(2):
            kp, km = kap.clone(), kap.clone()
            kp[c] *= 1 + h
            km[c] *= 1 - h
            fd = (loss(u0, kp, rp) - loss(u0, km, rp)).item() / (2 * h * kap[c].item())
            assert kr.grad[c].item() == pytest.approx(fd, rel=1e-5, abs=1e-12)
        rpp, rpm = rp.clone(), rp.clone()
        rpp[1] += h
        rpm[1] -= h
        fd = (loss(u0, kap, rpp) - loss(u0, kap, rpm)).item() / (2 * h)
        assert rr.grad[1].item() == pytest.approx(fd, rel=1e-5, abs=1e-12)
        v = torch.tensor(inputs.random_field(tuple(u0.shape), workload=114), dtype=torch.float64, device="cuda")
        fd = (loss(u0 + h * v, kap, rp) - loss(u0 - h * v, kap, rp)).item() / (2 * h)
        assert (u0r.grad * v).sum().item() == pytest.approx(fd, rel=1e-5)
