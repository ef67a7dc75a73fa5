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
@pytest.mark.parametrize("precision,bar", [("fp64", 1e-9), ("fp64split", 1e-9), ("fp64split32", 1e-5), ("tf32x3", 1e-5),
                                           ("bf16x6", 1e-5)])
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


def fhn_window_grads(torch, n, steps, precision, u0, target, every=20):
    """Gradients of 0.5 ||u(T) - target||^2 over a 3D FitzHugh-Nagumo window (the
    bench's adjoint workload parameters) through autograd.solve."""
    from paper_2601_06849_gb300 import autograd as AG

    dt = torch.float64 if precision in etd.F64_PRECISIONS else torch.float32
    u0r = torch.tensor(u0, dtype=dt, device="cuda").requires_grad_(True)
    kr = torch.tensor([1e-3, 5e-3], dtype=torch.float64, requires_grad=True)
    rr = torch.tensor([1.0, 0.01, 0.5, 0.1], dtype=torch.float64, requires_grad=True)
    u = AG.solve(u0r, kr, rr, d=3, n=n, q=0.0, dt=1e-2, n_steps=steps, precision=precision, reaction="fhn",
                 checkpoint_every=every)
    loss = 0.5 * ((u - torch.tensor(target, dtype=dt, device="cuda")) ** 2).sum()
    loss.backward()
    return kr.grad.numpy(), rr.grad.numpy(), u0r.grad.double().cpu().numpy()


@pytest.mark.gpu
@pytest.mark.parametrize("precision,bar", [("fp64split", 1e-8), ("fp64split32", 1e-5), ("bf16x6", 3e-4),
                                           ("tf32x3", 3e-3)])
def test_adjoint_long_window_against_fp64(precision, bar):
    """200 steps (10 checkpoint segments) of 3D FitzHugh-Nagumo, n = 24: each
    gradient (dL/dkappa, dL/d eps, dL/du0) against the FP64 path, relative to its
    largest entry. The FP32-field paths carry FP32 fields through the window and
    the adjoint, so their bounds here are stated errors, not the 1e-5 bar; for
    scale, rounding u0 to FP32 alone moves dL/du0 of the FP64 path by 5e-6 to
    1.4e-5 on this problem, so no FP32-field path can reach 1e-5 on u0 over such
    a window. The FP64-split path (FP64 fields) is held to 1e-8, its four-slice
    variant (32-bit products, FP64 fields) to the adjoint bar of 1e-5."""
    torch = need_gpu()
    n, steps = 24, 200
    u0 = inputs.fhn_uniform(n, 3, workload=115)
    target = inputs.fhn_uniform(n, 3, workload=116, lo=-0.05, hi=0.05)
    ref = fhn_window_grads(torch, n, steps, "fp64", u0, target)
    got = fhn_window_grads(torch, n, steps, precision, u0, target)
    assert rel_err(got[0], ref[0]) < bar  # kappa_u, kappa_v
    assert abs(got[1][1] - ref[1][1]) < bar * abs(ref[1][1])  # eps
    assert rel_err(got[2], ref[2]) < bar  # u0


@pytest.mark.gpu
def test_adjoint_fp64split_matches_finite_differences():
    """The FP64-split path: adjoint gradients against central differences of its
    own forward run (3D FitzHugh-Nagumo, 40 steps, two checkpoint segments)."""
    torch = need_gpu()
    from paper_2601_06849_gb300 import autograd as AG

    n, steps, tau = 16, 40, 1e-2
    rp = torch.tensor([1.0, 0.01, 0.5, 0.1], dtype=torch.float64)
    kap = torch.tensor([1e-3, 5e-3], dtype=torch.float64)
    u0 = torch.tensor(inputs.fhn_uniform(n, 3, workload=112), dtype=torch.float64, device="cuda")
    target = torch.tensor(inputs.fhn_uniform(n, 3, workload=113), dtype=torch.float64, device="cuda")

    def loss(u0_, kap_, rp_):
        u = AG.solve(u0_, kap_, rp_, d=3, n=n, q=0.0, dt=tau, n_steps=steps, precision="fp64split", reaction="fhn",
                     checkpoint_every=20)
        return 0.5 * ((u - target) ** 2).sum()

    u0r = u0.clone().requires_grad_(True)
    kr = kap.clone().requires_grad_(True)
    rr = rp.clone().requires_grad_(True)
    loss(u0r, kr, rr).backward()
    h = 1e-5
    with torch.no_grad():
        for c in range(2):
            kp, km = kap.clone(), kap.clone()
            kp[c] *= 1 + h
            km[c] *= 1 - h
            fd = (loss(u0, kp, rp) - loss(u0, km, rp)).item() / (2 * h * kap[c].item())
            assert kr.grad[c].item() == pytest.approx(fd, rel=1e-5, abs=1e-12)
        v = torch.tensor(inputs.random_field(tuple(u0.shape), workload=114), dtype=torch.float64, device="cuda")
        fd = (loss(u0 + h * v, kap, rp) - loss(u0 - h * v, kap, rp)).item() / (2 * h)
        assert (u0r.grad * v).sum().item() == pytest.approx(fd, rel=1e-5)
