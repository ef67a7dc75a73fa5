"""Full ETD2RK-DS steps through the C ABI against the FP64 CPU oracle.

Error metric (relative, whole field): max |U_gpu - U_oracle| / max |U_oracle|,
per component. Every precision carries the spectral state with more than FP32
precision (FP64, or double-float pairs in the FP32 paths), so the error of the
returned field is set by the transforms:
  fp64    1e-10                 the FP64 bar
  tf32x3  1e-6                  the split-precision bar (output transform: 3-piece split)
  tf32x6  1e-6                  same, three-piece split in every pass
  fp32    4 sqrt(n) 2^-24       FP32 round-to-nearest sums of n terms in each output pass
  tf32    3e-3                  one TF32 product: 11-bit operands (2^-11 = 4.9e-4 per pass)
  bf16x6  1e-6                  three BF16 pieces (24 bits) in every pass
  fp64split 1e-10               FP64 fields; products of six balanced 8-bit slices, exact accumulation
  fp64split40 3e-8              the same with five slices: operands rounded 2^8 more coarsely
                                (40 instead of 48 bits below the row's scale), so fp64split's
                                bar scaled by 2^8
  fp64split32 1e-6              four slices (32 bits): fp64split's bar scaled by 2^16 would be
                                6.6e-6; the mode is meant for the split-precision bar, 1e-6
  bf16x3  3e-6                  two BF16 pieces (16 bits, 2^-17 = 7.6e-6 per operand) in the
                                per-step passes, reaching the state through tau f: over the
                                N tau <= 0.2 of these runs <= 0.2 * 7.6e-6 on top of the 1e-6 bar
Sizes span several 128-row tiles, ragged tails and padded rows (n % 4 != 0).
"""
import numpy as np
import pytest

from gpu_util import need_gpu, rel_err
from oracle import oracle as O
from oracle import spectral as S
from paper_2601_06849_gb300 import etd, inputs

TOL = {"fp64": 1e-10, "fp64split": 1e-10, "fp64split40": 3e-8, "fp64split32": 1e-6, "tf32x3": 1e-6, "tf32x6": 1e-6, "tf32": 3e-3, "bf16x6": 1e-6,
       "bf16x3": 3e-6}


def tol(precision, n):
    if precision == "fp32":
        return 4 * np.sqrt(n) * 2.0 ** -24
    return TOL[precision]
FHN = (1.0, 0.01, 0.5, 0.1)  # c3, eps, a, b of the 2D FitzHugh-Nagumo workload


def run_gpu(torch, d, n, kappa, q, tau, u0, steps, precision, reaction, rp=(), pade=2, kappa_comp=None):
    ncomp = u0.shape[0]
    plan = etd.Plan(d, n, kappa, q, tau, pade=pade, precision=precision, reaction=reaction, rx_params=rp,
                    n_comp=ncomp, kappa_comp=kappa_comp)
    u = torch.tensor(u0, dtype=plan.dtype, device="cuda")
    plan.step(u, steps)
    plan.sync()
    out = u.double().cpu().numpy()
    plan.close()
    return out


def oracle_ref(d, n, kappa, q, tau, u0, steps, reaction, rp=(), pade=2):
    return O.run(O.Problem(d=d, n=n, kappa=tuple(kappa), q=q, tau=tau, pade=pade, reaction=reaction, rp=rp),
                 u0, steps)


@pytest.mark.gpu
@pytest.mark.parametrize("precision", ["fp64", "fp64split", "fp64split40", "fp64split32", "tf32x3", "tf32x6", "fp32", "tf32", "bf16x3",
                                       "bf16x6"])
def test_allen_cahn_2d_n64_100_steps(precision):
    """2D Allen-Cahn, n = 64, kappa = 0.01, q = 0, tau = 1e-3, 100 steps."""
    torch = need_gpu()
    n = 64
    u0 = inputs.allen_cahn_2d(64, workload=0)
    ref = oracle_ref(2, 64, (0.01,), 0.0, 1e-3, u0, 100, "allen_cahn")
    got = run_gpu(torch, 2, 64, 0.01, 0.0, 1e-3, u0, 100, precision, "allen_cahn")
    assert rel_err(got, ref) < tol(precision, n)


@pytest.mark.gpu
@pytest.mark.parametrize("precision", ["fp64", "fp64split", "fp64split40", "fp64split32", "tf32x3", "tf32x6", "fp32", "tf32", "bf16x3",
                                       "bf16x6"])
@pytest.mark.parametrize("n", [300, 129])
def test_fhn_2d_ragged(precision, n):
    """2D FitzHugh-Nagumo with the workload's parameters on grids with ragged tiles."""
    torch = need_gpu()
    u0 = inputs.fhn_uniform(n, 2, workload=1)
    ref = oracle_ref(2, n, (1e-3, 5e-3), 0.0, 1e-2, u0, 20, "fhn", FHN)
    got = run_gpu(torch, 2, n, 1e-3, 0.0, 1e-2, u0, 20, precision, "fhn", FHN, kappa_comp=(1e-3, 5e-3))
    for c in range(2):
        assert rel_err(got[c], ref[c]) < tol(precision, n)


@pytest.mark.gpu
@pytest.mark.parametrize("precision", ["fp64", "fp64split", "fp64split40", "fp64split32", "tf32x3", "fp32", "bf16x3", "bf16x6"])
@pytest.mark.parametrize("n", [48, 33])
def test_allen_cahn_3d(precision, n):
    """3D Allen-Cahn, kappa = 1e-3, q = 0.1, tau = 5e-3, Gaussian bump."""
    torch = need_gpu()
    u0 = inputs.gaussian_bump(n, 3)
    ref = oracle_ref(3, n, (1e-3,), 0.1, 5e-3, u0, 10, "allen_cahn")
    got = run_gpu(torch, 3, n, 1e-3, 0.1, 5e-3, u0, 10, precision, "allen_cahn")
    assert rel_err(got, ref) < tol(precision, n)


@pytest.mark.gpu
@pytest.mark.parametrize("precision", ["fp64", "fp64split", "fp64split40", "fp64split32", "tf32x3", "tf32x6", "bf16x6"])
def test_fhn_3d_two_components(precision):
    torch = need_gpu()
    n = 40
    u0 = inputs.fhn_uniform(n, 3, workload=4)
    ref = oracle_ref(3, n, (1e-3, 5e-3), 0.05, 1e-2, u0, 8, "fhn", FHN)
    got = run_gpu(torch, 3, n, 1e-3, 0.05, 1e-2, u0, 8, precision, "fhn", FHN, kappa_comp=(1e-3, 5e-3))
    for c in range(2):
        assert rel_err(got[c], ref[c]) < tol(precision, n)


@pytest.mark.gpu
@pytest.mark.parametrize("precision", ["fp64", "fp64split", "tf32x3"])
@pytest.mark.parametrize("d,n", [(2, 96), (3, 30)])
def test_pade04(precision, d, n):
    torch = need_gpu()
    u0 = inputs.allen_cahn_2d(n, workload=5) if d == 2 else inputs.gaussian_bump(n, 3)
    ref = oracle_ref(d, n, (0.01,), 0.2, 2e-3, u0, 15, "allen_cahn", pade=4)
    got = run_gpu(torch, d, n, 0.01, 0.2, 2e-3, u0, 15, precision, "allen_cahn", pade=4)
    assert rel_err(got, ref) < tol(precision, n)


@pytest.mark.gpu
@pytest.mark.parametrize("precision", ["fp64", "fp64split", "tf32x3", "bf16x6"])
@pytest.mark.parametrize("d,n", [(2, 80), (3, 36)])
def test_exact_exponential(precision, d, n):
    """eq. (9)-(10) with exact exponentials against the FP64 Sylvester oracle
    (whose factor grids are pinned to quadrature of the phi integrals). With
    kappa = 1e-3, q = 0.1, tau = 5e-3 the products tau lambda_k run from about
    2.5e-4 to 0.13, so both the series and the closed-form branches of E_3 are used."""
    torch = need_gpu()
    tau, steps = 5e-3, 12
    u0 = inputs.allen_cahn_2d(n, workload=6) if d == 2 else inputs.gaussian_bump(n, 3)
    P = O.Problem(d=d, n=n, kappa=(1e-3,), q=0.1, tau=tau, reaction="allen_cahn")
    ref = S.run(P, u0, steps, react=lambda t, u: u - u ** 3, kind="exact")
    got = run_gpu(torch, d, n, 1e-3, 0.1, tau, u0, steps, precision, "allen_cahn", pade="exact")
    assert rel_err(got, ref) < tol(precision, n)


@pytest.mark.gpu
@pytest.mark.parametrize("precision", ["fp64", "fp64split", "fp64split40", "fp64split32", "tf32x3"])
@pytest.mark.parametrize("d", [2, 3])
def test_smallest_grid(precision, d):
    torch = need_gpu()
    n = 2
    u0 = inputs.random_field((2,) + (2,) * d, workload=7, scale=0.2)
    ref = oracle_ref(d, 2, (0.3, 0.1), 0.0, 1e-2, u0, 5, "fhn", FHN)
    got = run_gpu(torch, d, 2, 0.3, 0.0, 1e-2, u0, 5, precision, "fhn", FHN, kappa_comp=(0.3, 0.1))
    assert rel_err(got, ref) < tol(precision, n)


@pytest.mark.gpu
def test_linear_reaction_two_components():
    torch = need_gpu()
    n = 50
    u0 = inputs.random_field((2, n, n), workload=8)
    ref = oracle_ref(2, n, (0.02, 0.02), 0.3, 1e-2, u0, 10, "linear", (0.7,))
    got = run_gpu(torch, 2, n, 0.02, 0.3, 1e-2, u0, 10, "tf32x3", "linear", (0.7,))
    assert rel_err(got, ref) < tol("tf32x3", n)


@pytest.mark.gpu
def test_split_calls_resume_and_repeat_bitwise():
    """step(5) + step(5) agrees with step(10) (the carried spectral state resumes;
    only the accurate output transform of the first call differs), and a second
    run of the same calls is bit-identical (deterministic reductions)."""
    torch = need_gpu()
    n = 130
    u0 = inputs.fhn_uniform(n, 2, workload=9)
    plan = etd.Plan(2, n, 1e-3, 0.0, 1e-2, precision="tf32x3", reaction="fhn", rx_params=FHN, n_comp=2,
                    kappa_comp=(1e-3, 5e-3))
    a = torch.tensor(u0, dtype=torch.float32, device="cuda")
    b = a.clone()
    plan.step(a, 10)
    plan.invalidate()
    plan.step(b, 5)
    plan.step(b, 5)
    plan.sync()
    assert rel_err(b.double().cpu().numpy(), a.double().cpu().numpy()) < 1e-6
    c = torch.tensor(u0, dtype=torch.float32, device="cuda")
    plan.invalidate()
    plan.step(c, 10)
    plan.sync()
    assert torch.equal(a, c)
    plan.close()


@pytest.mark.gpu
def test_host_entry_point_and_stats():
    torch = need_gpu()
    n = 100
    u0 = inputs.fhn_uniform(n, 2, workload=10)
    ref = oracle_ref(2, n, (1e-3, 5e-3), 0.0, 1e-2, u0, 6, "fhn", FHN)
    plan = etd.Plan(2, n, 1e-3, 0.0, 1e-2, precision="tf32x3", reaction="fhn", rx_params=FHN, n_comp=2,
                    kappa_comp=(1e-3, 5e-3))
    host = torch.tensor(u0, dtype=torch.float32).pin_memory()
    plan.step_host(host, 6)
    assert rel_err(host.double().numpy(), ref) < tol("tf32x3", n)
    dev = host.cuda()
    m, bad = plan.stats(dev)
    assert bad == 0 and m == pytest.approx(float(np.abs(host.numpy()).max()), rel=1e-7)
    dev[0, 3, 4] = float("nan")
    dev[1, 0, 0] = float("inf")
    m2, bad2 = plan.stats(dev)
    assert bad2 == 2
    plan.close()


@pytest.mark.gpu
def test_host_loop_keeps_state_and_notices_edits():
    """etd_step_host in a loop: handing back the field it returned keeps the
    carried spectral state (the result equals one device call of all the steps);
    an edited field is noticed and stepped from scratch."""
    torch = need_gpu()
    n = 96
    u0 = inputs.fhn_uniform(n, 2, workload=12)
    kw = dict(precision="bf16x6", reaction="fhn", rx_params=FHN, n_comp=2, kappa_comp=(1e-3, 5e-3))
    plan = etd.Plan(2, n, 1e-3, 0.0, 1e-2, **kw)
    host = torch.tensor(u0, dtype=torch.float32).pin_memory()
    for _ in range(3):
        plan.step_host(host, 4)
    dplan = etd.Plan(2, n, 1e-3, 0.0, 1e-2, **kw)
    dev = torch.tensor(u0, dtype=torch.float32, device="cuda")
    for _ in range(3):
        dplan.step(dev, 4)
    dplan.sync()
    assert torch.equal(host, dev.cpu())  # same carried state, same launches
    ref = oracle_ref(2, n, (1e-3, 5e-3), 0.0, 1e-2, u0, 12, "fhn", FHN)
    assert rel_err(host.double().numpy(), ref) < 1e-6
    # an edit: the next call must rebuild the state from the edited field
    host[0, 10, 10] += 0.05
    edited = host.double().numpy().copy()
    plan.step_host(host, 4)
    ref2 = oracle_ref(2, n, (1e-3, 5e-3), 0.0, 1e-2, edited, 4, "fhn", FHN)
    assert rel_err(host.double().numpy(), ref2) < 1e-6
    plan.close()
    dplan.close()


@pytest.mark.gpu
def test_bad_field_arguments():
    torch = need_gpu()
    plan = etd.Plan(2, 64, 0.01, 0.0, 1e-3, precision="tf32x3")
    with pytest.raises(etd.EtdError):
        plan.step(torch.zeros((1, 64, 65), device="cuda"))
    host = torch.zeros((1, 64, 64))
    with pytest.raises(etd.EtdError) as ei:
        etd.etd_step(plan.handle, host.data_ptr(), 1)
    assert ei.value.status == etd.ETD_ERR_INVALID_ARG
    # alignment: device fields must start on a 16-byte boundary (4-byte offset
    # refused, 16-byte offset taken)
    buf = torch.zeros(64 * 64 + 8, device="cuda")
    with pytest.raises(etd.EtdError) as ei:
        etd.etd_step(plan.handle, buf[1:].data_ptr(), 1)
    assert ei.value.status == etd.ETD_ERR_INVALID_ARG
    etd.etd_step(plan.handle, buf[4:].data_ptr(), 1)
    plan.sync()
    plan.close()


@pytest.mark.gpu
@pytest.mark.parametrize("precision", ["bf16x6", "fp64", "fp64split"])
@pytest.mark.parametrize("d,n", [(2, 96), (3, 40)])
def test_fused_reaction_across_calls_and_interleaved_transforms(precision, d, n):
    """Allen-Cahn is evaluated in the transform epilogues (f(W) in the pass that
    makes W, f(U+) for the next step in the pass that returns U+, also across
    calls on the same field). Calls that overwrite the plan's operand buffers
    in between (etd_transform) must make the next step evaluate f(U) afresh:
    3 + 2 + 3 steps with a transform between the calls equal 8 steps of the oracle."""
    torch = need_gpu()
    u0 = inputs.allen_cahn_2d(n, workload=13) if d == 2 else inputs.gaussian_bump(n, 3)
    tau = 1e-3 if d == 2 else 5e-3
    plan = etd.Plan(d, n, 0.01, 0.1, tau, precision=precision, reaction="allen_cahn")
    u = torch.tensor(u0, dtype=plan.dtype, device="cuda")
    other = torch.tensor(inputs.random_field(u0.shape, workload=14), dtype=plan.dtype, device="cuda")
    plan.step(u, 3)
    plan.step(u, 2)
    plan.transform(other)
    plan.step(u, 3)
    plan.sync()
    ref = oracle_ref(d, n, (0.01,), 0.1, tau, u0, 8, "allen_cahn")
    assert rel_err(u.double().cpu().numpy(), ref) < tol(precision, n)
    plan.close()


@pytest.mark.gpu
@pytest.mark.parametrize("precision", ["fp64split", "fp64split40", "fp64split32"])
def test_fp64split_2d_n1024_fhn(precision):
    """The FP64-split tensor-core paths on a 2D FitzHugh-Nagumo grid of n = 1024
    (K = 1024: 32 k-blocks of exact level sums per tile) within their bars."""
    torch = need_gpu()
    n, steps = 1024, 10
    u0 = inputs.fhn_uniform(n, 2, workload=15)
    ref = oracle_ref(2, n, (1e-3, 5e-3), 0.0, 1e-2, u0, steps, "fhn", FHN)
    got = run_gpu(torch, 2, n, 1e-3, 0.0, 1e-2, u0, steps, precision, "fhn", FHN, kappa_comp=(1e-3, 5e-3))
    for c in range(2):
        assert rel_err(got[c], ref[c]) < TOL[precision]
