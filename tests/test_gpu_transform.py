"""Step a2 alone: the spectral transform through the C ABI against its plain
definition T(X) = P^T X P (2D) / the three mode products (3D), in FP64."""
import numpy as np
import pytest

from gpu_util import need_gpu, rel_err, sine_basis
from paper_2601_06849_gb300 import etd, inputs

# bound on max|T_gpu - T| / max|T| for one transform (2 or 3 chained passes)
# fp64split: operands rounded to 48 bits below their row's power-of-two scale
# (2^-49 relative to the row's max; P to 47 bits), products of level 6 and below
# dropped (each term under 2^-49 of the scales' product): a few 2^-47 relative to
# max |T| per pass (a CPU emulation of the same arithmetic gives 1.7e-14 on
# Gaussian data at n = 512), 2e-13 per pass allowed, d passes.
# fp64split40 / fp64split32: the same with 40 / 32 bits, 2^8 / 2^16 times coarser.
# fp64: FP64 sums of n products on both sides (kernel and NumPy reference), whose
# worst-case rounding error grows as n u (gamma_n); 1e-13 holds up to n = 512 and
# is scaled by n / 512 beyond (1.7e-13 measured at n = 1100, 2.3e-13 at n = 1537).
TOL = {"fp64": 1e-13, "fp32": 1e-5, "tf32x3": 2e-6, "tf32x6": 2e-6, "tf32": 5e-3, "bf16x3": 2e-6, "bf16x6": 2e-6,
       "fp64split": 2e-13, "fp64split40": 2e-13 * 256, "fp64split32": 2e-13 * 65536}


def reference(x, d):
    n = x.shape[-1]
    P = sine_basis(n)
    if d == 2:
        return np.einsum("yl,cyx,xk->clk", P, x, P, optimize=True)
    return np.einsum("zp,yl,czyx,xk->cplk", P, P, x, P, optimize=True)


def test_sine_basis_diagonalises_operator():
    """The closed-form basis is orthogonal and diagonalises tridiag(-1, 2, -1) (CPU check)."""
    n = 37
    P = sine_basis(n)
    A = 2 * np.eye(n) - np.eye(n, k=1) - np.eye(n, k=-1)
    D = P.T @ A @ P
    lam = 4 * np.sin(np.arange(1, n + 1) * np.pi / (2 * (n + 1))) ** 2
    np.testing.assert_allclose(P.T @ P, np.eye(n), atol=1e-13)
    np.testing.assert_allclose(D, np.diag(lam), atol=1e-12)


@pytest.mark.gpu
@pytest.mark.parametrize("precision", ["fp64", "fp32", "tf32x3", "tf32x6", "tf32", "bf16x3", "bf16x6", "fp64split",
                                       "fp64split40", "fp64split32"])
@pytest.mark.parametrize("d,n,ncomp", [(2, 64, 1), (2, 200, 2), (2, 37, 1), (3, 24, 1), (3, 45, 2), (2, 520, 1),
                                       (2, 2, 1), (2, 1100, 1), (2, 1537, 2)])
def test_transform_matches_definition(precision, d, n, ncomp):
    torch = need_gpu()
    x = inputs.random_field((ncomp,) + (n,) * d, workload=40, sub=n)
    plan = etd.Plan(d, n, 0.01, 0.0, 1e-3, precision=precision, reaction="linear", n_comp=ncomp)
    dt = plan.dtype
    xt = torch.tensor(x, dtype=dt, device="cuda")
    out = plan.transform(xt)
    plan.sync()
    ref = reference(xt.double().cpu().numpy(), d)
    bound = TOL[precision] * (d if precision.startswith("fp64split") else 1)
    if precision == "fp64":
        bound *= max(1.0, n / 512)
    assert rel_err(out.cpu().numpy(), ref) < bound
    back = plan.transform(out)
    plan.sync()
    assert rel_err(back.cpu().numpy(), xt.double().cpu().numpy()) < 2 * bound
    plan.close()


@pytest.mark.gpu
@pytest.mark.parametrize("n", [96, 1031])
def test_fp64split_scales_per_component_and_keeps_nan(n):
    """The slices' scale is per operand row: a component a million times smaller
    than the other keeps its own relative accuracy, a row of zeros stays zero; a
    NaN in one component makes that component's transform NaN and leaves the other
    intact. (n = 96: one warp slices a row; n = 1031, odd: one block per row.)"""
    torch = need_gpu()
    x = inputs.random_field((2, n, n), workload=41)
    x[1] *= 1e-6
    x[1, 3, :] = 0.0
    plan = etd.Plan(2, n, 0.01, 0.0, 1e-3, precision="fp64split", reaction="linear", n_comp=2)
    xt = torch.tensor(x, dtype=torch.float64, device="cuda")
    out = plan.transform(xt)
    plan.sync()
    ref = reference(x, 2)
    for c in range(2):
        assert rel_err(out[c].cpu().numpy(), ref[c]) < 2 * TOL["fp64split"]
    xt[0, 5, 7] = float("nan")
    out = plan.transform(xt)
    plan.sync()
    assert torch.isnan(out[0]).all()
    assert rel_err(out[1].cpu().numpy(), ref[1]) < 2 * TOL["fp64split"]
    plan.close()
