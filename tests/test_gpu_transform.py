"""Step a2 alone: the spectral transform through the C ABI against its plain
definition T(X) = P^T X P (2D) / the three mode products (3D), in FP64."""
import numpy as np
import pytest

from gpu_util import need_gpu, rel_err, sine_basis
from paper_2601_06849_gb300 import etd, inputs

# bound on max|T_gpu - T| / max|T| for one transform (2 or 3 chained passes)
TOL = {"fp64": 1e-13, "fp32": 1e-5, "tf32x3": 2e-6, "tf32x6": 2e-6, "tf32": 5e-3, "bf16x3": 2e-6, "bf16x6": 2e-6}


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
@pytest.mark.parametrize("precision", ["fp64", "fp32", "tf32x3", "tf32x6", "tf32", "bf16x3", "bf16x6"])
@pytest.mark.parametrize("d,n,ncomp", [(2, 64, 1), (2, 200, 2), (2, 37, 1), (3, 24, 1), (3, 45, 2), (2, 520, 1),
                                       (2, 2, 1)])
def test_transform_matches_definition(precision, d, n, ncomp):
    torch = need_gpu()
    x = inputs.random_field((ncomp,) + (n,) * d, workload=40, sub=n)
    plan = etd.Plan(d, n, 0.01, 0.0, 1e-3, precision=precision, reaction="linear", n_comp=ncomp)
    dt = torch.float64 if precision == "fp64" else torch.float32
    xt = torch.tensor(x, dtype=dt, device="cuda")
    out = plan.transform(xt)
    plan.sync()
    ref = reference(xt.double().cpu().numpy(), d)
    assert rel_err(out.cpu().numpy(), ref) < TOL[precision]
    back = plan.transform(out)
    plan.sync()
    assert rel_err(back.cpu().numpy(), xt.double().cpu().numpy()) < 2 * TOL[precision]
    plan.close()
