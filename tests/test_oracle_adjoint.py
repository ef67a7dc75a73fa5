"""Pins of the FP64 adjoint oracle (the paper has no adjoint; these check it
against the mathematics: central finite differences of the forward step, the
dot-product identity of a linear step, and agreement of its forward step with
the LU oracle)."""
import numpy as np
import pytest

from oracle import adjoint as A
from oracle import oracle as O
from paper_2601_06849_gb300 import inputs

FHN = (1.0, 0.3, 0.5, 0.1)


def problem(d, n, kind, pade=2):
    kap = (0.02, 0.05) if kind == "fhn" else (0.03,)
    rp = FHN if kind == "fhn" else ((0.7,) if kind == "linear" else ())
    return O.Problem(d=d, n=n, kappa=kap, q=0.2, tau=0.03, pade=pade, reaction=kind, rp=rp)


@pytest.mark.parametrize("d,n,kind,pade", [(2, 9, "fhn", 2), (3, 6, "allen_cahn", 2), (2, 8, "linear", 4)])
def test_forward_matches_lu_oracle(d, n, kind, pade):
    P = problem(d, n, kind, pade)
    u0 = inputs.random_field((P.ncomp,) + (n,) * d, workload=95, scale=0.4)
    np.testing.assert_allclose(A.run(P, u0, 4)[-1], O.run(P, u0, 4), atol=1e-12)


def loss(P, u0, N, target):
    return 0.5 * float(np.sum((A.run(P, u0, N)[-1] - target) ** 2))


@pytest.mark.parametrize("d,n,kind,pade", [(2, 7, "fhn", 2), (3, 5, "allen_cahn", 2), (2, 6, "linear", 4),
                                           (3, 4, "fhn", 4)])
def test_gradients_match_central_differences(d, n, kind, pade):
    P = problem(d, n, kind, pade)
    N = 5
    u0 = inputs.random_field((P.ncomp,) + (n,) * d, workload=96, scale=0.4)
    target = inputs.random_field(u0.shape, workload=97, scale=0.1)
    uN = A.run(P, u0, N)[-1]
    ubar0, gk, gth = A.adjoint_run(P, u0, N, uN - target)
    h = 1e-6
    # initial state, a few random directions
    for k in range(3):
        v = inputs.random_field(u0.shape, workload=98, sub=k)
        fd = (loss(P, u0 + h * v, N, target) - loss(P, u0 - h * v, N, target)) / (2 * h)
        assert np.sum(ubar0 * v) == pytest.approx(fd, rel=1e-6, abs=1e-10)
    # diffusivities
    for c in range(P.ncomp):
        kp, km = list(P.kappa), list(P.kappa)
        kp[c] += h * P.kappa[c]
        km[c] -= h * P.kappa[c]
        Pp = O.Problem(**{**P.__dict__, "kappa": tuple(kp)})
        Pm = O.Problem(**{**P.__dict__, "kappa": tuple(km)})
        fd = (loss(Pp, u0, N, target) - loss(Pm, u0, N, target)) / (2 * h * P.kappa[c])
        assert gk[c] == pytest.approx(fd, rel=1e-5, abs=1e-10)
    # reaction parameters
    for i in range(len(gth)):
        rp_p, rp_m = list(P.rp), list(P.rp)
        step = h * max(abs(P.rp[i]), 1.0)
        rp_p[i] += step
        rp_m[i] -= step
        Pp = O.Problem(**{**P.__dict__, "rp": tuple(rp_p)})
        Pm = O.Problem(**{**P.__dict__, "rp": tuple(rp_m)})
        fd = (loss(Pp, u0, N, target) - loss(Pm, u0, N, target)) / (2 * step)
        assert gth[i] == pytest.approx(fd, rel=1e-5, abs=1e-10)


def test_linear_step_dot_product_identity():
    """For f = c u the step is linear: <J v, w> = <v, J^T w> exactly."""
    P = problem(2, 8, "linear")
    v = inputs.random_field((1, 8, 8), workload=99, sub=1)
    w = inputs.random_field((1, 8, 8), workload=99, sub=2)
    Jv = A.run(P, v, 3)[-1]
    JTw, _, _ = A.adjoint_run(P, v, 3, w)
    assert np.sum(Jv * w) == pytest.approx(np.sum(v * JTw), rel=1e-12)
