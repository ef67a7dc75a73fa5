"""Pins of the CPU oracle to facts fixed by the paper and by the mathematics.

None of these compares the oracle with itself: each expected value comes from
the paper's printed tables, a closed form, a dense assembly of the operators
written from Section 2.1, or an invariant. A dropped term, a wrong sign or
index, a transposed axis or a missing tau in the oracle fails at least one.
"""
import os

import numpy as np
import pytest

from oracle import oracle as O
from oracle import spectral as S
from paper_2601_06849_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def closed_rationals(pade, x):
    """Polynomial forms of E_1, E_2, E_3 (Section 3.1 and the P_{0,4} variant of Section 5)."""
    x = np.asarray(x, dtype=np.float64)
    if pade == 2:
        den = x * x + 2 * x + 2
        return 2 / den, (x + 2) / den, (x + 1) / den
    den = x ** 4 + 4 * x ** 3 + 12 * x ** 2 + 24 * x + 24
    return 24 / den, (x ** 3 + 4 * x ** 2 + 12 * x + 24) / den, (x ** 3 + 3 * x ** 2 + 8 * x + 12) / den


def eig1d(n, kappa, q, d):
    """Discrete sine-mode eigenvalues of A_x: (4 kappa/h^2) sin^2(k pi h/2) + q/d, k = 1..n."""
    h = 1.0 / (n + 1)
    k = np.arange(1, n + 1)
    return 4 * kappa / h ** 2 * np.sin(k * np.pi * h / 2) ** 2 + q / d


# ----------------------------------------------------------------- rationals

@pytest.mark.parametrize("pade", [2, 4])
def test_partial_fractions_equal_polynomial_forms(pade):
    xs = np.concatenate([[0.0], np.logspace(-6, 4, 60)])
    want = closed_rationals(pade, xs)
    for ell in (1, 2, 3):
        got = np.array([O.rational(pade, ell, x) for x in xs])
        np.testing.assert_allclose(got, want[ell - 1], rtol=1e-13, atol=1e-16)


@pytest.mark.parametrize("pade,order", [(2, 3), (4, 5)])
def test_pade_factors_approximate_phi_functions(pade, order):
    """E_1 ~ e^{-x}, E_2 ~ (1-e^{-x})/x, E_3 ~ (x-1+e^{-x})/x^2: P_{0,2} matches
    e^{-x} through x^2, P_{0,4} through x^4, so halving x cuts the error of E_1
    by 2^order."""
    xs = np.array([0.02, 0.01, 0.005]) if pade == 2 else np.array([0.04, 0.02, 0.01])
    e1 = np.array([O.rational(pade, 1, x) for x in xs])
    err = np.abs(e1 - np.exp(-xs))
    ratios = err[:-1] / err[1:]
    np.testing.assert_allclose(np.log2(ratios), order, atol=0.1)
    assert O.rational(pade, 1, 0.0) == pytest.approx(1.0, abs=1e-15)
    assert O.rational(pade, 2, 0.0) == pytest.approx(1.0, abs=1e-15)
    assert O.rational(pade, 3, 0.0) == pytest.approx(0.5, abs=1e-15)


def test_p04_poles_are_quartic_roots():
    poles, res = O.pade_data(4)
    assert len(poles) == 2 and np.all(poles.imag > 0)
    D = lambda s: s ** 4 + 4 * s ** 3 + 12 * s ** 2 + 24 * s + 24
    for s in poles:
        assert abs(D(s)) < 1e-11
    ref = np.sort_complex(np.roots([1, 4, 12, 24, 24]))
    ref = ref[ref.imag > 0]
    np.testing.assert_allclose(np.sort_complex(poles), np.sort_complex(ref), rtol=1e-12)


def test_factors_in_unit_interval():
    xs = np.logspace(-8, 5, 200)
    for pade in (2, 4):
        for ell in (1, 2):
            v = np.array([O.rational(pade, ell, x) for x in xs])
            assert np.all(v > 0) and np.all(v <= 1.0 + 1e-15)


# ---------------------------------- exact exponential factors, eq. (9)-(10)

def phi_quadrature(x):
    """(e^{-x}, int_0^1 e^{-x(1-s)} ds, int_0^1 s e^{-x(1-s)} ds) by 40-digit
    quadrature of the integral forms of eq. (9)-(10) (the integrals whose closed
    forms the scheme uses), independent of any closed form or series."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 40
    X = mp.mpf(float(x))
    f2 = lambda s: mp.exp(-X * (1 - s))
    f3 = lambda s: s * mp.exp(-X * (1 - s))
    # the integrands live within ~1/x of s = 1: give the quadrature that breakpoint
    pts = [0, 1 - mp.mpf(80) / X, 1] if X > 80 else [0, 1]
    return float(mp.exp(-X)), float(mp.quad(f2, pts)), float(mp.quad(f3, pts))


EXACT_XS = np.concatenate([[0.0, 1e-12, 1e-7, 9.99e-4, 1.0001e-3, 0.0499, 0.0501, 0.0999, 0.1001, 0.5, 1.0,
                            30.0, 1e3], np.logspace(-10, 3, 27)])


def test_exact_factors_equal_phi_integrals():
    """Both branches of the exact-exponential grids (series below the switch,
    expm1 forms above) against quadrature of the integral definitions, at
    points on both sides of every switch (1e-3, 0.05, 0.1)."""
    e1, e2, e3 = S.rational_grids("exact", EXACT_XS)
    for i, x in enumerate(EXACT_XS):
        r1, r2, r3 = phi_quadrature(x) if x > 0 else (1.0, 1.0, 0.5)
        assert abs(e1[i] - r1) <= 1e-15 * r1, x
        assert abs(e2[i] - r2) <= 1e-14 * r2, x
        assert abs(e3[i] - r3) <= 1e-14 * r3, x


def test_exact_factors_recurrences_and_limits():
    """phi_{l+1}(x) = (1 - phi_l(x)) / x (with phi_0 = e^{-x}) where no
    cancellation occurs, the limits 1, 1, 1/2 at x = 0, and the Pade factors of
    Section 3.1 / Section 5 converging to them near 0 (E_1 to e^{-x} with order
    3 / 5)."""
    xs = np.linspace(1.0, 50.0, 50)
    e1, e2, e3 = S.rational_grids("exact", xs)
    np.testing.assert_allclose(e2, (1 - e1) / xs, rtol=1e-14)
    np.testing.assert_allclose(e3, (1 - e2) / xs, rtol=1e-13)
    z = S.rational_grids("exact", np.array([0.0]))
    assert (z[0][0], z[1][0], z[2][0]) == (1.0, 1.0, 0.5)
    # E_{l+1} = (1 - E_l)/x for the Pade factors too, so each step down the
    # recurrence costs one order: E_1, E_2, E_3 err by O(x^3), O(x^2), O(x) (P_{0,2})
    for pade, order in ((2, 3), (4, 5)):
        h = np.array([0.02, 0.01])
        ex = S.rational_grids("exact", h)
        pa = S.rational_grids(pade, h)
        for ell in range(3):
            err = np.abs(ex[ell] - pa[ell])
            assert abs(np.log2(err[0] / err[1]) - (order - ell)) < 0.1, (pade, ell)


@pytest.mark.parametrize("d,n,modes", [(2, 20, [(1, 1), (4, 17)]), (3, 9, [(2, 1, 3), (9, 9, 9)])])
def test_exact_scheme_f0_modes_decay_by_exponential(d, n, modes):
    """f = 0, exact-exponential grids: each sine mode is multiplied per step by
    exp(-tau (lambda_kx + lambda_ky [+ lambda_kz]))."""
    kappa, q, tau, N = 0.03, 0.4, 0.02, 6
    lam = eig1d(n, kappa, q, d)
    P = O.Problem(d=d, n=n, kappa=(kappa,), q=q, tau=tau, pade=2, reaction="none")
    u0 = np.zeros((n,) * d)
    want = np.zeros((n,) * d)
    for w, m in enumerate(modes):
        shape = inputs.sine_mode(n, d, m)
        rate = sum(lam[k - 1] for k in m)
        u0 += (w + 1) * shape
        want += (w + 1) * np.exp(-tau * rate * N) * shape
    got = S.run(P, u0[None], N, react=lambda t, u: np.zeros_like(u), kind="exact")[0]
    np.testing.assert_allclose(got, want, atol=1e-13 * np.abs(u0).max())


def test_exact_scheme_linear_reaction_modal_recurrence():
    """f = c u on one sine mode with the exact grids: the scalar recurrence of
    eq. (9)-(10) with phi_1, phi_2 taken from quadrature."""
    n, kappa, q, tau, c, N = 16, 0.02, 0.4, 0.05, 1.3, 8
    lam = eig1d(n, kappa, q, 2)
    m = (3, 5)
    _, p1, p2 = phi_quadrature(tau * lam[m[0] - 1])
    e1x = np.exp(-tau * lam[m[0] - 1])
    s = np.exp(-tau * lam[m[1] - 1])
    a = 1.0
    for _ in range(N):
        w = e1x * s * a + tau * p1 * s * c * a
        a = w + tau * p2 * (c * w - s * c * a)
    P = O.Problem(d=2, n=n, kappa=(kappa,), q=q, tau=tau, pade=2, reaction="linear", rp=(c,))
    got = S.run(P, inputs.sine_mode(n, 2, m)[None], N, react=lambda t, u: c * u, kind="exact")[0]
    np.testing.assert_allclose(got, a * inputs.sine_mode(n, 2, m), atol=1e-14)


def discrete_manufactured_error(kind, N, n=31, d=2, lam=1.0, coarse=16):
    """E(N) against the exact solution of the semi-discrete problem: psi built
    with the discrete eigenvalue of sin(pi x) (A_h u0 = d mu_1 u0), so that
    u_h(t) = e^{-lam t} u0 solves u' + A_h u = u (1 - u^2) + psi exactly and the
    error is the time discretisation alone (the quantity the convergence
    theorems of Section 4 bound)."""
    h = 1.0 / (n + 1)
    mu1 = 4 / h ** 2 * np.sin(np.pi * h / 2) ** 2
    u0 = inputs.sine_mode(n, d, (1,) * d)

    def react(t, u):
        ue = np.exp(-lam * t) * u0
        return u * (1 - u * u) + ((-lam + d * mu1) * ue - ue * (1 - ue * ue))[None]

    P = O.Problem(d=d, n=n, kappa=(1.0,), q=0.0, tau=1.0 / N, pade=2, reaction="none")
    u, E, per = u0[None].copy(), 0.0, N // coarse
    for c in range(coarse):
        u = S.run(P, u, per, t0=c * per / N, react=react, kind=kind)
        E = max(E, np.abs(u[0] - np.exp(-lam * (c + 1) * per / N) * u0).max())
    return E


def test_exact_scheme_second_order():
    """The exact-exponential ETD2RK-DS scheme converges with order 2 in tau
    (the convergence theorem for eq. (9)-(10) in Section 4)."""
    E = np.array([discrete_manufactured_error("exact", N) for N in (16, 32, 64, 128)])
    eoc = np.log2(E[:-1] / E[1:])
    assert np.all(eoc > 1.85) and np.all(eoc < 2.1), eoc


# ------------------------------------------------- closed forms on sine modes

@pytest.mark.parametrize("d,n,modes,pade,q", [
    (2, 31, [(1, 1), (3, 7), (31, 2)], 2, 0.0),
    (2, 24, [(2, 5), (24, 24)], 4, 0.7),
    (3, 12, [(1, 2, 3), (12, 1, 5)], 2, 0.3),
    (3, 9, [(4, 4, 9)], 4, 0.0),
])
def test_f0_sine_modes_decay_by_pade_factor(d, n, modes, pade, q):
    """f = 0: each mode prod sin(k pi x) is multiplied per step by
    E_1(tau lambda_kx) E_1(tau lambda_ky) [E_1(tau lambda_kz)]."""
    kappa, tau, N = 0.05, 0.01, 7
    lam = eig1d(n, kappa, q, d)
    P = O.Problem(d=d, n=n, kappa=(kappa,), q=q, tau=tau, pade=pade, reaction="none")
    u0 = np.zeros((n,) * d)
    want = np.zeros((n,) * d)
    for w, m in enumerate(modes):
        shape = inputs.sine_mode(n, d, m)
        amp = 1.0
        for k in m:
            amp *= closed_rationals(pade, tau * lam[k - 1])[0]
        u0 += (w + 1) * shape
        want += (w + 1) * amp ** N * shape
    got = O.run(P, u0[None], N)[0]
    np.testing.assert_allclose(got, want, atol=1e-13 * np.abs(u0).max())


@pytest.mark.parametrize("d,pade", [(2, 2), (2, 4), (3, 2)])
def test_linear_reaction_modal_recurrence(d, pade):
    """f = c u on one sine mode: eq. (13)-(14) reduce to a scalar recurrence
    a -> w = e1x s a + tau e2x s c a;  a+ = w + tau e3x (c w - s c a), s = E_1(A_2)."""
    n, kappa, q, tau, c, N = 16, 0.02, 0.4, 0.02, 1.7, 9
    lam = eig1d(n, kappa, q, d)
    m = (3, 5, 2)[:d]
    e1x, e2x, e3x = [g[m[0] - 1] for g in closed_rationals(pade, tau * lam)]
    s = 1.0
    for k in m[1:]:
        s *= closed_rationals(pade, tau * lam[k - 1])[0]
    a = 1.0
    for _ in range(N):
        w = e1x * s * a + tau * e2x * s * c * a
        a = w + tau * e3x * (c * w - s * c * a)
    P = O.Problem(d=d, n=n, kappa=(kappa,), q=q, tau=tau, pade=pade, reaction="linear", rp=(c,))
    got = O.run(P, inputs.sine_mode(n, d, m)[None], N)[0]
    np.testing.assert_allclose(got, a * inputs.sine_mode(n, d, m), atol=1e-13)


def test_fhn_linear_modal_recurrence_two_components():
    """FitzHugh-Nagumo with c3 = 0, b = 0 is linear: f = M (u, v), M = [[1, -1],
    [eps, -eps a]]. With per-component kappa the modal recurrence uses each
    component's own grids (Example 5.3 block operators)."""
    n, ku, kv, tau, N = 20, 0.01, 0.3, 0.01, 11
    eps, a_ = 0.7, 0.5
    M = np.array([[1.0, -1.0], [eps, -eps * a_]])
    m = (2, 3)
    gr = []
    for kap in (ku, kv):
        lam = eig1d(n, kap, 0.0, 2)
        e = closed_rationals(2, tau * lam)
        gr.append((e[0][m[0] - 1], e[1][m[0] - 1], e[2][m[0] - 1], e[0][m[1] - 1]))
    amp = np.array([1.0, -0.4])
    for _ in range(N):
        F = M @ amp
        W = np.array([g[0] * g[3] * amp[c] + tau * g[1] * g[3] * F[c] for c, g in enumerate(gr)])
        FW = M @ W
        amp = np.array([W[c] + tau * g[2] * (FW[c] - g[3] * F[c]) for c, g in enumerate(gr)])
    shape = inputs.sine_mode(n, 2, m)
    P = O.Problem(d=2, n=n, kappa=(ku, kv), q=0.0, tau=tau, reaction="fhn", rp=(0.0, eps, a_, 0.0))
    got = O.run(P, np.stack([shape, -0.4 * shape]), N)
    np.testing.assert_allclose(got[0], amp[0] * shape, atol=1e-13)
    np.testing.assert_allclose(got[1], amp[1] * shape, atol=1e-13)


# ---------------------------------------------------- dense Kronecker operators

def dense_ops(d, n, kappa, q):
    """A_1 and the A_2 pieces as dense Kronecker products (Section 2.1 and
    Section 3.1): x fastest, so I_y (x) A_x acts inside each x row."""
    A = S.operator_1d(n, kappa, q, d)
    I = np.eye(n)
    if d == 2:
        return np.kron(I, A), [np.kron(A, I)]
    return np.kron(I, np.kron(I, A)), [np.kron(I, np.kron(A, I)), np.kron(A, np.kron(I, I))]


def dense_rational(pade, ell, X):
    I = np.eye(X.shape[0])
    if pade == 2:
        D = X @ X + 2 * X + 2 * I
        num = [2 * I, X + 2 * I, X + I][ell - 1]
    else:
        X2 = X @ X
        X3 = X2 @ X
        D = X2 @ X2 + 4 * X3 + 12 * X2 + 24 * X + 24 * I
        num = [24 * I, X3 + 4 * X2 + 12 * X + 24 * I, X3 + 3 * X2 + 8 * X + 12 * I][ell - 1]
    return np.linalg.solve(D, num)


def react_np(kind, rp):
    if kind == "allen_cahn":
        return lambda t, u: u - u ** 3
    if kind == "fhn":
        c3, eps, a_, b = rp
        return lambda t, u: np.stack([u[0] - c3 * u[0] ** 3 - u[1], eps * (u[0] - a_ * u[1] - b)])
    raise ValueError(kind)


@pytest.mark.parametrize("d,n,pade,kind", [(2, 7, 2, "allen_cahn"), (2, 6, 4, "fhn"), (3, 5, 2, "fhn"),
                                           (3, 6, 4, "allen_cahn")])
def test_dense_kronecker_scheme(d, n, pade, kind):
    """eq. (13)-(16) applied literally with dense matrices equal the sliced LU oracle."""
    q, tau, N = 0.6, 0.03, 4
    kap = (0.05,) if kind == "allen_cahn" else (0.05, 0.2)
    rp = () if kind == "allen_cahn" else (1.0, 0.3, 0.5, 0.1)
    f = react_np(kind, rp)
    u0 = inputs.random_field((len(kap),) + (n,) * d, workload=90, scale=0.5)
    Nn = n ** d
    ops = []
    for k in kap:
        A1, A2s = dense_ops(d, n, k, q)
        S2 = np.eye(Nn)
        for A2 in A2s:
            S2 = S2 @ dense_rational(pade, 1, tau * A2)
        ops.append((dense_rational(pade, 1, tau * A1), dense_rational(pade, 2, tau * A1),
                    dense_rational(pade, 3, tau * A1), S2))
    u = u0.reshape(len(kap), Nn).copy()
    for step in range(N):
        F = f(step * tau, u)
        W = np.stack([Q1 @ S2 @ u[c] + tau * Q2 @ S2 @ F[c] for c, (Q1, Q2, Q3, S2) in enumerate(ops)])
        FW = f((step + 1) * tau, W)
        u = np.stack([W[c] + tau * Q3 @ (FW[c] - S2 @ F[c]) for c, (Q1, Q2, Q3, S2) in enumerate(ops)])
    P = O.Problem(d=d, n=n, kappa=kap, q=q, tau=tau, pade=pade, reaction=kind, rp=rp)
    got = O.run(P, u0, N)
    np.testing.assert_allclose(got.reshape(len(kap), Nn), u, atol=1e-12, rtol=0)


@pytest.mark.parametrize("d,n,pade,kind", [(2, 24, 2, "fhn"), (2, 17, 4, "allen_cahn"), (3, 10, 2, "allen_cahn"),
                                           (3, 9, 4, "fhn")])
def test_lu_equals_sylvester(d, n, pade, kind):
    """Section 5 reports identical values from the LU and the Sylvester routes."""
    kap = (0.01,) if kind == "allen_cahn" else (0.01, 0.05)
    rp = () if kind == "allen_cahn" else (1.0, 0.2, 0.5, 0.1)
    P = O.Problem(d=d, n=n, kappa=kap, q=0.25, tau=0.02, pade=pade, reaction=kind, rp=rp)
    u0 = inputs.random_field((len(kap),) + (n,) * d, workload=91, scale=0.6)
    a = O.run(P, u0, 6)
    b = S.run(P, u0, 6, react=react_np(kind, rp))
    np.testing.assert_allclose(a, b, atol=1e-12, rtol=0)


# ----------------------------------------------- printed E(N) of Example 5.1

def load_golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.strip()
            if line and not line.startswith("#"):
                p, N, E = line.split()
                rows.append((int(p), int(N), float(E)))
    return rows


def manufactured_error(d, n, N, pade, coarse):
    """E(N) of Section 5: max over the coarse times S_coarse of ||u - U||_inf."""
    u0 = inputs.sine_mode(n, d, (1,) * d)
    P = O.Problem(d=d, n=n, kappa=(1.0,), q=0.0, tau=1.0 / N, pade=pade, reaction="ac_manufactured", rp=(1.0,))
    u, E, per = u0[None].copy(), 0.0, N // coarse
    for c in range(coarse):
        u = O.run(P, u, per, t0=c * per / N)
        E = max(E, np.abs(u[0] - np.exp(-(c + 1) * per / N) * u0).max())
    return E


def three_sig(x):
    return float(f"{x:.2E}")


@pytest.mark.parametrize("pade,N,E", load_golden("table1_ex51_2d.txt"))
def test_table1_allen_cahn_2d(pade, N, E):
    assert three_sig(manufactured_error(2, 511, N, pade, 16)) == pytest.approx(E, rel=1e-9)


@pytest.mark.parametrize("pade,N,E", load_golden("table2_ex51_3d.txt"))
def test_table2_allen_cahn_3d(pade, N, E):
    assert three_sig(manufactured_error(3, 79, N, pade, 10)) == pytest.approx(E, rel=1e-9)


# --------------------------------------------------------------- invariants

def test_second_order_in_time():
    """Remark after Theorem 4.6 and Tables 1-2: the observed order is about 2."""
    E = [manufactured_error(2, 63, N, 2, 16) for N in (32, 64, 128)]
    eoc = np.log2(np.array(E[:-1]) / np.array(E[1:]))
    assert np.all(eoc > 1.7) and np.all(eoc < 2.2), eoc


def test_allen_cahn_stays_bounded():
    """Section 4 remark: Allen-Cahn data with |u0| <= 1 stay in [-1, 1] up to O(tau)."""
    n, tau = 40, 0.01
    u0 = inputs.rng(92).uniform(-1.0, 1.0, size=(1, n, n))
    P = O.Problem(d=2, n=n, kappa=(1e-3,), q=0.0, tau=tau, reaction="allen_cahn")
    u = O.run(P, u0, 300)
    assert np.abs(u).max() <= 1.0 + 5 * tau


def test_reflection_symmetry_each_axis():
    """The split is not x<->y symmetric, but x -> 1-x (and y -> 1-y) is preserved."""
    n = 21
    r = inputs.random_field((2, n, n), workload=93, scale=0.3)
    u0 = r + r[:, :, ::-1]
    u0 = u0 + u0[:, ::-1, :]
    P = O.Problem(d=2, n=n, kappa=(0.01, 0.04), q=0.1, tau=0.02, reaction="fhn", rp=(1.0, 0.1, 0.5, 0.1))
    u = O.run(P, u0, 10)
    np.testing.assert_allclose(u, u[:, :, ::-1], atol=1e-13)
    np.testing.assert_allclose(u, u[:, ::-1, :], atol=1e-13)


def test_fp32_shadow_tracks_fp64():
    n = 32
    u0 = inputs.allen_cahn_2d(n)
    P = O.Problem(d=2, n=n, kappa=(0.01,), q=0.0, tau=1e-3, reaction="allen_cahn")
    a = O.run(P, u0, 20)
    b = O.run(P, u0, 20, precision="f32")
    err = np.abs(a - b).max() / np.abs(a).max()
    assert 1e-9 < err < 1e-5


@pytest.fixture(scope="module")
def singular_reference():
    return singular_trajectory(512)


def singular_trajectory(N, n=511, d=2, coarse=16):
    """The Example 5.2 run at the coarse times S_coarse (kappa = 1, q = 1, rho = 0.1)."""
    u = 0.99 * inputs.sine_mode(n, d, (1,) * d)[None]
    P = O.Problem(d=d, n=n, kappa=(1.0,), q=1.0, tau=1.0 / N, reaction="singular", rp=(0.1,))
    out, per = [], N // coarse
    for c in range(coarse):
        u = O.run(P, u, per, t0=c * per / N)
        out.append(u)
    return out


@pytest.mark.parametrize("pade,N,E", load_golden("table4_ex52_2d.txt"))
def test_table4_singular_source_2d(pade, N, E, singular_reference):
    tr = singular_trajectory(N)
    err = max(np.abs(a - b).max() for a, b in zip(tr, singular_reference))
    assert three_sig(err) == pytest.approx(E, rel=1e-9)


@pytest.fixture(scope="module")
def singular_reference_3d():
    return singular_trajectory(320, n=79, d=3, coarse=10)


@pytest.mark.parametrize("pade,N,E", load_golden("table4b_ex52_3d.txt"))
def test_table4b_singular_source_3d(pade, N, E, singular_reference_3d):
    tr = singular_trajectory(N, n=79, d=3, coarse=10)
    err = max(np.abs(a - b).max() for a, b in zip(tr, singular_reference_3d))
    assert three_sig(err) == pytest.approx(E, rel=1e-9)
