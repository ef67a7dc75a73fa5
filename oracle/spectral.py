"""Sylvester (diagonalisation) form of the ETD2RK-DS step, plain NumPy, FP64.

TEST INFRASTRUCTURE (same rules as oracle.py). This is the paper's second
implementation route (Section 3.3.2 and Algorithms 1-2 in matrix-matrix form,
Remark 2 of Section 3.4): A_x = P_x D_x P_x^T from a LAPACK symmetric
eigensolver, each E_l(tau A) applied as P diag(E_l(tau lambda)) P^T along one
axis. The rational factors are evaluated from their polynomial forms (P_{0,2}:
Section 3.1; P_{0,4}: Section 5), not from the partial fractions the LU oracle
uses, and the exact-exponential grids of eq. (9)-(10) are offered as a third
choice ("exact"). It exists to check LU == spectral (the paper reports identical
values) and to serve as the oracle of the exact-exponential variant.
"""
from __future__ import annotations

import numpy as np


def rational_grids(kind, x):
    """(E1, E2, E3)(x) for kind in {2, 4, 'exact'}; x = tau * lambda >= 0."""
    x = np.asarray(x, dtype=np.float64)
    if kind == 2:
        den = x * x + 2 * x + 2
        return 2 / den, (x + 2) / den, (x + 1) / den
    if kind == 4:
        den = x ** 4 + 4 * x ** 3 + 12 * x ** 2 + 24 * x + 24
        return 24 / den, (x ** 3 + 4 * x ** 2 + 12 * x + 24) / den, (x ** 3 + 3 * x ** 2 + 8 * x + 12) / den
    if kind == "exact":
        # eq. (9)-(10): E1 = e^{-x}, E2 = (1 - e^{-x})/x = int_0^1 e^{-x(1-s)} ds,
        # E3 = (x - 1 + e^{-x})/x^2 = int_0^1 s e^{-x(1-s)} ds. Written with expm1,
        # E2 loses nothing; E3's numerator x + expm1(-x) ~ x^2/2 still cancels
        # (relative error about 2 eps / x), so below x = 0.1 E3 is the Taylor
        # series sum_{j>=0} (-x)^j / (j+2)!, 16 terms (truncation < 1e-20 there).
        e1 = np.exp(-x)
        pos = x > 0
        xs = np.where(pos, x, 1.0)
        e2 = np.where(pos, -np.expm1(-xs) / xs, 1.0)
        small = x < 0.1
        series = np.zeros_like(x)
        term = np.full_like(x, 0.5)
        for j in range(16):
            series = series + term
            term = term * (-x) / (j + 3)
        xl = np.where(small, 1.0, x)
        e3 = np.where(small, series, (xl + np.expm1(-xl)) / xl ** 2)
        return e1, e2, e3
    raise ValueError(kind)


def operator_1d(n, kappa, q, d):
    """A = (1/h^2) tridiag(-kappa, 2 kappa + (q/d) h^2, -kappa), h = 1/(n+1)."""
    h = 1.0 / (n + 1)
    A = np.zeros((n, n))
    idx = np.arange(n)
    A[idx, idx] = (2 * kappa + (q / d) * h * h) / (h * h)
    A[idx[1:], idx[:-1]] = -kappa / (h * h)
    A[idx[:-1], idx[1:]] = -kappa / (h * h)
    return A


def _apply_axis(P, g, field, axis):
    """P diag(g) P^T applied along array axis ``axis``."""
    M = (P * g[None, :]) @ P.T
    return np.moveaxis(np.tensordot(M, field, axes=([1], [axis])), 0, axis)


def run(problem, u, nsteps, t0=0.0, react=None, kind=None):
    """Advance u (ncomp, n, n[, n]) by nsteps Sylvester-form steps.

    ``react(t, u) -> f`` evaluates the reaction on the whole stacked field;
    ``kind`` overrides problem.pade (use "exact" for eq. (9)-(10))."""
    d, n, tau = problem.d, problem.n, problem.tau
    kind = problem.pade if kind is None else kind
    u = np.array(u, dtype=np.float64, copy=True)
    grids = []
    for kap in problem.kappa:
        lam, P = np.linalg.eigh(operator_1d(n, kap, problem.q, d))
        grids.append((P, rational_grids(kind, tau * lam)))
    x_axis = d  # array axes: 0 = comp, then z/y, x last
    y_axis = d - 1
    for step in range(nsteps):
        tn = t0 + step * tau
        F = react(tn, u)
        W = np.empty_like(u)
        Bs = []
        for c, (P, (e1, e2, e3)) in enumerate(grids):
            a, b = u[c], F[c]
            if d == 3:  # z pass first (Algorithm 2, step 3.1)
                a, b = _apply_axis(P, e1, a, 0), _apply_axis(P, e1, b, 0)
            a, b = _apply_axis(P, e1, a, y_axis - 1), _apply_axis(P, e1, b, y_axis - 1)
            W[c] = _apply_axis(P, e1, a, x_axis - 1) + tau * _apply_axis(P, e2, b, x_axis - 1)
            Bs.append(b)
        FW = react(tn + tau, W)
        for c, (P, (e1, e2, e3)) in enumerate(grids):
            u[c] = W[c] + tau * _apply_axis(P, e3, FW[c] - Bs[c], x_axis - 1)
    return u
