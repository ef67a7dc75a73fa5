"""FP64 adjoint of the Pade ETD2RK-DS step, plain NumPy.

TEST INFRASTRUCTURE (same rules as oracle.py). The paper has no adjoint; this
is the reverse-mode derivative of its step (eq. (13)-(16)) written out. With
S = E_1(tau A_2) (3D: E_1(tau A_2^y) E_1(tau A_2^z)) and X_l = E_l(tau A_1), all
symmetric and commuting, per component c (its own kappa_c):

    forward:  F = f(U);  W = X1 S U + tau X2 S F;  G = f(W) - S F;  U+ = W + tau X3 G
    backward (given U+bar):
        Gbar = tau X3 U+bar
        Wbar = U+bar + J_f(W)^T Gbar
        Fbar = tau X2 S Wbar - S Gbar
        Ubar = X1 S Wbar + J_f(U)^T Fbar
    d/dkappa_c = <U+bar, tau dX3 G> - <Gbar, dS F> + <Wbar, d(X1 S) U + tau d(X2 S) F>
    d/dtheta   = <Gbar, d_theta f(W)> + <Fbar, d_theta f(U)>

Operators are applied through a LAPACK eigendecomposition of A_x; their kappa
derivatives use dE_l(tau lambda)/dkappa = tau mu E_l'(tau lambda), mu = dlambda/dkappa.
Reactions: "none", "linear" (c u; theta = c), "allen_cahn", "fhn" (theta = c3, eps, a, b).
"""
from __future__ import annotations

import numpy as np

from . import spectral


def _rational_and_derivative(pade, x):
    """(E1, E2, E3) and their x-derivatives for P_{0,2} / P_{0,4}."""
    x = np.asarray(x, dtype=np.float64)
    if pade == 2:
        D, dD = x * x + 2 * x + 2, 2 * x + 2
        N = [2 + 0 * x, x + 2, x + 1]
        dN = [0 * x, 1 + 0 * x, 1 + 0 * x]
    else:
        D = x ** 4 + 4 * x ** 3 + 12 * x ** 2 + 24 * x + 24
        dD = 4 * x ** 3 + 12 * x ** 2 + 24 * x + 24
        N = [24 + 0 * x, x ** 3 + 4 * x ** 2 + 12 * x + 24, x ** 3 + 3 * x ** 2 + 8 * x + 12]
        dN = [0 * x, 3 * x ** 2 + 8 * x + 12, 3 * x ** 2 + 6 * x + 8]
    E = [Nl / D for Nl in N]
    dE = [(dNl * D - Nl * dD) / D ** 2 for Nl, dNl in zip(N, dN)]
    return E, dE


class _Ops:
    """Per-component operators X_l, S and their kappa derivatives."""

    def __init__(self, problem, kappa):
        d, n, tau = problem.d, problem.n, problem.tau
        A = spectral.operator_1d(n, kappa, problem.q, d)
        lam, P = np.linalg.eigh(A)
        mu = np.diag(P.T @ spectral.operator_1d(n, 1.0, 0.0, d) @ P)  # dlambda/dkappa
        E, dE = _rational_and_derivative(problem.pade, tau * lam)
        self.d, self.P, self.tau = d, P, tau
        self.E = E
        self.dE = [tau * mu * g for g in dE]  # d E_l(tau lambda) / d kappa

    def _axis(self, g, f, axis):
        return spectral._apply_axis(self.P, g, f, axis)

    def X(self, l, f, deriv=False):
        g = (self.dE if deriv else self.E)[l - 1]
        return self._axis(g, f, self.d - 1)

    def S(self, f):
        f = self._axis(self.E[0], f, self.d - 2)
        if self.d == 3:
            f = self._axis(self.E[0], f, 0)
        return f

    def dS(self, f):
        """d/dkappa of S applied to f (product rule over the y and z factors)."""
        y = self.d - 2
        if self.d == 2:
            return self._axis(self.dE[0], f, y)
        a = self._axis(self.E[0], self._axis(self.dE[0], f, y), 0)
        b = self._axis(self.dE[0], self._axis(self.E[0], f, y), 0)
        return a + b


def react(kind, rp, U):
    if kind == "none":
        return np.zeros_like(U)
    if kind == "linear":
        return rp[0] * U
    if kind == "allen_cahn":
        return U - U ** 3
    if kind == "fhn":
        c3, eps, a, b = rp
        return np.stack([U[0] - c3 * U[0] ** 3 - U[1], eps * (U[0] - a * U[1] - b)])
    raise ValueError(kind)


def react_vjp(kind, rp, U, V):
    """J_f(U)^T V."""
    if kind == "none":
        return np.zeros_like(V)
    if kind == "linear":
        return rp[0] * V
    if kind == "allen_cahn":
        return (1 - 3 * U ** 2) * V
    if kind == "fhn":
        c3, eps, a, b = rp
        return np.stack([(1 - 3 * c3 * U[0] ** 2) * V[0] + eps * V[1], -V[0] - eps * a * V[1]])
    raise ValueError(kind)


def react_dtheta(kind, rp, U, V):
    """<V, d f(U) / d theta> for every reaction parameter theta (list)."""
    if kind == "linear":
        return [float(np.sum(V * U))]
    if kind == "fhn":
        c3, eps, a, b = rp
        return [float(np.sum(V[0] * -U[0] ** 3)), float(np.sum(V[1] * (U[0] - a * U[1] - b))),
                float(np.sum(V[1] * -eps * U[1])), float(np.sum(V[1] * -eps))]
    return []


def forward_step(problem, ops, U):
    kind, rp, tau = problem.reaction, tuple(problem.rp), problem.tau
    F = react(kind, rp, U)
    SU = np.stack([o.S(U[c]) for c, o in enumerate(ops)])
    SF = np.stack([o.S(F[c]) for c, o in enumerate(ops)])
    W = np.stack([o.X(1, SU[c]) + tau * o.X(2, SF[c]) for c, o in enumerate(ops)])
    G = react(kind, rp, W) - SF
    Un = np.stack([W[c] + tau * o.X(3, G[c]) for c, o in enumerate(ops)])
    return Un, dict(F=F, W=W, G=G)


def adjoint_step(problem, ops, U, Ubar_next):
    """(Ubar, dL/dkappa per component, dL/dtheta) for one step from state U."""
    kind, rp, tau = problem.reaction, tuple(problem.rp), problem.tau
    _, fw = forward_step(problem, ops, U)
    F, W, G = fw["F"], fw["W"], fw["G"]
    Gbar = np.stack([tau * o.X(3, Ubar_next[c]) for c, o in enumerate(ops)])
    Wbar = Ubar_next + react_vjp(kind, rp, W, Gbar)
    Fbar = np.stack([tau * o.X(2, o.S(Wbar[c])) - o.S(Gbar[c]) for c, o in enumerate(ops)])
    Ubar = np.stack([o.X(1, o.S(Wbar[c])) for c, o in enumerate(ops)]) + react_vjp(kind, rp, U, Fbar)
    gk = []
    for c, o in enumerate(ops):
        dX1SU = o.X(1, o.S(U[c]), deriv=True) + o.X(1, o.dS(U[c]))
        dX2SF = o.X(2, o.S(F[c]), deriv=True) + o.X(2, o.dS(F[c]))
        gk.append(float(np.sum(Ubar_next[c] * tau * o.X(3, G[c], deriv=True)) - np.sum(Gbar[c] * o.dS(F[c])) +
                        np.sum(Wbar[c] * (dX1SU + tau * dX2SF))))
    gth = [x + y for x, y in zip(react_dtheta(kind, rp, W, Gbar), react_dtheta(kind, rp, U, Fbar))]
    return Ubar, gk, gth


def run(problem, u0, nsteps):
    """Forward trajectory [U^0 .. U^N] with the same operators the adjoint uses."""
    ops = [_Ops(problem, k) for k in problem.kappa]
    traj = [np.array(u0, dtype=np.float64)]
    for _ in range(nsteps):
        traj.append(forward_step(problem, ops, traj[-1])[0])
    return traj


def adjoint_run(problem, u0, nsteps, ubar_final):
    """Ubar^0 and the accumulated parameter gradients of L with dL/dU^N = ubar_final."""
    ops = [_Ops(problem, k) for k in problem.kappa]
    traj = [np.array(u0, dtype=np.float64)]
    for _ in range(nsteps - 1):
        traj.append(forward_step(problem, ops, traj[-1])[0])
    ubar = np.array(ubar_final, dtype=np.float64)
    gk = np.zeros(len(ops))
    gth = None
    for step in reversed(range(nsteps)):
        ubar, gk_s, gth_s = adjoint_step(problem, ops, traj[step], ubar)
        gk += gk_s
        gth = np.array(gth_s) if gth is None else gth + np.array(gth_s)
    return ubar, gk, (gth if gth is not None else np.zeros(0))
