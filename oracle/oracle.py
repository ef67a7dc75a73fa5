"""ctypes front end of the plain CPU oracle (etd_oracle.c).

TEST INFRASTRUCTURE. Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
module. The product library never calls it.

The oracle advances the Pade ETD2RK-DS scheme (eq. (13)-(16) of Section 3.1)
with one LU/Thomas solve per 1D line per pole (Section 3.3.1), in the order of
Algorithm 1 (2D) and Algorithm 2 (3D), in FP64; the same code built in FP32 is
the "shadow" used to measure the error floor of FP32 storage.

Reaction kinds and their parameters ``rp``:

===================  ===============================================  =====================
kind                 f                                                rp
===================  ===============================================  =====================
``none``             0                                                --
``linear``           c u (each component)                             (c,)
``allen_cahn``       u - u^3                                          --
``fhn``              (u - c3 u^3 - v,  eps (u - a v - b))             (c3, eps, a, b)
``ac_manufactured``  u (1 - u^2) + psi(x, t), Example 5.1             (lambda,)
``singular``         rho u / (1 - u), Example 5.2                     (rho,)
===================  ===============================================  =====================
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass, field
from typing import Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_SOURCES = ("etd_oracle.c", "etd_oracle_step.h")

REACTIONS = {"none": 0, "linear": 1, "allen_cahn": 2, "fhn": 3, "ac_manufactured": 4, "singular": 5}


class _Problem(ctypes.Structure):
    _fields_ = [
        ("d", ctypes.c_int),
        ("n", ctypes.c_int),
        ("ncomp", ctypes.c_int),
        ("pade", ctypes.c_int),
        ("reaction", ctypes.c_int),
        ("pad_", ctypes.c_int),
        ("kappa", ctypes.c_double * 2),
        ("q", ctypes.c_double),
        ("tau", ctypes.c_double),
        ("rp", ctypes.c_double * 8),
    ]


@dataclass
class Problem:
    """One reaction-diffusion problem on (0,1)^d with n interior points per axis."""

    d: int
    n: int
    kappa: Sequence[float]
    q: float
    tau: float
    pade: int = 2
    reaction: str = "allen_cahn"
    rp: Sequence[float] = field(default_factory=tuple)

    @property
    def ncomp(self) -> int:
        return len(self.kappa)

    def shape(self):
        return (self.ncomp,) + (self.n,) * self.d

    def _c(self) -> _Problem:
        p = _Problem()
        p.d, p.n, p.ncomp, p.pade = self.d, self.n, self.ncomp, self.pade
        p.reaction = REACTIONS[self.reaction]
        for i, k in enumerate(self.kappa):
            p.kappa[i] = float(k)
        p.q, p.tau = float(self.q), float(self.tau)
        for i, v in enumerate(self.rp):
            p.rp[i] = float(v)
        return p


_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (C, OpenMP) into oracle/_build/liboracle.so."""
    os.makedirs(_BUILD, exist_ok=True)
    srcs = [os.path.join(_HERE, s) for s in _SOURCES]
    if not force and os.path.exists(_SO):
        so_t = os.path.getmtime(_SO)
        if all(os.path.getmtime(s) <= so_t for s in srcs):
            return _SO
    tmp = _SO + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=gnu11", "-fopenmp", "-fPIC", "-shared", "-o", tmp, srcs[0], "-lm"]
    subprocess.run(cmd, check=True, cwd=_HERE)
    os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            dp = ctypes.POINTER(ctypes.c_double)
            fp = ctypes.POINTER(ctypes.c_float)
            L.oracle_run_f64.argtypes = [ctypes.POINTER(_Problem), dp, ctypes.c_int, ctypes.c_double]
            L.oracle_run_f64.restype = ctypes.c_int
            L.oracle_run_f32.argtypes = [ctypes.POINTER(_Problem), fp, ctypes.c_int, ctypes.c_double]
            L.oracle_run_f32.restype = ctypes.c_int
            L.oracle_rational.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double]
            L.oracle_rational.restype = ctypes.c_double
            L.oracle_pade_data.argtypes = [ctypes.c_int, dp, dp, dp, dp]
            L.oracle_pade_data.restype = ctypes.c_int
            L.oracle_set_threads.argtypes = [ctypes.c_int]
            L.oracle_max_threads.restype = ctypes.c_int
            _lib = L
        return _lib


def set_threads(n: int) -> None:
    lib().oracle_set_threads(int(n))


def max_threads() -> int:
    return int(lib().oracle_max_threads())


def run(problem: Problem, u: np.ndarray, nsteps: int, t0: float = 0.0, precision: str = "f64") -> np.ndarray:
    """Return u advanced by ``nsteps`` steps of size tau from time t0.

    ``u`` has shape (ncomp, n, n) or (ncomp, n, n, n) in [comp][z][y][x] order
    (x fastest, Section 2.1 vectorisation). The input is not modified.
    """
    dt = np.float64 if precision == "f64" else np.float32
    out = np.ascontiguousarray(np.array(u, dtype=dt, copy=True)).reshape(problem.shape())
    p = problem._c()
    if precision == "f64":
        rc = lib().oracle_run_f64(ctypes.byref(p), out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), int(nsteps), float(t0))
    else:
        rc = lib().oracle_run_f32(ctypes.byref(p), out.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), int(nsteps), float(t0))
    if rc != 0:
        raise ValueError(f"oracle rejected the problem {problem}")
    return out


def rational(pade: int, ell: int, x: float) -> float:
    """E_ell(x) through the partial fractions the oracle uses."""
    return float(lib().oracle_rational(int(pade), int(ell), float(x)))


def pade_data(pade: int):
    """(poles, residues[ell][pole]) of the order-``pade`` factors, upper-half-plane poles."""
    s_re, s_im = (ctypes.c_double * 2)(), (ctypes.c_double * 2)()
    r_re, r_im = (ctypes.c_double * 6)(), (ctypes.c_double * 6)()
    npol = lib().oracle_pade_data(int(pade), s_re, s_im, r_re, r_im)
    poles = np.array([complex(s_re[p], s_im[p]) for p in range(npol)])
    res = np.array([[complex(r_re[l * 2 + p], r_im[l * 2 + p]) for p in range(npol)] for l in range(3)])
    return poles, res
