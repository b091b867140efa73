"""FP64 CPU oracle for the Runge–Kutta DG method with the jump filter (arXiv 2407.19169).

TEST INFRASTRUCTURE ONLY: the test-suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` use this package. The CUDA library never imports, links or calls it. The C sources
(``orc_*.c``) follow the paper's steps in its order and notation; this module only marshals numpy
arrays through ctypes.

Parity status per function (see the tests under ``tests/`` for each pin):
  - Legendre values/derivatives, Gauss rules: pinned to closed forms.
  - Projection: pinned by exact reproduction of polynomials.
  - DG residual, SSP-RK3: pinned by convergence orders, conservation, L2 energy decay, and by the
    paper's Table 1 "without filter" errors.
  - Jump filter (1D and 2D): pinned by hand-computed single-cell factors and by the paper's Table 1
    "with filter" errors.
  - Exact Riemann solver: pinned by Rankine–Hugoniot and isentropic relations.
"""
from __future__ import annotations

import ctypes as C
import dataclasses
import os

import numpy as np

from . import build as _build

EQ_ADVECTION, EQ_BURGERS, EQ_EULER = 0, 1, 2
BC_PERIODIC, BC_OUTFLOW = 0, 1
BASIS_Q, BASIS_P = 0, 1
IC_SINE, IC_RIEMANN1D, IC_ENTROPY1D, IC_QUADRANT2D, IC_VORTEX2D, IC_ZERO = range(6)
EX_BURGERS, EX_ADVECTION, EX_RIEMANN1D, EX_ENTROPY1D, EX_VORTEX2D = range(5)
FILTER_JUMP, FILTER_GLOBAL, FILTER_OEDG = range(3)


class _Problem(C.Structure):
    _fields_ = [("dim", C.c_int), ("nx", C.c_int), ("ny", C.c_int),
                ("x0", C.c_double), ("x1", C.c_double), ("y0", C.c_double), ("y1", C.c_double),
                ("bc", C.c_int * 4), ("k", C.c_int), ("basis", C.c_int), ("eq", C.c_int),
                ("gamma", C.c_double), ("adv", C.c_double * 2), ("filter", C.c_int),
                ("cfl", C.c_double), ("nq", C.c_int), ("filter_dt_mode", C.c_int), ("positivity", C.c_int),
                ("hybrid", C.c_int), ("filter_kind", C.c_int), ("filter_study", C.c_int)]


@dataclasses.dataclass
class Problem:
    dim: int = 1
    nx: int = 16
    ny: int = 1
    x0: float = 0.0
    x1: float = 1.0
    y0: float = 0.0
    y1: float = 1.0
    bc: tuple = (BC_PERIODIC,) * 4
    k: int = 2
    basis: int = BASIS_Q
    eq: int = EQ_BURGERS
    gamma: float = 1.4
    adv: tuple = (1.0, 0.0)
    filter: int = 1
    cfl: float = 0.1
    nq: int = 0
    filter_dt_mode: int = 0
    positivity: int = 0
    hybrid: int = 0
    filter_kind: int = 0
    filter_study: int = 0

    def c(self) -> _Problem:
        s = _Problem()
        for f in dataclasses.fields(self):
            val = getattr(self, f.name)
            if f.name == "bc":
                s.bc = (C.c_int * 4)(*val)
            elif f.name == "adv":
                s.adv = (C.c_double * 2)(*val)
            else:
                setattr(s, f.name, val)
        return s

    @property
    def nvars(self) -> int:
        return (3 if self.dim == 1 else 4) if self.eq == EQ_EULER else 1

    @property
    def nmodes(self) -> int:
        if self.dim == 1:
            return self.k + 1
        if self.basis == BASIS_P:
            return (self.k + 1) * (self.k + 2) // 2
        return (self.k + 1) ** 2

    @property
    def ncell(self) -> int:
        return self.nx * (self.ny if self.dim == 2 else 1)

    @property
    def shape(self):
        return (self.nvars, self.nmodes, self.ncell)

    @property
    def hx(self) -> float:
        return (self.x1 - self.x0) / self.nx

    @property
    def hy(self) -> float:
        return (self.y1 - self.y0) / self.ny if self.dim == 2 else 1.0


_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        D, I, P = C.c_double, C.c_int, C.POINTER(_Problem)
        dp = C.POINTER(C.c_double)
        sig = {
            "orc_legendre": (D, [I, D]), "orc_legendre_deriv": (D, [I, I, D]),
            "orc_gauss": (I, [I, dp, dp]), "orc_legendre_norm": (D, [I]),
            "orc_flux": (None, [P, I, dp, dp]), "orc_wave_speed": (D, [P, I, dp]),
            "orc_enthalpy": (D, [P, dp]), "orc_pressure": (D, [P, dp]),
            "orc_project": (I, [P, I, dp, I, I, dp]), "orc_max_rate": (D, [P, dp]),
            "orc_dt": (D, [P, dp, D, D]), "orc_residual": (None, [P, dp, dp]),
            "orc_filter": (None, [P, dp, D, dp]), "orc_filter_sigma": (None, [P, dp, dp]),
            "orc_positivity": (None, [P, dp]),
            "orc_oedg_norms": (None, [P, dp, dp]),
            "orc_jump_indicator": (None, [P, dp, dp]), "orc_hybrid": (None, [P, dp, D, dp]),
            "orc_rk_stage": (None, [P, I, dp, dp, D, dp]), "orc_step": (I, [P, dp, D]),
            "orc_advance": (I, [P, dp, D, D, C.c_long, dp, C.POINTER(C.c_long)]),
            "orc_check_physical": (I, [P, dp]), "orc_mass": (None, [P, dp, dp]),
            "orc_energy": (D, [P, dp]),
            "orc_burgers_exact": (D, [D, D, D, D, D, D, D]),
            "orc_riemann_exact": (I, [D, dp, dp, D, dp]),
            "orc_vortex_exact": (None, [D, D, D, D, D, D, D, D, D, D, D, dp]),
            "orc_errors": (I, [P, dp, I, dp, I, D, I, I, dp, dp, dp]),
            "orc_eval": (None, [P, dp, I, D, D, dp]),
            "orc_set_threads": (None, [I]), "orc_get_threads": (I, []),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _dp(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _arr(x) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(x, dtype=np.float64))


def set_threads(n: int) -> None:
    lib().orc_set_threads(int(n))


def legendre(n, x):
    return lib().orc_legendre(int(n), float(x))


def legendre_deriv(n, m, x):
    return lib().orc_legendre_deriv(int(n), int(m), float(x))


def gauss(n):
    x = np.zeros(n)
    w = np.zeros(n)
    if lib().orc_gauss(int(n), _dp(x), _dp(w)):
        raise ValueError("bad Gauss order")
    return x, w


def legendre_norm(n):
    return lib().orc_legendre_norm(int(n))


def flux(p: Problem, direction: int, u):
    u = _arr(u)
    f = np.zeros(p.nvars)
    pc = p.c()
    lib().orc_flux(C.byref(pc), int(direction), _dp(u), _dp(f))
    return f


def wave_speed(p: Problem, direction: int, u):
    u = _arr(u)
    pc = p.c()
    return lib().orc_wave_speed(C.byref(pc), int(direction), _dp(u))


def enthalpy(p: Problem, u):
    u = _arr(u)
    pc = p.c()
    return lib().orc_enthalpy(C.byref(pc), _dp(u))


def zeros(p: Problem) -> np.ndarray:
    return np.zeros(p.shape)


def project(p: Problem, ic: int, params, nq_init: int = 0) -> np.ndarray:
    u = zeros(p)
    prm = _arr(params if len(params) else [0.0])
    pc = p.c()
    if lib().orc_project(C.byref(pc), int(ic), _dp(prm), len(params), int(nq_init), _dp(u)):
        raise ValueError("bad initial condition for this problem")
    return u


def max_rate(p: Problem, u) -> float:
    u = _arr(u)
    pc = p.c()
    return lib().orc_max_rate(C.byref(pc), _dp(u))


def dt(p: Problem, u, t: float = 0.0, T: float = float("inf")) -> float:
    u = _arr(u)
    pc = p.c()
    return lib().orc_dt(C.byref(pc), _dp(u), float(t), float(T))


def residual(p: Problem, u) -> np.ndarray:
    u = _arr(u)
    R = np.zeros_like(u)
    pc = p.c()
    lib().orc_residual(C.byref(pc), _dp(u), _dp(R))
    return R


def filter(p: Problem, u, dt_: float) -> np.ndarray:  # noqa: A001 - the paper's name
    u = _arr(u)
    out = np.zeros_like(u)
    pc = p.c()
    lib().orc_filter(C.byref(pc), _dp(u), float(dt_), _dp(out))
    return out


def oedg_norms(p: Problem, u) -> np.ndarray:
    """||u_v - avg(u_v)||_inf per variable (the OEDG coefficient's normaliser)."""
    u = _arr(u)
    out = np.zeros(p.nvars)
    pc = p.c()
    lib().orc_oedg_norms(C.byref(pc), _dp(u), _dp(out))
    return out


def positivity(p: Problem, u) -> np.ndarray:
    """Zhang–Shu positivity-preserving limiter applied to a copy of u."""
    u = _arr(u).copy()
    pc = p.c()
    lib().orc_positivity(C.byref(pc), _dp(u))
    return u


def jump_indicator(p: Problem, u) -> np.ndarray:
    """eta_j of Algorithm 1 per cell (first conservative variable)."""
    u = _arr(u)
    eta = np.zeros(p.ncell)
    pc = p.c()
    lib().orc_jump_indicator(C.byref(pc), _dp(u), _dp(eta))
    return eta


def hybrid(p: Problem, u, dt_: float) -> np.ndarray:
    """u^hyd of Algorithm 1 from a DG solution u: troubled cells blended with the jump filter."""
    u = _arr(u)
    out = np.zeros_like(u)
    pc = p.c()
    lib().orc_hybrid(C.byref(pc), _dp(u), float(dt_), _dp(out))
    return out


def filter_sigma(p: Problem, u) -> np.ndarray:
    """sigma per (mode, cell): 1D sigma_j^l, 2D sigma^{p,q}."""
    u = _arr(u)
    s = np.zeros((p.nmodes, p.ncell))
    pc = p.c()
    lib().orc_filter_sigma(C.byref(pc), _dp(u), _dp(s))
    return s


def rk_stage(p: Problem, s: int, un, us, dt_: float) -> np.ndarray:
    un, us = _arr(un), _arr(us)
    out = np.zeros_like(us)
    pc = p.c()
    lib().orc_rk_stage(C.byref(pc), int(s), _dp(un), _dp(us), float(dt_), _dp(out))
    return out


def step(p: Problem, u, dt_: float) -> np.ndarray:
    u = _arr(u).copy()
    pc = p.c()
    if lib().orc_step(C.byref(pc), _dp(u), float(dt_)):
        raise FloatingPointError("non-physical state")
    return u


def advance(p: Problem, u, t0: float, T: float, max_steps: int = 1 << 62):
    u = _arr(u).copy()
    t = C.c_double(0.0)
    n = C.c_long(0)
    pc = p.c()
    rc = lib().orc_advance(C.byref(pc), _dp(u), float(t0), float(T), int(max_steps), C.byref(t), C.byref(n))
    if rc:
        raise FloatingPointError("non-physical state after %d steps" % n.value)
    return u, t.value, n.value


def check_physical(p: Problem, u) -> bool:
    u = _arr(u)
    pc = p.c()
    return lib().orc_check_physical(C.byref(pc), _dp(u)) == 0


def mass(p: Problem, u) -> np.ndarray:
    u = _arr(u)
    m = np.zeros(p.nvars)
    pc = p.c()
    lib().orc_mass(C.byref(pc), _dp(u), _dp(m))
    return m


def energy(p: Problem, u) -> float:
    u = _arr(u)
    pc = p.c()
    return lib().orc_energy(C.byref(pc), _dp(u))


def burgers_exact(x, t, a, b, w, phi, L):
    return lib().orc_burgers_exact(float(x), float(t), float(a), float(b), float(w), float(phi), float(L))


def riemann_exact(gamma, WL, WR, xi):
    WL, WR = _arr(WL), _arr(WR)
    W = np.zeros(3)
    if lib().orc_riemann_exact(float(gamma), _dp(WL), _dp(WR), float(xi), _dp(W)):
        raise ValueError("vacuum")
    return W


def vortex_exact(gamma, x0, y0, beta, Lx, Ly, x, y, t):
    W = np.zeros(4)
    lib().orc_vortex_exact(float(gamma), float(x0), float(y0), float(beta), float(Lx), float(Ly),
                           0.0, 0.0, float(x), float(y), float(t), _dp(W))
    return W


def errors(p: Problem, u, kind: int, params, t: float, var: int = 0, nq_err: int = 0):
    """(L1, L2, Linf) of variable ``var`` against an exact solution, unnormalised integrals."""
    u = _arr(u)
    prm = _arr(params)
    l1, l2, li = C.c_double(), C.c_double(), C.c_double()
    pc = p.c()
    if lib().orc_errors(C.byref(pc), _dp(u), int(kind), _dp(prm), len(params), float(t), int(nq_err),
                        int(var), C.byref(l1), C.byref(l2), C.byref(li)):
        raise ValueError("bad exact-solution request")
    return l1.value, l2.value, li.value


def evaluate(p: Problem, u, cell: int, xi: float, eta: float = 0.0) -> np.ndarray:
    u = _arr(u)
    val = np.zeros(p.nvars)
    pc = p.c()
    lib().orc_eval(C.byref(pc), _dp(u), int(cell), float(xi), float(eta), _dp(val))
    return val


__all__ = [n for n in dir() if not n.startswith("_")]
os.environ.setdefault("OMP_WAIT_POLICY", "PASSIVE")
