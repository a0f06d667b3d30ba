"""Plain FP64 CPU oracle for the relativistic lattice Boltzmann time step (arXiv:1608.03004).

TEST INFRASTRUCTURE ONLY. The oracle checks the CUDA path; it is not part of it. Only ``tests/``,
``__graft_entry__.smoke()`` and the ``cpu_baseline`` leg / ``--impl reference`` arm of ``bench.py`` may
import it. It shares no code with ``paper_1608_03004_gb300`` and imports nothing from it.

The arithmetic lives in ``rlb_oracle.c`` (plain C, one function per step of the method, each citing the
paper's section or equation); this module only compiles it with gcc and marshals numpy arrays.

Every function here has a pin in ``tests/test_oracle_*.py`` against something other than the oracle
itself (library quadrature, brute-force integrals, closed forms, conservation, exact solutions).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rlb_oracle.c")
_LIB = os.path.join(_HERE, "liborc.so")
_lock = threading.Lock()
_lib = None

OK, EINVAL, ENOMEM, ENONPHYS = 0, 1, 2, 4
BC_OPEN, BC_PERIODIC = 0, 1
FIELDS = ("N0", "Nz", "T00", "T0z", "Tzz", "e", "beta", "n")


class OracleError(RuntimeError):
    pass


class Params(ctypes.Structure):
    _fields_ = [
        ("Qp", ctypes.c_int),
        ("Qxi", ctypes.c_int),
        ("Np", ctypes.c_int),
        ("Nv", ctypes.c_int),
        ("Nx", ctypes.c_int),
        ("dx", ctypes.c_double),
        ("dt", ctypes.c_double),
        ("tau", ctypes.c_double),
        ("bc", ctypes.c_int),
    ]


def build(force: bool = False) -> str:
    """Compile rlb_oracle.c into liborc.so next to it (plain -O2, no fast-math)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fno-fast-math", "-ffp-contract=off",
               "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            dp = ctypes.POINTER(ctypes.c_double)
            pp = ctypes.POINTER(Params)
            lib.orc_quadrature.argtypes = [ctypes.c_int, ctypes.c_int, dp, dp, dp, dp]
            lib.orc_legendre_P.argtypes = [ctypes.c_int, ctypes.c_double]
            lib.orc_legendre_P.restype = ctypes.c_double
            lib.orc_laguerre1_L.argtypes = [ctypes.c_int, ctypes.c_double]
            lib.orc_laguerre1_L.restype = ctypes.c_double
            lib.orc_moments_cell.argtypes = [ctypes.c_int, ctypes.c_int, dp, dp, dp, ctypes.c_long, dp]
            lib.orc_landau.argtypes = [dp, dp]
            lib.orc_hhat.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double]
            lib.orc_hhat.restype = ctypes.c_double
            lib.orc_feq_cell.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, dp, dp, dp, dp,
                                         ctypes.c_double, ctypes.c_double, ctypes.c_double, dp, ctypes.c_long]
            lib.orc_weno5.argtypes = [ctypes.c_double] * 5
            lib.orc_weno5.restype = ctypes.c_double
            lib.orc_weno5_population.argtypes = [ctypes.c_double] * 6
            lib.orc_weno5_population.restype = ctypes.c_double
            lib.orc_weno5_indicators.argtypes = [ctypes.c_double] * 5 + [dp]
            lib.orc_rhs.argtypes = [pp, dp, dp]
            lib.orc_step.argtypes = [pp, dp, ctypes.c_long]
            lib.orc_init.argtypes = [pp, dp, dp, dp, dp]
            lib.orc_fields.argtypes = [pp, dp, dp]
            lib.orc_init_riemann.argtypes = [pp, ctypes.c_double, dp, dp]
            _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _check(st: int, what: str):
    if st != OK:
        raise OracleError(f"{what} failed with status {st}")


def quadrature(Qp: int, Qxi: int):
    """(pbar, w^p, xi, w^xi): generalised Gauss-Laguerre (alpha=1) and Gauss-Legendre, ascending."""
    lib = _load()
    pbar, wp = np.zeros(Qp), np.zeros(Qp)
    xi, wxi = np.zeros(Qxi), np.zeros(Qxi)
    _check(lib.orc_quadrature(Qp, Qxi, _ptr(pbar), _ptr(wp), _ptr(xi), _ptr(wxi)), "quadrature")
    return pbar, wp, xi, wxi


def legendre_P(n: int, x: float) -> float:
    return _load().orc_legendre_P(n, x)


def laguerre1_L(n: int, x: float) -> float:
    return _load().orc_laguerre1_L(n, x)


def moments_cell(Qp: int, Qxi: int, F: np.ndarray) -> np.ndarray:
    """(N0, Nz, T00, T0z, Tzz) of one cell's populations F[s], s = i*Qxi + j."""
    pbar, _, xi, _ = quadrature(Qp, Qxi)
    F = np.ascontiguousarray(F, dtype=np.float64)
    out = np.zeros(5)
    _load().orc_moments_cell(Qp, Qxi, _ptr(pbar), _ptr(xi), _ptr(F), 1, _ptr(out))
    return out


def landau(mom) -> np.ndarray:
    """(e, beta, n, T) from (N0, Nz, T00, T0z, Tzz)."""
    mom = np.ascontiguousarray(mom, dtype=np.float64)
    out = np.zeros(4)
    _check(_load().orc_landau(_ptr(mom), _ptr(out)), "landau")
    return out


def hhat(m: int, k: int, beta: float) -> float:
    """(2k+1)/2 * int_{-1}^{1} P_k(xi) (1 - beta xi)^(-m) dxi."""
    return _load().orc_hhat(m, k, beta)


def feq_cell(Qp: int, Qxi: int, Np: int, Nv: int, n: float, T: float, beta: float) -> np.ndarray:
    """Truncated, quadrature-weighted equilibrium F^eq[s] of one cell."""
    pbar, wp, xi, wxi = quadrature(Qp, Qxi)
    out = np.zeros(Qp * Qxi)
    _check(_load().orc_feq_cell(Qp, Qxi, Np, Nv, _ptr(pbar), _ptr(wp), _ptr(xi), _ptr(wxi), n, T, beta,
                                _ptr(out), 1), "feq_cell")
    return out


def weno5(vm2, vm1, v0, vp1, vp2) -> float:
    """Jiang-Shu WENO5 interface value (eps = 1e-6), samples in wind order."""
    return _load().orc_weno5(vm2, vm1, v0, vp1, vp2)


def weno5_population(ws, vm2, vm1, v0, vp1, vp2) -> float:
    """WENO5 of a population whose quadrature weight factor is ws (the scheme on F / ws, scaled back)."""
    return _load().orc_weno5_population(ws, vm2, vm1, v0, vp1, vp2)


def weno5_indicators(vm2, vm1, v0, vp1, vp2) -> np.ndarray:
    """The smoothness indicators (beta_0, beta_1, beta_2) of the three candidate stencils, samples in wind
    order."""
    out = np.zeros(3)
    _load().orc_weno5_indicators(vm2, vm1, v0, vp1, vp2, _ptr(out))
    return out


def params(Qp=3, Qxi=8, Np=2, Nv=5, Nx=400, dx=None, dt=None, tau=1e-3, bc=BC_OPEN) -> Params:
    """Run parameters; the default time step is min(0.5 dx, 0.9 tau), the stable rule for SSP-RK3 with WENO5
    advection and stiff relaxation at |v| <= 0.63 (tests/test_stability.py)."""
    dx = 1.0 / Nx if dx is None else dx
    tau = 0.0 if (tau is None or not np.isfinite(tau)) else tau
    if dt is None:
        dt = 0.5 * dx if tau <= 0 else min(0.5 * dx, 0.9 * tau)
    return Params(Qp, Qxi, Np, Nv, Nx, dx, dt, tau, bc)


def init(p: Params, P, n, v) -> np.ndarray:
    """F[Q][Nx] = F^eq of the per-cell state (P, n, v), Eq. (condinit)."""
    P, n, v = (np.ascontiguousarray(a, dtype=np.float64) for a in (P, n, v))
    F = np.zeros((p.Qp * p.Qxi, p.Nx))
    _check(_load().orc_init(ctypes.byref(p), _ptr(P), _ptr(n), _ptr(v), _ptr(F)), "init")
    return F


def init_riemann(p: Params, left=(1.0, 1.0, 0.0), right=(0.1, 0.125, 0.0), xleft=-0.5) -> np.ndarray:
    """Riemann data (P, n, v) left/right of x = 0 on cell centres; a centre on x = 0 takes the mean F."""
    st = np.array(list(left) + list(right), dtype=np.float64)
    F = np.zeros((p.Qp * p.Qxi, p.Nx))
    _check(_load().orc_init_riemann(ctypes.byref(p), float(xleft), _ptr(st), _ptr(F)), "init_riemann")
    return F


def step(p: Params, F: np.ndarray, nsteps: int) -> np.ndarray:
    """nsteps SSP-RK3 steps; returns a new array."""
    F = np.array(F, dtype=np.float64, order="C", copy=True)
    _check(_load().orc_step(ctypes.byref(p), _ptr(F), int(nsteps)), "step")
    return F


def rhs(p: Params, F: np.ndarray) -> np.ndarray:
    F = np.ascontiguousarray(F, dtype=np.float64)
    L = np.zeros_like(F)
    _check(_load().orc_rhs(ctypes.byref(p), _ptr(F), _ptr(L)), "rhs")
    return L


def fields(p: Params, F: np.ndarray) -> np.ndarray:
    """[8][Nx]: N0, Nz, T00, T0z, Tzz, e, beta, n (Landau)."""
    F = np.ascontiguousarray(F, dtype=np.float64)
    out = np.zeros((8, p.Nx))
    _check(_load().orc_fields(ctypes.byref(p), _ptr(F), _ptr(out)), "fields")
    return out
