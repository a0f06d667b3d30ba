"""Gradients of an oracle run by central differences.

TEST INFRASTRUCTURE ONLY, under the same rules as the rest of ``oracle/``: only ``tests/``, ``smoke()`` and
bench.py's CPU legs may use it, and it imports nothing from the CUDA package.

A run is the oracle's: F0 = F^eq of per-cell (P, n, v) (Eq. (condinit) with Eq. (feqtrunc)), nsteps SSP-RK3
steps of Eq. (Boltz) with the time step dt held fixed, then the fields of every cell (section "Relativistic
lattice Boltzmann equation"): the five conserved moments N^0, N^z, T^00, T^0z, T^zz (rows = 5, the default)
or those and the Landau-frame e, beta, n (rows = 8). A loss is any function of those rows. The gradient is
the definition of the derivative evaluated with a finite step:
    dL/dq ~ (L(q + h) - L(q - h)) / (2h),
for q = log(tau) or one cell's P, n or v. Its truncation error is h^2 L'''/6 and its rounding error about
eps_machine |L| / h, i.e. about 1e-9 of |L| at h = 1e-6; the oracle's own arithmetic is not changed.
"""
from __future__ import annotations

import math

import numpy as np

from . import Params, fields, init, step


def _with_tau(p: Params, tau: float) -> Params:
    """Same run parameters (dt included) with another relaxation time."""
    return Params(p.Qp, p.Qxi, p.Np, p.Nv, p.Nx, p.dx, p.dt, tau, p.bc)


def run_moments(p: Params, P, n, v, nsteps: int, rows: int = 5) -> np.ndarray:
    """[rows][Nx] fields (the conserved moments, then e, beta, n) after nsteps steps from F^eq(P, n, v)."""
    F = step(p, init(p, P, n, v), nsteps)
    return fields(p, F)[:rows]


def run_moments_from_state(p: Params, F0, nsteps: int) -> np.ndarray:
    """[5][Nx] conserved moments after nsteps steps from the state F0 [Q][Nx]."""
    return fields(p, step(p, F0, nsteps))[:5]


def grad_log_tau(p: Params, P, n, v, nsteps: int, loss, h: float = 1e-6, rows: int = 5) -> float:
    """dL/dlog(tau) at fixed dt by central differences (the oracle's tau must be finite and positive)."""
    lt = math.log(p.tau)
    lp = loss(run_moments(_with_tau(p, math.exp(lt + h)), P, n, v, nsteps, rows))
    lm = loss(run_moments(_with_tau(p, math.exp(lt - h)), P, n, v, nsteps, rows))
    return (lp - lm) / (2.0 * h)


def grad_log_tau_from_state(p: Params, F0, nsteps: int, loss, h: float = 1e-6) -> float:
    """dL/dlog(tau) at fixed dt and fixed initial state F0, by central differences."""
    lt = math.log(p.tau)
    lp = loss(run_moments_from_state(_with_tau(p, math.exp(lt + h)), F0, nsteps))
    lm = loss(run_moments_from_state(_with_tau(p, math.exp(lt - h)), F0, nsteps))
    return (lp - lm) / (2.0 * h)


def grad_field(p: Params, P, n, v, nsteps: int, loss, which: str, cells, h: float = 1e-6,
               rows: int = 5) -> np.ndarray:
    """dL/dq(x) for q in {"P", "n", "v"} at the given cells, by central differences."""
    base = {"P": np.array(P, dtype=np.float64), "n": np.array(n, dtype=np.float64),
            "v": np.array(v, dtype=np.float64)}
    out = np.zeros(len(cells))
    for k, x in enumerate(cells):
        vals = []
        for sgn in (1.0, -1.0):
            f = {key: arr.copy() for key, arr in base.items()}
            f[which][x] += sgn * h
            vals.append(loss(run_moments(p, f["P"], f["n"], f["v"], nsteps, rows)))
        out[k] = (vals[0] - vals[1]) / (2.0 * h)
    return out
