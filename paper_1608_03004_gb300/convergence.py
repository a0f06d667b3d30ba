"""The paper's convergence study in the quadrature order (section "Numerical results", Eq. (err), Fig. 2(b)).

For each relaxation time tau, Sod tubes with several polar orders Qxi are advanced to the same time in one
handle; the density n(x) of each is compared with the profile of a reference order (Qxi = 200 in the paper):
    epsilon(Qxi, tau) = max_x |n(x) - n_ref(x)| / Delta n,   Delta n = n_L - n_R = 0.875.
The paper prints "max{z}" in Eq. (err); it is read as the maximum over the grid of the absolute deviation.
n is the Landau density of the model (the density that enters the equilibrium). The default grid is the
paper's: L_z = 10000 nodes on the unit domain with dt = 0.5e-4 (CFL 0.5); on coarser grids (dx > tau) the
shock is not resolved and sub-cell shifts between orders dominate epsilon at small tau.

    python -m paper_1608_03004_gb300.convergence          # prints the table (needs a GPU)
"""
from __future__ import annotations

import math
from typing import Dict, Sequence

import numpy as np

from . import binding as rb
from . import workloads as W

DELTA_N = W.SOD_LEFT[1] - W.SOD_RIGHT[1]  # 0.875
DEFAULT_TAUS = (1e-4, 1e-3, 1e-2, 1e-1, 1.0)
DEFAULT_QXI = (4, 6, 8, 12, 16, 24, 32, 48, 64)


def density_profiles(tau: float, qxis: Sequence[int], Nx: int, t_end: float, storage: int = rb.STORAGE_F64):
    """Landau density of Sod tubes with the given polar orders at t_end (one handle, one launch per stage)."""
    specs = [W.sod_tube(Nx, q, tau) for q in qxis]
    dt = specs[0].dt
    nsteps = int(round(t_end / dt))
    tubes = [rb.Tube(s.Qp, s.Qxi, s.Np, s.Nv, s.Nx, s.dx, s.dt, s.tau if math.isfinite(s.tau) else math.inf,
                     s.bc, storage) for s in specs]
    states = np.array([list(s.left) + list(s.right) for s in specs])
    with rb.rlb_init_riemann(tubes, states, np.array([s.x_left for s in specs])) as h:
        rb.rlb_step(h, nsteps)
        f = rb.rlb_moments(h)
    n = f[rb.FIELDS.index("n")].reshape(len(qxis), Nx)
    return {q: n[k] for k, q in enumerate(qxis)}, nsteps * dt


def epsilon_table(taus: Sequence[float] = DEFAULT_TAUS, qxis: Sequence[int] = DEFAULT_QXI, qxi_ref: int = 200,
                  Nx: int = 10000, t_end: float = 0.25) -> Dict[float, Dict[int, float]]:
    """epsilon(Qxi, tau) of Eq. (err) against the Qxi = qxi_ref profile."""
    out = {}
    for tau in taus:
        prof, _ = density_profiles(tau, list(qxis) + [qxi_ref], Nx, t_end)
        ref = prof[qxi_ref]
        out[tau] = {q: float(np.max(np.abs(prof[q] - ref)) / DELTA_N) for q in qxis}
    return out


def smallest_converged(table_row: Dict[int, float], threshold: float = 0.01):
    """Smallest order whose epsilon is below the threshold and stays below it for every larger order."""
    qs = sorted(table_row)
    for k, q in enumerate(qs):
        if all(table_row[p] < threshold for p in qs[k:]):
            return q
    return None


if __name__ == "__main__":
    tab = epsilon_table()
    qs = list(next(iter(tab.values())).keys())
    print("tau \\ Qxi " + " ".join(f"{q:>8d}" for q in qs) + "   converged at")
    for tau, row in tab.items():
        print(f"{tau:9.0e} " + " ".join(f"{row[q]:8.4f}" for q in qs) + f"   {smallest_converged(row)}")
