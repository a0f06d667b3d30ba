"""Seeded synthetic workloads (tube descriptions and initial states). No step of the method lives here.

Each workload is a list of ``TubeSpec``: grid, quadrature orders, relaxation time, time step and an initial
condition, either Riemann data (left/right states of Eq. (condinit), section "Riemann problem") or per-cell
(P, n, v) arrays. Tests feed the same specs to the CUDA path and to the oracle; the benchmark times them.

Workloads (sizes as stated):
  * ``sod_small``: the paper's Sod tube (P, n, v) = (1, 1, 0) | (0.1, 0.125, 0) on x in [-0.5, 0.5],
    Nx = 400, Qp = 3, Qxi = 8 (24 velocities), tau = 1e-3, CFL 0.5 (dt = min(1.25e-3, 0.9 tau) = 9e-4,
    444 steps to t = 0.4).
  * ``sod_sweep``: the relaxation-time sweep, Nx = 4096, tau in {1e-4, 1e-3, 1e-2, 1e-1, 1, 10, inf} x
    Qxi in {8, 32, 128, 200}, Qp = 3: 28 tubes, 31.65 M velocity nodes; dt = min(0.5 dx, 0.9 tau).
  * ``batched_tubes``: 256 tubes, seed 160803004: Nx ~ U[1024, 16384], log10 tau ~ U[-4, 1],
    Qxi in {8, 16, 32, 64}, P_L ~ U[0.5, 2], P_R = P_L U(0.01, 0.5), n_L = P_L, n_R = P_R / 0.8 (the paper
    is silent on n; this keeps its T_L = 1, T_R = 0.8 and reproduces (1, 0.125) at P = (1, 0.1));
    dt = min(0.5 dx, 0.45 tau) (the strong shocks reach |v| ~ 0.8).
  * ``gaussian_bumps``: Nx = 2048, Qxi = 32, per-cell pressure 1 + sum of seed-fixed Gaussian bumps of
    relative amplitude 0.05, n = P, v = 0; ``perturbed`` multiplies P and n by a second seed-fixed set of
    bumps (the inverse problem's target state).
  * ``stress``: one Sod tube, Nx = 1,048,576, Qxi = 128 (384 velocities), tau = 1e-2.
  * ``random_smooth``: seeded smooth periodic (P, n, v) profiles for parity tests.
  * ``fast_flow``: smooth periodic states whose speed reaches vmax (0.9 .. 0.99), where the Landau-frame
    extraction of e and u^mu cancels; ``rarefied``: P and n down to 1e-4 of their largest value.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence

import numpy as np

SOD_LEFT = (1.0, 1.0, 0.0)
SOD_RIGHT = (0.1, 0.125, 0.0)
BC_OPEN, BC_PERIODIC = 0, 1
SWEEP_TAUS = (1e-4, 1e-3, 1e-2, 1e-1, 1.0, 10.0, math.inf)
SWEEP_QXI = (8, 32, 128, 200)
BATCH_SEED = 160803004


@dataclasses.dataclass
class TubeSpec:
    Nx: int
    Qxi: int
    tau: float
    dt: float
    dx: float
    Qp: int = 3
    Np: int = 2
    Nv: int = 5
    bc: int = BC_OPEN
    x_left: float = -0.5
    left: Optional[Sequence[float]] = SOD_LEFT    # Riemann data ...
    right: Optional[Sequence[float]] = SOD_RIGHT
    P: Optional[np.ndarray] = None                # ... or per-cell (P, n, v)
    n: Optional[np.ndarray] = None
    v: Optional[np.ndarray] = None

    @property
    def Q(self) -> int:
        return self.Qp * self.Qxi

    @property
    def riemann(self) -> bool:
        return self.P is None


STIFF_SOD = 0.9     # dt <= 0.9 tau: SSP-RK3 + WENO5 at CFL 0.5 stays stable up to |v| ~ 0.63
STIFF_STRONG = 0.45  # dt <= 0.45 tau: up to |v| ~ 0.9 (strong shocks of the batched workload)


def cfl_dt(dx: float, tau: float, cfl: float = 0.5, stiff: float = STIFF_SOD) -> float:
    """Time step rule of the workloads: min(cfl dx, stiff tau). With WENO5 advection at CFL 0.5 the SSP-RK3
    step is stable for collision stiffness dt gamma (1 + |v|) / tau <= 1.977, hence stiff <= 0.989 for |v| <= 0.6."""
    dt = cfl * dx
    if tau is not None and math.isfinite(tau) and tau > 0:
        dt = min(dt, stiff * tau)
    return dt


def sod_tube(Nx: int, Qxi: int, tau: float, Qp: int = 3, Np: int = 2, Nv: int = 5, cfl: float = 0.5,
             bc: int = BC_OPEN, x_left: float = -0.5, length: float = 1.0, left=SOD_LEFT,
             right=SOD_RIGHT, stiff: float = STIFF_SOD) -> TubeSpec:
    dx = length / Nx
    return TubeSpec(Nx=Nx, Qxi=Qxi, tau=tau, dt=cfl_dt(dx, tau, cfl, stiff), dx=dx, Qp=Qp, Np=Np, Nv=Nv, bc=bc,
                    x_left=x_left, left=tuple(left), right=tuple(right))


def sod_small() -> List[TubeSpec]:
    return [sod_tube(400, 8, 1e-3)]


def sod_sweep(Nx: int = 4096, taus=SWEEP_TAUS, qxis=SWEEP_QXI) -> List[TubeSpec]:
    return [sod_tube(Nx, q, t) for t in taus for q in qxis]


def batched_tubes(ntubes: int = 256, seed: int = BATCH_SEED) -> List[TubeSpec]:
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(ntubes):
        Nx = int(rng.integers(1024, 16384, endpoint=True))
        tau = float(10.0 ** rng.uniform(-4, 1))
        Qxi = int(rng.choice([8, 16, 32, 64]))
        PL = float(rng.uniform(0.5, 2.0))
        PR = PL * float(rng.uniform(0.01, 0.5))
        out.append(sod_tube(Nx, Qxi, tau, left=(PL, PL, 0.0), right=(PR, PR / 0.8, 0.0), stiff=STIFF_STRONG))
    return out


def gaussian_bumps(Nx: int = 2048, Qxi: int = 32, tau: float = 0.05, amplitude: float = 0.05, seed: int = 4,
                   nbumps: int = 5) -> TubeSpec:
    rng = np.random.default_rng(seed)
    dx = 1.0 / Nx
    x = -0.5 + (np.arange(Nx) + 0.5) * dx
    P = np.ones(Nx)
    for _ in range(nbumps):
        c, w = rng.uniform(-0.3, 0.3), rng.uniform(0.02, 0.08)
        P += amplitude * rng.uniform(0.5, 1.0) * np.exp(-0.5 * ((x - c) / w) ** 2)
    return TubeSpec(Nx=Nx, Qxi=Qxi, tau=tau, dt=cfl_dt(dx, tau), dx=dx, P=P, n=P.copy(), v=np.zeros(Nx))


def perturbed(base: TubeSpec, seed: int, amplitude: float = 0.05, nbumps: int = 5) -> TubeSpec:
    """The per-cell state of `base` with its pressure perturbed by seed-fixed Gaussian bumps of relative
    amplitude `amplitude` (n follows P, so the temperature is kept); the target of the inverse problem."""
    rng = np.random.default_rng(seed)
    x = base.x_left + (np.arange(base.Nx) + 0.5) * base.dx
    f = np.ones(base.Nx)
    for _ in range(nbumps):
        c, w = rng.uniform(-0.3, 0.3), rng.uniform(0.02, 0.08)
        f += amplitude * rng.uniform(0.5, 1.0) * np.exp(-0.5 * ((x - c) / w) ** 2)
    return dataclasses.replace(base, P=base.P * f, n=base.n * f, v=base.v.copy())


def stress(Nx: int = 1 << 20, Qxi: int = 128, tau: float = 1e-2) -> TubeSpec:
    return sod_tube(Nx, Qxi, tau)


def random_smooth(Nx: int, Qxi: int, tau: float, seed: int, bc: int = BC_PERIODIC, vmax: float = 0.5,
                  Qp: int = 3, Np: int = 2, Nv: int = 5, cfl: float = 0.5) -> TubeSpec:
    """Smooth random periodic profiles: P in [0.3, 1.7], n in [0.3, 1.7], |v| <= vmax (few Fourier modes)."""
    rng = np.random.default_rng(seed)
    dx = 1.0 / Nx
    x = (np.arange(Nx) + 0.5) * dx

    def field(amp):
        f = np.zeros(Nx)
        for k in range(1, 4):
            f += rng.uniform(-1, 1) * np.sin(2 * np.pi * k * x + rng.uniform(0, 2 * np.pi)) / k
        return amp * f / max(np.max(np.abs(f)), 1e-12)

    P = 1.0 + field(0.7)
    n = 1.0 + field(0.7)
    v = field(vmax)
    return TubeSpec(Nx=Nx, Qxi=Qxi, tau=tau, dt=cfl_dt(dx, tau, cfl), dx=dx, Qp=Qp, Np=Np, Nv=Nv, bc=bc,
                    x_left=0.0, P=P, n=n, v=v)


def _stiff_for(vmax: float, limit: float = 1.8) -> float:
    """dt / tau that keeps dt gamma (1 + vmax) / tau at `limit`, inside the SSP-RK3 + WENO5 stability bound
    (1.977 at CFL 0.5) for every direction of a flow of speed vmax."""
    return limit * math.sqrt(1.0 - vmax * vmax) / (1.0 + vmax)


def fast_flow(Nx: int, Qxi: int, tau: float, vmax: float, seed: int, uniform: bool = False,
              bc: int = BC_PERIODIC, stiff_limit: float = 0.25) -> TubeSpec:
    """Smooth periodic states at speeds up to vmax: v = vmax sin(2 pi x + phase) (both directions) with P and n
    varying by +-30 %, or with uniform=True a near-uniform flow v = vmax - 0.002 (1 + sin(2 pi x + phase)) with
    P and n varying by +-5 %. The time step keeps dt gamma (1 + vmax) / tau at stiff_limit: near |v| = 1 the
    collision rate gamma (1 - v xi) / tau grows with the speed it acts on, and steps at the linear stability
    bound (1.8 here) run away within a few steps at |v| >= 0.97."""
    rng = np.random.default_rng(seed)
    dx = 1.0 / Nx
    x = (np.arange(Nx) + 0.5) * dx
    ph = rng.uniform(0, 2 * np.pi, 3)
    amp = 0.05 if uniform else 0.3
    P = 1.0 + amp * np.sin(2 * np.pi * x + ph[0])
    n = 1.0 + amp * np.sin(4 * np.pi * x + ph[1])
    if uniform:
        v = vmax - 0.002 * (1.0 + np.sin(2 * np.pi * x + ph[2]))
    else:
        v = vmax * np.sin(2 * np.pi * x + ph[2])
    return TubeSpec(Nx=Nx, Qxi=Qxi, tau=tau, dt=cfl_dt(dx, tau, stiff=_stiff_for(vmax, stiff_limit)), dx=dx,
                    bc=bc, x_left=0.0, P=P, n=n, v=v)


def rarefied(Nx: int, Qxi: int, tau: float, seed: int, floor: float = 1e-4, vmax: float = 0.3,
             bc: int = BC_PERIODIC) -> TubeSpec:
    """Smooth periodic states with rarefied cells: P = floor^(1/2 + sin(2 pi x + phase)/2) spans [floor, 1]
    on a log scale, n = P / T with T = 1 + 0.2 sin(...), |v| <= vmax."""
    rng = np.random.default_rng(seed)
    dx = 1.0 / Nx
    x = (np.arange(Nx) + 0.5) * dx
    ph = rng.uniform(0, 2 * np.pi, 3)
    P = floor ** (0.5 + 0.5 * np.sin(2 * np.pi * x + ph[0]))
    T = 1.0 + 0.2 * np.sin(2 * np.pi * x + ph[1])
    v = vmax * np.sin(2 * np.pi * x + ph[2])
    return TubeSpec(Nx=Nx, Qxi=Qxi, tau=tau, dt=cfl_dt(dx, tau, stiff=_stiff_for(vmax)), dx=dx, bc=bc,
                    x_left=0.0, P=P, n=P / T, v=v)


def strong_shock(Nx: int, Qxi: int, tau: float, ratio: float = 0.01) -> TubeSpec:
    """Riemann tube with P_R / P_L = ratio (the strongest shocks of the batched workload), the batch's n and
    time-step rules."""
    return sod_tube(Nx, Qxi, tau, left=(1.0, 1.0, 0.0), right=(ratio, ratio / 0.8, 0.0), stiff=STIFF_STRONG)


def total_nodes(specs: Sequence[TubeSpec]) -> int:
    """Velocity nodes per step, sum of Nx * Q."""
    return int(sum(s.Nx * s.Q for s in specs))
