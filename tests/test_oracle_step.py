"""Pins for the oracle's full time step (Eq. (Boltz) with WENO5 + SSP-RK3, section "Numerical results").

* The collision conserves N^mu and T^{mu nu} (Landau frame, Landau density).
* One SSP-RK3 step of a spatially uniform state relaxes F - F^eq by exactly the stability polynomial
  1 + z + z^2/2 + z^3/6, z = -dt gamma (1 - beta xi_j) / tau, of the Shu-Osher scheme.
* Periodic grids conserve sum_x N^0, T^00 and T^0z to round-off (flux form + conservative collision).
* Mirror symmetry x -> -x, xi -> -xi.
* Ballistic regime (tau -> infinity): converges to the exact discrete free-streaming solution.
* Hydrodynamic regime (tau -> 0): approaches the exact ideal-hydro (P = e/3) Riemann solution.
* The paper's printed shock width at tau = 1e-4, dz = 1e-4, Qxi = 6 (golden fixture).
"""
import json
import math
import os

import numpy as np
import pytest

import exact
import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def uniform_state(rng, Qxi, Nx, beta_target=0.3):
    """A spatially uniform, non-equilibrium state: an equilibrium plus a positive random perturbation."""
    F = oracle.feq_cell(3, Qxi, 2, 5, 0.8, 0.9, beta_target)
    F = F * (1 + 0.3 * rng.uniform(-1, 1, F.size))
    return np.repeat(F[:, None], Nx, axis=1)


def conserved(p, F):
    f = oracle.fields(p, F)
    return np.array([f[0].sum(), f[2].sum(), f[3].sum()])


def test_collision_conserves_moments():
    rng = np.random.default_rng(21)
    Qxi, Nx = 8, 6
    p = oracle.params(Qxi=Qxi, Nx=Nx, tau=1e-3, bc=oracle.BC_PERIODIC)
    F = uniform_state(rng, Qxi, Nx)
    L = oracle.rhs(p, F)
    pbar, _, xi, _ = oracle.quadrature(3, Qxi)
    P = np.repeat(pbar, Qxi)[:, None]
    X = np.tile(xi, 3)[:, None]
    rate_scale = np.abs(L).max() * F.shape[0] * 10
    # N^0, T^00 and T^0z are conserved; N^z and T^zz are not
    for w in (P, P * P, P * P * X):
        assert np.max(np.abs((L * w).sum(axis=0))) < 1e-14 * rate_scale
    assert np.max(np.abs((L * P * X).sum(axis=0))) > 1e-3
    # and the collision is genuinely active
    assert np.abs(L).max() > 1.0


def test_rk3_relaxation_factor():
    """F0 = F^eq + delta with delta orthogonal to (1 - beta xi)^k pbar^a xi^b (a = 1, 2; b <= 2; k <= 3), so
    that no stage changes N^mu or T^{mu nu}, the Landau frame stays put and each velocity relaxes linearly."""
    rng = np.random.default_rng(22)
    Qxi, Nx, tau, n, T, beta = 8, 4, 1e-3, 0.8, 0.9, 0.45
    p = oracle.params(Qxi=Qxi, Nx=Nx, dx=1.0 / 64, dt=1.1e-3, tau=tau, bc=oracle.BC_PERIODIC)
    pbar, _, xi, _ = oracle.quadrature(3, Qxi)
    P = np.repeat(pbar, Qxi)
    X = np.tile(xi, 3)
    rows = [P**a * X**b * (1 - beta * X) ** k for a in (1, 2) for b in range(3) for k in range(4)]
    _, _, Vt = np.linalg.svd(np.array(rows))
    null = Vt[np.linalg.matrix_rank(np.array(rows)):]
    Feq = oracle.feq_cell(3, Qxi, 2, 5, n, T, beta)
    delta = null.T @ rng.normal(size=null.shape[0])
    delta *= 0.2 * Feq.min() / np.abs(delta).max()
    F0 = np.repeat((Feq + delta)[:, None], Nx, axis=1)
    np.testing.assert_allclose(oracle.landau(oracle.moments_cell(3, Qxi, F0[:, 0]))[1:], [beta, n, T], rtol=1e-13)
    F1 = oracle.step(p, F0, 1)
    g = 1 / math.sqrt(1 - beta * beta)
    z = -p.dt * g * (1 - beta * X) / tau
    R = 1 + z + z * z / 2 + z**3 / 6
    # round-off of F itself bounds the comparison; a wrong RK weight or rate would miss by ~|delta| ~ 1e-6
    np.testing.assert_allclose(F1[:, 0] - Feq, R * delta, rtol=0, atol=2e-15 * np.abs(Feq).max())
    assert np.abs(delta).max() > 1e8 * 2e-15 * np.abs(Feq).max()
    assert np.max(np.abs(F1 - F1[:, :1])) == 0.0  # uniform state stays uniform


def sod_periodic_state(Nx):
    x = (np.arange(Nx) + 0.5) / Nx
    P = np.where(np.abs(x - 0.5) < 0.25, 1.0, 0.1) * (1 + 0.1 * np.sin(2 * np.pi * x))
    n = np.where(np.abs(x - 0.5) < 0.25, 1.0, 0.125)
    v = 0.2 * np.sin(4 * np.pi * x)
    return P, n, v


@pytest.mark.parametrize("tau", [1e-2, np.inf])
def test_periodic_conservation(tau):
    Nx, Qxi = 96, 8
    p = oracle.params(Qxi=Qxi, Nx=Nx, tau=tau, bc=oracle.BC_PERIODIC)
    F = oracle.init(p, *sod_periodic_state(Nx))
    c0 = conserved(p, F)
    G = oracle.step(p, F, 150)
    c1 = conserved(p, G)
    assert np.max(np.abs(c1 - c0) / np.abs(c0).max()) < 1e-13
    assert np.max(np.abs(G - F)) > 1e-3  # the state did evolve


def test_mirror_symmetry():
    Nx, Qxi = 64, 8
    p = oracle.params(Qxi=Qxi, Nx=Nx, tau=1e-2)
    x = -0.5 + (np.arange(Nx) + 0.5) / Nx
    P = 1.0 + 0.5 * np.tanh(10 * x) + 0.2 * np.exp(-200 * (x - 0.1) ** 2)
    n = 1.0 - 0.3 * np.tanh(8 * x)
    v = 0.3 * np.exp(-100 * x * x)
    F = oracle.init(p, P, n, v)
    Fm = oracle.init(p, P[::-1], n[::-1], -v[::-1])
    G = oracle.step(p, F, 30)
    Gm = oracle.step(p, Fm, 30)
    # mirror: x -> Nx-1-x and xi_j -> xi_{Qxi-1-j}
    Gm_back = Gm.reshape(3, Qxi, Nx)[:, ::-1, ::-1].reshape(3 * Qxi, Nx)
    np.testing.assert_allclose(G, Gm_back, rtol=1e-12, atol=1e-14 * np.abs(G).max())


def test_ballistic_converges_to_free_streaming():
    Qxi, t = 8, 0.2
    pbar, wp, xi, wxi = oracle.quadrature(3, Qxi)
    errs = []
    for Nx in (100, 400):
        p = oracle.params(Qxi=Qxi, Nx=Nx, tau=np.inf)
        F = oracle.init_riemann(p)
        steps = int(round(t / p.dt))
        G = oracle.step(p, F, steps)
        f = oracle.fields(p, G)
        x = -0.5 + (np.arange(Nx) + 0.5) / Nx
        ref = exact.free_streaming_moments(pbar, wp, xi, wxi, 1.0, 1.0, 0.125, 0.8, x, steps * p.dt)
        errs.append(np.mean(np.abs(f[:5] - ref), axis=1))
    errs = np.array(errs)
    # first-order-like convergence at the moving jumps (L1 error ~ dx^0.8)
    assert np.all(errs[1] < 0.45 * errs[0]), errs
    assert np.all(errs[1] < 3e-3 * np.array([1.0, 1.0, 3.0, 3.0, 3.0])), errs


def test_ballistic_continuum_is_eckart_density():
    """Eq. (ballistic) is the Eckart density sqrt(N0^2 - Nz^2) of free streaming; its gap to the discrete
    free-streaming solution shrinks as Qxi grows and is small at Qxi = 200 (Fig. 1(b) caption)."""
    z = np.linspace(-0.24, 0.24, 25)
    t = 0.25
    gaps = []
    for Qxi in (16, 64, 200):
        pbar, wp, xi, wxi = oracle.quadrature(3, Qxi)
        m = exact.free_streaming_moments(pbar, wp, xi, wxi, 1.0, 1.0, 0.125, 0.8, z, t)
        nE = np.sqrt(m[0] ** 2 - m[1] ** 2)
        gaps.append(np.max(np.abs(nE - exact.n_ballistic(z, t, 1.0, 0.125))))
    assert gaps[0] > gaps[1] > gaps[2]
    assert gaps[2] < 5e-3


@pytest.mark.slow
def test_hydro_limit_approaches_ideal_riemann_solution():
    Nx, t = 400, 0.4
    xs = -0.5 + (np.arange(Nx) + 0.5) / Nx
    e_ex, v_ex, n_ex, _ = exact.riemann_ideal(1.0, 1.0, 0.1, 0.125, xs / t)
    errs = {}
    for tau in (1e-2, 1e-3):
        p = oracle.params(Qxi=8, Nx=Nx, tau=tau)
        F = oracle.init_riemann(p)
        G = oracle.step(p, F, int(round(t / p.dt)))
        f = oracle.fields(p, G)
        errs[tau] = np.array([np.mean(np.abs(f[5] - e_ex)), np.mean(np.abs(f[6] - v_ex)),
                              np.mean(np.abs(f[7] - n_ex))])
    assert np.all(errs[1e-3] < 0.6 * errs[1e-2]), errs
    assert np.all(errs[1e-3] < np.array([0.02, 0.006, 0.01])), errs


@pytest.mark.slow
def test_paper_shock_width():
    """Section "Numerical results": at tau = 1e-4, dt = 0.5e-4, L_z = 10000 (dz = 1e-4), Np = 2, Nv = 5,
    Qxi = 6 the shock is about 6-7 grid nodes wide. Run on a window around the membrane; signals travel at
    speed <= 1, so at t = 0.02 the window edges (0.02 and 0.03 away) see only the undisturbed states."""
    with open(os.path.join(GOLDEN, "paper_values.json")) as fh:
        g = json.load(fh)["shock_width"]
    dx, Nx = 1.0 / g["L_z"], 500
    p = oracle.params(Qxi=g["Qxi"], Np=g["N_p"], Nv=g["N_v"], Nx=Nx, dx=dx, dt=g["dt"], tau=g["tau"])
    F = oracle.init_riemann(p, xleft=-0.02)
    G = oracle.step(p, F, 400)
    e = oracle.fields(p, G)[5]
    x = -0.02 + (np.arange(Nx) + 0.5) * dx
    _, _, _, info = exact.riemann_ideal(1.0, 1.0, 0.1, 0.125, np.array([0.0]))
    estar, eR = 3 * info["Pstar"], 0.3
    frac = (e - eR) / (estar - eR)
    right = x > 0.5 * (info["vstar"] + info["vshock"]) * 0.02  # beyond the contact
    width = int(np.sum(right & (frac > 0.02) & (frac < 0.98)))
    lo, hi = g["nodes"]
    assert lo - 2 <= width <= hi + 2, width


def test_paper_initial_states():
    with open(os.path.join(GOLDEN, "paper_values.json")) as fh:
        g = json.load(fh)["riemann"]
    assert g["n_L"] - g["n_R"] == pytest.approx(g["delta_n"])
    p = oracle.params(Qxi=8, Nx=4)
    F = oracle.init_riemann(p, left=(g["P_L"], g["n_L"], g["u_L"]), right=(g["P_R"], g["n_R"], g["u_R"]))
    f = oracle.fields(p, F)
    np.testing.assert_allclose(f[7], [1.0, 1.0, 0.125, 0.125], rtol=1e-14)
    np.testing.assert_allclose(f[5], [3.0, 3.0, 0.3, 0.3], rtol=1e-14)


def test_strong_shock_with_many_directions_stays_physical():
    """A 60:1 density jump with Qxi = 64 (weak collisions): WENO5 limited on the weight-normalised populations
    keeps every cell physical; with eps fixed on the weighted populations the small-weight directions fall back
    to the linear scheme and its undershoot drives the low-density moments negative at the first step."""
    Nx, Qxi, tau = 64, 64, 1.72e-2
    dx = 1.0 / 10000
    p = oracle.params(Qxi=Qxi, Nx=Nx, dx=dx, dt=0.5 * dx, tau=tau)
    F = oracle.init_riemann(p, left=(1.53, 1.53, 0.0), right=(0.0245, 0.0306, 0.0), xleft=-32 * dx)
    G = oracle.step(p, F, 30)
    f = oracle.fields(p, G)
    assert np.all(f[5] > 0) and np.all(f[7] > 0) and np.all(np.abs(f[6]) < 1)
