"""Pins for the oracle's central-difference gradients (oracle/gradient.py).

1. Uniform relaxation, closed form. A spatially uniform state at rest whose distribution is anisotropic but
   even in xi has no advection (equal neighbours give equal fluxes) and keeps beta = 0, n = N^0, e = T^00
   (the collision conserves N^mu and T^0mu, section "Relativistic lattice Boltzmann equation"), so F^eq is
   fixed and every SSP-RK3 step multiplies F - F^eq by R(z) = 1 + z + z^2/2 + z^3/6, z = -dt/tau. Hence
   T^zz_N = T^zz_eq + R^N (T^zz_0 - T^zz_eq), T^zz_eq = T^00/3, and dT^zz_N/dlog(tau) follows in closed form.
2. Conservation (periodic tube). Sum_x N^0, sum_x T^00 and sum_x T^0z are constant in time, so their
   gradients with respect to the initial fields are those of the initial moments of the perfect fluid:
   N^0 = n gamma, T^00 = (4 gamma^2 - 1) P, T^0z = 4 P gamma^2 v; at v = 0: dT^00/dP = 3, dN^0/dn = 1,
   dT^0z/dv = 4P, and none depends on tau.
"""
import math

import numpy as np
import pytest

import oracle
from oracle import gradient as og


def test_uniform_relaxation_log_tau_gradient_closed_form():
    Nx, Qxi, N = 6, 8, 8
    p = oracle.params(Qxi=Qxi, Nx=Nx, tau=0.03, dt=0.01, bc=oracle.BC_PERIODIC)
    feq = oracle.feq_cell(3, Qxi, 2, 5, 0.8, 1.3, 0.0)
    _, _, xi, _ = oracle.quadrature(3, Qxi)
    p2 = 0.5 * (3 * xi**2 - 1)  # Legendre P_2: even in xi, keeps T^0z = 0
    F0 = np.tile((feq * (1.0 + 0.08 * np.tile(p2, 3)))[:, None], (1, Nx))
    m0 = oracle.moments_cell(3, Qxi, F0[:, 0])
    T00, Tzz0 = m0[2], m0[4]
    assert abs(m0[3]) < 1e-15 * T00
    Tzz_eq = T00 / 3.0
    z = -p.dt / p.tau
    R = 1 + z + z * z / 2 + z**3 / 6
    dR = 1 + z + z * z / 2
    # the closed form of the state itself, checked first
    mN = og.run_moments_from_state(p, F0, N)
    np.testing.assert_allclose(mN[4], Tzz_eq + R**N * (Tzz0 - Tzz_eq), rtol=1e-13)
    exact = Nx * (Tzz0 - Tzz_eq) * N * R ** (N - 1) * dR * (p.dt / p.tau)
    loss = lambda m: float(np.sum(m[4]))  # noqa: E731
    got = og.grad_log_tau_from_state(p, F0, N, loss)
    # central-difference error budget: rounding eps |L| / h (about 1e-9 |L| at h = 1e-6) plus h^2 terms
    L = loss(mN)
    assert abs(got - exact) <= 1e-8 * abs(L) + 1e-7 * abs(exact), (got, exact)
    assert abs(exact) > 1e-3 * abs(L)  # the gradient is well above the error budget


@pytest.fixture(scope="module")
def smooth_run():
    Nx, Qxi = 16, 8
    x = (np.arange(Nx) + 0.5) / Nx
    P = 1.0 + 0.3 * np.sin(2 * np.pi * x) + 0.1 * np.cos(4 * np.pi * x)
    n = 1.0 + 0.2 * np.cos(2 * np.pi * x + 0.4)
    v = np.zeros(Nx)
    p = oracle.params(Qxi=Qxi, Nx=Nx, tau=0.05, dt=0.5 / Nx, bc=oracle.BC_PERIODIC)
    return p, P, n, v


@pytest.mark.parametrize("row,which,expected", [(2, "P", lambda P: 3.0 + 0 * P), (2, "n", lambda P: 0 * P),
                                                (0, "n", lambda P: 1.0 + 0 * P), (0, "P", lambda P: 0 * P),
                                                (3, "v", lambda P: 4.0 * P)])
def test_conserved_sums_have_the_initial_gradients(smooth_run, row, which, expected):
    p, P, n, v = smooth_run
    cells = [0, 5, 11]
    loss = lambda m: float(np.sum(m[row]))  # noqa: E731
    g = og.grad_field(p, P, n, v, 12, loss, which, cells)
    np.testing.assert_allclose(g, expected(P[cells]), rtol=1e-6, atol=1e-6)
    assert abs(og.grad_log_tau(p, P, n, v, 12, loss)) < 1e-6


def test_nonconserved_loss_depends_on_tau(smooth_run):
    """Sanity of the setting: a non-conserved moment does respond to tau (the pins above are not vacuous)."""
    p, P, n, v = smooth_run
    g = og.grad_log_tau(p, P, n, v, 12, lambda m: float(np.sum(m[4] ** 2)))
    assert abs(g) > 1e-4
    assert math.isfinite(g)
