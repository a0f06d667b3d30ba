"""Pins for the oracle's Landau-frame solve and WENO5 reconstruction.

Landau frame (section "Relativistic lattice Boltzmann equation", T^mu_nu u^nu = -e u^mu): the closed form is
checked against a library eigen-solver on generic (non-equilibrium) tensors and by a round trip through the
perfect-fluid form. WENO5 (section "Numerical results", cited Jiang-Shu scheme): checked against the linear
fifth-order upwind formula it must reduce to, against exact reconstruction of linear data, and against the
ENO property on a step.
"""
import math

import numpy as np
import pytest

import oracle


def random_moments(rng, Qxi=8):
    F = rng.uniform(0.0, 1.0, 3 * Qxi) * rng.uniform(0.01, 1.0)
    return oracle.moments_cell(3, Qxi, F)


def test_landau_matches_eigensolver():
    rng = np.random.default_rng(7)
    for _ in range(200):
        mom = random_moments(rng)
        N0, Nz, T00, T0z, Tzz = mom
        e, beta, n, T = oracle.landau(mom)
        M = np.array([[-T00, T0z], [-T0z, Tzz]])  # T^mu_nu, signature (-,+)
        w, V = np.linalg.eig(M)
        # the eigenvector with u^0 > |u^z| (timelike) belongs to eigenvalue -e
        ok = [k for k in range(2) if abs(V[0, k]) > abs(V[1, k])]
        assert len(ok) == 1
        k = ok[0]
        assert -w[k].real == pytest.approx(e, rel=1e-13)
        assert V[1, k].real / V[0, k].real == pytest.approx(beta, rel=1e-12, abs=1e-15)
        g = 1 / math.sqrt(1 - beta * beta)
        assert n == pytest.approx(g * (N0 - beta * Nz), rel=1e-15)
        assert T == pytest.approx(e / (3 * n), rel=1e-15)
        # residual of T^mu_nu u^nu = -e u^mu
        u = np.array([g, g * beta])
        assert np.max(np.abs(M @ u + e * u)) < 1e-13 * T00


def test_landau_round_trip():
    rng = np.random.default_rng(11)
    for _ in range(100):
        n, T, beta = rng.uniform(0.05, 3), rng.uniform(0.2, 3), rng.uniform(-0.97, 0.97)
        g = 1 / math.sqrt(1 - beta**2)
        P = n * T
        e = 3 * P
        mom = [n * g, n * g * beta, 4 * P * g * g - P, 4 * P * g * g * beta, 4 * P * g * g * beta**2 + P]
        out = oracle.landau(mom)
        np.testing.assert_allclose(out, [e, beta, n, T], rtol=1e-12, atol=1e-15)


def test_landau_rejects_nonphysical():
    with pytest.raises(oracle.OracleError):
        oracle.landau([1.0, 0.0, 1.0, 2.0, 1.0])  # |T0z| > (T00 + Tzz)/2
    with pytest.raises(oracle.OracleError):
        oracle.landau([1.0, 0.0, -1.0, 0.0, 0.0])


def linear_weno(vm2, vm1, v0, vp1, vp2):
    return (2 * vm2 - 13 * vm1 + 47 * v0 + 27 * vp1 - 3 * vp2) / 60.0


def test_weno_reduces_to_linear_scheme_for_tiny_data():
    """When beta_k << eps the nonlinear weights are the linear ones (1, 6, 3)/10: fifth-order upwind."""
    rng = np.random.default_rng(3)
    for _ in range(100):
        v = 1e-9 * rng.normal(size=5)
        got = oracle.weno5(*v)
        assert got == pytest.approx(linear_weno(*v), rel=1e-6, abs=1e-22)


def test_weno_exact_on_linear_data():
    """Linear data make all smoothness indicators equal, so the interface value is exact."""
    rng = np.random.default_rng(4)
    for _ in range(100):
        a, g = rng.normal(), rng.normal() * 10
        v = [a + g * k for k in (-2, -1, 0, 1, 2)]
        assert oracle.weno5(*v) == pytest.approx(a + 0.5 * g, rel=1e-13, abs=1e-13)


def test_weno_constant_preserved():
    for c in (0.0, 1.0, -3.5, 1e-7):
        assert oracle.weno5(c, c, c, c, c) == pytest.approx(c, rel=1e-15, abs=0)


def test_weno_eno_on_step():
    """A jump between v0 and vp1: only the fully upwind stencil (v_-2..v_0) is smooth and it dominates."""
    assert abs(oracle.weno5(0, 0, 0, 1, 1) - 0.0) < 1e-10
    assert abs(oracle.weno5(1, 1, 1, 0, 0) - 1.0) < 1e-10
    # a jump between v_-1 and v_0: the reconstruction stays within the data range (no overshoot > 1e-10)
    r = oracle.weno5(0, 0, 1, 1, 1)
    assert -1e-10 <= r <= 1 + 1e-10


def test_weno_mirror_symmetry():
    rng = np.random.default_rng(5)
    for _ in range(50):
        v = rng.normal(size=5)
        # reflecting the data and the wind gives the same interface value
        a = oracle.weno5(*v)
        b = oracle.weno5(*v[::-1])
        c = oracle.weno5(*(-v))
        assert c == pytest.approx(-a, rel=1e-14, abs=1e-14)
        assert np.isfinite(b)


def test_population_weno_is_the_scheme_on_normalised_values():
    """The population form applies the eps = 1e-6 scheme to F / ws and scales the result back."""
    rng = np.random.default_rng(6)
    for _ in range(200):
        ws = 10.0 ** rng.uniform(-6, 0)
        g = rng.normal(size=5) * 10.0 ** rng.uniform(-3, 1)
        got = oracle.weno5_population(ws, *(ws * g))
        assert got == pytest.approx(ws * oracle.weno5(*g), rel=1e-12, abs=1e-300)
