"""Pins for the oracle's truncated equilibrium, Eq. (feqtrunc) built from Eq. (feqMJ).

* hhat_{m,k} (Legendre coefficients of (1 - beta xi)^-m) against brute-force extended-precision quadrature
  and against closed forms at k = 0 (2/(1-b^2), 2/(1-b^2)^2, (2 + 2b^2/3)/(1-b^2)^3 for the integrals).
* Exact recovery, Eq. (mom_feq): the quadrature moments of F^eq equal the perfect-fluid N^mu = n u^mu and
  T^{mu nu} = (e+P) u^mu u^nu + P g^{mu nu}, P = nT, e = 3P (section "Relativistic lattice Boltzmann
  equation"), for random states.
* Every moment int d^3p/p^0 pbar^a xi^b f^eq with a <= Np and b <= Nv equals the same moment of the
  untruncated Maxwell-Juttner distribution, integrated directly (mpmath) from Eq. (feqMJ).
"""
import math

import numpy as np
import pytest

import oracle

mp = pytest.importorskip("mpmath")
mp.mp.dps = 40


def brute_hhat(m, k, beta):
    f = lambda x: mp.legendre(k, x) * (1 - beta * x) ** (-m)
    return float((2 * k + 1) / mp.mpf(2) * mp.quad(f, [-1, 0, 1]))


@pytest.mark.parametrize("beta", [-0.9, -0.47, -0.1, 1e-3, 0.3, 0.6, 0.9])
def test_hhat_against_brute_force(beta):
    for m in (2, 3, 4):
        scale = max(1.0, abs(brute_hhat(m, 0, beta)))
        for k in range(8):
            assert abs(oracle.hhat(m, k, beta) - brute_hhat(m, k, beta)) <= 2e-15 * scale, (m, k)


@pytest.mark.parametrize("beta", [-0.95, -0.5, 0.0, 0.25, 0.7, 0.95])
def test_hhat_closed_forms_k0(beta):
    g2 = 1.0 / (1.0 - beta * beta)
    # (1/2) int (1 - b x)^-m dx for m = 2, 3, 4
    assert oracle.hhat(2, 0, beta) == pytest.approx(g2, rel=2e-15)
    assert oracle.hhat(3, 0, beta) == pytest.approx(g2**2, rel=2e-15)
    assert oracle.hhat(4, 0, beta) == pytest.approx((1 + beta * beta / 3) * g2**3, rel=2e-15)


def test_hhat_rest_frame_and_parity():
    for m in (2, 3, 4):
        assert oracle.hhat(m, 0, 0.0) == 1.0
        for k in range(1, 6):
            assert oracle.hhat(m, k, 0.0) == 0.0
            for b in (0.2, 0.8):  # h_m(xi; -b) = h_m(-xi; b)
                assert oracle.hhat(m, k, -b) == pytest.approx((-1) ** k * oracle.hhat(m, k, b), rel=1e-15)


def perfect_fluid(n, T, beta):
    g = 1.0 / math.sqrt(1 - beta * beta)
    P = n * T
    e = 3 * P
    return np.array([n * g, n * g * beta, (e + P) * g * g - P, (e + P) * g * g * beta, (e + P) * g * g * beta**2 + P])


@pytest.mark.parametrize("Qxi", [4, 6, 8, 32, 200])
def test_exact_moment_recovery(Qxi):
    rng = np.random.default_rng(1608 + Qxi)
    for _ in range(12):
        n = rng.uniform(0.05, 3.0)
        T = rng.uniform(0.3, 2.5)
        beta = rng.uniform(-0.95, 0.95)
        F = oracle.feq_cell(3, Qxi, 2, 5, n, T, beta)
        mom = oracle.moments_cell(3, Qxi, F)
        exp = perfect_fluid(n, T, beta)
        scale = np.array([exp[0], exp[0], exp[2], exp[2], exp[2]])
        assert np.all(np.abs(mom - exp) <= 3e-14 * scale), (n, T, beta, mom - exp)


def test_rest_frame_special_case():
    for n, T in [(1.0, 1.0), (0.125, 0.8), (2.0, 0.4)]:
        mom = oracle.moments_cell(3, 8, oracle.feq_cell(3, 8, 2, 5, n, T, 0.0))
        assert mom[0] == pytest.approx(n, rel=1e-14)
        assert mom[2] == pytest.approx(3 * n * T, rel=1e-14)
        assert abs(mom[1]) < 1e-15 and abs(mom[3]) < 1e-15
        assert mom[4] == pytest.approx(n * T, rel=1e-14)


def mj_moment(a, b, n, T, beta):
    """int d^3p/p^0 pbar^a xi^b f_MJ, f_MJ = n/(8 pi T^3) exp(-pbar gamma (1 - beta xi)/T), Eq. (feqMJ).

    d^3p/p^0 = pbar dpbar dxi dphi; the pbar integral is (a+1)! / Lambda^(a+2), Lambda = (1 - beta xi)/s,
    s = T/gamma; the xi integral is done by mpmath."""
    g = 1 / mp.sqrt(1 - mp.mpf(beta) ** 2)
    s = mp.mpf(T) / g
    ang = mp.quad(lambda x: x**b * (1 - beta * x) ** (-(a + 2)), [-1, 0, 1])
    return float(2 * mp.pi * n / (8 * mp.pi * mp.mpf(T) ** 3) * math.factorial(a + 1) * s ** (a + 2) * ang)


@pytest.mark.parametrize("beta", [-0.6, 0.0, 0.35, 0.8])
def test_truncated_moments_equal_maxwell_juttner(beta):
    n, T, Qxi = 0.7, 0.9, 12  # Nv + b < 2 Qxi and a + Np < 2 Qp keep every sum exact
    pbar, _, xi, _ = oracle.quadrature(3, Qxi)
    F = oracle.feq_cell(3, Qxi, 2, 5, n, T, beta).reshape(3, Qxi)
    for a in range(3):
        for b in range(6):
            got = np.sum(F * (pbar[:, None] ** a) * (xi[None, :] ** b))
            ref = mj_moment(a, b, n, T, beta)
            assert abs(got - ref) <= 1e-13 * max(abs(mj_moment(a, 0, n, T, beta)), 1e-300), (a, b, got, ref)


def test_truncation_is_not_the_full_distribution():
    """Moments beyond the truncation orders differ from Maxwell-Juttner (the projection is genuine)."""
    n, T, beta, Qxi = 0.7, 0.9, 0.6, 12
    pbar, _, xi, _ = oracle.quadrature(3, Qxi)
    F = oracle.feq_cell(3, Qxi, 2, 5, n, T, beta).reshape(3, Qxi)
    got = np.sum(F * pbar[:, None] * xi[None, :] ** 7)
    ref = mj_moment(1, 7, n, T, beta)
    assert abs(got - ref) > 1e-6 * abs(ref)


def test_feq_rejects_nonphysical():
    with pytest.raises(oracle.OracleError):
        oracle.feq_cell(3, 8, 2, 5, 1.0, 1.0, 1.0)
    with pytest.raises(oracle.OracleError):
        oracle.feq_cell(3, 8, 2, 5, -1.0, 1.0, 0.0)
