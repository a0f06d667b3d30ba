"""Pins for the oracle's quadrature (section "Discretization of the momentum space using quadrature rules").

Nodes and weights are checked against library routines (scipy, numpy) and against the exactness property
the paper states: the polar rule integrates powers of xi below 2 Qxi exactly, the radial rule (weight
pbar e^-pbar) integrates powers of pbar below 2 Qp exactly.
"""
import math

import numpy as np
import pytest
from numpy.polynomial import legendre as npleg
from scipy.special import eval_genlaguerre, roots_genlaguerre

import oracle


@pytest.mark.parametrize("Qp", [1, 2, 3, 4, 6])
def test_laguerre_nodes_weights_match_library(Qp):
    pbar, wp, _, _ = oracle.quadrature(Qp, 4)
    x, w = roots_genlaguerre(Qp, 1)
    np.testing.assert_allclose(pbar, x, rtol=1e-13)
    np.testing.assert_allclose(wp, w, rtol=1e-12)
    # nodes are zeros of L^(1)_Qp
    assert np.all(np.abs(eval_genlaguerre(Qp, 1, pbar)) < 1e-11 * np.maximum(1, pbar) ** Qp)


@pytest.mark.parametrize("Qxi", [1, 2, 4, 5, 6, 8, 16, 32])
def test_legendre_nodes_weights_match_library(Qxi):
    _, _, xi, wxi = oracle.quadrature(3, Qxi)
    x, w = npleg.leggauss(Qxi)
    np.testing.assert_allclose(xi, x, rtol=0, atol=2e-15)
    np.testing.assert_allclose(wxi, w, rtol=1e-12)
    c = np.zeros(Qxi + 1)
    c[-1] = 1
    assert np.max(np.abs(npleg.legval(xi, c))) < 1e-13


@pytest.mark.parametrize("Qxi", [64, 128, 200, 256])
def test_legendre_high_order_against_extended_precision(Qxi):
    """At high order numpy's weights carry ~1e-11 relative error near the ends; pin against mpmath."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 30
    _, _, xi, wxi = oracle.quadrature(3, Qxi)
    x, _ = npleg.leggauss(Qxi)
    np.testing.assert_allclose(xi, x, rtol=0, atol=2e-15)
    for j in list(range(0, Qxi, 17)) + [Qxi - 1]:
        r = mp.mpf(xi[j])
        for _ in range(6):  # Newton with P_n' = n (x P_n - P_{n-1}) / (x^2 - 1)
            p, pm = mp.legendre(Qxi, r), mp.legendre(Qxi - 1, r)
            r -= p * (r * r - 1) / (Qxi * (r * p - pm))
        w = 2 * (1 - r**2) / ((Qxi + 1) ** 2 * mp.legendre(Qxi + 1, r) ** 2)
        assert abs(xi[j] - float(r)) <= 2e-16
        assert abs(wxi[j] / float(w) - 1) < 2e-13


@pytest.mark.parametrize("Qp", [2, 3, 4])
def test_radial_rule_exactness(Qp):
    pbar, wp, _, _ = oracle.quadrature(Qp, 4)
    for k in range(2 * Qp):  # int_0^inf pbar^(k+1) e^-pbar = (k+1)!
        assert abs(np.sum(wp * pbar**k) - math.factorial(k + 1)) < 1e-12 * math.factorial(k + 1)


@pytest.mark.parametrize("Qxi", [4, 7, 8, 200])
def test_polar_rule_exactness(Qxi):
    _, _, xi, wxi = oracle.quadrature(3, Qxi)
    for k in range(2 * Qxi):
        exact = 2.0 / (k + 1) if k % 2 == 0 else 0.0
        assert abs(np.sum(wxi * xi**k) - exact) < 5e-14 * max(1.0, 2.0 / (k + 1)) * (1 + k)


def test_printed_polar_weight_is_garbled():
    """Eq. (polarInt) prints 2(1-xi_j)^2 in the numerator; with 2(1-xi_j^2) the rule is Gauss-Legendre.

    The printed form is not symmetric in xi and does not sum to 2, so the reading 1 - xi_j^2 is forced."""
    Qxi = 8
    _, _, xi, wxi = oracle.quadrature(3, Qxi)
    P9 = np.array([oracle.legendre_P(Qxi + 1, t) for t in xi])
    printed = 2 * (1 - xi) ** 2 / ((Qxi + 1) ** 2 * P9**2)
    read = 2 * (1 - xi**2) / ((Qxi + 1) ** 2 * P9**2)
    assert abs(printed.sum() - 2) > 0.1
    np.testing.assert_allclose(read, wxi, rtol=1e-13)


def test_invalid_orders_rejected():
    with pytest.raises(oracle.OracleError):
        oracle.quadrature(0, 8)
    with pytest.raises(oracle.OracleError):
        oracle.quadrature(3, 0)
