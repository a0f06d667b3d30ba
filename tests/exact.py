"""Closed-form solutions used to pin the oracle (independent of it and of the CUDA path).

* ``riemann_ideal``: exact Riemann solution of ideal relativistic hydrodynamics with P = e/3 for a left
  state and a right state at rest with P_L > P_R (rarefaction moving left, shock moving right). This is the
  tau -> 0 limit of the kinetic model (section "Numerical results", hydrodynamic regime).
  - Rarefaction: the Riemann invariant atanh(v) + (sqrt(3)/4) ln e is constant through the fan; inside it
    the C- characteristic passes through the origin, x/t = (v - c_s)/(1 - v c_s), c_s = 1/sqrt(3).
    Isentropic flow of the massless Boltzmann gas keeps T^3/n fixed, so n ~ e^(3/4).
  - Shock (P = e/3): in the shock frame the up- and down-stream speeds satisfy v1 v2 = 1/3; with the
    pre-shock gas at rest the shock moves at v1, the post-shock gas at v = (3 v1^2 - 1)/(2 v1) and
    P2/P1 = (9 v1^2 - 1)/(3 (1 - v1^2)); particle number across it: n2 = n1 gamma1 v1 / (gamma2 v2).
  - Contact: P and v continuous.
* ``n_ballistic``: the paper's Eq. (ballistic), density in the free-streaming limit.
* ``free_streaming_moments``: moments of the discrete-velocity free-streaming solution F_j(x - xi_j t, 0)
  for two-state initial data, given the quadrature (exact solution of the tau -> infinity equation).
"""
from __future__ import annotations

import numpy as np
from scipy.optimize import brentq

CS = 1.0 / np.sqrt(3.0)


def _shock_from_v1(v1, PR):
    P2 = PR * (9 * v1 * v1 - 1) / (3 * (1 - v1 * v1))
    vpost = (3 * v1 * v1 - 1) / (2 * v1)
    return P2, vpost


def riemann_ideal(PL, nL, PR, nR, xt):
    """(e, v, n) at self-similar coordinate xt = x/t for the Sod-type problem (both states at rest)."""
    assert PL > PR > 0
    eL = 3 * PL

    def v_rare(P):
        return np.tanh(np.sqrt(3.0) / 4.0 * np.log(eL / (3 * P)))

    def mismatch(v1):
        P2, vpost = _shock_from_v1(v1, PR)
        return v_rare(P2) - vpost

    v1 = brentq(mismatch, CS * (1 + 1e-12), 1 - 1e-12, xtol=1e-15, rtol=1e-15, maxiter=500)
    Pstar, vstar = _shock_from_v1(v1, PR)
    estar = 3 * Pstar
    # densities
    nL_star = nL * (estar / eL) ** 0.75
    v2 = 1.0 / (3 * v1)
    g1, g2 = 1 / np.sqrt(1 - v1 * v1), 1 / np.sqrt(1 - v2 * v2)
    nR_star = nR * g1 * v1 / (g2 * v2)
    xt = np.asarray(xt, dtype=float)
    e = np.empty_like(xt)
    v = np.empty_like(xt)
    n = np.empty_like(xt)
    head = -CS
    tail = (vstar - CS) / (1 - vstar * CS)
    for k, s in np.ndenumerate(xt):
        if s <= head:
            e[k], v[k], n[k] = eL, 0.0, nL
        elif s <= tail:
            vv = (s + CS) / (1 + s * CS)
            ee = eL * np.exp(-4.0 / np.sqrt(3.0) * np.arctanh(vv))
            e[k], v[k], n[k] = ee, vv, nL * (ee / eL) ** 0.75
        elif s <= vstar:
            e[k], v[k], n[k] = estar, vstar, nL_star
        elif s <= v1:
            e[k], v[k], n[k] = estar, vstar, nR_star
        else:
            e[k], v[k], n[k] = 3 * PR, 0.0, nR
    return e, v, n, dict(Pstar=Pstar, vstar=vstar, vshock=v1, tail=tail, head=head)


def n_ballistic(z, t, nL, nR):
    """Eq. (ballistic): density profile in the free-streaming regime."""
    z = np.asarray(z, dtype=float)
    a = z / t
    inner = np.sqrt(((nL + nR) / 2 - (nL - nR) / 2 * a) ** 2 - ((nL - nR) / 4) ** 2 * (1 - a * a) ** 2)
    return np.where(z < -t, nL, np.where(z > t, nR, inner))


def free_streaming_moments(pbar, wp, xi, wxi, nL, TL, nR, TR, z, t):
    """(N0, Nz, T00, T0z, Tzz) of F_j(z - xi_j t, 0) for rest-frame equilibria left/right of z = 0.

    At rest the projected equilibrium needs no angular projection (h_m = 1), so
    F_ij = n/(4 T^3) w^p_i w^xi_j (s^2 L_0 + ...) with s = T: the radial projection of exp(-pbar (1/T - 1))
    onto L^(1)_l, l <= 2, written out from the Laguerre generating function. Computed here independently.
    """
    def feq_rest(n, T):
        lam = 1.0 / T
        A = [(lam - 1) ** l / lam ** (l + 2) for l in range(3)]
        L = [np.ones_like(pbar), 2 - pbar, 0.5 * (pbar * pbar - 6 * pbar + 6)]
        rad = sum(A[l] * L[l] for l in range(3))
        return n / (4 * T ** 3) * (wp * rad)[:, None] * wxi[None, :]

    FL, FR = feq_rest(nL, TL), feq_rest(nR, TR)
    z = np.atleast_1d(np.asarray(z, dtype=float))
    out = np.zeros((5, z.size))
    P = pbar[:, None]
    X = xi[None, :]
    for k, zz in enumerate(z):
        left = (zz - xi * t) < 0
        F = np.where(left[None, :], FL, FR)
        out[:, k] = [(F * P).sum(), (F * P * X).sum(), (F * P * P).sum(), (F * P * P * X).sum(),
                     (F * P * P * X * X).sum()]
    return out
