"""Pins for the oracle's WENO5 reconstruction against the definition of the cited scheme.

The paper only cites its fifth-order WENO scheme (section "Numerical results"); the oracle reads it as the
Jiang-Shu scheme. These tests rebuild every part of that scheme from its definition with numpy polynomials,
independently of the oracle's written-out coefficients:
  - candidate k is the quadratic whose cell averages (cell width h = 1) match the data on stencil k, evaluated
    at the downwind face of the centre cell;
  - its smoothness indicator is beta_k = sum_{l=1,2} h^(2l-1) int_cell (d^l p_k / dx^l)^2 dx over the centre
    cell;
  - the linear weights d_k are the unique weights for which sum_k d_k p_k(face) is the face value of the
    quartic through all five cell averages (solved for here, not typed in);
  - alpha_k = d_k / (eps + beta_k)^2 with eps = 1e-6, w_k = alpha_k / sum alpha.
A convergence study on smooth periodic data measures the order of the whole scheme in the oracle's step.
Planted errors (a copy of the oracle with one constant of the indicators or the linear weights changed,
compiled on the CPU) show that each pin detects the mistakes it is meant to.
"""
import ctypes
import functools
import os
import re
import subprocess

import numpy as np
import pytest
from numpy.polynomial import Polynomial

import oracle

STENCILS = ((-2, -1, 0), (-1, 0, 1), (0, 1, 2))  # cells of the candidates, in wind order; the centre cell is 0


def quadratic_from_averages(vals, cells):
    """The quadratic whose averages over the unit cells centred on `cells` are `vals`."""
    A = np.zeros((3, 3))
    for r, m in enumerate(cells):
        for d in range(3):
            prim = Polynomial([0.0] * d + [1.0]).integ()
            A[r, d] = prim(m + 0.5) - prim(m - 0.5)
    return Polynomial(np.linalg.solve(A, vals))


def quartic_from_averages(v):
    A = np.zeros((5, 5))
    for r, m in enumerate(range(-2, 3)):
        for d in range(5):
            prim = Polynomial([0.0] * d + [1.0]).integ()
            A[r, d] = prim(m + 0.5) - prim(m - 0.5)
    return Polynomial(np.linalg.solve(A, v))


def candidates(v):
    return [quadratic_from_averages([v[c + 2] for c in cells], cells) for cells in STENCILS]


def indicators_by_definition(v):
    out = []
    for p in candidates(v):
        b = 0.0
        for l in (1, 2):  # h^(2l-1) = 1 at h = 1
            d = p.deriv(l)
            prim = (d * d).integ()
            b += prim(0.5) - prim(-0.5)
        out.append(b)
    return np.array(out)


@functools.lru_cache(maxsize=1)
def linear_weights_by_definition():
    """d_k with sum_k d_k p_k(1/2) = quartic(1/2) for all data: a linear system over random samples."""
    rng = np.random.default_rng(20)
    rows, rhs = [], []
    for _ in range(12):
        v = rng.normal(size=5)
        rows.append([p(0.5) for p in candidates(v)])
        rhs.append(quartic_from_averages(v)(0.5))
    d, res, rank, _ = np.linalg.lstsq(np.array(rows), np.array(rhs), rcond=None)
    assert rank == 3 and np.max(np.abs(np.array(rows) @ d - rhs)) < 1e-12  # exact: the weights exist
    return tuple(d)


def weno_by_definition(v, eps=1e-6):
    q = np.array([p(0.5) for p in candidates(v)])
    alpha = np.array(linear_weights_by_definition()) / (eps + indicators_by_definition(v)) ** 2
    return float(np.dot(alpha, q) / alpha.sum())


def test_linear_weights_are_the_textbook_ones():
    """The weights solved for above are (1, 6, 3)/10: the definition test below uses the solved ones."""
    np.testing.assert_allclose(linear_weights_by_definition(), [0.1, 0.6, 0.3], rtol=1e-12)


def indicator_error(fn, n=200, seed=1):
    rng = np.random.default_rng(seed)
    worst = 0.0
    for _ in range(n):
        v = rng.normal(size=5) * 10.0 ** rng.uniform(-3, 3)
        got, ref = fn(*v), indicators_by_definition(v)
        worst = max(worst, float(np.max(np.abs(got - ref) / np.abs(ref))))
    return worst


def test_indicators_match_their_integral_definition():
    assert indicator_error(oracle.weno5_indicators) < 1e-13


def test_interface_value_matches_the_definition():
    """The whole nonlinear reconstruction (candidates, derived linear weights, indicators, alpha_k) on random
    data whose indicators are far above eps, so that every part of the weights matters."""
    rng = np.random.default_rng(2)
    for _ in range(200):
        v = rng.normal(size=5)
        assert oracle.weno5(*v) == pytest.approx(weno_by_definition(v), rel=1e-12, abs=1e-14)
    # smooth data (indicators close to each other): the weights stay near the linear ones
    for _ in range(50):
        a, b, c = rng.normal(size=3)
        v = [a + b * 0.1 * k + c * 0.01 * k * k for k in range(-2, 3)]
        assert oracle.weno5(*v) == pytest.approx(weno_by_definition(v), rel=1e-12, abs=1e-14)


# ---- convergence order of the oracle's step on smooth periodic data ----------------------------------------

def _profile(y):
    return 1.0 + 0.5 * np.sin(2 * np.pi * y) + 0.2 * np.cos(4 * np.pi * y)


def advection_error(Nx, step=None, t=0.25, Qxi=4):
    """Mean and max error (normalised populations) of ballistic periodic transport to time t against the exact
    translate, with dt proportional to dx^(5/3) so that the third-order time error stays below the spatial
    one."""
    pbar, wp, xi, wxi = oracle.quadrature(3, Qxi)
    dx = 1.0 / Nx
    x = -0.5 + (np.arange(Nx) + 0.5) * dx
    dt = 0.1 * dx * (Nx / 32.0) ** (-2.0 / 3.0)
    n = int(np.ceil(t / dt))
    p = oracle.params(Qp=3, Qxi=Qxi, Nx=Nx, dt=t / n, tau=None, bc=oracle.BC_PERIODIC)
    ws = 0.5 * np.outer(wp, wxi).ravel()
    speeds = np.tile(xi, 3)
    F0 = ws[:, None] * _profile(x[None, :])
    F = (step or oracle.step)(p, F0, n)
    err = np.abs(F - ws[:, None] * _profile(x[None, :] - speeds[:, None] * t)) / ws[:, None]
    return float(err.mean()), float(err.max())


def convergence_orders(step=None):
    e = [advection_error(n, step)[0] for n in (64, 128, 256)]
    return np.log2(e[0] / e[1]), np.log2(e[1] / e[2])


def test_weno_convergence_order():
    """Fifth order in space: measured L1 orders 5.03 (64 -> 128 cells) and 5.42 (128 -> 256); the Jiang-Shu
    weights with eps = 1e-6 approach the linear ones only as the grid resolves the profile."""
    o1, o2 = convergence_orders()
    assert o1 > 4.7 and o2 > 4.7, (o1, o2)


# ---- planted errors: a copy of the oracle with one constant changed, compiled here ------------------------

_SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle", "rlb_oracle.c")


def _mutant(tmp_path, func, old, new, tag):
    """Compile a copy of the oracle in which `old` is replaced by `new` inside function `func` only."""
    src = open(_SRC).read()
    m = re.search(r"static [a-z]+ " + func + r"\(.*?\n}\n", src, re.S)
    assert m and old in m.group(0), f"{old!r} not found in {func}"
    body = m.group(0).replace(old, new)
    cfile = tmp_path / f"orc_{tag}.c"
    cfile.write_text(src[:m.start()] + body + src[m.end():])
    so = tmp_path / f"orc_{tag}.so"
    subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fno-fast-math", "-ffp-contract=off", "-o",
                    str(so), str(cfile), "-lm"], check=True)
    lib = ctypes.CDLL(str(so))
    dp = ctypes.POINTER(ctypes.c_double)
    lib.orc_weno5_indicators.argtypes = [ctypes.c_double] * 5 + [dp]
    lib.orc_step.argtypes = [ctypes.POINTER(oracle.Params), dp, ctypes.c_long]
    return lib


def _indicators_of(lib):
    def fn(*v):
        out = np.zeros(3)
        lib.orc_weno5_indicators(*v, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
        return out
    return fn


def _step_of(lib):
    def step(p, F, n):
        F = np.array(F, dtype=np.float64, order="C", copy=True)
        assert lib.orc_step(ctypes.byref(p), F.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), int(n)) == 0
        return F
    return step


@pytest.mark.parametrize("old,new", [("13.0 / 12.0", "13.0 / 3.0"), ("0.25 *", "1.0 *"),
                                     ("13.0 / 12.0", "1.0")])
def test_indicator_pin_detects_changed_constants(tmp_path, old, new):
    """13/3 in place of 13/12, 1 in place of 1/4, or both weights 1: each passes the linear-limit, linear-data,
    constant, ENO and mirror tests, and each fails the definition pin."""
    lib = _mutant(tmp_path, "weno5_indicators", old, new, "ind")
    assert indicator_error(_indicators_of(lib), n=20) > 1e-3


def test_convergence_pin_detects_a_wrong_linear_weight(tmp_path):
    """With 0.5 in place of the central linear weight 0.6 the scheme drops to third order."""
    lib = _mutant(tmp_path, "weno5_eps", "0.6 /", "0.5 /", "lin")
    o1, o2 = convergence_orders(_step_of(lib))
    assert o2 < 3.5, (o1, o2)
