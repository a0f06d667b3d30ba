"""Time-step rule: linear stability of SSP-RK3 for WENO5 advection plus the Anderson-Witting relaxation.

For one velocity the semi-discrete equation is dF/dt = -(xi/dx) D F - k F with k = gamma (1 - beta xi)/tau.
In the smooth limit WENO5 is the linear fifth-order upwind scheme, whose Fourier symbol is computed here; the
step is stable when |R(nu sym(theta) - k dt)| <= 1 for all theta, R(z) = 1 + z + z^2/2 + z^3/6, nu = |xi| dt/dx.
This pins the time-step rule of the library and of the workloads: dt = min(cfl dx, 0.9 tau) is stable at
cfl 0.5 up to |v| ~ 0.63, whereas a 1.25 tau cap (stable on the real axis alone) is not once |v| ~ 0.47 and
|xi| ~ 1 - the instability seen in long hydrodynamic runs with many directions.
"""
import numpy as np

from paper_1608_03004_gb300 import workloads as W

TH = np.linspace(0.0, 2.0 * np.pi, 8001)


def max_growth(nu, kdt):
    E = lambda m: np.exp(1j * m * TH)
    phi = (2 * E(-2) - 13 * E(-1) + 47 * E(0) + 27 * E(1) - 3 * E(2)) / 60.0
    z = nu * (-(phi - phi * E(-1))) - kdt
    return np.abs(1 + z + z * z / 2 + z**3 / 6).max()


def test_pure_advection_is_stable_at_cfl_half():
    assert max_growth(0.5, 0.0) <= 1 + 1e-12


def test_pure_relaxation_limit_is_the_real_axis_bound():
    assert max_growth(0.0, 2.51) <= 1 + 1e-12
    assert max_growth(0.0, 2.52) > 1


def test_workload_rule_is_stable_up_to_v_063():
    v = 0.63
    g = 1 / np.sqrt(1 - v * v)
    kdt = W.STIFF_SOD * g * (1 + v)  # the fastest relaxation rate times the capped dt
    assert max_growth(0.5, kdt) <= 1 + 1e-12


def test_strong_shock_rule_is_stable_up_to_v_09():
    v = 0.9
    g = 1 / np.sqrt(1 - v * v)
    assert max_growth(0.5, W.STIFF_STRONG * g * (1 + v)) <= 1 + 1e-12


def test_a_125_tau_cap_is_unstable_at_sod_speeds():
    v = 0.47
    g = 1 / np.sqrt(1 - v * v)
    assert max_growth(0.495, 1.22 * g * (1 + v)) > 1.01  # dt = 1.22 tau at Nx = 4096, tau = 1e-4, |xi| = 0.99


def _limit(nu):
    """Largest k dt with max_growth(nu, k dt) <= 1, by bisection on the numpy symbol above."""
    lo, hi = 0.0, 3.0
    for _ in range(40):
        mid = 0.5 * (lo + hi)
        lo, hi = (mid, hi) if max_growth(nu, mid) <= 1 + 1e-12 else (lo, mid)
    return lo


def test_library_stiffness_limit_matches_the_linear_analysis():
    import shutil

    import pytest

    from paper_1608_03004_gb300 import binding, build
    if shutil.which("nvcc") is None and not build.os.path.exists(build.LIB):
        pytest.skip("no nvcc and no prebuilt library")
    build.build()
    for nu in (0.0, 0.1, 0.25, 0.4, 0.5):
        assert binding.rlb_stiffness_limit(nu) == pytest.approx(_limit(nu), rel=1e-6), nu
    # the real-axis bound of SSP-RK3, 1 + z + z^2/2 + z^3/6 = -1 at z = -2.5127
    assert binding.rlb_stiffness_limit(0.0) == pytest.approx(2.5127453266, rel=1e-9)
    assert max_growth(1.5, 0.0) > 1 and binding.rlb_stiffness_limit(1.5) == 0.0  # advection alone is unstable
    assert binding.rlb_stiffness_limit(-1.0) == 0.0


def test_library_stiffness_limit_falls_with_the_courant_number():
    """Advection takes part of the stable region, so the room left for the collision shrinks as nu grows,
    down to 0 past the advective limit of SSP-RK3 with WENO5 (about 1.43)."""
    import shutil

    import pytest

    from paper_1608_03004_gb300 import binding, build
    if shutil.which("nvcc") is None and not build.os.path.exists(build.LIB):
        pytest.skip("no nvcc and no prebuilt library")
    build.build()
    nus = np.linspace(0.0, 1.4, 15)
    lims = np.array([binding.rlb_stiffness_limit(nu) for nu in nus])
    assert np.all(np.diff(lims) < 0), lims
    assert lims[-1] > 0.0 and binding.rlb_stiffness_limit(1.45) == 0.0
