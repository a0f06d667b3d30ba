"""Reduced-precision storage (FP32, BF16) against the FP64 oracle: every result states its error.

F is stored in FP32 or BF16; advection, equilibrium evaluation, collision and the Runge-Kutta combination run
in FP32; the moments are compensated FP32 sums reduced in FP64 and the Landau frame is solved in FP64.
Target: FP32 energy density within 1e-5 relative of the FP64 oracle, read normwise,
max_x |e - e_ref| / max_x |e_ref|, and also held for the mean pointwise error (|e - e_ref| / e_ref averaged
over cells). The worst single cell is recorded as well: on the Sod run to t = 0.4 (444 steps) it sits on the
shock and contact, where a shift of a fraction of a cell dominates, at 1.9e-5 for e and 3.3e-5 for T^xx,
above the target; it is bounded at 5e-5 to catch regressions. BF16 (unit roundoff 2^-8) loses several per
cent on average and up to ~50 % at the waves over a few hundred steps (measured: e mean 6.0 %, T^xx mean
5.3 %, worst T^xx 50.4 % on the contact): its rounding noise, relative 2^-9 of each weight-normalised
population, is far above the limiter's sqrt(eps) = 1e-3, so the WENO weights follow the noise (normwise e
9.3 %, T^xx 25 %). Its errors are measured and bounded loosely. The regime where the e, u^mu extraction cancels (flows at |v| up to 0.99,
rarefied cells, strong shocks) has its own test that states both storages' errors there. The errors found
are printed (pytest -s).
"""
import math

import numpy as np
import pytest

import harness as H
import oracle
from paper_1608_03004_gb300 import binding as rb
from paper_1608_03004_gb300 import workloads as W

pytestmark = pytest.mark.gpu

# (field index, name) of the fields the precision targets are stated for
E, V, TXX = 5, 6, 4


def run(specs, nsteps, storage):
    with H.gpu_init(specs, storage) as h:
        rb.rlb_step(h, nsteps)
        rb.rlb_sync(h)
        return H.split_fields(specs, rb.rlb_moments(h)), H.split_state(specs, rb.rlb_get_state(h))


def errors(f, ref):
    re = np.abs(f[E] - ref[E]) / np.abs(ref[E])
    rt = np.abs(f[TXX] - ref[TXX]) / np.abs(ref[TXX])
    return {
        "e_norm": float(np.max(np.abs(f[E] - ref[E])) / np.max(np.abs(ref[E]))),
        "Txx_norm": float(np.max(np.abs(f[TXX] - ref[TXX])) / np.max(np.abs(ref[TXX]))),
        "e_rel_mean": float(np.mean(re)), "e_rel_max": float(np.max(re)),
        "Txx_rel_mean": float(np.mean(rt)), "Txx_rel_max": float(np.max(rt)),
        "v_abs_max": float(np.max(np.abs(f[V] - ref[V]))),
    }


# (normwise bound, mean pointwise bound, worst-cell bound) per storage; FP32's first two are the 1e-5 target
BOUNDS = {rb.STORAGE_F32: (1e-5, 1e-5, 5e-5), rb.STORAGE_BF16: (0.35, 0.1, 0.65)}


def check_bounds(err, storage):
    norm_b, mean_b, max_b = BOUNDS[storage]
    # the 1e-5 target is the energy density's; T^xx is held to twice it (measured 0.99e-5 to 1.09e-5 normwise on
    # the Sod run, depending on the rounding of the kernel's constants)
    assert err["e_norm"] <= norm_b and err["Txx_norm"] <= 2 * norm_b, err
    assert err["e_rel_mean"] <= mean_b and err["Txx_rel_mean"] <= mean_b, err
    assert err["e_rel_max"] <= max_b and err["Txx_rel_max"] <= max_b and err["v_abs_max"] <= max_b, err


@pytest.mark.parametrize("storage", [rb.STORAGE_F32, rb.STORAGE_BF16])
def test_sod_small_full_run_against_oracle(storage):
    s = W.sod_small()[0]
    nsteps = int(round(0.4 / s.dt))  # to t = 0.4
    (f,), _ = run([s], nsteps, storage)
    _, fr = H.oracle_run(s, nsteps)
    err = errors(f, fr)
    print(f"storage {storage}: Sod Nx=400 Q=24 t=0.4 ({nsteps} steps) errors vs FP64 oracle {err}")
    check_bounds(err, storage)


@pytest.mark.parametrize("storage", [rb.STORAGE_F32, rb.STORAGE_BF16])
def test_moving_and_ballistic_batch_against_oracle(storage):
    specs = [W.random_smooth(150, 16, 2e-2, seed=3, vmax=0.6), W.sod_tube(200, 32, math.inf),
             W.random_smooth(90, 8, 1e-3, seed=4, bc=W.BC_OPEN)]
    # one handle takes per-cell states: give the Sod tube its cell states (no centre on the membrane)
    x = -0.5 + (np.arange(200) + 0.5) / 200
    specs[1].P = np.where(x < 0, 1.0, 0.1)
    specs[1].n = np.where(x < 0, 1.0, 0.125)
    specs[1].v = np.zeros(200)
    nsteps = 40
    fg, _ = run(specs, nsteps, storage)
    for s, f in zip(specs, fg):
        _, fr = H.oracle_run(s, nsteps)
        err = errors(f, fr)
        print(f"storage {storage}: Nx={s.Nx} Qxi={s.Qxi} tau={s.tau} errors vs FP64 oracle {err}")
        check_bounds(err, storage)


# The regime where the Landau-frame extraction cancels: (name, spec, steps, FP32 bounds (e_norm, T^xx_norm),
# BF16 bounds or None where BF16 cannot hold the state). Measured, FP32: |v| <= 0.97 e_norm 7.6e-5 (T^xx 3.5e-7),
# |v| = 0.99 e_norm 1.9e-2 (T^xx 1.6e-5), rarefied 9.7e-7, strong shock 6.0e-7. Near |v| = 1 the condition
# number of e with respect to the moments (1.4e3 at 0.97, 1.3e4 at 0.99, measured with the oracle) times the
# FP32 rounding of the stored populations and of the FP32 equilibrium sum sets the error: FP64 moments and an
# FP64 Landau solve cannot undo the storage rounding, so the 1e-5 target is missed there and met elsewhere.
# BF16 rounding of the initial equilibrium at |v| >= 0.97 leaves T^{mu nu} without a timelike eigenvector in
# part of the cells (38 of 128 at 0.97, 72 at 0.99, checked on the CPU): such states are refused (RLB_EINVAL).
HARD = [("fast flow, |v| <= 0.97", lambda: W.fast_flow(128, 16, 2e-2, 0.97, seed=97), 10, (3e-4, 1e-5), None),
        ("near-uniform flow at |v| = 0.99", lambda: W.fast_flow(128, 16, 2e-2, 0.99, seed=100, uniform=True), 10,
         (0.06, 1e-4), None),
        ("rarefied cells, P down to 1e-4", lambda: W.rarefied(128, 16, 1e-2, seed=6), 40, (1e-5, 1e-5),
         (0.1, 0.1)),
        ("strong shock, P_R / P_L = 0.01", lambda: W.strong_shock(200, 16, 1e-2), 40, (1e-5, 1e-5), (0.05, 0.05))]


@pytest.mark.parametrize("storage", [rb.STORAGE_F32, rb.STORAGE_BF16])
@pytest.mark.parametrize("case", range(len(HARD)))
def test_hard_regime_errors_against_oracle(storage, case):
    name, make, nsteps, b32, b16 = HARD[case]
    s = make()
    bounds = b32 if storage == rb.STORAGE_F32 else b16
    if bounds is None:
        with pytest.raises(rb.RlbError) as ei:
            run([s], nsteps, storage)
        assert ei.value.status == rb.EINVAL
        print(f"storage {storage}: {name}: refused (the rounded state has no Landau frame)")
        return
    (f,), _ = run([s], nsteps, storage)
    _, fr = H.oracle_run(s, nsteps)
    err = errors(f, fr)
    print(f"storage {storage}: {name}, {nsteps} steps, errors vs FP64 oracle {err}")
    assert err["e_norm"] <= bounds[0] and err["Txx_norm"] <= bounds[1], err


def test_state_round_trip_rounds_to_storage():
    s = W.random_smooth(77, 8, 1e-2, seed=8)
    F = H.oracle_init(s).ravel()
    for storage in (rb.STORAGE_F32, rb.STORAGE_BF16):
        with H.gpu_init([s], storage) as h:
            rb.rlb_set_state(h, F)
            got = rb.rlb_get_state(h)
        if storage == rb.STORAGE_F32:
            np.testing.assert_array_equal(got, F.astype(np.float32).astype(np.float64))
        else:
            assert np.max(np.abs(got - F) / np.abs(F)) <= 2.0**-8  # unit roundoff of an 8-bit significand
            # values are bf16: 8 significant bits, the low 16 bits of the float pattern are zero
            assert np.all((got.astype(np.float32).view(np.uint32) & 0xFFFF) == 0)


def test_mixed_storage_in_one_handle_rejected():
    a, b = W.sod_tube(64, 8, 1e-3), W.sod_tube(64, 8, 1e-3)
    tubes = [H.to_tube(a, rb.STORAGE_F32), H.to_tube(b, rb.STORAGE_F64)]
    with pytest.raises(rb.RlbError) as ei:
        rb.rlb_init_riemann(tubes, np.array([list(a.left) + list(a.right)] * 2), np.array([-0.5, -0.5]))
    assert ei.value.status == rb.EINVAL


@pytest.mark.parametrize("storage", [rb.STORAGE_F32, rb.STORAGE_BF16])
def test_orders_and_grids_of_the_warp_tiles(storage):
    """The reduced-precision kernel's paths in one handle: warp tiles of 120 cells (a warp holds 128, the
    4-cell halo in its edge lanes) whose cells all lie inside the tube (vector loads: the second tile of 244
    cells ends exactly at the tube's end, 367 has two such tiles), that reach past an end by a cell (243) or
    more (127, 129, 257), or shorter than a tile (60, 9, 3, 2, 1 cells), open and periodic boundaries, odd Qxi
    (a xi = 0 node), the generic orders (Np = 3, Nv = 8: 9 coefficient columns per radial node), and tubes of
    different orders sharing the per-warp shared-memory layout."""
    specs = [W.random_smooth(127, 8, 2e-2, seed=11, bc=W.BC_OPEN),
             W.random_smooth(128, 5, 1e-2, seed=12),
             W.random_smooth(244, 8, 1e-2, seed=20, bc=W.BC_OPEN),
             W.random_smooth(243, 6, 1e-2, seed=21),
             W.random_smooth(367, 5, 2e-2, seed=22, bc=W.BC_OPEN),
             W.random_smooth(129, 16, 5e-3, seed=13, bc=W.BC_OPEN),
             W.random_smooth(257, 4, 3e-2, seed=14, Qp=4, Np=3, Nv=5),
             W.random_smooth(60, 6, 1e-2, seed=15, Qp=4, Np=3, Nv=8, bc=W.BC_OPEN),
             W.random_smooth(9, 7, 2e-2, seed=16),
             W.random_smooth(3, 8, 1e-2, seed=17),
             W.random_smooth(2, 8, 1e-2, seed=18, bc=W.BC_OPEN),
             W.random_smooth(1, 8, 1e-2, seed=19, bc=W.BC_OPEN)]
    nsteps = 10
    fg, _ = run(specs, nsteps, storage)
    for s, f in zip(specs, fg):
        _, fr = H.oracle_run(s, nsteps)
        err = errors(f, fr)
        print(f"storage {storage}: Nx={s.Nx} Qp={s.Qp} Np={s.Np} Nv={s.Nv} Qxi={s.Qxi} bc={s.bc} errors {err}")
        check_bounds(err, storage)


def _window_step_errors(specs, storage, before, xs_of, halo=9):
    """One GPU step after `before` steps against one FP64 oracle step from the same (stored) state, on
    windows of +-halo cells around the cells xs_of(index, spec) of each tube; the state stays on the device
    and only the windows travel. Returns the worst error relative to each row's largest value."""
    import torch

    tot = sum(s.Q * s.Nx for s in specs)
    with H.gpu_init(specs, storage) as h:
        rb.rlb_step(h, before)
        A = torch.empty(tot, dtype=torch.float64, device="cuda")
        rb.rlb_get_state(h, A)
        rb.rlb_step(h, 1)
        B = torch.empty(tot, dtype=torch.float64, device="cuda")
        rb.rlb_get_state(h, B)
    worst, p = 0.0, 0
    for k, s in enumerate(specs):
        a = A[p:p + s.Q * s.Nx].view(s.Q, s.Nx)
        b = B[p:p + s.Q * s.Nx].view(s.Q, s.Nx)
        scale = b.abs().amax(dim=1).cpu().numpy()
        for x in xs_of(k, s):
            lo, hi = max(0, x - halo), min(s.Nx, x + halo + 1)
            sub = W.TubeSpec(Nx=hi - lo, Qxi=s.Qxi, tau=s.tau, dt=s.dt, dx=s.dx, Qp=s.Qp, Np=s.Np, Nv=s.Nv, bc=s.bc)
            ref = oracle.step(H.to_params(sub), np.ascontiguousarray(a[:, lo:hi].cpu().numpy()), 1)
            got = b[:, x].cpu().numpy()
            worst = max(worst, float(np.max(np.abs(got - ref[:, x - lo]) / scale)))
        p += s.Q * s.Nx
    return worst


# one step from the same stored state: FP32 arithmetic and the storage rounding of the output; FP64 storage
# is held to the parity bar of the FP64 path
ONE_STEP = {rb.STORAGE_F64: H.RTOL, rb.STORAGE_F32: 2e-6, rb.STORAGE_BF16: 2.0**-7}


@pytest.mark.parametrize("storage", [rb.STORAGE_F64, rb.STORAGE_F32, rb.STORAGE_BF16])
def test_stress_tube_full_size_one_step(storage):
    """The stress tube at full size (Nx = 2^20, Q = 384) in each storage (FP64: one CTA per tile; FP32/BF16:
    one CTA per group of warp tiles): after 20 steps, the next step at the membrane, at the waves and at
    random cells against the oracle."""
    s = W.stress()
    rng = np.random.default_rng(5)
    mid = s.Nx // 2

    def xs(k, sp):
        return [mid - 1, mid, mid + 3, mid - 15, mid + 15, 0, sp.Nx - 1] + list(rng.integers(0, sp.Nx, 4))

    err = _window_step_errors([s], storage, 20, xs)
    print(f"storage {storage}: stress tube one-step error vs FP64 oracle {err:.3e}")
    assert err <= ONE_STEP[storage], err


def test_batched_tubes_full_size_one_step():
    """The 256-tube batch of the benchmark (FP32, 203 M velocity nodes): after 20 steps, the next step of
    every 16th tube near its membrane and at random cells against the oracle."""
    specs = W.batched_tubes()
    rng = np.random.default_rng(6)

    def xs(k, sp):
        if k % 16:
            return []
        m = sp.Nx // 2
        return [m - 1, m, m + 5, 0, sp.Nx - 1] + list(rng.integers(0, sp.Nx, 2))

    err = _window_step_errors(specs, rb.STORAGE_F32, 20, xs)
    print(f"batched tubes one-step error vs FP64 oracle {err:.3e}")
    assert err <= ONE_STEP[rb.STORAGE_F32], err
