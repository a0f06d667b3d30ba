"""GPU unit tests of the stage kernels' device arithmetic (csrc/rlb_device_math.cuh):
* rcp_nr: hardware reciprocal approximation + one cubic Newton-Raphson step, against IEEE division (numpy);
* weno5_pair + weno5_combine (WENO5 with indicators per pair of differences, then three pairs per
  interface) for both wind directions, against the oracle's textbook Jiang-Shu formula on random, smooth,
  stepped and tiny data;
* the double-float limiter of the FP64 stage kernel (df_split, weno5_pair_df, weno5_combine6_df) on the same
  data, and the split's round trip."""
import ctypes
import os
import shutil
import subprocess
import tempfile

import numpy as np
import pytest

import oracle
from paper_1608_03004_gb300 import build as B

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def shim():
    out = os.path.join(tempfile.mkdtemp(prefix="rlb_dm_"), "libdm.so")
    subprocess.run([B.nvcc(), B.ARCH, "-O3", "-std=c++17", "-shared", "-Xcompiler", "-fPIC", "-o", out,
                    os.path.join(HERE, "gpu_src", "device_math_check.cu")], check=True)
    lib = ctypes.CDLL(out)
    lib.dm_eval.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]
    yield lib
    shutil.rmtree(os.path.dirname(out), ignore_errors=True)


def run(lib, which, x, n):
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.empty(n)
    assert lib.dm_eval(which, x.ctypes.data, y.ctypes.data, n) == 0
    return y


def test_reciprocal_within_two_ulp(shim):
    rng = np.random.default_rng(1)
    d = np.exp(rng.uniform(-60, 60, 1 << 20))
    r = run(shim, 0, d, d.size)
    rel = np.abs(r * d - 1.0)
    assert rel.max() <= 2.5 * 2.0**-53 * 2, rel.max()


def test_weno5_matches_oracle(shim):
    rng = np.random.default_rng(2)
    cases = []
    for scale in (1e-8, 1e-3, 1.0, 10.0):
        cases.append(scale * rng.normal(size=(4000, 5)))                      # rough data
        base = rng.uniform(0.1, 1.0, size=(4000, 1)) * scale
        cases.append(base + 1e-3 * scale * np.cumsum(rng.normal(size=(4000, 5)), axis=1))  # smooth
        step = np.where(np.arange(5) >= rng.integers(1, 5, size=(4000, 1)), 1.0, 0.1) * scale
        cases.append(step)                                                    # jumps
    v = np.concatenate(cases)
    scale = np.max(np.abs(v), axis=1)
    # wind toward +x: memory order is wind order
    got = run(shim, 1, v, v.shape[0])
    ref = np.array([oracle.weno5(*row) for row in v])
    assert (np.abs(got - ref) / scale).max() < 1e-14
    # wind toward -x: the oracle sees the samples in reverse (wind) order
    got = run(shim, 2, v, v.shape[0])
    ref = np.array([oracle.weno5(*row[::-1]) for row in v])
    assert (np.abs(got - ref) / scale).max() < 1e-14


def weno_cases():
    rng = np.random.default_rng(2)
    cases = []
    for scale in (1e-8, 1e-3, 1.0, 10.0):
        cases.append(scale * rng.normal(size=(4000, 5)))                      # rough data
        base = rng.uniform(0.1, 1.0, size=(4000, 1)) * scale
        cases.append(base + 1e-3 * scale * np.cumsum(rng.normal(size=(4000, 5)), axis=1))  # smooth
        step = np.where(np.arange(5) >= rng.integers(1, 5, size=(4000, 1)), 1.0, 0.1) * scale
        cases.append(step)                                                    # jumps
    return np.concatenate(cases)


def test_weno5_double_float_limiter_matches_oracle(shim):
    """The FP64 stage kernel's limiter in double-float (about 47-bit significands, section on the limiter in
    rlb_device_math.cuh): the interface value stays within 6e-14 of the five samples' scale of the oracle's
    FP64 formula. The bound is twice the largest error of a numpy emulation of the same arithmetic on these
    cases (2.9e-14, rough data; smooth data and jumps stay near 1e-15): the relative error of the indicators
    and of 6 G is a few 2^-46, times the spread of the candidates."""
    v = weno_cases()
    scale = np.max(np.abs(v), axis=1)
    for which, order in ((3, slice(None)), (4, slice(None, None, -1))):
        got = run(shim, which, v, v.shape[0])
        ref = np.array([oracle.weno5(*row[order]) for row in v])
        err = np.abs(got - ref) / scale
        print(f"double-float limiter, mode {which}: max {err.max():.2e}")
        assert np.all(np.isfinite(got)) and err.max() < 6e-14, err.max()


def test_double_float_split_round_trip(shim):
    """df_split keeps the top 47 significant bits of a double (hi + lo, both truncated): the widened sum is
    within 2^-46 relative for |d| >= 2^-80, within 2^-23 for 2^-126 <= |d| < 2^-80 (where lo is subnormal or
    dropped, and df_widen reads a subnormal float as 0), and 0 below; zero stays zero and signs are kept."""
    rng = np.random.default_rng(3)
    d = rng.normal(size=20000) * 10.0 ** rng.uniform(-40, 30, 20000)
    d = np.concatenate([d, [0.0, -3.0, 1.0, -(2.0 ** -100), 2.0 ** -103, 2.0 ** 127, 1e-39]])
    got = run(shim, 5, d, d.size)
    a = np.abs(d)
    full, hi_only, tiny = a >= 2.0 ** -80, (a >= 2.0 ** -126) & (a < 2.0 ** -80), a < 2.0 ** -126
    assert full.sum() > 12000 and hi_only.sum() > 1000 and tiny.sum() > 100
    assert np.all(np.abs(got[full] - d[full]) <= 2.0 ** -46 * a[full])
    assert np.all(np.abs(got[hi_only] - d[hi_only]) <= 2.0 ** -23 * a[hi_only])
    assert np.all(got[tiny] == 0.0)
    nz = full | hi_only
    assert np.all(np.sign(got[nz]) == np.sign(d[nz]))


def test_fp64_fma_rate_bounds_the_derived_peak():
    """The FP64 stage kernel is bound by the FP64 pipe; its roofline takes 2 FMAs per SM per clock at the
    maximum SM clock (2070 MHz) as the peak. A loop of independent FMA chains measures the rate: it cannot
    exceed that peak (the denominator is not an underestimate) and reaches at least half of it even on a
    GPU held below its maximum clock."""
    out = os.path.join(tempfile.mkdtemp(prefix="rlb_fp64_"), "libfp64.so")
    subprocess.run([B.nvcc(), B.ARCH, "-O3", "-std=c++17", "-shared", "-Xcompiler", "-fPIC", "-o", out,
                    os.path.join(HERE, "gpu_src", "fp64_rate.cu")], check=True)
    lib = ctypes.CDLL(out)
    lib.fp64_rate.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]
    rate, nsm = ctypes.c_double(), ctypes.c_int()
    assert lib.fp64_rate(4096, 8, ctypes.byref(rate), ctypes.byref(nsm)) == 0
    shutil.rmtree(os.path.dirname(out), ignore_errors=True)
    per_sm_clock = rate.value / (nsm.value * 2070e6)
    print(f"FP64 FMA rate {rate.value * 2 / 1e12:.3f} TFLOP/s on {nsm.value} SMs = "
          f"{per_sm_clock:.2f} FMA per SM per clock at 2070 MHz")
    assert 1.0 <= per_sm_clock <= 2.05, per_sm_clock
