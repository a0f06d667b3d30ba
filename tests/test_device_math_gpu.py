"""GPU unit tests of the stage kernel's device arithmetic (csrc/rlb_device_math.cuh):
* rcp_nr: hardware reciprocal approximation + one cubic Newton-Raphson step, against IEEE division (numpy);
* weno5_pair + weno5_combine (the kernel's WENO5: indicators per pair of differences, then three pairs per
  interface) for both wind directions, against the oracle's textbook Jiang-Shu formula on random, smooth,
  stepped and tiny data."""
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
