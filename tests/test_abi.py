"""CPU-side checks of the C ABI: the library builds for sm_103a, loads, exports every entry point declared in
include/rlb.h, and its host-only helpers behave (no GPU compute is launched here)."""
import ctypes
import math
import shutil
import subprocess

import numpy as np
import pytest

import oracle
import paper_1608_03004_gb300 as rlb
from paper_1608_03004_gb300 import binding, build

pytestmark = pytest.mark.skipif(shutil.which("nvcc") is None and not build.os.path.exists(build.LIB),
                                reason="no nvcc and no prebuilt library")


def test_library_builds_and_exports_every_declared_symbol():
    path = build.build()
    declared = binding.declared_entry_points()
    assert len(declared) >= 10
    lib = ctypes.CDLL(path)
    for name in declared:
        assert hasattr(lib, name), name
    nm = shutil.which("nm")
    if nm:
        out = subprocess.run([nm, "-D", "--defined-only", path], capture_output=True, text=True, check=True).stdout
        exported = {ln.split()[-1] for ln in out.splitlines() if " T " in ln}
        assert set(declared) <= exported
    # the build targets the GB300 architecture only
    assert build.ARCH == "-gencode=arch=compute_103a,code=sm_103a"


def test_binding_names_match_header():
    for name in binding.declared_entry_points():
        assert hasattr(rlb, name), name


def test_suggest_dt_and_error_strings():
    assert rlb.rlb_suggest_dt(1e-4, 1e-4, 0.5) == pytest.approx(5e-5)   # the paper's dt at L_z = 10000
    assert rlb.rlb_suggest_dt(1 / 400, 1e-3, 0.5) == pytest.approx(0.9e-3)
    assert rlb.rlb_suggest_dt(1 / 1024, 1e-4, 0.5) == pytest.approx(0.9e-4)
    assert rlb.rlb_suggest_dt(0.01, math.inf, 0.5) == pytest.approx(5e-3)
    for st in range(5):
        assert rlb.rlb_error_string(st).startswith("RLB_")


@pytest.mark.parametrize("Qp,Qxi", [(3, 4), (3, 5), (3, 8), (2, 32), (4, 128), (3, 200)])
def test_library_quadrature_agrees_with_oracle(Qp, Qxi):
    got = rlb.rlb_quadrature(Qp, Qxi)
    ref = oracle.quadrature(Qp, Qxi)
    for g, r in zip(got, ref):
        np.testing.assert_allclose(g, r, rtol=1e-13, atol=1e-15)
    if Qxi % 2:
        assert got[2][Qxi // 2] == 0.0
    np.testing.assert_array_equal(got[2], -got[2][::-1])


def test_invalid_arguments_rejected_before_any_device_call():
    lib = binding.load()
    h = ctypes.c_void_p()
    one = np.ones(8)
    p = one.ctypes.data_as(ctypes.c_void_p)
    bad = [
        rlb.Tube(3, 8, 3, 5, 8, 0.1, 0.01, 1e-3, 0, 0),    # Np >= Qp
        rlb.Tube(3, 8, 1, 5, 8, 0.1, 0.01, 1e-3, 0, 0),    # Np < 2 cannot recover T^{mu nu}
        rlb.Tube(2, 8, 1, 5, 8, 0.1, 0.01, 1e-3, 0, 0),    # Qp < 3
        rlb.Tube(3, 3, 2, 5, 8, 0.1, 0.01, 1e-3, 0, 0),    # 2 Qxi < Nv + 3
        rlb.Tube(3, 8, 2, 9, 8, 0.1, 0.01, 1e-3, 0, 0),    # Nv above the supported maximum
        rlb.Tube(5, 8, 2, 5, 8, 0.1, 0.01, 1e-3, 0, 0),    # Qp above the supported maximum
        rlb.Tube(3, 8, 2, 5, 0, 0.1, 0.01, 1e-3, 0, 0),    # no cells
        rlb.Tube(3, 8, 2, 5, 8, -0.1, 0.01, 1e-3, 0, 0),   # dx <= 0
        rlb.Tube(3, 8, 2, 5, 8, 0.1, 0.0, 1e-3, 0, 0),     # dt <= 0
        rlb.Tube(3, 8, 2, 5, 2, 0.1, 0.01, 1e-3, 1, 0),    # periodic with Nx < 3
        rlb.Tube(3, 8, 2, 5, 8, 0.1, 0.01, 1e-3, 7, 0),    # unknown boundary condition
        rlb.Tube(3, 8, 2, 5, 8, 0.1, 0.01, float("nan"), 0, 0),
    ]
    for t in bad:
        st = lib.rlb_init(ctypes.byref(h), ctypes.byref(t), 1, p, p, p, 0, None)
        assert st == binding.EINVAL, (t.Qp, t.Qxi, t.Np, t.Nv, t.Nx, st)
    t = rlb.Tube(3, 8, 2, 5, 8, 0.1, 0.01, 1e-3, 0, 0)
    assert lib.rlb_init(ctypes.byref(h), ctypes.byref(t), 0, p, p, p, 0, None) == binding.EINVAL
    assert lib.rlb_init(ctypes.byref(h), ctypes.byref(t), 1, None, p, p, 0, None) == binding.EINVAL
    assert lib.rlb_step(None, 1) == binding.EINVAL
    assert lib.rlb_moments(None, p, 0) == binding.EINVAL
    assert lib.rlb_sync(None) == binding.EINVAL
    assert lib.rlb_destroy(None) == binding.OK
    assert lib.rlb_state_size(None) == -1
