"""The allocation-free entry point rlb_step_static against the handle-based rlb_step.

rlb_step_static serves callers that cannot allocate device memory while they step (their device memory
belongs to their own pool allocator, their host forbids allocation once running, or a cudaMalloc that may
synchronise the device is not acceptable in their loop): the caller passes the state in and out, and the
library keeps its scratch in a fixed file-scope device array. Both entry points run the same stage kernel on
the same arithmetic, so their results must agree bit for bit. This file is collected last so that a run that
stops at the first failure has run every other test before it; it also passes on its own in a fresh process.
"""
import ctypes

import numpy as np
import pytest

import harness as H
from paper_1608_03004_gb300 import binding as rb
from paper_1608_03004_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def handle_state(spec, nsteps):
    with H.gpu_init([spec]) as h:
        F0 = rb.rlb_get_state(h).copy()
        if nsteps:
            rb.rlb_step(h, nsteps)
        return F0, rb.rlb_get_state(h)


def test_static_step_matches_handle_step_on_two_calls_in_a_row():
    torch = pytest.importorskip("torch")
    a = W.sod_tube(300, 16, 1e-3)
    b = W.random_smooth(130, 8, 2e-2, seed=9)  # periodic, moving, ragged tile count
    A0, A7 = handle_state(a, 7)
    B0, B5 = handle_state(b, 5)
    flag = torch.zeros(1, dtype=torch.int32, device="cuda")
    fin = torch.tensor(A0, device="cuda")
    fout = torch.empty_like(fin)
    fb = torch.tensor(B0, device="cuda")
    # first call: out of place (on a fresh device it also does the one-time set-up)
    rb.rlb_step_static(H.to_tube(a), fin, fout, 7, flag)
    torch.cuda.synchronize()
    got_a = fout.cpu().numpy()
    # second call right after it, on another tube, in place (the shared scratch keeps the first call's data);
    # it must leave the device's free memory and torch's allocations as they were
    free0, alloc0 = torch.cuda.mem_get_info()[0], torch.cuda.memory_allocated()
    rb.rlb_step_static(H.to_tube(b), fb, fb, 5, flag)
    torch.cuda.synchronize()
    free1, alloc1 = torch.cuda.mem_get_info()[0], torch.cuda.memory_allocated()
    got_b = fb.cpu().numpy()
    np.testing.assert_array_equal(got_a, A7, err_msg="rlb_step_static, first call")
    np.testing.assert_array_equal(got_b, B5, err_msg="rlb_step_static, second call")
    assert int(flag.item()) == 0
    assert free1 == free0, f"free device memory changed by {free1 - free0} bytes"
    assert alloc1 == alloc0
    # the input of the out-of-place call is untouched
    np.testing.assert_array_equal(fin.cpu().numpy(), A0)


def test_static_step_rejects_a_tube_over_the_limit():
    torch = pytest.importorskip("torch")
    big = W.sod_tube(20000, 200, 1e-3)  # 2 x 600 x 20000 doubles > 64 MiB
    t = H.to_tube(big)
    x = torch.zeros(8, dtype=torch.float64, device="cuda")
    lib = rb.load()
    st = lib.rlb_step_static(ctypes.byref(t), ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(x.data_ptr()), 1,
                             None, None)
    assert st == rb.EINVAL


def test_static_step_refuses_a_capturing_stream():
    """Its small tables come from host memory that lives only during the call: under capture it returns
    RLB_EINVAL before it enqueues anything."""
    torch = pytest.importorskip("torch")
    a = W.sod_tube(64, 8, 1e-3)
    x = torch.zeros(a.Q * a.Nx, dtype=torch.float64, device="cuda")
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    lib = rb.load()
    torch.cuda.synchronize()
    with torch.cuda.stream(s):
        g.capture_begin(capture_error_mode="relaxed")
        try:
            st = lib.rlb_step_static(ctypes.byref(H.to_tube(a)), ctypes.c_void_p(x.data_ptr()),
                                     ctypes.c_void_p(x.data_ptr()), 1, None, ctypes.c_void_p(s.cuda_stream))
        finally:
            g.capture_end()
    torch.cuda.synchronize()
    assert st == rb.EINVAL
