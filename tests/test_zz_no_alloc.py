"""The allocation-free entry point rlb_step_static against the handle-based rlb_step.

rlb_step_static serves callers that cannot allocate device memory while they step (their device memory
belongs to their own pool allocator, their host forbids allocation once running, or a cudaMalloc that may
synchronise the device is not acceptable in their loop): the caller passes the state in and out, and the
library keeps its scratch in a fixed file-scope device array. This file is collected last so that a run that
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
    # first call: out of place
    fin = torch.tensor(A0, device="cuda")
    fout = torch.empty_like(fin)
    rb.rlb_step_static(H.to_tube(a), fin, fout, 7, flag)
    torch.cuda.synchronize()
    got_a = fout.cpu().numpy().reshape(a.Q, a.Nx)
    # second call right after it, on another tube, in place (the shared scratch keeps the first call's data)
    fb = torch.tensor(B0, device="cuda")
    rb.rlb_step_static(H.to_tube(b), fb, fb, 5, flag)
    torch.cuda.synchronize()
    got_b = fb.cpu().numpy().reshape(b.Q, b.Nx)
    H.assert_state_parity(got_a, A7.reshape(a.Q, a.Nx), what="rlb_step_static, first call")
    H.assert_state_parity(got_b, B5.reshape(b.Q, b.Nx), what="rlb_step_static, second call")
    assert int(flag.item()) == 0
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
