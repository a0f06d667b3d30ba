"""Thin ctypes binding of librlb (include/rlb.h): the same entry points, argument marshalling only.

Every step of the time step runs in the CUDA library. There is no Python or CPU fallback: if librlb.so
is missing or cannot be loaded, every call raises. Host arrays are numpy float64; device buffers are
torch CUDA tensors (float64, contiguous), passed by pointer. PyTorch supplies device memory and the stream.
"""
from __future__ import annotations

import ctypes
import os
import re
import threading
from typing import Iterable, Sequence

import numpy as np

from . import build as _build

OK, EINVAL, ENOMEM, ECUDA, ENONPHYS = 0, 1, 2, 3, 4
BC_OPEN, BC_PERIODIC, BC_HALO_LEFT, BC_HALO_RIGHT = 0, 1, 2, 4
STORAGE_F64, STORAGE_F32, STORAGE_BF16 = 0, 1, 2
STORAGE = {"f64": STORAGE_F64, "f32": STORAGE_F32, "bf16": STORAGE_BF16}
FIELDS = ("N0", "Nx", "T00", "T0x", "Txx", "e", "v", "n")
NFIELDS = len(FIELDS)
F_N0, F_NX, F_T00, F_T0X, F_TXX, F_E, F_V, F_N = range(NFIELDS)

_lib = None
_lock = threading.Lock()


class RlbError(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = status
        super().__init__(f"{what}: {rlb_error_string(status)}")


class Tube(ctypes.Structure):
    """rlb_tube: one tube's quadrature orders, grid, time step, relaxation time, boundary condition and
    storage of F (STORAGE_F64, STORAGE_F32 or STORAGE_BF16)."""

    _fields_ = [
        ("Qp", ctypes.c_int32),
        ("Qxi", ctypes.c_int32),
        ("Np", ctypes.c_int32),
        ("Nv", ctypes.c_int32),
        ("Nx", ctypes.c_int64),
        ("dx", ctypes.c_double),
        ("dt", ctypes.c_double),
        ("tau", ctypes.c_double),
        ("bc", ctypes.c_int32),
        ("storage", ctypes.c_int32),
    ]

    @classmethod
    def make(cls, Nx: int, Qxi: int, tau: float, dt: float | None = None, dx: float | None = None, Qp: int = 3,
             Np: int = 2, Nv: int = 5, bc: int = BC_OPEN, cfl: float = 0.5, storage: int = STORAGE_F64) -> "Tube":
        dx = 1.0 / Nx if dx is None else dx
        tau_c = float(tau) if (tau is not None and np.isfinite(tau)) else float("inf")
        dt = rlb_suggest_dt(dx, tau_c, cfl) if dt is None else dt
        return cls(Qp, Qxi, Np, Nv, Nx, dx, dt, tau_c, bc, storage)


SCHED_TILE, SCHED_STRIDE, SCHED_COUNTER = 0, 1, 2
ORDER_COST, ORDER_INTERLEAVE = 0, 1


class Launch(ctypes.Structure):
    """rlb_launch: scheduling of a handle's steps (never changes results)."""

    _fields_ = [("schedule", ctypes.c_int32), ("ctas_per_sm", ctypes.c_int32), ("graph_steps", ctypes.c_int32),
                ("order", ctypes.c_int32), ("split", ctypes.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


def library_path() -> str:
    return _build.LIB


def load():
    """Load librlb.so (building it first if a source changed and nvcc is available)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.LIB
        if _build.stale():
            try:
                _build.build()
            except Exception as exc:  # noqa: BLE001 - report the build failure, never fall back
                if not os.path.exists(path):
                    raise RuntimeError(f"librlb.so is not built and the build failed: {exc}") from exc
        if not os.path.exists(path):
            raise RuntimeError("librlb.so is not built: run paper_1608_03004_gb300.build.build()")
        lib = ctypes.CDLL(path)
        vp, dp, ip = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.c_int32
        tp = ctypes.POINTER(Tube)
        sig = {
            "rlb_init": ([ctypes.POINTER(vp), tp, ip, vp, vp, vp, ip, vp], ctypes.c_int),
            "rlb_init_riemann": ([ctypes.POINTER(vp), tp, ip, dp, dp, vp], ctypes.c_int),
            "rlb_step": ([vp, ctypes.c_int64], ctypes.c_int),
            "rlb_moments": ([vp, vp, ip], ctypes.c_int),
            "rlb_get_state": ([vp, vp, ip], ctypes.c_int),
            "rlb_set_state": ([vp, vp, ip], ctypes.c_int),
            "rlb_sync": ([vp], ctypes.c_int),
            "rlb_destroy": ([vp], ctypes.c_int),
            "rlb_state_size": ([vp], ctypes.c_int64),
            "rlb_error_string": ([ctypes.c_int], ctypes.c_char_p),
            "rlb_suggest_dt": ([ctypes.c_double, ctypes.c_double, ctypes.c_double], ctypes.c_double),
            "rlb_quadrature": ([ip, ip, dp, dp, dp, dp], ctypes.c_int),
            "rlb_step_static": ([tp, vp, vp, ctypes.c_int64, vp, vp], ctypes.c_int),
            "rlb_get_launch": ([vp, ctypes.POINTER(Launch)], ctypes.c_int),
            "rlb_set_launch": ([vp, ctypes.POINTER(Launch)], ctypes.c_int),
            "rlb_autotune": ([vp, ip, ctypes.POINTER(Launch), dp], ctypes.c_int),
            "rlb_record": ([vp, ctypes.c_int64, ip], ctypes.c_int),
            "rlb_stiffness_limit": ([ctypes.c_double], ctypes.c_double),
            "rlb_warnings": ([vp, ctypes.POINTER(ctypes.c_uint32)], ctypes.c_int),
            "rlb_backward": ([vp, vp, vp, dp], ctypes.c_int),
            "rlb_moments_vjp": ([vp, vp, vp], ctypes.c_int),
            "rlb_fields_vjp": ([vp, vp, vp], ctypes.c_int),
            "rlb_halo_size": ([vp], ctypes.c_int64),
            "rlb_halo_pack": ([vp, ctypes.c_int32, vp], ctypes.c_int),
            "rlb_halo_unpack": ([vp, ctypes.c_int32, vp], ctypes.c_int),
            "rlb_stage": ([vp, ctypes.c_int32], ctypes.c_int),
            "rlb_init_vjp": ([vp, vp, vp, vp, vp, vp, vp, vp], ctypes.c_int),
        }
        for name, (args, res) in sig.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = res
        _lib = lib
        return lib


def declared_entry_points() -> list[str]:
    """Names of the functions declared in include/rlb.h."""
    hdr = os.path.join(_build.ROOT, "include", "rlb.h")
    text = open(hdr).read()
    return sorted(set(re.findall(r"^\s*(?:const\s+)?[a-z_0-9]+\s*\*?\s*(rlb_[a-z_]+)\s*\(", text, re.M)))


def _check(st: int, what: str):
    if st != OK:
        raise RlbError(st, what)


def _is_cuda_tensor(a) -> bool:
    return hasattr(a, "is_cuda") and bool(a.is_cuda)


def _dev_ptr(t, n: int | None = None):
    import torch

    if t.dtype != torch.float64 or not t.is_contiguous():
        raise ValueError("device buffers must be contiguous float64 CUDA tensors")
    if n is not None and t.numel() < n:
        raise ValueError(f"device buffer holds {t.numel()} doubles, {n} needed")
    return ctypes.c_void_p(t.data_ptr())


def _host(a, n: int | None = None) -> np.ndarray:
    arr = np.ascontiguousarray(a, dtype=np.float64)
    if n is not None and arr.size != n:
        raise ValueError(f"host array holds {arr.size} doubles, {n} needed")
    return arr


def _stream(stream):
    if stream is not None:
        return ctypes.c_void_p(int(stream))
    try:
        import torch

        if torch.cuda.is_available():
            return ctypes.c_void_p(int(torch.cuda.current_stream().cuda_stream))
    except ImportError:
        pass
    return ctypes.c_void_p(0)


class Handle:
    """An rlb_handle plus the tube list it was created with (for output sizes)."""

    def __init__(self, ptr: ctypes.c_void_p, tubes: Sequence[Tube]):
        self.ptr = ptr
        self.tubes = list(tubes)
        self.nx_total = int(sum(t.Nx for t in tubes))
        self.state_size = int(sum(t.Qp * t.Qxi * t.Nx for t in tubes))

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        rlb_destroy(self)

    def __del__(self):
        if getattr(self, "ptr", None) and _lib is not None:
            _lib.rlb_destroy(self.ptr)
            self.ptr = None


def _tube_array(tubes):
    if isinstance(tubes, Tube):
        tubes = [tubes]
    tubes = list(tubes)
    arr = (Tube * len(tubes))(*tubes)
    return tubes, arr


def rlb_init(tubes: Tube | Iterable[Tube], P, n, v, stream=None) -> Handle:
    """Create a handle; F = truncated equilibrium of per-cell (P, n, v) (host arrays or CUDA tensors)."""
    lib = load()
    tubes, arr = _tube_array(tubes)
    nx = int(sum(t.Nx for t in tubes))
    if all(_is_cuda_tensor(a) for a in (P, n, v)):
        ptrs = [_dev_ptr(a, nx) for a in (P, n, v)]
        on_dev = 1
        keep = ptrs
    else:
        keep = [_host(a, nx) for a in (P, n, v)]
        ptrs = [a.ctypes.data_as(ctypes.c_void_p) for a in keep]
        on_dev = 0
    h = ctypes.c_void_p()
    _check(lib.rlb_init(ctypes.byref(h), arr, len(tubes), ptrs[0], ptrs[1], ptrs[2], on_dev, _stream(stream)),
           "rlb_init")
    del keep
    return Handle(h, tubes)


def rlb_init_riemann(tubes: Tube | Iterable[Tube], states, x_left, stream=None) -> Handle:
    """Create a handle for Riemann data: states[b] = (P_L, n_L, v_L, P_R, n_R, v_R), x_left[b] = domain edge."""
    lib = load()
    tubes, arr = _tube_array(tubes)
    st = _host(np.reshape(states, (-1,)), 6 * len(tubes))
    xl = _host(np.reshape(x_left, (-1,)), len(tubes))
    h = ctypes.c_void_p()
    dp = ctypes.POINTER(ctypes.c_double)
    _check(lib.rlb_init_riemann(ctypes.byref(h), arr, len(tubes), st.ctypes.data_as(dp), xl.ctypes.data_as(dp),
                                _stream(stream)), "rlb_init_riemann")
    return Handle(h, tubes)


def rlb_step(h: Handle, nsteps: int = 1) -> None:
    _check(load().rlb_step(h.ptr, int(nsteps)), "rlb_step")


def rlb_moments(h: Handle, out=None):
    """Fields [8][sum Nx] (N0, Nx, T00, T0x, Txx, e, v, n). out: None (new numpy array), numpy or CUDA tensor."""
    lib = load()
    n = NFIELDS * h.nx_total
    if out is not None and _is_cuda_tensor(out):
        _check(lib.rlb_moments(h.ptr, _dev_ptr(out, n), 1), "rlb_moments")
        return out
    res = np.empty((NFIELDS, h.nx_total)) if out is None else out
    if not (isinstance(res, np.ndarray) and res.dtype == np.float64 and res.flags.c_contiguous and res.size == n):
        raise ValueError("out must be a contiguous float64 array of 8 * sum(Nx) values")
    _check(lib.rlb_moments(h.ptr, res.ctypes.data_as(ctypes.c_void_p), 0), "rlb_moments")
    return res


def rlb_get_state(h: Handle, out=None):
    """Packed state (tube by tube, [Q][Nx] each) into a new numpy array, a numpy array or a CUDA tensor."""
    lib = load()
    if out is not None and _is_cuda_tensor(out):
        _check(lib.rlb_get_state(h.ptr, _dev_ptr(out, h.state_size), 1), "rlb_get_state")
        return out
    res = np.empty(h.state_size) if out is None else out
    if not (isinstance(res, np.ndarray) and res.dtype == np.float64 and res.flags.c_contiguous
            and res.size == h.state_size):
        raise ValueError("out must be a contiguous float64 array of rlb_state_size values")
    _check(lib.rlb_get_state(h.ptr, res.ctypes.data_as(ctypes.c_void_p), 0), "rlb_get_state")
    return res


def rlb_set_state(h: Handle, F) -> None:
    lib = load()
    if _is_cuda_tensor(F):
        _check(lib.rlb_set_state(h.ptr, _dev_ptr(F, h.state_size), 1), "rlb_set_state")
    else:
        arr = _host(np.reshape(F, (-1,)), h.state_size)
        _check(lib.rlb_set_state(h.ptr, arr.ctypes.data_as(ctypes.c_void_p), 0), "rlb_set_state")


def rlb_sync(h: Handle) -> None:
    _check(load().rlb_sync(h.ptr), "rlb_sync")


def rlb_destroy(h: Handle) -> None:
    if h.ptr:
        _check(load().rlb_destroy(h.ptr), "rlb_destroy")
        h.ptr = None


def rlb_state_size(h: Handle) -> int:
    return int(load().rlb_state_size(h.ptr))


def rlb_error_string(status: int) -> str:
    try:
        return load().rlb_error_string(int(status)).decode()
    except Exception:  # noqa: BLE001 - message formatting only
        return f"status {status}"


def rlb_suggest_dt(dx: float, tau: float, cfl: float = 0.5) -> float:
    return float(load().rlb_suggest_dt(float(dx), float(tau), float(cfl)))


WARN_STIFF = 1


def rlb_stiffness_limit(nu: float) -> float:
    """Largest k dt for which SSP-RK3 with (linear) WENO5 advection at Courant number nu damps every mode."""
    return float(load().rlb_stiffness_limit(float(nu)))


def rlb_warnings(h: Handle) -> int:
    """Read and clear the handle's sticky warning bits (WARN_STIFF: the collision was too stiff for dt)."""
    bits = ctypes.c_uint32()
    _check(load().rlb_warnings(h.ptr, ctypes.byref(bits)), "rlb_warnings")
    return int(bits.value)


def rlb_quadrature(Qp: int, Qxi: int):
    """The library's own (pbar, w^p, xi, w^xi)."""
    lib = load()
    out = [np.zeros(Qp), np.zeros(Qp), np.zeros(Qxi), np.zeros(Qxi)]
    dp = ctypes.POINTER(ctypes.c_double)
    _check(lib.rlb_quadrature(Qp, Qxi, *[a.ctypes.data_as(dp) for a in out]), "rlb_quadrature")
    return tuple(out)


def rlb_step_static(tube: Tube, F_in, F_out, nsteps: int, flag=None, stream=None) -> None:
    """Allocation-free step of one tube (rlb_step_static): F_in, F_out (may be the same tensor) and the optional
    int32 flag are CUDA tensors owned by the caller; no device memory is allocated by the library. Meant for
    callers that cannot allocate device memory while they step (see include/rlb.h)."""
    n = tube.Qp * tube.Qxi * tube.Nx
    fp = None
    if flag is not None:
        import torch

        if flag.dtype != torch.int32 or not flag.is_cuda:
            raise ValueError("flag must be an int32 CUDA tensor")
        fp = ctypes.c_void_p(flag.data_ptr())
    _check(load().rlb_step_static(ctypes.byref(tube), _dev_ptr(F_in, n), _dev_ptr(F_out, n), int(nsteps), fp,
                                  _stream(stream)), "rlb_step_static")


def halo_dtype(h: Handle):
    """torch dtype of a handle's exchange buffer (its storage type)."""
    import torch

    return {STORAGE_F64: torch.float64, STORAGE_F32: torch.float32, STORAGE_BF16: torch.bfloat16}[h.tubes[0].storage]


def rlb_halo_size(h: Handle) -> int:
    """Elements of the handle's exchange buffer (rlb_halo_size)."""
    return int(load().rlb_halo_size(h.ptr))


def _halo_buf(h: Handle, buf):
    import torch

    if not isinstance(buf, torch.Tensor) or not buf.is_cuda or not buf.is_contiguous() or buf.dtype != halo_dtype(h):
        raise ValueError("exchange buffers must be contiguous CUDA tensors of the handle's storage type")
    if buf.numel() < rlb_halo_size(h):
        raise ValueError(f"exchange buffer holds {buf.numel()} elements, {rlb_halo_size(h)} needed")
    return ctypes.c_void_p(buf.data_ptr())


def rlb_halo_pack(h: Handle, stage: int, send) -> None:
    """Edge cells of stage `stage`'s input of every slab into send (rlb_halo_pack)."""
    _check(load().rlb_halo_pack(h.ptr, int(stage), _halo_buf(h, send)), "rlb_halo_pack")


def rlb_halo_unpack(h: Handle, stage: int, recv) -> None:
    """Ghost cells of stage `stage`'s input of every slab from recv (rlb_halo_unpack)."""
    _check(load().rlb_halo_unpack(h.ptr, int(stage), _halo_buf(h, recv)), "rlb_halo_unpack")


def rlb_stage(h: Handle, stage: int) -> None:
    """One Runge-Kutta stage of the current step (rlb_stage)."""
    _check(load().rlb_stage(h.ptr, int(stage)), "rlb_stage")


def rlb_get_launch(h: Handle) -> Launch:
    out = Launch()
    _check(load().rlb_get_launch(h.ptr, ctypes.byref(out)), "rlb_get_launch")
    return out


def rlb_set_launch(h: Handle, cfg: Launch | dict) -> None:
    if isinstance(cfg, dict):
        cfg = Launch(**cfg)
    _check(load().rlb_set_launch(h.ptr, ctypes.byref(cfg)), "rlb_set_launch")


def rlb_autotune(h: Handle, trial_steps: int = 3):
    """Time every launch shape on this handle's tubes and keep the fastest; returns (Launch, ms per step)."""
    best = Launch()
    ms = ctypes.c_double()
    _check(load().rlb_autotune(h.ptr, int(trial_steps), ctypes.byref(best), ctypes.byref(ms)), "rlb_autotune")
    return best, ms.value


# ---------------------------------------------------------------------------------------------------------
# Adjoint (FP64 handles): device buffers are contiguous float64 CUDA tensors
# ---------------------------------------------------------------------------------------------------------

def rlb_record(h: Handle, nsteps: int, every: int) -> None:
    """rlb_step(h, nsteps) keeping a checkpoint every `every` steps for rlb_backward."""
    _check(load().rlb_record(h.ptr, int(nsteps), int(every)), "rlb_record")


def rlb_backward(h: Handle, seed, grad_state=None):
    """Reverse sweep over the last rlb_record. seed: dL/dF of the final state (packed, CUDA tensor).
    Returns (grad_state tensor or None, numpy array of dL/dlog(tau) per tube)."""
    glt = np.zeros(len(h.tubes))
    gp = None if grad_state is None else _dev_ptr(grad_state, h.state_size)
    _check(load().rlb_backward(h.ptr, _dev_ptr(seed, h.state_size), gp,
                               glt.ctypes.data_as(ctypes.POINTER(ctypes.c_double))), "rlb_backward")
    return grad_state, glt


def rlb_moments_vjp(h: Handle, grad_moments, seed):
    """seed (packed, CUDA) = dL/dF from grad_moments [5][sum Nx] (CUDA): the adjoint of the five moments."""
    _check(load().rlb_moments_vjp(h.ptr, _dev_ptr(grad_moments, 5 * h.nx_total), _dev_ptr(seed, h.state_size)),
           "rlb_moments_vjp")
    return seed


def rlb_fields_vjp(h: Handle, grad_fields, seed):
    """seed (packed, CUDA) = dL/dF from grad_fields [RLB_NFIELDS][sum Nx] (CUDA): the adjoint of the five
    moments and of the Landau-frame e, v, n at the handle's current state."""
    _check(load().rlb_fields_vjp(h.ptr, _dev_ptr(grad_fields, NFIELDS * h.nx_total),
                                 _dev_ptr(seed, h.state_size)), "rlb_fields_vjp")
    return seed


def rlb_init_vjp(h: Handle, P, n, v, grad_state, grad_P, grad_n, grad_v) -> None:
    """dL/dP, dL/dn, dL/dv of the initial fields (CUDA, field layout) from dL/dF of the initial state."""
    m = h.nx_total
    _check(load().rlb_init_vjp(h.ptr, _dev_ptr(P, m), _dev_ptr(n, m), _dev_ptr(v, m),
                               _dev_ptr(grad_state, h.state_size), _dev_ptr(grad_P, m), _dev_ptr(grad_n, m),
                               _dev_ptr(grad_v, m)), "rlb_init_vjp")
