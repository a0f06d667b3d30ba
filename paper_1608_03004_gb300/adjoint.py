"""Gradients of a run of the time step, through torch.autograd.

A run starts from the truncated equilibrium of per-cell fields (P, n, v) (Eq. (condinit) with Eq. (feqtrunc))
and takes nsteps SSP-RK3 steps of Eq. (Boltz) with each tube's time step held fixed; its output is the fields
of every cell: the five conserved moments (N^0, N^x, T^00, T^0x, T^xx) and the Landau-frame e, v, n. The
backward pass is the library's hand-written adjoint: rlb_record keeps a checkpoint every `every` steps,
rlb_backward recomputes each segment from its checkpoint and runs the transposed stage kernels backwards,
rlb_fields_vjp seeds it from the fields' gradient (through the Landau frame on the device) and rlb_init_vjp
carries the result back to (P, n, v). Argument marshalling only: every step runs in the CUDA library.
"""
from __future__ import annotations

import math
from typing import Sequence

import torch

from . import binding as rb


def _with_tau(tubes: Sequence[rb.Tube], log_tau) -> list:
    out = []
    for t, lt in zip(tubes, log_tau):
        tau = math.exp(float(lt)) if math.isfinite(float(lt)) else math.inf
        out.append(rb.Tube(t.Qp, t.Qxi, t.Np, t.Nv, t.Nx, t.dx, t.dt, tau, t.bc, rb.STORAGE_F64))
    return out


class _Run(torch.autograd.Function):
    @staticmethod
    def forward(ctx, log_tau, P, n, v, tubes, nsteps, every):
        tb = _with_tau(tubes, log_tau.detach().cpu().tolist())
        P_, n_, v_ = (a.detach().contiguous() for a in (P, n, v))
        h = rb.rlb_init(tb, P_, n_, v_)
        rb.rlb_record(h, nsteps, every)
        fields = torch.empty((rb.NFIELDS, h.nx_total), dtype=torch.float64, device=P.device)
        rb.rlb_moments(h, fields)
        ctx.h = h
        ctx.lt_device = log_tau.device
        ctx.save_for_backward(P_, n_, v_)
        return fields

    @staticmethod
    def backward(ctx, grad_f):
        h = ctx.h
        P, n, v = ctx.saved_tensors
        seed = torch.empty(h.state_size, dtype=torch.float64, device=P.device)
        rb.rlb_fields_vjp(h, grad_f.contiguous(), seed)
        gF = torch.empty_like(seed)
        _, glt = rb.rlb_backward(h, seed, gF)
        gP, gn, gv = torch.empty_like(P), torch.empty_like(n), torch.empty_like(v)
        rb.rlb_init_vjp(h, P, n, v, gF, gP, gn, gv)
        rb.rlb_destroy(h)
        ctx.h = None
        return (torch.as_tensor(glt, dtype=torch.float64, device=ctx.lt_device), gP, gn, gv, None, None, None)


def run_fields(log_tau, P, n, v, tubes: Sequence[rb.Tube], nsteps: int, every: int = 50):
    """Fields [RLB_NFIELDS][sum Nx] (N^0, N^x, T^00, T^0x, T^xx, e, v, n) after nsteps steps from
    F = F^eq(P, n, v), differentiable in log_tau ([ntubes], float64) and in P, n, v ([sum Nx] float64 CUDA
    tensors, tube after tube). Each tube's relaxation time is exp(log_tau[b]) (inf: ballistic); its dt is taken
    from `tubes` and held fixed."""
    return _Run.apply(log_tau, P, n, v, list(tubes), int(nsteps), int(every))


def run_moments(log_tau, P, n, v, tubes: Sequence[rb.Tube], nsteps: int, every: int = 50):
    """The five conserved moments [5][sum Nx] of run_fields."""
    return run_fields(log_tau, P, n, v, tubes, nsteps, every)[:5]
