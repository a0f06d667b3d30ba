"""Domain decomposition of one tube into x-slabs, the method's one exchange step.

Every Runge-Kutta stage of the step (section "Numerical results": SSP-RK3 with WENO5 advection) reads three
cells beyond each cell, so a tube split into slabs needs, before each stage, the three edge cells of all Q
velocities of each neighbouring slab: 3 Q values per side and neighbour (2 x 3 x Q x element size bytes per
slab boundary and stage). A slab is a tube with RLB_BC_HALO_LEFT and/or RLB_BC_HALO_RIGHT; the library packs a
slab's edge cells (rlb_halo_pack), sets its ghost cells (rlb_halo_unpack) and runs one stage (rlb_stage). This
module holds the host side: the slab bounds, the exchange schedule (which block goes to which neighbour) and
the transport, within one process (LocalExchange: slabs as handles of one GPU, device copies) or between
processes (DistExchange: torch.distributed point-to-point, NCCL between GPUs, gloo between CPU processes).
Argument marshalling and data movement only: every step of the method runs in the CUDA library.

Block layout of a slab's buffers (the library's): one block of Q x 3 elements per halo side, left first. In a
send buffer the left block holds the slab's cells 0..2 and the right block its cells Nx-3..Nx-1; in a receive
buffer the left block holds the ghost cells -3..-1 (the left neighbour's last three cells) and the right
block the ghost cells Nx..Nx+2 (the right neighbour's first three).
"""
from __future__ import annotations

import dataclasses
from typing import List, Optional, Sequence, Tuple

from . import binding as rb

HALO = 3  # WENO5 reaches three cells on each side


def slab_bounds(Nx: int, parts: int) -> List[Tuple[int, int]]:
    """Cell ranges [a, b) of `parts` slabs of Nx cells, sizes differing by at most one, each at least 3."""
    if parts < 1 or Nx < HALO * parts:
        raise ValueError(f"{Nx} cells cannot make {parts} slabs of at least {HALO} cells")
    base, extra = divmod(Nx, parts)
    out, a = [], 0
    for p in range(parts):
        b = a + base + (1 if p < extra else 0)
        out.append((a, b))
        a = b
    return out


@dataclasses.dataclass(frozen=True)
class SlabSchedule:
    """Neighbours and halo sides of the slabs of one tube: a chain with open outer ends, or a ring (the tube is
    periodic). One slab of a periodic tube is its own neighbour on both sides."""

    parts: int
    periodic: bool = False

    def left(self, p: int) -> Optional[int]:
        if p > 0:
            return p - 1
        return self.parts - 1 if self.periodic else None

    def right(self, p: int) -> Optional[int]:
        if p < self.parts - 1:
            return p + 1
        return 0 if self.periodic else None

    def bc(self, p: int) -> int:
        """Boundary flags of slab p (RLB_BC_HALO_* on the sides with a neighbour, open otherwise)."""
        return (rb.BC_HALO_LEFT if self.left(p) is not None else 0) | (
            rb.BC_HALO_RIGHT if self.right(p) is not None else 0)


def slab_tubes(tube: rb.Tube, parts: int) -> Tuple[List[rb.Tube], List[Tuple[int, int]], SlabSchedule]:
    """The slabs of `tube` (open or periodic) as tubes of their own: same orders, grid spacing, time step,
    relaxation time and storage, with halo boundary flags. Returns (tubes, cell ranges, schedule)."""
    if tube.bc not in (rb.BC_OPEN, rb.BC_PERIODIC):
        raise ValueError("only an open or periodic tube is split into slabs")
    sched = SlabSchedule(parts, tube.bc == rb.BC_PERIODIC)
    bounds = slab_bounds(int(tube.Nx), parts)
    tubes = [rb.Tube(tube.Qp, tube.Qxi, tube.Np, tube.Nv, b - a, tube.dx, tube.dt, tube.tau, sched.bc(p),
                     tube.storage) for p, (a, b) in enumerate(bounds)]
    return tubes, bounds, sched


def blocks(buf, bc: int, q3: int):
    """(left block, right block) views of a slab's buffer (None for a side without a halo)."""
    k = 0
    left = right = None
    if bc & rb.BC_HALO_LEFT:
        left = buf[k:k + q3]
        k += q3
    if bc & rb.BC_HALO_RIGHT:
        right = buf[k:k + q3]
    return left, right


class LocalExchange:
    """The slabs of one tube as handles in one process (one GPU): receive blocks filled by device copies from the
    neighbours' send blocks."""

    def __init__(self, sched: SlabSchedule, q3: int):
        self.sched, self.q3 = sched, q3

    def __call__(self, sends: Sequence, recvs: Sequence) -> None:
        s = self.sched
        for p in range(s.parts):
            rl, rr = blocks(recvs[p], s.bc(p), self.q3)
            if rl is not None:  # the left neighbour's last cells: its right send block
                rl.copy_(blocks(sends[s.left(p)], s.bc(s.left(p)), self.q3)[1])
            if rr is not None:  # the right neighbour's first cells: its left send block
                rr.copy_(blocks(sends[s.right(p)], s.bc(s.right(p)), self.q3)[0])


class DistExchange:
    """One slab per process of a torch.distributed group (rank p holds slab p). The transfers go in two phases in
    the same order on every rank, so that point-to-point messages between a pair of ranks match also without
    tags (NCCL) and when both neighbours are the same rank (a ring of two): phase 1 sends the right block to the
    right neighbour and receives the left ghosts from the left one; phase 2 sends the left block to the left
    neighbour and receives the right ghosts from the right one."""

    def __init__(self, sched: SlabSchedule, rank: int, q3: int, group=None):
        self.sched, self.rank, self.q3, self.group = sched, rank, q3, group

    def __call__(self, send, recv) -> None:
        import torch.distributed as dist

        s, p = self.sched, self.rank
        sl, sr = blocks(send, s.bc(p), self.q3)
        rl, rr = blocks(recv, s.bc(p), self.q3)
        if s.parts == 1:  # one periodic slab: its own neighbour
            rl.copy_(sr)
            rr.copy_(sl)
            return
        ops = []
        if sr is not None:
            ops.append(dist.P2POp(dist.isend, sr.contiguous(), s.right(p), self.group, tag=1))
        if rl is not None:
            ops.append(dist.P2POp(dist.irecv, rl, s.left(p), self.group, tag=1))
        if sl is not None:
            ops.append(dist.P2POp(dist.isend, sl.contiguous(), s.left(p), self.group, tag=2))
        if rr is not None:
            ops.append(dist.P2POp(dist.irecv, rr, s.right(p), self.group, tag=2))
        if ops:
            for w in dist.batch_isend_irecv(ops):
                w.wait()


def step_slabs(handles: Sequence[rb.Handle], exchange, sends: Sequence, recvs: Sequence, nsteps: int) -> None:
    """nsteps steps of every slab handle: before each of the three stages, pack the stage input's edge cells,
    exchange, unpack the ghost cells, then run the stage. `exchange(sends, recvs)` for a LocalExchange (all slabs
    here), `exchange(send, recv)` for a DistExchange (one slab per process, one handle)."""
    local = isinstance(exchange, LocalExchange)
    for _ in range(int(nsteps)):
        for st in range(3):
            for h, s in zip(handles, sends):
                rb.rlb_halo_pack(h, st, s)
            if local:
                exchange(sends, recvs)
            else:
                exchange(sends[0], recvs[0])
            for h, r in zip(handles, recvs):
                rb.rlb_halo_unpack(h, st, r)
            for h in handles:
                rb.rlb_stage(h, st)


class GraphStep:
    """One step of all slabs of one process (every stage's pack, exchange, unpack and stage) captured once as a
    CUDA graph, then replayed: a step costs one graph launch instead of five launches per slab and stage from
    the host, the cost that bounds the slab path when the stages are short. The slab handles must launch on
    `stream` (created with stream=stream.cuda_stream): the capture runs there, and so does every replay. The
    send and receive buffers are captured by address and must stay alive. LocalExchange only (device copies)."""

    def __init__(self, handles: Sequence[rb.Handle], exchange: LocalExchange, sends: Sequence, recvs: Sequence,
                 stream):
        import torch

        if not isinstance(exchange, LocalExchange):
            raise TypeError("GraphStep captures the device copies of a LocalExchange")
        self.stream = stream
        self.graph = torch.cuda.CUDAGraph()
        torch.cuda.synchronize()
        with torch.cuda.graph(self.graph, stream=stream):
            step_slabs(handles, exchange, sends, recvs, 1)

    def __call__(self, nsteps: int) -> None:
        import torch

        with torch.cuda.stream(self.stream):
            for _ in range(int(nsteps)):
                self.graph.replay()
