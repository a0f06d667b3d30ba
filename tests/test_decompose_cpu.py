"""Domain decomposition on CPU ranks: the slab bounds and exchange schedule of paper_1608_03004_gb300.decompose
with gloo process groups on 127.0.0.1 (world sizes 2 and 3, open and periodic tubes, ragged slabs).

Each rank holds one slab and advances it with the oracle: before each Runge-Kutta stage it packs the edge cells
of the stage input in the library's block layout, exchanges them through decompose.DistExchange, extends its
slab by the received ghost cells and takes the oracle's right-hand side of Eq. (Boltz) on the extended slab
(the cells of a slab see exactly the values they see in the undivided tube: WENO5 reaches three cells), then
the oracle's SSP-RK3 combination. The assembled slabs must be bit-identical to the oracle's run of the whole
tube; a schedule that swapped a block, a side or a neighbour would not be.
"""
import os
import socket
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as tmp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from paper_1608_03004_gb300 import decompose as D  # noqa: E402


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def make_case(periodic):
    """(spec, oracle params, initial F) of the test tube: a smooth moving state, 50 ragged-sliceable cells."""
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    import harness as H
    from paper_1608_03004_gb300 import workloads as W

    bc = W.BC_PERIODIC if periodic else W.BC_OPEN
    s = W.random_smooth(50, 6, 2e-2, seed=31, bc=bc, vmax=0.4)
    return s, H.to_params(s), H.oracle_init(s)


def oracle_slab_steps(rank, world, periodic, nsteps):
    """Advance this rank's slab by nsteps steps, exchanging halos over the default process group."""
    import oracle
    from paper_1608_03004_gb300 import binding as rb

    s, p, F0 = make_case(periodic)
    tube = rb.Tube(s.Qp, s.Qxi, s.Np, s.Nv, s.Nx, s.dx, s.dt, s.tau, s.bc, rb.STORAGE_F64)
    _, bounds, sched = D.slab_tubes(tube, world)
    a, b = bounds[rank]
    bc = sched.bc(rank)
    Q, q3 = s.Q, 3 * s.Q
    nsides = bin(bc).count("1")
    send = torch.zeros(nsides * q3, dtype=torch.float64)
    recv = torch.zeros(nsides * q3, dtype=torch.float64)
    ex = D.DistExchange(sched, rank, q3)
    dt = p.dt

    def rhs(G):
        sl, sr = D.blocks(send, bc, q3)
        if sl is not None:
            sl.copy_(torch.from_numpy(np.ascontiguousarray(G[:, :3]).ravel()))
        if sr is not None:
            sr.copy_(torch.from_numpy(np.ascontiguousarray(G[:, -3:]).ravel()))
        ex(send, recv)
        rl, rr = D.blocks(recv, bc, q3)
        parts = ([rl.numpy().reshape(Q, 3)] if rl is not None else []) + [G] + (
            [rr.numpy().reshape(Q, 3)] if rr is not None else [])
        E = np.ascontiguousarray(np.concatenate(parts, axis=1))
        pe = oracle.Params(p.Qp, p.Qxi, p.Np, p.Nv, E.shape[1], p.dx, p.dt, p.tau, oracle.BC_OPEN)
        k = 3 if rl is not None else 0
        return oracle.rhs(pe, E)[:, k:k + G.shape[1]]

    F = np.ascontiguousarray(F0[:, a:b])
    for _ in range(nsteps):  # the oracle's Shu-Osher combination, operation for operation
        F1 = F + dt * rhs(F)
        F2 = 0.75 * F + 0.25 * (F1 + dt * rhs(F1))
        F = F / 3.0 + 2.0 / 3.0 * (F2 + dt * rhs(F2))
    return a, b, F


def _rank_main(rank, world, port, periodic, nsteps, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        a, b, F = oracle_slab_steps(rank, world, periodic, nsteps)
        out[rank] = (a, b, F.tobytes(), F.shape)
        dist.barrier()
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world,periodic", [(2, False), (3, False), (2, True), (3, True)])
def test_slab_exchange_over_gloo_is_bit_identical_to_the_whole_tube(world, periodic):
    import oracle

    nsteps = 6
    mgr = tmp.Manager()
    out = mgr.dict()
    tmp.spawn(_rank_main, args=(world, free_port(), periodic, nsteps, out), nprocs=world, join=True)
    s, p, F0 = make_case(periodic)
    ref = oracle.step(p, F0, nsteps)
    got = np.zeros_like(ref)
    for rank in range(world):
        a, b, buf, shape = out[rank]
        got[:, a:b] = np.frombuffer(buf, dtype=np.float64).reshape(shape)
    np.testing.assert_array_equal(got, ref)


def test_slab_bounds_and_schedule():
    assert D.slab_bounds(50, 3) == [(0, 17), (17, 34), (34, 50)]
    assert D.slab_bounds(9, 3) == [(0, 3), (3, 6), (6, 9)]
    with pytest.raises(ValueError):
        D.slab_bounds(8, 3)
    chain, ring = D.SlabSchedule(3), D.SlabSchedule(3, periodic=True)
    assert [chain.left(p) for p in range(3)] == [None, 0, 1]
    assert [chain.right(p) for p in range(3)] == [1, 2, None]
    assert [ring.left(p) for p in range(3)] == [2, 0, 1]
    assert [ring.right(p) for p in range(3)] == [1, 2, 0]
    from paper_1608_03004_gb300 import binding as rb

    assert [chain.bc(p) for p in range(3)] == [rb.BC_HALO_RIGHT, rb.BC_HALO_LEFT | rb.BC_HALO_RIGHT,
                                               rb.BC_HALO_LEFT]
    assert all(ring.bc(p) == rb.BC_HALO_LEFT | rb.BC_HALO_RIGHT for p in range(3))
    buf = torch.arange(12.0)
    left, right = D.blocks(buf, rb.BC_HALO_LEFT | rb.BC_HALO_RIGHT, 6)
    assert left.tolist() == list(range(6)) and right.tolist() == list(range(6, 12))
    left, right = D.blocks(buf[:6], rb.BC_HALO_RIGHT, 6)
    assert left is None and right.tolist() == list(range(6))


def test_local_exchange_moves_each_block_to_the_right_neighbour():
    """LocalExchange (slabs of one process): slab p's left ghosts are slab p-1's right send block, its right
    ghosts slab p+1's left send block; a ring closes over the ends."""
    from paper_1608_03004_gb300 import binding as rb

    for periodic in (False, True):
        sched = D.SlabSchedule(3, periodic)
        q3 = 2
        sends = [torch.tensor([10.0 * p + k for k in range(bin(sched.bc(p)).count("1") * q3)]) for p in range(3)]
        recvs = [torch.zeros_like(x) for x in sends]
        D.LocalExchange(sched, q3)(sends, recvs)
        for p in range(3):
            rl, rr = D.blocks(recvs[p], sched.bc(p), q3)
            if sched.left(p) is not None:
                assert rl.tolist() == D.blocks(sends[sched.left(p)], sched.bc(sched.left(p)), q3)[1].tolist()
            if sched.right(p) is not None:
                assert rr.tolist() == D.blocks(sends[sched.right(p)], sched.bc(sched.right(p)), q3)[0].tolist()
        assert (sched.left(0) is None) == (not periodic) and rb.BC_HALO_LEFT & sched.bc(1)
