"""Domain decomposition on one GPU: a tube split into x-slabs, one handle per slab, halos exchanged before every
Runge-Kutta stage (rlb_halo_pack / device copies / rlb_halo_unpack / rlb_stage, decompose.LocalExchange). Each
slab's cells see exactly the values they see in the undivided tube, so the assembled result must be bit-identical
to the whole tube advanced by rlb_step, in every storage type. This is the data path a multi-GPU run takes,
with the device copies in place of NCCL transfers.
"""
import numpy as np
import pytest
import torch

import harness as H
from paper_1608_03004_gb300 import binding as rb
from paper_1608_03004_gb300 import decompose as D
from paper_1608_03004_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def slab_run(spec, storage, parts, nsteps):
    tube = H.to_tube(spec, storage)
    tubes, bounds, sched = D.slab_tubes(tube, parts)
    handles = [rb.rlb_init([t], spec.P[a:b], spec.n[a:b], spec.v[a:b]) for t, (a, b) in zip(tubes, bounds)]
    dtype = rb.halo_dtype(handles[0])
    sends = [torch.zeros(rb.rlb_halo_size(h), dtype=dtype, device="cuda") for h in handles]
    recvs = [torch.zeros_like(x) for x in sends]
    D.step_slabs(handles, D.LocalExchange(sched, 3 * spec.Q), sends, recvs, nsteps)
    out = np.zeros((spec.Q, spec.Nx))
    for h, (a, b) in zip(handles, bounds):
        out[:, a:b] = rb.rlb_get_state(h).reshape(spec.Q, b - a)
        rb.rlb_destroy(h)
    return out


def whole_run(spec, storage, nsteps):
    with H.gpu_init([spec], storage) as h:
        rb.rlb_step(h, nsteps)
        return rb.rlb_get_state(h).reshape(spec.Q, spec.Nx)


@pytest.mark.parametrize("storage", [rb.STORAGE_F64, rb.STORAGE_F32, rb.STORAGE_BF16])
@pytest.mark.parametrize("parts,periodic", [(2, False), (3, False), (2, True), (4, True)])
def test_slabs_are_bit_identical_to_the_whole_tube(storage, parts, periodic):
    """250 cells (ragged slabs, none a multiple of a tile), a moving smooth state, 7 steps."""
    spec = W.random_smooth(250, 8, 2e-2, seed=40 + parts, bc=W.BC_PERIODIC if periodic else W.BC_OPEN, vmax=0.5)
    np.testing.assert_array_equal(slab_run(spec, storage, parts, 7), whole_run(spec, storage, 7))


def test_sod_slabs_with_a_three_cell_slab():
    """The paper's Sod tube as per-cell states, split 3 | 197 | 200 (the smallest slab allowed, three cells:
    its ghosts on both sides reach into both neighbours), 20 steps through the shock's formation."""
    spec = W.sod_tube(400, 8, 1e-3)
    x = spec.x_left + (np.arange(spec.Nx) + 0.5) * spec.dx
    spec.P, spec.n, spec.v = np.where(x < 0, 1.0, 0.1), np.where(x < 0, 1.0, 0.125), np.zeros(spec.Nx)
    tube = H.to_tube(spec)
    sched = D.SlabSchedule(3)
    bounds = [(0, 3), (3, 200), (200, 400)]
    handles = [rb.rlb_init([rb.Tube(tube.Qp, tube.Qxi, tube.Np, tube.Nv, b - a, tube.dx, tube.dt, tube.tau,
                                    sched.bc(p), tube.storage)], spec.P[a:b], spec.n[a:b], spec.v[a:b])
               for p, (a, b) in enumerate(bounds)]
    sends = [torch.zeros(rb.rlb_halo_size(h), dtype=torch.float64, device="cuda") for h in handles]
    recvs = [torch.zeros_like(x_) for x_ in sends]
    D.step_slabs(handles, D.LocalExchange(sched, 3 * spec.Q), sends, recvs, 20)
    got = np.concatenate([rb.rlb_get_state(h).reshape(spec.Q, b - a) for h, (a, b) in zip(handles, bounds)], axis=1)
    for h in handles:
        rb.rlb_destroy(h)
    np.testing.assert_array_equal(got, whole_run(spec, rb.STORAGE_F64, 20))


@pytest.mark.parametrize("storage", [rb.STORAGE_F64, rb.STORAGE_F32])
def test_slab_steps_replayed_from_a_cuda_graph(storage):
    """One step of four slabs (packs, device copies, unpacks, stages) captured as a CUDA graph and replayed 7
    times: bit-identical to the undivided tube, as the launched path is."""
    spec = W.random_smooth(250, 8, 2e-2, seed=47, bc=W.BC_PERIODIC, vmax=0.5)
    tube = H.to_tube(spec, storage)
    tubes, bounds, sched = D.slab_tubes(tube, 4)
    stream = torch.cuda.Stream()
    handles = [rb.rlb_init([t], spec.P[a:b], spec.n[a:b], spec.v[a:b], stream=stream.cuda_stream)
               for t, (a, b) in zip(tubes, bounds)]
    dtype = rb.halo_dtype(handles[0])
    sends = [torch.zeros(rb.rlb_halo_size(h), dtype=dtype, device="cuda") for h in handles]
    recvs = [torch.zeros_like(x_) for x_ in sends]
    step = D.GraphStep(handles, D.LocalExchange(sched, 3 * spec.Q), sends, recvs, stream)
    step(7)
    stream.synchronize()
    got = np.concatenate([rb.rlb_get_state(h).reshape(spec.Q, b - a) for h, (a, b) in zip(handles, bounds)], axis=1)
    for h in handles:
        rb.rlb_destroy(h)
    np.testing.assert_array_equal(got, whole_run(spec, storage, 7))


def test_three_stages_make_one_step_and_slabs_refuse_rlb_step():
    spec = W.random_smooth(130, 8, 2e-2, seed=5)
    with H.gpu_init([spec]) as h:
        for st in range(3):
            rb.rlb_stage(h, st)
        staged = rb.rlb_get_state(h)
    np.testing.assert_array_equal(staged, whole_run(spec, rb.STORAGE_F64, 1).ravel())
    t = rb.Tube(3, 8, 2, 5, 64, 1 / 64, 0.5 / 64, 0.02, rb.BC_HALO_LEFT | rb.BC_HALO_RIGHT, rb.STORAGE_F64)
    with rb.rlb_init([t], np.ones(64), np.ones(64), np.zeros(64)) as h:
        assert rb.rlb_halo_size(h) == 2 * 3 * 24
        with pytest.raises(rb.RlbError) as ei:
            rb.rlb_step(h, 1)
        assert ei.value.status == rb.EINVAL
