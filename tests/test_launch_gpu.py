"""Launch shapes (persistent schedules, CUDA-graph replay, tile order, work items per tile) and the autotuner.

Scheduling never changes the arithmetic: every shape must reproduce the default launch bit for bit, for the
FP64 and the FP32 kernels, on a batch of uneven tubes (different Nx, Qxi, tau, boundary conditions)."""
import math

import numpy as np
import pytest

import harness as H
from paper_1608_03004_gb300 import binding as rb
from paper_1608_03004_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def batch():
    return [W.random_smooth(300, 8, 1e-2, seed=1), W.random_smooth(130, 32, math.inf, seed=2),
            W.random_smooth(517, 5, 3e-3, seed=3, bc=W.BC_OPEN), W.random_smooth(64, 16, 1e-1, seed=4),
            W.random_smooth(1000, 4, 2e-2, seed=5)]


SHAPES = [
    dict(schedule=rb.SCHED_TILE, ctas_per_sm=0, graph_steps=0, order=rb.ORDER_INTERLEAVE, split=0),
    dict(schedule=rb.SCHED_TILE, ctas_per_sm=0, graph_steps=0, order=rb.ORDER_COST, split=1),
    dict(schedule=rb.SCHED_TILE, ctas_per_sm=0, graph_steps=0, order=rb.ORDER_COST, split=3),
    dict(schedule=rb.SCHED_STRIDE, ctas_per_sm=0, graph_steps=0, order=rb.ORDER_COST, split=0),
    dict(schedule=rb.SCHED_STRIDE, ctas_per_sm=1, graph_steps=3, order=rb.ORDER_INTERLEAVE, split=8),
    dict(schedule=rb.SCHED_COUNTER, ctas_per_sm=0, graph_steps=0, order=rb.ORDER_COST, split=1),
    dict(schedule=rb.SCHED_COUNTER, ctas_per_sm=2, graph_steps=4, order=rb.ORDER_COST, split=5),
    dict(schedule=rb.SCHED_TILE, ctas_per_sm=0, graph_steps=7, order=rb.ORDER_COST, split=0),
]


@pytest.mark.parametrize("storage", [rb.STORAGE_F64, rb.STORAGE_F32])
def test_every_launch_shape_is_bit_identical(storage):
    specs = batch()
    nsteps = 11  # not a multiple of the graph lengths: graph replays plus a remainder of plain launches
    with H.gpu_init(specs, storage) as h:
        rb.rlb_step(h, nsteps)
        ref = rb.rlb_get_state(h)
    for shape in SHAPES:
        with H.gpu_init(specs, storage) as h:
            rb.rlb_set_launch(h, shape)
            assert rb.rlb_get_launch(h).as_dict() == shape
            rb.rlb_step(h, nsteps)
            np.testing.assert_array_equal(rb.rlb_get_state(h), ref, err_msg=str(shape))


def test_autotune_keeps_the_state_and_the_results():
    specs = batch()
    with H.gpu_init(specs, rb.STORAGE_F32) as h:
        rb.rlb_step(h, 2)
        before = rb.rlb_get_state(h)
        best, ms = rb.rlb_autotune(h, 2)
        assert ms > 0 and best.schedule in (0, 1, 2) and best.order in (0, 1)
        np.testing.assert_array_equal(rb.rlb_get_state(h), before)
        rb.rlb_step(h, 5)
        tuned = rb.rlb_get_state(h)
    with H.gpu_init(specs, rb.STORAGE_F32) as h:
        rb.rlb_step(h, 7)
        np.testing.assert_array_equal(rb.rlb_get_state(h), tuned)


def test_autotune_fp64_tries_the_split_and_keeps_the_results():
    """FP64 handle with few tiles (the automatic split is above 1, so the tuner also tries split = 1): the
    tuned shape reproduces the default launch bit for bit."""
    specs = batch()
    with H.gpu_init(specs, rb.STORAGE_F64) as h:
        rb.rlb_step(h, 2)
        before = rb.rlb_get_state(h)
        best, ms = rb.rlb_autotune(h, 2)
        assert ms > 0 and best.split in (0, 1)
        np.testing.assert_array_equal(rb.rlb_get_state(h), before)
        rb.rlb_step(h, 5)
        tuned = rb.rlb_get_state(h)
    with H.gpu_init(specs, rb.STORAGE_F64) as h:
        rb.rlb_step(h, 7)
        np.testing.assert_array_equal(rb.rlb_get_state(h), tuned)


def test_bad_launch_shapes_rejected():
    with H.gpu_init([W.sod_tube(64, 8, 1e-3)]) as h:
        for bad in (dict(schedule=3, ctas_per_sm=0, graph_steps=0, order=0),
                    dict(schedule=0, ctas_per_sm=-1, graph_steps=0, order=0),
                    dict(schedule=0, ctas_per_sm=0, graph_steps=65, order=0),
                    dict(schedule=0, ctas_per_sm=0, graph_steps=0, order=2),
                    dict(schedule=0, ctas_per_sm=0, graph_steps=0, order=0, split=9),
                    dict(schedule=0, ctas_per_sm=0, graph_steps=0, order=0, split=-1)):
            with pytest.raises(rb.RlbError) as ei:
                rb.rlb_set_launch(h, bad)
            assert ei.value.status == rb.EINVAL
        with pytest.raises(rb.RlbError):
            rb.rlb_autotune(h, 0)
