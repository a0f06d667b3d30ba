"""The CPU samples bench.py times the oracle on (cpu_baseline leg and reference arm): windows cut from the
workload's tubes, never above their node budget except for the first window, so that shrinking the budget
shrinks the sample."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
from paper_1608_03004_gb300 import workloads as W  # noqa: E402


def test_small_workload_is_taken_whole():
    specs = W.sod_small()
    sample, what = bench.cpu_sample(specs)
    assert sample is specs and "every tube" in what


def test_windows_respect_the_budget_and_shrink_with_it():
    specs, _ = bench.workload("sweep")
    for window in (4096, 512):
        sizes = []
        for budget in (24_000_000, 5_000_000, 1_180_000, 200_000, 50_000):
            sample, _ = bench.cpu_sample(specs, max_nodes=budget, window=window)
            nodes = W.total_nodes(sample)
            assert len(sample) >= 1
            assert nodes <= budget or len(sample) == 1
            assert all(s.Nx <= window for s in sample)
            # each window keeps its tube's orders, grid spacing, time step and relaxation time
            for s in sample:
                assert any(s.Qxi == t.Qxi and s.dx == t.dx and s.dt == t.dt and s.tau == t.tau for t in specs)
            sizes.append(nodes)
        assert sizes == sorted(sizes, reverse=True), sizes


def test_windows_are_centred_on_the_membrane():
    specs, _ = bench.workload("sweep")
    sample, _ = bench.cpu_sample(specs, max_nodes=2_000_000, window=1024)
    for s in sample:
        assert abs(s.x_left + 0.5 * s.Nx * s.dx) < 1e-15  # x = 0 at the middle of the window
