#!/usr/bin/env python3
"""Benchmark of the GB300 RLB time step: G velocity-node updates/s.

Headline workload (default ``stress``, the largest single-GPU configuration): one Sod tube, (P, n, v) =
(1, 1, 0) | (0.1, 0.125, 0) on [-0.5, 0.5], Nx = 1,048,576, Qp = 3, Qxi = 128 (384 velocities, 402.7 M
velocity nodes), tau = 1e-2, CFL 0.5, open boundaries, FP64. A step is one SSP-RK3 time step (three launches
of the stage kernel). One velocity-node update = one velocity at one cell over one step.

With no --workload the line also carries, under "extra", a full record (value, ms_per_step, roofline, e2e,
clocks) of each other configuration: the stress tube in FP32 and BF16 storage, autotuned (with the ratio to
FP64 on the same tube), the 256-tube batch autotuned in FP32 and in FP64 (and their ratio), the relaxation-time sweep
(Nx = 4096, tau in {1e-4, 1e-3, 1e-2, 1e-1, 1, 10, inf} x Qxi in {8, 32, 128, 200}, 28 tubes) in FP64, and
one gradient of the inverse problem on Gaussian bumps.

    python bench.py [--steps K] [--warmup W] [--workload sweep|small|stress|batched|gradient|gradient_batch]
                    [--precision f64|f32|bf16] [--impl ours|reference] [--no-extras]

--precision f32/bf16 stores F in that type (FP32 arithmetic, compensated moments reduced in FP64, FP64 Landau
solve); its roofline is HBM (algorithmic 8 x element size bytes per velocity node per step).

--workload gradient: one gradient of the inverse problem on Gaussian bumps (Nx = 2048, Q = 3 x 32, 1000 steps,
checkpoints every 50 steps): the loss is 1/2 |e(x) - e*(x)|^2 of the final energy density at tau = 0.08
against the run at tau* = 0.05 from the initial pressure perturbed by a second set of Gaussian bumps
(amplitude 0.05); the gradient is taken with respect to log(tau) and the initial fields, through the adjoint
(rlb_fields_vjp carries dL/de through the Landau frame); gradient_batch: 64 such tubes (bump seeds 4 .. 67)
in one handle. A step is one gradient; one update = one velocity node carried one time step forward and
back.

Prints one JSON line. Under torchrun every rank advances its own copy of the workload (weak scaling, no
collective on the data path); the time is the max over ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import multiprocessing as mp
import os
import re
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from paper_1608_03004_gb300 import workloads as W  # noqa: E402

METRIC = "G velocity-node updates/s"
UNIT = "G updates/s"
# Algorithmic flops per velocity-node per RK stage (FMA = 2): WENO5 interface value 54 (the first difference 1,
# the limiter 53), flux difference and xi/dx 2, equilibrium (Nv+1 = 6 FMAs) 12, collision 5, Runge-Kutta
# combination 5, moment reduction 6. Per-cell work (Landau solve, Legendre series) is not counted, so these are
# lower bounds. The FP64 stage kernel runs the limiter's 53 in double-float on the FP32 pipe; the other 31 run
# on the FP64 pipe, which bounds the kernel.
FLOPS_PER_NODE_STAGE = 84
FP64_FLOPS_PER_NODE_STAGE = 31
# Algorithmic HBM bytes per velocity node per step with one launch per stage: stage inputs read once
# (1 + 2 + 2 doubles), outputs written once (3 doubles).
BYTES_PER_NODE_STEP = 64
# ncu summaries by (kernel kind, workload): bench.py reports a kernel's DRAM traffic per launch only from the summary
# taken on that workload while the kernel's sources still hash to the recorded value
PROFILES = {("adjoint", "gradient"): os.path.join(ROOT, "profiles", "rlb_adjoint_kernel_gradient.md"),
            ("f64", "stress"): os.path.join(ROOT, "profiles", "rlb_stage_kernel_stress.md"),
            ("f64", "sweep"): os.path.join(ROOT, "profiles", "rlb_stage_kernel_sod_sweep.md"),
            ("f32", "stress"): os.path.join(ROOT, "profiles", "rlb_stage_rp_kernel_f32_stress.md"),
            ("bf16", "stress"): os.path.join(ROOT, "profiles", "rlb_stage_rp_kernel_bf16_stress.md")}
_CSRC = os.path.join(ROOT, "paper_1608_03004_gb300", "csrc")
_SHARED = [os.path.join(_CSRC, "rlb_device_math.cuh"), os.path.join(_CSRC, "rlb_internal.h")]
KERNEL_SRCS = {"adjoint": [os.path.join(_CSRC, "rlb_adjoint.cuh"), os.path.join(_CSRC, "rlb_stage.cuh")] + _SHARED,
               "f64": [os.path.join(_CSRC, "rlb_stage.cuh")] + _SHARED,
               "f32": [os.path.join(_CSRC, "rlb_stage_rp.cuh"), os.path.join(_CSRC, "rlb_stage.cuh")] + _SHARED,
               "bf16": [os.path.join(_CSRC, "rlb_stage_rp.cuh"), os.path.join(_CSRC, "rlb_stage.cuh")] + _SHARED}
ESIZE = {"f64": 8, "f32": 4, "bf16": 2}
EXTRA_STEPS = 40  # timed steps of each extra configuration (after the headline's warm-up count)
CPU_SAMPLE_NODES = 24_000_000  # bound on the velocity nodes the oracle advances per CPU sample step
REF_BUDGET_S = 120.0  # the reference arm's whole run (warm-up and timed steps) on the host cores
GRAD_METRIC = "G velocity-node gradient updates/s"
GRAD_UNIT = "G gradient updates/s"
GRAD_STEPS, GRAD_EVERY, GRAD_TAU, GRAD_TAU_STAR = 1000, 50, 0.08, 0.05
GRAD_TARGET_SEED = 5  # bumps of the target's initial pressure perturbation (tube k: seed 5 + k)
GRAD_CPU_STEPS = 4  # steps of each oracle run in the gradient workloads' CPU samples (two runs per gradient)
# Algorithmic FP64 flops per velocity node per adjoint stage (FMA = 2, a division counted as one flop):
# WENO5 interface derivative 130 (candidates 16, indicator terms 18, eps + beta_k 18, alpha_k and weights 11,
# Phi 5, kappa_k 12, their products with the indicator terms 12, the five partials 38), adjoint flux 3, slot
# products 5, gather 4, collision and moment weights 15, output 5, equilibrium and the Lam / S0 / S1 sums 33,
# moments 6.
ADJ_FLOPS_PER_NODE_STAGE = 201


def workload(name: str, nx: int | None = None, ntubes: int | None = None):
    if name == "sweep":
        return W.sod_sweep(), ("Sod tube sweep: Nx=4096, tau in {1e-4,1e-3,1e-2,1e-1,1,10,inf} x Qxi in "
                               "{8,32,128,200}, Qp=3, Np=2, Nv=5, CFL 0.5 (dt=min(0.5dx,0.9tau)), open BC")
    if name == "small":
        return W.sod_small(), "Sod tube: Nx=400, Qp=3, Qxi=8, tau=1e-3, CFL 0.5, open BC"
    if name == "stress":
        n = nx or (1 << 20)
        return [W.stress(Nx=n)], f"Sod tube: Nx={n}, Qp=3, Qxi=128, tau=1e-2, CFL 0.5, open BC"
    if name == "batched":
        return W.batched_tubes(), ("256 shock tubes, seed 160803004: Nx ~ U[1024,16384], log10 tau ~ U[-4,1], "
                                   "Qxi in {8,16,32,64}, Qp=3, P_L ~ U[0.5,2], P_R = P_L U(0.01,0.5), "
                                   "dt=min(0.5dx,0.45tau), open BC")
    if name == "gradient":
        return [W.gaussian_bumps(tau=GRAD_TAU)], ("inverse problem on Gaussian bumps: Nx=2048, Qp=3, Qxi=32, "
                                                  "Np=2, Nv=5, dt=0.5dx, open BC; loss 1/2 |e(x) - e*(x)|^2 of the "
                                                  "final energy density at tau=0.08 against the run at tau*=0.05 "
                                                  "from P perturbed by Gaussian bumps (amplitude 0.05, seed 5); "
                                                  "1000 steps, checkpoints every 50, FP64")
    if name == "gradient_batch":
        m = ntubes or 64
        return [W.gaussian_bumps(tau=GRAD_TAU, seed=4 + k) for k in range(m)], (
            f"{m} inverse problems on Gaussian bumps (seeds 4..{3 + m}): Nx=2048, Qp=3, Qxi=32, Np=2, Nv=5, "
            "dt=0.5dx, open BC, e(x) at tau=0.08 against the runs at tau*=0.05 from perturbed P (seeds "
            f"5..{4 + m}), 1000 steps, checkpoints every 50")
    raise SystemExit(f"unknown workload {name}")


# ---------------------------------------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.rows = []
        self.proc = None
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) == 8:
                self.rows.append(parts)

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm = [float(r[0]) for r in self.rows if _num(r[0])]
        mx = [float(r[1]) for r in self.rows if _num(r[1])]
        reasons = set()
        for r in self.rows:
            for name, val in zip(("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"),
                                 r[4:8]):
                if val.lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(self.rows)}


def _num(s: str) -> bool:
    try:
        float(s)
        return True
    except ValueError:
        return False


# ---------------------------------------------------------------------------------------------------------
# oracle on the host cores (cpu_baseline leg and the reference arm)
# ---------------------------------------------------------------------------------------------------------

def _oracle_worker(conn, specs):
    """Holds the oracle states of its tubes: 'step' advances them by one time step, 'mark' keeps the current
    states, 'step_mark' advances the kept states by one step (leaving the kept states as they were)."""
    sys.path.insert(0, ROOT)
    import oracle

    params, states = [], []
    for s in specs:
        tau = s.tau if (s.tau is not None and math.isfinite(s.tau)) else 0.0
        p = oracle.Params(s.Qp, s.Qxi, s.Np, s.Nv, s.Nx, s.dx, s.dt, tau, s.bc)
        params.append(p)
        states.append(oracle.init_riemann(p, s.left, s.right, s.x_left))
    conn.send("ready")
    kept = None
    while True:
        msg = conn.recv()
        if msg == "stop":
            break
        if msg == "mark":
            kept = [st.copy() for st in states]
            conn.send(0.0)
            continue
        t0 = time.perf_counter()
        for k, p in enumerate(params):
            if msg == "step_mark":
                oracle.step(p, kept[k], 1)  # returns a new array; the kept state is not changed
            else:
                states[k] = oracle.step(p, states[k], 1)
        conn.send(time.perf_counter() - t0)


class OraclePool:
    """Static partition of the tubes over worker processes (spawned: no fork after CUDA initialisation)."""

    def __init__(self, specs, nproc: int):
        import oracle

        oracle.build()  # once, before the workers load it
        nproc = max(1, min(nproc, len(specs)))
        groups = [[] for _ in range(nproc)]
        load = [0] * nproc
        for s in sorted(specs, key=lambda s: -s.Nx * s.Q):  # greedy balance by velocity nodes
            k = load.index(min(load))
            groups[k].append(s)
            load[k] += s.Nx * s.Q
        ctx = mp.get_context("spawn")
        self.conns, self.procs = [], []
        for g in groups:
            a, b = ctx.Pipe()
            p = ctx.Process(target=_oracle_worker, args=(b, g), daemon=True)
            p.start()
            self.conns.append(a)
            self.procs.append(p)
        for c in self.conns:
            assert c.recv() == "ready"
        self.nproc = nproc

    def step(self, msg: str = "step") -> float:
        t0 = time.perf_counter()
        for c in self.conns:
            c.send(msg)
        for c in self.conns:
            c.recv()
        return time.perf_counter() - t0

    def close(self):
        for c in self.conns:
            c.send("stop")
        for p in self.procs:
            p.join(timeout=10)


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def cpu_sample(specs, max_nodes: int = CPU_SAMPLE_NODES, window: int = 4096, cores: int = 1):
    """The workload itself if small enough, else windows cut from its tubes around the membrane (each window
    an independent tube with the same orders, grid spacing, time step and relaxation time), taken from the
    tubes in turn while they fit in max_nodes velocity nodes (the first window always). The windows are made
    short enough (down to 64 cells) that the budget holds at least `cores` of them, so that one process per
    host core has work. Returns (specs, description)."""
    if W.total_nodes(specs) <= max_nodes:
        return specs, f"every tube of the workload ({W.total_nodes(specs)} velocity nodes)"
    qmax = max(s.Q for s in specs)
    window = max(64, min(window, max_nodes // (max(1, cores) * qmax)))
    out, nodes, k, misses = [], 0, 0, 0
    while misses < len(specs) and k < 10000:
        base = specs[k % len(specs)]
        k += 1
        nx = min(base.Nx, window)
        if out and nodes + nx * base.Q > max_nodes:
            misses += 1
            continue
        misses = 0
        win = W.TubeSpec(Nx=nx, Qxi=base.Qxi, tau=base.tau, dt=base.dt, dx=base.dx, Qp=base.Qp, Np=base.Np,
                         Nv=base.Nv, bc=base.bc, x_left=-0.5 * nx * base.dx, left=base.left, right=base.right)
        out.append(win)
        nodes += nx * base.Q
    return out, (f"{len(out)} windows of {out[0].Nx} cells cut around the membrane of the workload's tubes "
                 f"({nodes} velocity nodes)")


def cpu_baseline(specs, desc: str) -> dict:
    sample, what = cpu_sample(specs, cores=host_cores())
    pool = OraclePool(sample, host_cores())
    try:
        wall = pool.step()
    finally:
        pool.close()
    nodes = W.total_nodes(sample)
    # the same oracle on one core: one process advancing the first windows of the sample one after another
    # (as many as make about an eighth of the sample's nodes per core, at least one)
    few, per = [], max(1, nodes // (8 * pool.nproc))
    for s in sample:
        if few and W.total_nodes(few) + s.Nx * s.Q > per:
            break
        few.append(s)
    single = OraclePool(few, 1)
    try:
        wall1 = single.step()
    finally:
        single.close()
    return {"value": nodes / wall / 1e9, "unit": UNIT, "cores": pool.nproc, "kind": "oracle",
            "sample": f"one time step of {what} from the initial condition, plain C FP64 oracle, tubes split over "
                      f"{pool.nproc} processes",
            "seconds": wall,
            "single_core": {"value": W.total_nodes(few) / wall1 / 1e9, "unit": UNIT, "cores": 1,
                            "sample": f"one time step of the first {len(few)} of those windows "
                                      f"({W.total_nodes(few)} velocity nodes) in one process",
                            "seconds": wall1}}


# ---------------------------------------------------------------------------------------------------------
# roofline bookkeeping
# ---------------------------------------------------------------------------------------------------------

def measured_peaks() -> dict:
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh)
    except (OSError, ValueError):
        return {}


def kernel_sources_sha(kind: str) -> str:
    """First 16 hex digits of the sha256 of a kernel's sources (the value the ncu summaries record)."""
    h = hashlib.sha256()
    for src in KERNEL_SRCS[kind]:
        h.update(open(src, "rb").read())
    return h.hexdigest()[:16]


def ncu_traffic_per_launch(kind: str, workload: str):
    """DRAM bytes per stage launch from the committed ncu summary of this kernel on this workload, if it was taken
    on the current kernel sources."""
    path = PROFILES.get((kind, workload))
    try:
        text = open(path).read() if path else None
    except OSError:
        return None
    m_wl = re.search(r"^\s*workload:\s*(\S+)", text or "", re.M)
    if not m_wl or m_wl.group(1) != workload:
        return None
    m_sha = re.search(r"kernel_source_sha256_16:\s*([0-9a-f]+)", text)
    m_tr = re.search(r"dram_bytes_per_stage_launch_full_size:\s*([0-9.eE+]+)", text)
    if not m_sha or not m_tr or m_sha.group(1) != kernel_sources_sha(kind):
        return None
    return float(m_tr.group(1))


# ---------------------------------------------------------------------------------------------------------
# ranks (torchrun): every rank advances its own replica of the workload; no collective on the data path
# ---------------------------------------------------------------------------------------------------------

def reduce_max_over_ranks(values, world: int, device: str = "cuda"):
    """Element-wise max of per-rank timings (the slowest rank sets the job time)."""
    if world <= 1:
        return list(values)
    import torch

    t = torch.tensor(list(values), dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return [float(v) for v in t.tolist()]


def whole_job_rate(nodes_per_rank: int, steps: int, world: int, max_seconds: float) -> float:
    """G velocity-node updates/s of the whole job: the units all ranks processed over the slowest rank's time."""
    return world * nodes_per_rank * steps / max_seconds / 1e9


def rank_prints(rank: int) -> bool:
    return rank == 0


# ---------------------------------------------------------------------------------------------------------
# arms
# ---------------------------------------------------------------------------------------------------------

def _oracle_fd_gradient_task(spec, nsteps: int) -> float:
    """Seconds for the oracle's central-difference dL/dlog(tau) of one tube over nsteps (two forward runs at
    tau exp(+-h), dt fixed, then the loss)."""
    sys.path.insert(0, ROOT)
    import oracle
    from oracle import gradient as og

    p = oracle.params(Qp=spec.Qp, Qxi=spec.Qxi, Np=spec.Np, Nv=spec.Nv, Nx=spec.Nx, dx=spec.dx, dt=spec.dt,
                      tau=spec.tau, bc=spec.bc)
    t0 = time.perf_counter()
    og.grad_log_tau(p, spec.P, spec.n, spec.v, nsteps, lambda m: 0.5 * float(np.sum(m[5] ** 2)), rows=8)
    return time.perf_counter() - t0


def oracle_gradient_sample(specs, nsteps: int):
    """The oracle's gradient (central differences in log tau) on up to one tube per host core for nsteps steps;
    returns (G gradient updates/s, cores, description)."""
    import concurrent.futures as cf

    import oracle

    oracle.build()
    cores = host_cores()
    sample = specs[:max(1, min(len(specs), cores))]
    with cf.ProcessPoolExecutor(max_workers=len(sample), mp_context=mp.get_context("spawn")) as ex:
        t0 = time.perf_counter()
        list(ex.map(_oracle_fd_gradient_task, sample, [nsteps] * len(sample)))
        wall = time.perf_counter() - t0
    nodes = W.total_nodes(sample)
    what = (f"dL/dlog(tau) of a loss of e(x) by central differences of the plain C FP64 oracle (two forward runs of {nsteps} "
            f"steps) on {len(sample)} of the workload's tubes ({nodes} velocity nodes), one process per tube")
    return nodes * nsteps / wall / 1e9, len(sample), what


def run_reference(args, specs, desc, rank):
    if not rank_prints(rank):  # under torchrun only rank 0 runs the CPU reference
        return
    if args.workload.startswith("gradient"):
        vals = []
        for k in range(args.warmup + args.steps):
            val, cores, what = oracle_gradient_sample(specs, GRAD_CPU_STEPS)
            if k >= args.warmup:
                vals.append(val)
        value = statistics.mean(vals)
        nodes = W.total_nodes(specs)
        line = {"impl": "reference", "metric": GRAD_METRIC, "value": value, "unit": GRAD_UNIT,
                "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": 1e3 * nodes * GRAD_STEPS / (value * 1e9), "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": desc, "velocity_nodes": nodes},
                "cpu_baseline": {"value": value, "unit": GRAD_UNIT, "cores": cores, "kind": "oracle",
                                 "sample": f"each step: {what}"},
                "e2e": {"value": value, "unit": GRAD_UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line), flush=True)
        return
    # The oracle's cost differs a lot between hosts (its long double arithmetic is hardware on x86, software on
    # Arm) and grows as the flow develops (its series run only in moving cells). So: W warm-up steps advance a
    # sample from the initial condition, and each of the K timed steps is one step from that same state, which
    # makes every timed step cost the same. The sample is shrunk (fewer windows, then shorter ones) until one
    # such step fits the run's per-step share of REF_BUDGET_S.
    per_step = REF_BUDGET_S / (args.warmup + args.steps)
    target = CPU_SAMPLE_NODES if args.warmup + args.steps <= 10 else 2_000_000
    cores = host_cores()
    pool = None
    for attempt in range(6):
        cand, what = cpu_sample(specs, max_nodes=target, cores=cores)
        pool = OraclePool(cand, cores)
        for _ in range(args.warmup):
            pool.step()
        pool.step("mark")
        t = pool.step("step_mark")
        if t <= per_step or attempt == 5:
            break
        pool.close()
        target = max(1, int(W.total_nodes(cand) * per_step / t * 0.8))
    specs = cand
    try:
        times = [pool.step("step_mark") for _ in range(args.steps)]
    finally:
        pool.close()
    nodes = W.total_nodes(specs)
    total = sum(times)
    value = nodes * args.steps / total / 1e9
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": desc, "velocity_nodes_per_step": nodes},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": pool.nproc, "kind": "oracle",
                             "sample": f"each step: one time step of {what}, from the state after the "
                                       f"{args.warmup} warm-up steps, plain C FP64 oracle, tubes split over "
                                       f"{pool.nproc} processes"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def measure(args, specs, desc, precision, autotune, steps, warmup, rank, world, workload_name, e2e=True):
    """Time `steps` steps of the workload in one handle (after `warmup` steps) with CUDA events on the launching
    stream and return the record: value, ms_per_step, roofline of the stage kernel, e2e through the C ABI with
    host buffers, clocks sampled during the timed steps."""
    import torch

    from paper_1608_03004_gb300 import binding as rb

    dev = torch.cuda.current_device()
    storage = rb.STORAGE[precision]
    tubes = [rb.Tube(s.Qp, s.Qxi, s.Np, s.Nv, s.Nx, s.dx, s.dt, s.tau, s.bc, storage) for s in specs]
    states = np.array([list(s.left) + list(s.right) for s in specs])
    xl = np.array([s.x_left for s in specs])
    stream = torch.cuda.current_stream()
    nodes = W.total_nodes(specs)

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    h = rb.rlb_init_riemann(tubes, states, xl, stream=stream.cuda_stream)
    launch = None
    if autotune:
        best, _ = rb.rlb_autotune(h, 3)
        launch = best.as_dict()
    for _ in range(warmup):
        rb.rlb_step(h, 1)
    rb.rlb_sync(h)
    torch.cuda.synchronize()
    barrier()
    visible = os.environ.get("CUDA_VISIBLE_DEVICES", "").split(",")
    clocks = ClockSampler(int(visible[dev]) if dev < len(visible) and visible[dev].isdigit() else dev)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
    torch.cuda.synchronize()
    graph = launch is not None and launch["graph_steps"] > 0
    ev[0].record(stream)
    if graph:  # the tuned shape replays captured graphs: time the whole run as one
        rb.rlb_step(h, steps)
        ev[steps].record(stream)
    else:
        for k in range(steps):
            rb.rlb_step(h, 1)
            ev[k + 1].record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    barrier()
    run_ms = ev[0].elapsed_time(ev[steps]) if graph else sum(ev[k].elapsed_time(ev[k + 1]) for k in range(steps))
    total_ms = reduce_max_over_ranks([run_ms], world)[0]
    rb.rlb_sync(h)  # raises if any cell went non-physical during the timed steps

    # end to end through the public API with host buffers: H2D of the state from pinned memory, one step,
    # D2H of the fields, every step
    e2e_rec = None
    if e2e:
        e2e_steps = max(3, min(steps, 10))
        host_state = torch.empty(h.state_size, dtype=torch.float64, pin_memory=True).numpy()
        host_fields = torch.empty((rb.NFIELDS, h.nx_total), dtype=torch.float64, pin_memory=True).numpy()
        rb.rlb_get_state(h, host_state)
        torch.cuda.synchronize()
        barrier()
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            rb.rlb_set_state(h, host_state)
            rb.rlb_step(h, 1)
            rb.rlb_moments(h, host_fields)
        e2e_s = reduce_max_over_ranks([time.perf_counter() - t0], world)[0]
        e2e_rec = {"value": whole_job_rate(nodes, e2e_steps, world, e2e_s), "unit": UNIT,
                   "h2d_bytes_per_step": 8 * h.state_size, "d2h_bytes_per_step": 8 * rb.NFIELDS * h.nx_total,
                   "steps": e2e_steps, "api": "rlb_set_state(host) + rlb_step(1) + rlb_moments(host)"}
    rb.rlb_destroy(h)

    value = whole_job_rate(nodes, steps, world, total_ms * 1e-3)
    stage_ms = total_ms / (3 * steps)
    props = torch.cuda.get_device_properties(dev)
    peaks = measured_peaks()
    sm_max = clk.get("sm_max_mhz") or peaks.get("sm_max_mhz") or 2070.0
    hbm_peak = peaks.get("hbm_gbs", 6800.0)  # fallback: the profiling recipe's figure
    esize = ESIZE[precision]
    bytes_per_node_step = 8 * esize  # stage inputs read once (1 + 2 + 2), outputs written once (3)
    hbm_achieved = bytes_per_node_step * nodes / 3 / (stage_ms * 1e-3) / 1e9
    traffic = ncu_traffic_per_launch(precision, workload_name) if args.nx is None else None
    hbm = {"achieved_gbs": hbm_achieved, "peak_gbs": hbm_peak, "frac": hbm_achieved / hbm_peak,
           "note": f"{bytes_per_node_step} algorithmic bytes per velocity node per step, of measured copy"}
    if precision == "f64":
        # FP64: 2 DFMA per SM per clock on GB300 (measured with a DFMA loop: 1.99 per SM-clock at 2070 MHz,
        # 1.253 TFLOP/s; nominal 1.25 TFLOP/s), 4 flops per SM per clock
        fp64_peak = props.multi_processor_count * 4 * sm_max * 1e6 / 1e12
        achieved = FP64_FLOPS_PER_NODE_STAGE * nodes / (stage_ms * 1e-3) / 1e12
        method_rate = FLOPS_PER_NODE_STAGE * nodes / (stage_ms * 1e-3) / 1e12
        roofline = {"bound": "alu", "achieved": achieved, "peak": fp64_peak, "unit": "TFLOP/s",
                    "frac": achieved / fp64_peak, "traffic": traffic, "kernel": "rlb_stage_kernel",
                    "launch_ms": stage_ms,
                    "method_flops_tflops": method_rate,
                    "method_flops_vs_fp64_peak": method_rate / fp64_peak,
                    "note": "FP64 pipe; peak = SMs x 2 DFMA/clk x 2 flops x max SM clock (derived); achieved = the "
                            f"{FP64_FLOPS_PER_NODE_STAGE} algorithmic flops per velocity node and stage that run "
                            f"in FP64. The WENO5 limiter's other {FLOPS_PER_NODE_STAGE - FP64_FLOPS_PER_NODE_STAGE} "
                            "run in double-float on the FP32 pipe; method_flops_* count all "
                            f"{FLOPS_PER_NODE_STAGE} against the FP64 peak (above 1: faster than an all-FP64 "
                            "kernel can be)"}
    else:
        roofline = {"bound": "hbm", "achieved": hbm_achieved, "peak": hbm_peak, "unit": "GB/s",
                    "frac": hbm_achieved / hbm_peak, "traffic": traffic, "kernel": "rlb_stage_rp_kernel",
                    "launch_ms": stage_ms, "note": hbm["note"] + " (the burst copy figure of MEASURED_PEAKS)"}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": steps,
        "warmup": warmup, "ms_per_step": total_ms / steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": {"f64": "f64 (WENO5 limiter in double-float f32)", "f32": "f32 (moments f64)",
                  "bf16": "bf16 storage, f32 arithmetic (moments f64)"}[precision],
        "data": "synthetic",
        "config": {"workload": desc, "velocity_nodes_per_step": nodes, "tubes": len(specs),
                   "precision": precision, "launch": launch or "one CTA per tile, plain launches",
                   "l2": "inputs larger than L2: state %d B x nodes = %.0f MB per buffer, 3 buffers; no flush"
                         % (esize, esize * nodes / 1e6),
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
        "roofline": roofline,
        "hbm": hbm,
        "e2e": e2e_rec,
        "clocks": clk,
        "gpu_launches": 3 * steps,
    }
    return line


def run_ours(args, specs, desc, rank, world):
    line = measure(args, specs, desc, args.precision, args.autotune, args.steps, args.warmup, rank, world,
                   args.workload)
    if args.extras:
        line["extra"] = extras(args, rank, world, line)
    if rank_prints(rank) and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(specs, desc)
    if rank_prints(rank):
        print(json.dumps(line), flush=True)


def extras(args, rank, world, head):
    """The other configurations of the benchmark, each a full record on the headline's line: the stress tube in
    FP32 and BF16 storage and the 256-tube batch in FP32 and FP64 (each with the launch shape rlb_autotune
    picks), the relaxation-time sweep in FP64 and one gradient of the inverse problem. Ratios to the FP64 path
    on the same workload and GPU are added."""
    k = max(1, min(args.steps, EXTRA_STEPS))
    w = args.warmup
    out = {}
    stress_specs, stress_desc = workload("stress")
    for prec in ("f32", "bf16"):
        r = measure(args, stress_specs, stress_desc, prec, True, k, w, rank, world, "stress")
        r["vs_f64_same_workload"] = r["value"] / head["value"] if args.workload == "stress" else None
        out[f"stress_{prec}"] = r
    bspecs, bdesc = workload("batched")
    for prec in ("f32", "f64"):
        out[f"batched_{prec}"] = measure(args, bspecs, bdesc, prec, True, k, w, rank, world, "batched")
    out["batched_f32"]["vs_f64_same_workload"] = out["batched_f32"]["value"] / out["batched_f64"]["value"]
    sspecs, sdesc = workload("sweep")
    out["sweep_f64"] = measure(args, sspecs, sdesc, "f64", False, k, w, rank, world, "sweep")
    gspecs, gdesc = workload("gradient")
    gargs = argparse.Namespace(**vars(args))
    gargs.steps, gargs.warmup, gargs.tubes, gargs.no_cpu_baseline = 3, 3, None, True
    out["gradient_f64"] = run_gradient(gargs, gspecs, gdesc, rank, world, emit=False)
    return out


def run_slabs(args, specs, desc):
    """The stress tube split into args.slabs x-slabs on this one GPU (one handle per slab), advanced by the
    decomposition's data path: before every Runge-Kutta stage each slab packs its edge cells, the blocks go to
    the neighbours' receive buffers by device copies, the ghosts are unpacked, then the stage runs. The result is
    bit-identical to the undivided tube (tests/test_decompose_gpu.py), so the gap to the undivided tube's rate
    is the cost of the exchange and of launching per slab. The steps are timed twice: launched one call at a
    time from the host, then as a captured CUDA graph of one step replayed (decompose.GraphStep); `value` is the
    graph's. Same metric; one JSON line."""
    import torch

    from paper_1608_03004_gb300 import binding as rb
    from paper_1608_03004_gb300 import decompose as D

    (s,) = specs
    x = s.x_left + (np.arange(s.Nx) + 0.5) * s.dx
    P, n, v = (np.where(x < 0, s.left[k], s.right[k]).astype(np.float64) for k in range(3))
    tube = rb.Tube(s.Qp, s.Qxi, s.Np, s.Nv, s.Nx, s.dx, s.dt, s.tau, s.bc, rb.STORAGE[args.precision])
    tubes, bounds, sched = D.slab_tubes(tube, args.slabs)
    stream = torch.cuda.Stream()
    handles = [rb.rlb_init([t], P[a:b], n[a:b], v[a:b], stream=stream.cuda_stream) for t, (a, b) in zip(tubes, bounds)]
    dtype = rb.halo_dtype(handles[0])
    sends = [torch.zeros(rb.rlb_halo_size(h), dtype=dtype, device="cuda") for h in handles]
    recvs = [torch.zeros_like(t) for t in sends]
    ex = D.LocalExchange(sched, 3 * s.Q)
    torch.cuda.synchronize()
    visible = os.environ.get("CUDA_VISIBLE_DEVICES", "").split(",")
    clocks = ClockSampler(int(visible[0]) if visible[0].isdigit() else 0)

    def timed(run):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        run(args.steps)
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / args.steps

    with torch.cuda.stream(stream):
        D.step_slabs(handles, ex, sends, recvs, args.warmup)
        ms_launched = timed(lambda k: D.step_slabs(handles, ex, sends, recvs, k))
    graph = D.GraphStep(handles, ex, sends, recvs, stream)
    graph(args.warmup)
    ms = timed(graph)
    clk = clocks.stop()
    for h in handles:
        rb.rlb_sync(h)
        rb.rlb_destroy(h)
    nodes = W.total_nodes(specs)
    esize = ESIZE[args.precision]
    print(json.dumps({
        "metric": METRIC, "value": nodes / (ms * 1e-3) / 1e9, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": args.precision, "data": "synthetic",
        "config": {"workload": desc, "slabs": args.slabs, "slab_cells": [b - a for a, b in bounds],
                   "exchange": "before every stage: rlb_halo_pack, device copies of 3 Q cells per side, "
                               "rlb_halo_unpack, then rlb_stage per slab",
                   "halo_bytes_per_boundary_and_stage": 2 * 3 * s.Q * esize,
                   "ms_per_step_launched": ms_launched, "ms_per_step_graph": ms,
                   "parallelism": f"{args.slabs} x-slabs of one tube on one GPU"},
        "clocks": clk, "gpu_launches": 3 * args.steps * (3 * args.slabs),  # packs, unpacks, stages (+ copies)
    }), flush=True)


def run_gradient(args, specs, desc, rank, world, emit=True):
    """Gradients of the inverse problem through the adjoint: each step is one full gradient (set the initial
    state, rlb_record, the loss's seed, rlb_backward, rlb_init_vjp)."""
    import torch

    from paper_1608_03004_gb300 import adjoint
    from paper_1608_03004_gb300 import binding as rb

    dev = torch.cuda.current_device()
    stream = torch.cuda.current_stream()
    f64 = dict(dtype=torch.float64, device="cuda")
    mk = lambda s, tau: rb.Tube(s.Qp, s.Qxi, s.Np, s.Nv, s.Nx, s.dx, s.dt, tau, s.bc, rb.STORAGE_F64)  # noqa: E731
    tubes = [mk(s, GRAD_TAU) for s in specs]
    P, n, v = (np.concatenate([getattr(s, a) for s in specs]) for a in ("P", "n", "v"))
    Pd, nd, vd = (torch.tensor(a, **f64) for a in (P, n, v))
    nodes = W.total_nodes(specs)

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    # the targets: runs at tau* from the initial pressure perturbed by a second seed-fixed set of bumps
    tg = [W.perturbed(s, seed=GRAD_TARGET_SEED + k) for k, s in enumerate(specs)]
    Pt_, nt_, vt_ = (torch.tensor(np.concatenate([getattr(s, a) for s in tg]), **f64) for a in ("P", "n", "v"))
    with rb.rlb_init([mk(s, GRAD_TAU_STAR) for s in specs], Pt_, nt_, vt_) as hs:
        rb.rlb_step(hs, GRAD_STEPS)
        ft = torch.empty((rb.NFIELDS, hs.nx_total), **f64)
        rb.rlb_moments(hs, ft)
        target = ft[rb.F_E].clone()
    h = rb.rlb_init(tubes, Pd, nd, vd)
    F0 = torch.empty(h.state_size, **f64)
    rb.rlb_get_state(h, F0)
    fields = torch.empty((rb.NFIELDS, h.nx_total), **f64)
    gm = torch.zeros((rb.NFIELDS, h.nx_total), **f64)
    seed, gF = torch.empty(h.state_size, **f64), torch.empty(h.state_size, **f64)
    gP, gn, gv = (torch.empty(h.nx_total, **f64) for _ in range(3))
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(5)] for _ in range(args.steps)]

    def gradient(e=None):
        rb.rlb_set_state(h, F0)
        if e:
            e[0].record(stream)
        rb.rlb_record(h, GRAD_STEPS, args.every)
        if e:
            e[1].record(stream)
        rb.rlb_moments(h, fields)
        torch.sub(fields[rb.F_E], target, out=gm[rb.F_E])  # dL/de of L = 1/2 sum (e - target)^2
        rb.rlb_fields_vjp(h, gm, seed)
        if e:
            e[2].record(stream)
        _, glt = rb.rlb_backward(h, seed, gF)
        if e:
            e[3].record(stream)
        rb.rlb_init_vjp(h, Pd, nd, vd, gF, gP, gn, gv)
        if e:
            e[4].record(stream)
        return glt

    for _ in range(args.warmup):
        gradient()
    torch.cuda.synchronize()
    barrier()
    visible = os.environ.get("CUDA_VISIBLE_DEVICES", "").split(",")
    clocks = ClockSampler(int(visible[dev]) if dev < len(visible) and visible[dev].isdigit() else dev)
    for k in range(args.steps):
        glt = gradient(ev[k])
    torch.cuda.synchronize()
    clk = clocks.stop()
    barrier()
    total_ms = sum(e[0].elapsed_time(e[4]) for e in ev)
    record_ms = sum(e[0].elapsed_time(e[1]) for e in ev)
    backward_ms = sum(e[2].elapsed_time(e[3]) for e in ev)
    total_ms, record_ms, backward_ms = reduce_max_over_ranks([total_ms, record_ms, backward_ms], world)
    # the reverse sweep recomputes the recorded forward launches (unless the record kept the stage inputs),
    # then runs 3 GRAD_STEPS adjoint launches
    recompute_ms = record_ms if args.every < GRAD_STEPS else 0.0  # a kept record leaves nothing to recompute
    adj_launch_ms = max(backward_ms - recompute_ms, 1e-9) / (3 * GRAD_STEPS * args.steps)

    # end to end: the autograd call from host arrays (pinned H2D of P, n, v; D2H of the four gradients)
    e2e_steps = max(2, min(args.steps, 3))
    Ph, nh, vh = (torch.from_numpy(a).pin_memory() for a in (P, n, v))

    def user_gradient():
        lt = torch.full((len(tubes),), math.log(GRAD_TAU), dtype=torch.float64, requires_grad=True)
        Pt, nt, vt = (a.to("cuda", non_blocking=True).requires_grad_() for a in (Ph, nh, vh))
        f = adjoint.run_fields(lt, Pt, nt, vt, tubes, GRAD_STEPS, args.every)
        (0.5 * ((f[rb.F_E] - target) ** 2).sum()).backward()
        return [lt.grad.numpy(), Pt.grad.cpu().numpy(), nt.grad.cpu().numpy(), vt.grad.cpu().numpy()]

    user_gradient()  # warm-up: the first call loads torch's kernels for the loss and its backward
    torch.cuda.synchronize()
    barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        grads = user_gradient()
    e2e_s = reduce_max_over_ranks([time.perf_counter() - t0], world)[0]
    rb.rlb_destroy(h)
    assert all(np.all(np.isfinite(g)) for g in grads) and np.all(np.isfinite(glt))

    props = torch.cuda.get_device_properties(dev)
    sm_max = clk.get("sm_max_mhz") or measured_peaks().get("sm_max_mhz") or 2070.0
    fp64_peak = props.multi_processor_count * 4 * sm_max * 1e6 / 1e12
    achieved = ADJ_FLOPS_PER_NODE_STAGE * nodes / (adj_launch_ms * 1e-3) / 1e12
    tiles = sum((s.Nx + 59) // 60 for s in specs)
    line = {
        "metric": GRAD_METRIC, "value": whole_job_rate(nodes, GRAD_STEPS * args.steps, world, total_ms * 1e-3),
        "unit": GRAD_UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": total_ms / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64 (forward WENO5 limiter in double-float f32)", "data": "synthetic",
        "config": {"workload": desc, "velocity_nodes": nodes, "tubes": len(specs),
                   "step": ("one gradient: record 1000 steps with checkpoints every %d, seed, reverse sweep (recompute + "
                            "adjoint), initial-condition adjoint" % args.every) if args.every < GRAD_STEPS else
                           "one gradient: record 1000 steps keeping every stage input, seed, reverse sweep (adjoint "
                           "only), initial-condition adjoint",
                   "record_ms_per_step": record_ms / args.steps, "backward_ms_per_step": backward_ms / args.steps,
                   "adjoint_ctas_per_launch": tiles,
                   "l2": "state %.1f MB per buffer; checkpoints and the recomputed segment %.0f MB; no flush"
                         % (8 * nodes / 1e6, 8 * nodes * (-(-GRAD_STEPS // args.every) + 3 * min(args.every, GRAD_STEPS) + 1) / 1e6),
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": fp64_peak, "unit": "TFLOP/s",
                     "frac": achieved / fp64_peak,
                     "traffic": ncu_traffic_per_launch("adjoint", args.workload) if args.tubes is None else None,
                     "kernel": "rlb_adjoint_kernel",
                     "launch_ms": adj_launch_ms,
                     "note": f"{ADJ_FLOPS_PER_NODE_STAGE} algorithmic FP64 flops per velocity node per adjoint "
                             "stage; launch time = (reverse sweep - recompute) / adjoint launches; peak = SMs x 2 "
                             "DFMA/clk x 2 flops x max SM clock (derived)"},
        "e2e": {"value": whole_job_rate(nodes, GRAD_STEPS * e2e_steps, world, e2e_s), "unit": GRAD_UNIT,
                "h2d_bytes_per_step": 3 * 8 * h.nx_total, "d2h_bytes_per_step": 3 * 8 * h.nx_total + 8 * len(tubes),
                "steps": e2e_steps, "api": "adjoint.run_fields (torch.autograd) from pinned host fields, "
                                          "gradients read back"},
        "clocks": clk,
        "gpu_launches": 9 * GRAD_STEPS + 3,
    }
    if not emit:
        return line
    if rank_prints(rank) and not args.no_cpu_baseline:
        val, cores, what = oracle_gradient_sample(specs, GRAD_CPU_STEPS)
        line["cpu_baseline"] = {"value": val, "unit": GRAD_UNIT, "cores": cores, "kind": "oracle", "sample": what}
    if rank_prints(rank):
        print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None, help="default 100 for the stress tube, 200 for the other step workloads, 5 for the gradient workloads")
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=["sweep", "small", "stress", "batched", "gradient", "gradient_batch"],
                    default=None, help="default stress, with the other configurations as extras")
    ap.add_argument("--precision", choices=["f64", "f32", "bf16"], default=None,
                    help="default f64; f32 for the batched workload (FP32 storage, FP64 moments)")
    ap.add_argument("--autotune", action="store_true", help="pick the launch shape with rlb_autotune first "
                    "(default for the batched workload)")
    ap.add_argument("--nx", type=int, default=None, help="cells of the stress tube (default 1048576)")
    ap.add_argument("--tubes", type=int, default=None, help="tubes of the gradient_batch workload (default 64)")
    ap.add_argument("--every", type=int, default=GRAD_EVERY, help="checkpoint interval of the gradient workloads "
                    "(default 50; >= 1000 keeps every stage input and recomputes nothing)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="time the headline workload only")
    ap.add_argument("--slabs", type=int, default=0, help="with --workload stress: split the tube into this many "
                    "x-slabs on this GPU and time the decomposition's data path (halo exchange before every stage)")
    args = ap.parse_args()
    args.extras = args.workload is None and not args.no_extras
    if args.workload is None:
        args.workload = "stress"
    if args.steps is None:
        args.steps = 5 if args.workload.startswith("gradient") else (100 if args.workload == "stress" else 200)
    if args.warmup < 3:
        raise SystemExit("--warmup must be >= 3")
    if args.precision is None:
        args.precision = "f32" if args.workload == "batched" else "f64"
    if args.workload == "batched":
        args.autotune = True
    specs, desc = workload(args.workload, args.nx, args.tubes)
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.impl == "reference":
        run_reference(args, specs, desc, rank)
        return
    import torch

    if world > 1:
        local = int(os.environ.get("LOCAL_RANK", "0"))
        torch.cuda.set_device(local)
        torch.distributed.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    try:
        if args.slabs > 1:
            if args.workload != "stress" or world > 1:
                raise SystemExit("--slabs takes --workload stress on one GPU")
            run_slabs(args, specs, desc)
        elif args.workload.startswith("gradient"):
            run_gradient(args, specs, desc, rank, world)
        else:
            run_ours(args, specs, desc, rank, world)
    finally:
        if world > 1:
            torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
