#!/usr/bin/env python3
"""Benchmark: fiber node-updates/s of the full Strang split step on GB300.

Workload (per GPU): the full-scale bundle, 67,600 fibers (260 x 260) x 1481
nodes = 1.0e8 nodes, h = 0.01 cm, 200 motor units with exponential sizes,
Poisson firing at 10-30 Hz; seeded synthetic inputs.  One benchmark "step" is
one CUDA-graph launch of BENCH_SPLIT_STEPS = 100 split steps (each: CN half,
3 Heun substeps, CN half, for every fiber), i.e. 0.3 ms of simulated time.
The timed region runs --steps such graph launches with the state already
resident in HBM.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Under torchrun (N > 1) every rank simulates its own bundle (seed 5 + rank) on
its own GPU with no data-path communication (fibers are independent): weak
scaling, whole-job value = sum of node-updates over ranks / max time.

``--impl reference`` times the FP64 CPU oracle (the only reference
implementation of this method) on the host cores instead.

Secondary legs on the same GPU (each optional): the 7744-fiber bundle, the
ragged 20,000-fiber bundle with the autotuner and 1000-step graphs, the
learned-surrogate path timed while action potentials propagate, adaptive
computation, the scheme variants and the exp* approximation.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2107_07104_gb300 import workloads as W  # noqa: E402

METRIC = "fiber node-updates/s (full split step) at max|ΔVm|≤0.5 mV, plain FP32 vs surrogate"
UNIT = "node-updates/s"
WORKLOAD = "bundle 67600 fibers x 1481 nodes (260x260), 200 MUs, Poisson 10-30 Hz"
BENCH_SPLIT_STEPS = 100          # split steps per benchmark step (one CUDA-graph launch)
# Algorithmic work per node-update of the plain FP32 path (the method's operation counts):
BYTES_PER_NODE_UPDATE = 32.0     # read + write V, m, h, n (FP32) once per split step
FMA_OPS_PER_NODE_UPDATE = 238.0  # FP32 FMA-pipe operations of the method per split step
EX2_OPS_PER_NODE_UPDATE = 24.0   # 2^x special-function operations per split step (4 per HH RHS)
RCP_OPS_PER_NODE_UPDATE = 18.0   # 1/x special-function operations per split step (3 per HH RHS)
# Per-SM per-clock unit rates on GB300 (FP32 FMA lanes; XU pipe rates of
# ex2.approx and rcp.approx, which share the special-function pipe).
FP32_LANES_PER_SM = 128.0
EX2_PER_SM = 32.0
RCP_PER_SM = 16.0
NCU_SUMMARY = os.path.join("profiles", "split_step_kernel_bundle7744_ncu.md")


def _env_int(k, d):
    try:
        return int(os.environ.get(k, d))
    except ValueError:
        return d


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return json.load(f), "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int, period_ms: int = 50):
        self.gpu = gpu_index
        self.period = period_ms
        self.proc = None
        self.path = None

    def __enter__(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.out = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", str(self.period)],
                                         stdout=self.out, stderr=subprocess.DEVNULL)
            time.sleep(0.3)  # let the sampler start before the timed region
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.out.close()

    def summary(self):
        if self.proc is None or not self.path:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, smax, pw, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax.append(float(parts[2]))
                    pw.append(float(parts[3]))
                except ValueError:
                    continue
                for name, v in zip(names, parts[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(name)
        os.unlink(self.path)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm), "sample_period_ms": self.period, "power_w_max": max(pw) if pw else None}


def kernel_source_hash() -> str:
    import hashlib
    h = hashlib.sha256()
    for name in ("split_step_kernel.cuh", "split_step.cu", "hh_device.cuh", "fibers_internal.h", "solver_tables.cpp"):
        with open(os.path.join(ROOT, "paper_2107_07104_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def profile_fields():
    """Capture identity and DRAM figures of the committed ncu summary."""
    try:
        with open(os.path.join(ROOT, NCU_SUMMARY)) as f:
            text = f.read()
    except OSError:
        return {}
    fields = {}
    for line in text.splitlines():
        if line.startswith("- ") and ": " in line:
            k, v = line[2:].split(": ", 1)
            fields[k.strip()] = v.strip().strip("`")
    return fields


def dram_traffic_per_node_update(tune):
    """DRAM bytes per node-update of the step kernel from the committed ncu
    capture, or None when the kernel source or the launch shape has changed
    since the counters were taken."""
    fields = profile_fields()
    try:
        same = (fields.get("kernel source sha256[:16]") == kernel_source_hash()
                and int(fields.get("steps_per_launch", -1)) == tune["steps_per_launch"]
                and int(fields.get("nodes_per_thread", -1)) == tune["nodes_per_thread"]
                and int(fields.get("reaction_pairs", -1)) == tune["reaction_pairs"]
                and int(fields.get("ctas_per_sm", -1)) == tune["ctas_per_sm"])
        if not same:
            return None
        return float(fields["dram bytes per launch"]) / float(fields["node-updates per launch"])
    except (KeyError, ValueError):
        return None


WORKLOADS = {
    "bundle_67600": ("bundle 67600 fibers x 1481 nodes (260x260), 200 MUs, Poisson 10-30 Hz",
                     lambda rank: W.bundle_67600(seed=5 + rank, t_end_ms=100.0)),
    # smaller case for profiler captures (ncu) of the same kernel
    "bundle_7744": ("bundle 7744 fibers x 1481 nodes (88x88), 100 MUs, Poisson 10-30 Hz",
                    lambda rank: W.bundle_7744(seed=2 + rank, t_end_ms=20.0)),
}


def rank_workload(rank: int, name: str = "bundle_67600"):
    """Each rank simulates its own seeded bundle (the full-scale one unless
    named otherwise): fibers are independent, so ranks share nothing on the
    data path (weak scaling)."""
    return WORKLOADS[name][1](rank)


def aggregate_over_ranks(node_updates_local: float, seconds_local: float, dist, device=None):
    """(node-updates summed over ranks, wall seconds max over ranks)."""
    if dist is None:
        return node_updates_local, seconds_local
    import torch
    t = torch.tensor([seconds_local], dtype=torch.float64, device=device)
    n = torch.tensor([node_updates_local], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(n, op=dist.ReduceOp.SUM)
    return float(n.item()), float(t.item())


def dist_setup():
    world = _env_int("WORLD_SIZE", 1)
    rank = _env_int("RANK", 0)
    local = _env_int("LOCAL_RANK", 0)
    pg = None
    if world > 1:
        import torch.distributed as dist
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        backend = "nccl"
        try:
            import torch
            torch.cuda.set_device(local)
        except Exception:
            backend = "gloo"
        dist.init_process_group(backend=backend)
        pg = dist
    return world, rank, local, pg


def cpu_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def oracle_rate(w, fibers: int, steps: int):
    """Node-updates/s of the FP64 oracle on the first `fibers` fibers, all host cores."""
    import oracle
    sub = w.subset(np.arange(min(fibers, w.n_fibers)))
    state = oracle.init_state(sub.params, sub.total_nodes, sub.vm0)
    cores = cpu_cores()
    t0 = time.perf_counter()
    oracle.run(sub.params, sub.n_nodes, sub.mu_of_fiber, sub.junction, sub.mu_offsets, sub.fire_times, state, 0,
               steps, n_threads=cores)
    dt = time.perf_counter() - t0
    oracle_rate.last = (sub, state[:sub.total_nodes].copy())
    return sub.total_nodes * steps / dt, dt, cores, sub.total_nodes


def accuracy_vs_oracle(tune, steps):
    """The GPU path on the CPU-baseline sample (same fibers, same steps, the
    bench's launch shape) against the FP64 oracle's final V."""
    from paper_2107_07104_gb300 import fibers as F
    sub, v_ref = oracle_rate.last
    with F.Fibers.from_workload(sub, tuning=dict(tune, graph_steps=0)) as f:
        f.step(steps)
        v = f.read_vm().astype(np.float64)
    d = v - v_ref
    return {"fibers": int(sub.n_fibers), "split_steps": int(steps), "max_abs_mv": float(np.max(np.abs(d))),
            "rel_l2": float(np.linalg.norm(d) / np.linalg.norm(v_ref)), "tolerance_mv": 0.5,
            "nodes_above_rest_plus_15_mv": int(np.sum(v_ref > sub.params["Vrest"] + 15.0))}


def run_reference(args, world, rank):
    if rank != 0:
        return 0
    w = rank_workload(0)
    import oracle
    cores = cpu_cores()
    # size the per-step sample so that warm-up + timed steps take about 100 s
    rate, _, _, _ = oracle_rate(w, 64, 2)
    split = args.steps + args.warmup
    fibers = int(np.clip(rate * 100.0 / (1481.0 * split), 16, 1024))
    sub = w.subset(np.arange(fibers))
    state = oracle.init_state(sub.params, sub.total_nodes, sub.vm0)
    step = 0
    for _ in range(args.warmup):
        oracle.run(sub.params, sub.n_nodes, sub.mu_of_fiber, sub.junction, sub.mu_offsets, sub.fire_times, state,
                   step, 1, n_threads=cores)
        step += 1
    t0 = time.perf_counter()
    oracle.run(sub.params, sub.n_nodes, sub.mu_of_fiber, sub.junction, sub.mu_offsets, sub.fire_times, state, step,
               args.steps, n_threads=cores)
    dt = time.perf_counter() - t0
    value = sub.total_nodes * args.steps / dt
    sample = (f"first {fibers} of 67600 fibers x 1481 nodes, one split step per benchmark step "
              f"({args.steps} timed), FP64 oracle")
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": WORKLOAD, "sample": sample, "parallelism": "host threads"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def timed_graph_launches(fib, stream, dev, k, split_steps):
    """k benchmark steps (each `split_steps` split steps, one graph launch) with
    a CUDA event between launches on the launching stream: (total ms, per-launch ms)."""
    import torch
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(k + 1)]
    torch.cuda.synchronize(dev)
    ev[0].record(stream)
    for i in range(k):
        fib.step(split_steps)
        ev[i + 1].record(stream)
    ev[k].synchronize()
    per = [ev[i].elapsed_time(ev[i + 1]) for i in range(k)]
    return ev[0].elapsed_time(ev[k]), per


def run_gpu(args, world, rank, local, dist):
    import torch
    from paper_2107_07104_gb300 import fibers as F

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    w = rank_workload(rank, args.workload)
    workload_name = WORKLOADS[args.workload][0]
    total = w.total_nodes
    S = BENCH_SPLIT_STEPS
    stream = torch.cuda.Stream(device=dev)
    tuning = dict(nodes_per_thread=args.nodes_per_thread, warps_per_cta=args.warps_per_cta,
                  steps_per_launch=S, graph_steps=S, reaction_pairs=args.reaction_pairs,
                  ctas_per_sm=args.ctas_per_sm, warp_roles=args.warp_roles)

    def barrier():
        if dist is not None:
            dist.barrier()

    # ---- device-resident timing: K graph launches, state already in HBM ----
    fib = F.Fibers.from_workload(w, tuning=tuning, stream=stream)
    for _ in range(args.warmup):
        fib.step(S)
    fib.synchronize()
    launches0 = fib.kernel_launches
    barrier()
    torch.cuda.synchronize(dev)
    with ClockSampler(local) as clk:
        ms, per_launch = timed_graph_launches(fib, stream, dev, args.steps, S)
    torch.cuda.synchronize(dev)
    barrier()
    launches = fib.kernel_launches - launches0
    tune = fib.tuning
    vm = fib.read_vm()
    finite = bool(np.isfinite(vm).all())
    fib.close()
    split_steps = args.steps * S
    node_updates, t_max = aggregate_over_ranks(float(total) * split_steps, ms / 1e3, dist, dev)
    value = node_updates / t_max

    # ---- end to end through the C ABI with host buffers ---------------------
    # Timed: fibers_create and set_stimulus_times from host arrays (the
    # bundle's inputs), then every benchmark step one graph launch of S split
    # steps and a read of every node's V into pinned host memory
    # (read_vm_async into two alternating buffers: the copy of step k
    # overlaps the computation of step k + 1, and a buffer is reused only
    # after its previous read has arrived).  The timer stops when the last
    # read is in host memory.
    host_out = [torch.empty(total, dtype=torch.float32, pin_memory=True) for _ in range(2)]
    barrier()
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    fib2 = F.Fibers.from_workload(w, tuning=tune, stream=stream)
    t_create = time.perf_counter() - t0
    tickets = []
    for k in range(args.steps):
        fib2.step(S)
        if k >= 2:
            fib2.read_vm_wait(tickets[k - 2])
        tickets.append(fib2.read_vm_async(host_out[k % 2]))
    for t in tickets[-2:]:
        fib2.read_vm_wait(t)
    t_e2e = time.perf_counter() - t0
    e2e_finite = bool(np.isfinite(host_out[(args.steps - 1) % 2].numpy()).all())
    fib2.close()
    _, te = aggregate_over_ranks(float(total) * split_steps, t_e2e, dist, dev)
    e2e_value = node_updates / te
    h2d = 12 * w.n_fibers + 8 * (w.mu_offsets.size + w.fire_times.size)
    d2h = 4 * total * args.steps

    if rank != 0:
        return 0
    peaks, peak_kind = measured_peaks()
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    sm_max = float(peaks.get("sm_max_mhz", 2070.0)) * 1e6
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    per_gpu_rate = float(total) * split_steps / (ms / 1e3)
    clocks = clk.summary()
    # The dominant kernel: one split-step launch per graph (the graph's other
    # kernel is the 1-thread step-counter update).  Per-launch duration from
    # the events between graph launches.
    launch_ms = statistics.mean(per_launch)
    alg_bytes = BYTES_PER_NODE_UPDATE * total * S
    achieved_gbs = alg_bytes / (launch_ms * 1e-3) / 1e9
    traffic_per_nu = dram_traffic_per_node_update(tune)
    # ALU roofline: node-updates/s if the binding pipe (FP32 FMA or the
    # special-function XU pipe) ran at its full rate on every SM at the
    # maximum SM clock.
    fma_clk = FMA_OPS_PER_NODE_UPDATE / FP32_LANES_PER_SM
    xu_clk = EX2_OPS_PER_NODE_UPDATE / EX2_PER_SM + RCP_OPS_PER_NODE_UPDATE / RCP_PER_SM
    alu_peak = n_sm * sm_max / max(fma_clk, xu_clk)
    cpu = None
    accuracy = None
    if not args.no_cpu_baseline:
        rate, dt, cores, nodes = oracle_rate(w, args.cpu_fibers, args.cpu_steps)
        cpu = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"first {args.cpu_fibers} of {w.n_fibers} fibers x 1481 nodes, {args.cpu_steps} split steps "
                         f"({dt:.1f} s of FP64 oracle on {cores} threads)"}
        accuracy = accuracy_vs_oracle(tune, args.cpu_steps)
    legs = {}
    if not args.no_legs:
        legs["bundle_7744"] = bundle_7744_leg(args, stream, dev)
        legs["split_roles"] = split_roles_leg(args, stream, dev)
        legs["ragged_20000"] = ragged_leg(args, stream, dev)
        if not args.no_surrogate:
            legs["surrogate"] = surrogate_leg(args, stream, dev)
        legs["adaptive"] = adaptive_leg(args, stream, dev)
        legs["schemes"] = schemes_leg(args, stream, dev)
        legs["exp_approx"] = exp_approx_leg(args, stream, dev)
        legs["emg"] = emg_leg(args, stream, dev)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": (t_max * 1e3) / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": workload_name, "fibers": int(w.n_fibers), "nodes": int(total),
                   "bench_step": f"{S} split steps (one CUDA-graph launch of the split-step kernel, "
                                 f"{S * w.params['dt_split']:.1f} simulated ms)",
                   "split_steps_timed": split_steps,
                   "path": "plain FP32 (HH Heun x3 + CN/partitioned Thomas x2)",
                   "tuning": tune, "parallelism": f"replicas x{world} (independent fibers)",
                   "l2": f"state {4 * 4 * total / 1e9:.2f} GB > 129 MB L2, loaded from and stored to HBM by "
                         f"every launch"},
        "roofline": {
            "bound": "hbm", "achieved": achieved_gbs, "peak": hbm_peak, "unit": "GB/s",
            "frac": achieved_gbs / hbm_peak,
            "traffic": None if traffic_per_nu is None else traffic_per_nu * total * S,
            "traffic_source": (f"{NCU_SUMMARY}: ncu dram__bytes_read.sum + dram__bytes_write.sum per node-update "
                               f"of the same kernel source and launch shape, scaled to this launch"
                               if traffic_per_nu is not None else
                               "null: the kernel changed since the committed ncu capture"),
            "peak_kind": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)",
            "kernel": "split_step_kernel", "kernel_ms_per_launch": launch_ms, "launches_timed": len(per_launch),
            "kernel_ms_per_launch_median": statistics.median(per_launch),
            "kernel_ms_per_launch_spread": [min(per_launch), max(per_launch)],
            "algorithmic_bytes_per_launch": alg_bytes,
            "algorithmic_bytes": f"{BYTES_PER_NODE_UPDATE:.0f} B per node-update (read + write V, m, h, n in FP32) "
                                 f"x {total} nodes x {S} split steps per launch",
            "alu": {"bound": "alu", "achieved": per_gpu_rate / 1e9, "peak": alu_peak / 1e9,
                    "unit": "Gnode-updates/s", "frac": per_gpu_rate / alu_peak,
                    "peak_derivation": f"{n_sm} SMs x {sm_max / 1e6:.0f} MHz / max(FMA "
                                       f"{FMA_OPS_PER_NODE_UPDATE:.0f} ops / 128 lanes = {fma_clk:.3f} clk, XU "
                                       f"{EX2_OPS_PER_NODE_UPDATE:.0f} ex2 / 32 + {RCP_OPS_PER_NODE_UPDATE:.0f} "
                                       f"rcp / 16 = {xu_clk:.3f} clk) per node-update",
                    "note": "the state stays on chip for a whole launch, so DRAM traffic is about 1 % of the "
                            "algorithmic bytes and the special-function and FP32 pipes bind the kernel"},
        },
        "cpu_baseline": cpu,
        "accuracy_vs_oracle": accuracy,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d / args.steps,
                "d2h_bytes_per_step": d2h / args.steps,
                "includes": "fibers_create + set_stimulus_times from host arrays, then per benchmark step "
                            f"step({S}) and read_vm_async of every node's V into one of two pinned host "
                            "buffers (the copy overlaps the next step; timer stops when the last read has "
                            "arrived)",
                "create_s": t_create, "finite": e2e_finite},
        "gpu_launches": int(launches),
        "clocks": clocks,
        "finite": finite,
    }
    line.update(legs)
    print(json.dumps(line), flush=True)
    return 0


def activation_times(samples, dt):
    """First upward 0 mV crossing per node (linear interpolation), NaN if none."""
    s = np.asarray(samples, np.float64)
    cross = (s[:-1] < 0) & (s[1:] >= 0)
    t = np.full(s.shape[1], np.nan)
    idx = np.nonzero(cross.any(axis=0))[0]
    k = np.argmax(cross, axis=0)[idx]
    v0, v1 = s[k, idx], s[k + 1, idx]
    t[idx] = (k + 1 + (0.0 - v0) / (v1 - v0)) * dt
    return t


def time_steps(fib, stream, dev, steps, chunk):
    """ms for `steps` split steps enqueued as step(chunk) calls."""
    import torch
    torch.cuda.synchronize(dev)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps // chunk):
        fib.step(chunk)
    e1.record(stream)
    e1.synchronize()
    return e0.elapsed_time(e1)


def bundle_7744_leg(args, stream, dev, steps=1000):
    """The 7744-fiber bundle (88 x 88 x 1481): plain FP32 rate with 100-step graphs."""
    from paper_2107_07104_gb300 import fibers as F
    w = W.bundle_7744(seed=2, t_end_ms=20.0)
    hbm_peak = float(measured_peaks()[0].get("hbm_gbs", 6800.0))
    with F.Fibers.from_workload(w, tuning=dict(graph_steps=100), stream=stream) as fib:
        fib.step(300)
        ms = time_steps(fib, stream, dev, steps, 100)
        finite = bool(np.isfinite(fib.read_vm()).all())
    rate = float(w.total_nodes) * steps / (ms / 1e3)
    return {"workload": "bundle 7744 fibers x 1481 nodes (88x88), 100 MUs, Poisson 10-30 Hz",
            "node_updates_per_s": rate, "ms_per_split_step": ms / steps, "split_steps": steps, "finite": finite,
            "hbm_frac_at_32_bytes": rate * BYTES_PER_NODE_UPDATE / 1e9 / hbm_peak}


def split_roles_leg(args, stream, dev, steps=1000):
    """The launch shapes of the step kernel on the headline workload: the
    fused kernel and the two split-role shapes (reaction and diffusion on
    separate warps), each timed over the same steps in 100-step graphs."""
    from paper_2107_07104_gb300 import fibers as F
    w = rank_workload(0, args.workload)
    out = {"workload": WORKLOADS[args.workload][0], "split_steps": steps}
    for roles, name in ((1, "fused"), (2, "split roles, 2 fibers per CTA"), (3, "split roles, 8 fibers per CTA")):
        with F.Fibers.from_workload(w, tuning=dict(graph_steps=100, warp_roles=roles), stream=stream) as fib:
            fib.step(200)
            ms = time_steps(fib, stream, dev, steps, 100)
            finite = bool(np.isfinite(fib.read_vm()).all())
        out[name] = {"warp_roles": roles, "node_updates_per_s": float(w.total_nodes) * steps / (ms / 1e3),
                     "ms_per_split_step": ms / steps, "finite": finite}
    base = out["fused"]["node_updates_per_s"]
    for k in ("split roles, 2 fibers per CTA", "split roles, 8 fibers per CTA"):
        out[k]["vs_fused"] = out[k]["node_updates_per_s"] / base
    return out


def ragged_leg(args, stream, dev, steps=2000):
    """The ragged bundle (20,000 fibers of U{800..2000} nodes, V0 = rest +
    N(0, 0.5 mV)): the autotuner chooses the launch shape on the bundle's own
    fibers, then 1000-step CUDA graphs are timed."""
    from paper_2107_07104_gb300 import fibers as F
    w = W.ragged_20000(seed=3, t_end_ms=50.0)
    hbm_peak = float(measured_peaks()[0].get("hbm_gbs", 6800.0))
    with F.Fibers.from_workload(w, tuning=dict(graph_steps=1000), stream=stream) as fib:
        t0 = time.perf_counter()
        best = fib.autotune(20)
        t_tune = time.perf_counter() - t0
        fib.step(1000)
        ms = time_steps(fib, stream, dev, steps, 1000)
        finite = bool(np.isfinite(fib.read_vm()).all())
        tune = fib.tuning
    rate = float(w.total_nodes) * steps / (ms / 1e3)
    return {"workload": "ragged 20000 fibers x U{800..2000} nodes, 150 MUs, Poisson 10-40 Hz",
            "nodes": int(w.total_nodes), "node_updates_per_s": rate, "ms_per_split_step": ms / steps,
            "split_steps": steps, "graph_steps": 1000, "autotuned": tune, "autotune_s": t_tune,
            "finite": finite, "hbm_frac_at_32_bytes": rate * BYTES_PER_NODE_UPDATE / 1e9 / hbm_peak,
            "best": best}


def firing_subset(w, n=64, seed=9):
    """n fibers of the bundle whose motor unit fires (the accuracy sample)."""
    firing = [f for f in range(w.n_fibers) if w.mu_offsets[w.mu_of_fiber[f] + 1] > w.mu_offsets[w.mu_of_fiber[f]]]
    return w.subset(np.sort(np.random.default_rng(seed).choice(firing, min(n, len(firing)), replace=False)))


TRAJ_EVERY = 10


def trajectory(sub, mode=None, blob=None, **params):
    """V of every node of ``sub`` every TRAJ_EVERY split steps over its whole
    horizon, through the GPU path (FP32 unless ``mode``), with parameter
    overrides."""
    from paper_2107_07104_gb300 import fibers as F
    ws = sub.with_steps(sub.n_steps)
    ws.params = dict(sub.params, **params)
    with F.Fibers.from_workload(ws, mode=F.FIB_MODE_FP32 if mode is None else mode) as f:
        if blob is not None:
            F.fibers_load_surrogate(f.ctx, blob)
        rows = []
        for _ in range(ws.n_steps // TRAJ_EVERY):
            f.step(TRAJ_EVERY)
            rows.append(f.read_vm().astype(np.float64))
    return np.array(rows)


def agreement(a, b, sub):
    """How closely trajectory b follows the reference trajectory a."""
    dt = TRAJ_EVERY * sub.params["dt_split"]
    ta, tb = activation_times(a, dt), activation_times(b, dt)
    both = ~np.isnan(ta) & ~np.isnan(tb)
    return {"fibers": int(sub.n_fibers), "simulated_ms": sub.n_steps * sub.params["dt_split"],
            "activation_time_max_diff_ms": float(np.max(np.abs(ta[both] - tb[both]))) if both.any() else None,
            "activated_nodes": int((~np.isnan(ta)).sum()), "matched_nodes": int(both.sum()),
            "rel_l2": float(np.linalg.norm(a - b) / np.linalg.norm(a)),
            "max_abs_mv": float(np.max(np.abs(a - b)))}


def surrogate_leg(args, stream, dev, settle_ms=4.0, steps=300):
    """Surrogate and plain FP32 node-updates/s on the full-scale bundle, both
    timed from the same state after settle_ms of simulated time (action
    potentials propagating), and the share of node-updates the network took.
    Accuracy on held-out fibers (seed 4 of the 7744-fiber bundle, never seen
    in training) against the plain FP32 path."""
    from paper_2107_07104_gb300 import fibers as F
    from paper_2107_07104_gb300 import surrogate as S
    w = rank_workload(0)
    blob = S.load_blob()
    settle = int(round(settle_ms / w.params["dt_split"]))
    with F.Fibers.from_workload(w, tuning=dict(graph_steps=100), stream=stream) as fib:
        fib.step(settle)
        state = fib.read_state()
        ms_plain = time_steps(fib, stream, dev, steps, 100)
    with F.Fibers.from_workload(w, tuning=dict(graph_steps=100), stream=stream, mode=F.FIB_MODE_SURROGATE) as fib:
        F.fibers_load_surrogate(fib.ctx, blob)
        fib.write_state(state, settle)
        _, fb0 = fib.stats()
        ms_sur = time_steps(fib, stream, dev, steps, 100)
        _, fb1 = fib.stats()
        finite = bool(np.isfinite(fib.read_vm()).all())
    rate_p = float(w.total_nodes) * steps / (ms_plain / 1e3)
    rate_s = float(w.total_nodes) * steps / (ms_sur / 1e3)
    held = firing_subset(W.bundle_7744(seed=4, t_end_ms=20.0), n=32, seed=4)
    acc = agreement(trajectory(held), trajectory(held, mode=F.FIB_MODE_SURROGATE, blob=blob), held)
    return {"workload": WORKLOAD, "timed_from_ms": settle * w.params["dt_split"], "split_steps": steps,
            "surrogate_node_updates_per_s": rate_s, "plain_fp32_node_updates_per_s": rate_p,
            "surrogate_vs_plain": rate_s / rate_p, "finite": finite,
            "network_fraction_of_node_updates": 1.0 - (fb1 - fb0) / (float(w.total_nodes) * steps),
            "accuracy_vs_plain_fp32_held_out": acc,
            "weights": "paper_2107_07104_gb300/data/hh_surrogate.npy (trained on the GPU by this package)"}


def emg_leg(args, stream, dev, settle=1500, reps=5):
    """The fiber-to-3D coupling on the 7744-fiber bundle (88 x 88 fibers at
    0.05 cm, 14.8 cm long) with a 30 x 30 x 41 mesh (36,900 nodes): time of
    the mapping V3D and of the phi_e solve (FP64 conjugate gradients to 1e-8
    of the right-hand side) 4.5 ms into the run, next to one split step."""
    import torch
    from paper_2107_07104_gb300 import fibers as F
    w = W.bundle_7744(seed=2, t_end_ms=20.0)
    xy = W.fiber_grid_xy(88, 0.05)
    mp = W.box_mesh(xy, 14.8, 30, 41)
    mesh = F.make_mesh3d(mp["nx"], mp["ny"], mp["nz"], mp["origin"], mp["spacing"], 8.93, 6.7)
    with F.Fibers.from_workload(w, tuning=dict(graph_steps=100), stream=stream) as fib:
        fib.step(settle)
        t0 = time.perf_counter()
        emg = F.fibers_emg_create(fib.ctx, xy, 0.0, mesh)
        t_setup = time.perf_counter() - t0
        try:
            n3 = F.fibers_emg_nodes(emg)
            v3 = torch.empty(n3, dtype=torch.float64, device=dev)
            phi = torch.empty(n3, dtype=torch.float32, device=dev)
            F.fibers_emg_phi_e(emg, phi, rtol=1e-8)
            ms_map, ms_phi, its = [], [], []
            for _ in range(reps):
                torch.cuda.synchronize(dev)
                t0 = time.perf_counter()
                F.fibers_emg_vm3d(emg, v3)
                ms_map.append(1e3 * (time.perf_counter() - t0))
                t0 = time.perf_counter()
                it, res = F.fibers_emg_phi_e(emg, phi, rtol=1e-8)
                ms_phi.append(1e3 * (time.perf_counter() - t0))
                its.append(it)
            finite = bool(torch.isfinite(phi).all().item())
            peak = float(phi.abs().max().item())
        finally:
            F.fibers_emg_destroy(emg)
    return {"workload": "bundle 7744 fibers x 1481 nodes at 0.05 cm spacing, 3D mesh 30 x 30 x 41",
            "nodes_3d": int(n3), "fiber_nodes": int(w.total_nodes), "setup_s": t_setup,
            "vm3d_ms": statistics.median(ms_map), "phi_e_ms_incl_mapping": statistics.median(ms_phi),
            "cg_iterations": int(statistics.median(its)), "rtol": 1e-8, "max_abs_phi_e_mv": peak,
            "finite": finite, "timing": "host wall clock around each synchronising call"}


def exp_approx_leg(args, stream, dev, steps=500):
    """The thesis's exp* approximation (eq:apx-e-function) on the 7744-fiber
    bundle: node-updates/s, and its agreement with the exact-exponential FP32
    path on 64 firing fibers over 20 ms."""
    from paper_2107_07104_gb300 import fibers as F
    w = W.bundle_7744(seed=2, t_end_ms=20.0)
    wa = w.with_steps(w.n_steps)
    wa.params = dict(w.params, exp_approx=1)
    with F.Fibers.from_workload(wa, tuning=dict(graph_steps=100), stream=stream) as fib:
        fib.step(100)
        ms = time_steps(fib, stream, dev, steps, 100)
    with F.Fibers.from_workload(w, tuning=dict(graph_steps=100), stream=stream) as fib:
        fib.step(100)
        ms_p = time_steps(fib, stream, dev, steps, 100)
    sub = firing_subset(w)
    return {"workload": "bundle 7744 fibers x 1481 nodes", "node_updates_per_s": float(w.total_nodes) * steps / (ms / 1e3),
            "vs_plain_fp32": ms_p / ms,
            "accuracy_vs_plain_fp32": agreement(trajectory(sub), trajectory(sub, exp_approx=1), sub),
            "exp": "exp*(x) = (1 + x/1024)^1024 for every exponential of the rates (FP32 pipe, no ex2)"}


def adaptive_leg(args, stream, dev, steps=2000):
    """The 7744-fiber bundle with adaptive computation: node-updates/s counted
    over all nodes (the simulated work), the share of fiber-steps skipped,
    and the agreement with the plain path at the end of the timed region."""
    from paper_2107_07104_gb300 import fibers as F
    w = W.bundle_7744(seed=2, t_end_ms=20.0)
    wa = w.with_steps(w.n_steps)
    wa.params = dict(w.params)
    wa.params["flags"] = F.FIB_FLAG_ADAPTIVE
    warm = 200
    with F.Fibers.from_workload(wa, tuning=dict(graph_steps=100), stream=stream) as fib:
        fib.step(warm)
        fib.synchronize()
        s0 = F.fibers_adaptive_stats(fib.ctx)
        ms = time_steps(fib, stream, dev, steps, 100)
        s1 = F.fibers_adaptive_stats(fib.ctx)
        va = fib.read_vm().astype(np.float64)
    with F.Fibers.from_workload(w, tuning=dict(graph_steps=100), stream=stream) as ref:
        ref.step(warm)
        ms_p = time_steps(ref, stream, dev, steps, 100)
        vp = ref.read_vm().astype(np.float64)
    rate = float(w.total_nodes) * steps / (ms / 1e3)
    return {"workload": "bundle 7744 fibers x 1481 nodes", "node_updates_per_s": rate, "vs_plain_fp32": ms_p / ms,
            "timed_from_ms": warm * w.params["dt_split"], "split_steps": steps,
            "skipped_fiber_step_fraction": (s1 - s0) / float(w.n_fibers * steps),
            "equilibrium_test": "every component of every node changed <= 1e-5 relative over a launch's last "
                                "split step, and no pulse due in the next launch",
            "max_abs_mv_vs_plain_fp32_at_end": float(np.max(np.abs(va - vp)))}


# Scheme variants timed on the 7744-fiber bundle: (name, parameter
# overrides).  The two thesis configurations compare a first-order scheme at
# a small step with a second-order one at a large step; their accuracy
# against a fine reference is measured by the oracle tests, their cost here.
SCHEME_LEGS = [
    ("strang 1D-0D-1D, CN, dt 3e-3 (default)", {}),
    ("strang 0D-1D-0D, CN, dt 4e-3, dt_0D 2e-3, dt_1D 4e-3",
     dict(splitting=2, diffusion=0, dt_split=4e-3, dt_0d=2e-3, dt_1d=4e-3)),
    ("godunov 0D-1D, IE, dt 5e-4, dt_0D 1e-4, dt_1D 5e-4",
     dict(splitting=3, diffusion=1, dt_split=5e-4, dt_0d=1e-4, dt_1d=5e-4)),
    ("strang 0D-1D-0D, IE, dt 3e-3, dt_0D 5e-4, dt_1D 1.5e-3",
     dict(splitting=2, diffusion=1, dt_0d=5e-4, dt_1d=1.5e-3)),
]


def schemes_leg(args, stream, dev, sim_ms=3.0):
    """Each scheme variant on the 7744-fiber bundle over the same simulated
    interval: node-updates/s per split step and simulated milliseconds per second."""
    from paper_2107_07104_gb300 import fibers as F
    w = W.bundle_7744(seed=2, t_end_ms=20.0)
    out = {}
    for name, over in SCHEME_LEGS:
        ws = w.with_steps(w.n_steps)
        ws.params = dict(w.params)
        ws.params.update(over)
        dt = ws.params["dt_split"]
        steps = int(round(sim_ms / dt))
        steps -= steps % 50
        with F.Fibers.from_workload(ws, tuning=dict(graph_steps=50), stream=stream) as fib:
            fib.step(100)
            ms = time_steps(fib, stream, dev, steps, 50)
            finite = bool(np.all(np.isfinite(fib.read_vm())))
        out[name] = {"node_updates_per_s": float(w.total_nodes) * steps / (ms / 1e3), "ms_per_step": ms / steps,
                     "simulated_ms_per_s": steps * dt / (ms / 1e3), "steps": steps, "finite": finite}
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20, help=f"benchmark steps of {BENCH_SPLIT_STEPS} split steps")
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--nodes-per-thread", type=int, default=0)
    ap.add_argument("--warps-per-cta", type=int, default=0)
    ap.add_argument("--reaction-pairs", type=int, default=0, help="1 scalar, 2 packed FP32x2, 0 auto")
    ap.add_argument("--ctas-per-sm", type=int, default=0, help="register budget: 2, 3 or 4 CTAs per SM, 0 auto")
    ap.add_argument("--warp-roles", type=int, default=0,
                    help="1 fused step kernel, 2 split reaction/diffusion warps, 0 auto")
    ap.add_argument("--cpu-fibers", type=int, default=256)
    ap.add_argument("--cpu-steps", type=int, default=1500)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-legs", action="store_true", help="time the headline workload only")
    ap.add_argument("--no-surrogate", action="store_true")
    ap.add_argument("--workload", default="bundle_67600", choices=sorted(WORKLOADS),
                    help="headline workload (bundle_7744: the smaller case used for profiler captures)")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    world, rank, local, dist = dist_setup()
    try:
        if args.impl == "reference":
            return run_reference(args, world, rank)
        return run_gpu(args, world, rank, local, dist)
    finally:
        if dist is not None:
            dist.destroy_process_group()


if __name__ == "__main__":
    sys.exit(main())
