"""Helpers shared by the GPU parity tests: run the CUDA library and the FP64
oracle on the same seeded workload and compare what they produce."""
from __future__ import annotations

from typing import List, Optional, Sequence

import numpy as np

import oracle
from paper_2107_07104_gb300 import fibers as F
from paper_2107_07104_gb300 import workloads as W

# Tolerances for the FP32 path against the FP64 oracle over a trajectory.
MAX_ABS_MV = 0.5
REL_L2 = 1e-3
ACT_TIME_MS = 0.05


def gpu_checkpoints(w, checkpoints: Sequence[int], tuning: Optional[dict] = None, mode: int = F.FIB_MODE_FP32,
                    stream=None) -> np.ndarray:
    """V (float64) of every node after each checkpoint step count (ascending)."""
    out = []
    with F.Fibers.from_workload(w, tuning=tuning, mode=mode, stream=stream) as fib:
        done = 0
        for c in checkpoints:
            fib.step(c - done)
            done = c
            out.append(fib.read_vm().astype(np.float64))
    return np.array(out)


def oracle_checkpoints(w, checkpoints: Sequence[int], fibers: Optional[Sequence[int]] = None) -> np.ndarray:
    """Oracle V after each checkpoint, on all fibers or on a subset."""
    ww = w if fibers is None else w.subset(fibers)
    state = oracle.init_state(ww.params, ww.total_nodes, ww.vm0)
    out = []
    done = 0
    for c in checkpoints:
        oracle.run(ww.params, ww.n_nodes, ww.mu_of_fiber, ww.junction, ww.mu_offsets, ww.fire_times, state,
                   done, c - done)
        done = c
        out.append(state[:ww.total_nodes].copy())
    return np.array(out)


def select_fibers(w, values: np.ndarray, fibers: Sequence[int]) -> np.ndarray:
    """Columns of ``values`` (ragged node order of w) that belong to ``fibers``."""
    off = w.offsets()
    return np.concatenate([values[..., off[f]:off[f + 1]] for f in fibers], axis=-1)


def errors(gpu: np.ndarray, ref: np.ndarray):
    d = gpu - ref
    max_abs = float(np.max(np.abs(d))) if d.size else 0.0
    rel = float(np.linalg.norm(d) / max(np.linalg.norm(ref), 1e-300))
    return max_abs, rel


def activation_times(samples: np.ndarray, dt: float, threshold: float = 0.0) -> np.ndarray:
    """First upward crossing of `threshold` per node, linearly interpolated
    between samples taken every dt (sample i at time (i + 1) dt).  NaN if none."""
    s = samples
    below = s[:-1] < threshold
    above = s[1:] >= threshold
    cross = below & above
    t = np.full(s.shape[1], np.nan)
    any_c = cross.any(axis=0)
    k = np.argmax(cross, axis=0)
    idx = np.nonzero(any_c)[0]
    kk = k[idx]
    v0 = s[kk, idx]
    v1 = s[kk + 1, idx]
    t[idx] = (kk + 1 + (threshold - v0) / (v1 - v0)) * dt
    return t


EDGE_LENGTHS = [1, 2, 3, 4, 5, 7, 8, 9, 12, 13, 16, 17, 31, 32, 33, 47, 48, 49, 63, 64, 65, 127, 128, 129,
                255, 256, 257, 383, 384, 385, 511, 512, 513, 700]


def edge_workload(n_steps, seed=11, amp=None):
    """Fibers of 1..700 nodes: chunk-aligned and ragged tails, 1-3 node
    fibers, junctions at both ends, never-stimulated fibers, noisy start."""
    rng = np.random.default_rng(seed)
    lens = np.array(EDGE_LENGTHS, np.int32)
    n = lens.shape[0]
    w = W.small_ragged(seed, n, 1, 2, n_steps)
    w.n_nodes = lens
    w.junction = W.centre_junctions(rng, lens, 0.05)
    w.junction[3] = 0          # junction at the first node
    w.junction[10] = lens[10] - 1  # and at the last
    w.mu_of_fiber = rng.integers(-1, w.n_mu, size=n).astype(np.int32)  # -1: never stimulated
    w.vm0 = (w.params["Vrest"] + rng.normal(0, 0.5, size=int(lens.sum()))).astype(np.float32)
    if amp is not None:
        w.params["stim_amplitude"] = amp
    return w


def subset_indices(w, fibers) -> np.ndarray:
    off = w.offsets()
    return np.concatenate([np.arange(off[f], off[f + 1]) for f in fibers]).astype(np.int64)


def gpu_subset_trajectory(w, fibers, every: int, tuning: Optional[dict] = None, autotune: bool = False):
    """V (float64) of the nodes of `fibers` after every `every` split steps
    over the workload's horizon, through the CUDA path at full size; read_vm
    writes into device memory and the subset is picked out there.  Returns
    (samples, the launch shape that ran)."""
    import torch
    idx = torch.as_tensor(subset_indices(w, fibers), device="cuda")
    n_s = w.n_steps // every
    out = torch.empty((n_s, idx.numel()), dtype=torch.float32, device="cuda")
    buf = torch.empty(w.total_nodes, dtype=torch.float32, device="cuda")
    with F.Fibers.from_workload(w, tuning=tuning) as fib:
        if autotune:
            fib.autotune(20)
        for i in range(n_s):
            fib.step(every)
            F.read_vm(fib.ctx, buf)
            out[i] = buf.index_select(0, idx)
        shape = fib.tuning
    return out.cpu().numpy().astype(np.float64), shape


def oracle_subset_trajectory(w, fibers, every: int) -> np.ndarray:
    """Oracle V of `fibers` (run alone: fibers are independent) after every
    `every` split steps."""
    sub = w.subset(fibers)
    state = oracle.init_state(sub.params, sub.total_nodes, sub.vm0)
    n_s = w.n_steps // every
    return oracle.run(sub.params, sub.n_nodes, sub.mu_of_fiber, sub.junction, sub.mu_offsets, sub.fire_times,
                      state, 0, n_s * every, every)


def dense_parity(w, fibers, every: int, tuning: Optional[dict] = None, autotune: bool = False):
    """GPU and oracle trajectories of the subset (oracle in a host thread
    while the GPU runs), their errors and the activation-time difference."""
    import threading
    res = {}
    th = threading.Thread(target=lambda: res.setdefault("o", oracle_subset_trajectory(w, fibers, every)))
    th.start()
    g, shape = gpu_subset_trajectory(w, fibers, every, tuning, autotune)
    th.join()
    o = res["o"]
    mx, rel = errors(g, o)
    dt = every * w.params["dt_split"]
    tg, to = activation_times(g, dt), activation_times(o, dt)
    # a node activated on one side only must be one whose activation falls
    # within the tolerance of the last sample (the other side crosses after it)
    one_side = np.isnan(tg) != np.isnan(to)
    t_one = np.where(np.isnan(tg), to, tg)[one_side]
    t_last = g.shape[0] * dt
    same_set = bool(np.all(t_one >= t_last - ACT_TIME_MS - dt))
    fired = ~np.isnan(to) & ~np.isnan(tg)
    act = float(np.max(np.abs(tg[fired] - to[fired]))) if fired.any() else 0.0
    return dict(max_abs=mx, rel_l2=rel, act=act, same_activated=same_set, activated=int(fired.sum()),
                samples=int(g.shape[0]), shape=shape)
