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
