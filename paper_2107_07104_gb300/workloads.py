"""Seeded synthetic fiber-bundle workloads.

This module only *draws inputs*: fiber lengths, motor-unit (MU) membership,
neuromuscular-junction positions, MU firing trains and initial membrane
voltages.  It holds none of the method's arithmetic (no rates, no diffusion
matrices, no stimulus windows), so both the CUDA library and the FP64 oracle
can be fed from it without sharing method code.

Shapes follow the thesis's workloads (Maier 2021):
  * straight fibers discretised with h = 0.01 cm, i.e. 1481 nodes for a
    14.8 cm biceps fiber (section "Effect of the Mesh Width on the Action
    Potential Propagation Velocity", sec:action_potential_velocity);
  * MU sizes following the exponential progression q(k) = b^k / sum_l b^l of
    Eq. (eq:mus_q), with b = 1.02 for 100 MUs (the EMG mesh-width study) and
    b = R^(1/n_MU), R = 10, otherwise (the Enoka form quoted beside eq:mus_q);
  * junctions in a band at the fiber centre, node int(n/2)
    (sec:stimulation_times_callbacks), with a uniform jitter;
  * per-MU Poisson firing trains (stand-in for the motor-neuron model).

All randomness comes from numpy's PCG64 seeded per workload, so a workload is
fully determined by its name and seed.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence

import numpy as np

# --------------------------------------------------------------------------
# Model and discretisation constants used by every workload (units: cm, ms,
# mV, uA/cm^2, uF/cm^2, mS/cm^2, mS/cm).  Plain numbers only; each consumer
# derives what it needs (e.g. the leak reversal) with its own arithmetic.
# --------------------------------------------------------------------------
DEFAULT_PARAMS = dict(
    Cm=1.0,            # membrane capacitance, uF/cm^2
    gNa=120.0,         # max sodium conductance, mS/cm^2
    gK=36.0,           # max potassium conductance, mS/cm^2
    gL=0.3,            # leak conductance, mS/cm^2
    Vrest=-75.0,       # resting potential, mV
    ENa=-75.0 + 115.0,  # sodium reversal = Vrest + 115 mV (HH 1952 shifted)
    EK=-75.0 - 12.0,    # potassium reversal = Vrest - 12 mV
    EL=float("nan"),   # NaN: derive so that Vrest is an exact rest state
    sigma_eff=3.828,   # effective conductivity, mS/cm
    Am=500.0,          # surface-to-volume ratio, 1/cm
    h=0.01,            # mesh width, cm
    dt_split=3e-3,     # Strang splitting step, ms
    dt_0d=1e-3,        # Heun substep, ms
    dt_1d=1.5e-3,      # Crank-Nicolson step (= dt_split / 2), ms
    # 400 uA/cm^2 for 0.1 ms at 3 nodes is below the excitation threshold of
    # this discretisation (about 611 uA/cm^2 at h = 0.01 cm), so no action
    # potential would start; the workloads stimulate at twice threshold.
    stim_amplitude=1200.0,  # uA/cm^2
    stim_duration=0.1,     # ms
    stim_half_width=1,     # nodes j-1..j+1
    splitting=0,           # Strang, diffusion dt/2 - reaction dt - diffusion dt/2
    diffusion=0,           # Crank-Nicolson
    exp_approx=0,          # 1: rates use exp*(x) = (1 + x/1024)^1024 instead of exp
)


@dataclasses.dataclass
class Workload:
    """A complete, seeded input set for one simulation."""

    name: str
    params: dict
    n_nodes: np.ndarray        # int32 [n_fibers]
    mu_of_fiber: np.ndarray    # int32 [n_fibers]
    junction: np.ndarray       # int32 [n_fibers]
    mu_offsets: np.ndarray     # int64 [n_mu + 1] (CSR into fire_times)
    fire_times: np.ndarray     # float64 [n_fire], sorted within each MU, ms
    vm0: Optional[np.ndarray]  # float32 [sum(n_nodes)] initial V (mV) or None
    n_steps: int               # split steps to simulate
    seed: int

    @property
    def n_fibers(self) -> int:
        return int(self.n_nodes.shape[0])

    @property
    def n_mu(self) -> int:
        return int(self.mu_offsets.shape[0] - 1)

    @property
    def total_nodes(self) -> int:
        return int(self.n_nodes.astype(np.int64).sum())

    def offsets(self) -> np.ndarray:
        """Ragged start offset of each fiber in a concatenated node array."""
        off = np.zeros(self.n_fibers + 1, dtype=np.int64)
        np.cumsum(self.n_nodes, out=off[1:])
        return off

    def subset(self, fibers: Sequence[int], name: Optional[str] = None) -> "Workload":
        """The same simulation restricted to some fibers (fibers are independent)."""
        fibers = np.asarray(fibers, dtype=np.int64)
        off = self.offsets()
        vm0 = None
        if self.vm0 is not None:
            vm0 = np.concatenate([self.vm0[off[f]:off[f + 1]] for f in fibers]).astype(np.float32)
        return Workload(
            name=name or f"{self.name}[subset {len(fibers)}]",
            params=dict(self.params),
            n_nodes=self.n_nodes[fibers].copy(),
            mu_of_fiber=self.mu_of_fiber[fibers].copy(),
            junction=self.junction[fibers].copy(),
            mu_offsets=self.mu_offsets.copy(),
            fire_times=self.fire_times.copy(),
            vm0=vm0,
            n_steps=self.n_steps,
            seed=self.seed,
        )

    def with_steps(self, n_steps: int) -> "Workload":
        w = dataclasses.replace(self)
        w.n_steps = int(n_steps)
        return w


def n_steps_for(t_end_ms: float, dt_split: float) -> int:
    """Split steps needed to reach t_end: ceil(T / dt), guarding FP noise."""
    q = t_end_ms / dt_split
    return int(math.ceil(q - 1e-9))


def mu_size_probabilities(n_mu: int, b: float) -> np.ndarray:
    """Exponential MU size progression q(k) = b^k / sum_l b^l, k = 1..n_MU (Eq. mus_q)."""
    k = np.arange(1, n_mu + 1, dtype=np.float64)
    w = b ** k
    return w / w.sum()


def assign_mus(rng: np.random.Generator, n_fibers: int, n_mu: int, b: float) -> np.ndarray:
    """Multinomial MU assignment with the thesis's empty-MU repair.

    Each fiber draws its MU from q(k).  Every MU that ends up empty takes one
    fiber from the currently largest MU (the thesis reassigns one fiber to each
    empty MU after sampling).  Only possible when n_fibers >= n_mu.
    """
    q = mu_size_probabilities(n_mu, b)
    mu = rng.choice(n_mu, size=n_fibers, p=q).astype(np.int32)
    if n_fibers >= n_mu:
        counts = np.bincount(mu, minlength=n_mu)
        for k in np.nonzero(counts == 0)[0]:
            donor = int(np.argmax(counts))
            idx = np.nonzero(mu == donor)[0]
            take = int(idx[rng.integers(idx.shape[0])])
            mu[take] = k
            counts[donor] -= 1
            counts[k] += 1
    return mu


def poisson_trains(rng: np.random.Generator, rates_hz: np.ndarray, t_end_ms: float):
    """Independent homogeneous Poisson firing trains on [0, t_end) per MU (CSR)."""
    offsets = [0]
    times: List[float] = []
    for rate in rates_hz:
        mean_isi = 1000.0 / float(rate)
        t = rng.exponential(mean_isi)
        while t < t_end_ms:
            times.append(t)
            t += rng.exponential(mean_isi)
        offsets.append(len(times))
    return np.asarray(offsets, dtype=np.int64), np.asarray(times, dtype=np.float64)


def centre_junctions(rng: Optional[np.random.Generator], n_nodes: np.ndarray, jitter: float) -> np.ndarray:
    """Junction node per fiber: int((N-1)/2) plus a uniform +-jitter*(N-1) offset, clamped."""
    n = n_nodes.astype(np.int64)
    centre = (n - 1) // 2
    if rng is None or jitter == 0.0:
        return centre.astype(np.int32)
    off = np.rint(rng.uniform(-jitter, jitter, size=n.shape[0]) * (n - 1)).astype(np.int64)
    return np.clip(centre + off, 0, n - 1).astype(np.int32)


def bundle(name: str, n_fibers: int, n_nodes, n_mu: int, b: float, rate_lo: float, rate_hi: float,
           t_end_ms: float, seed: int, jitter: float = 0.05, v0_sigma: float = 0.0,
           params: Optional[dict] = None) -> Workload:
    """Generic seeded bundle.  ``n_nodes`` is an int or a (lo, hi) inclusive range."""
    p = dict(DEFAULT_PARAMS if params is None else params)
    rng = np.random.default_rng(seed)
    if isinstance(n_nodes, tuple):
        lens = rng.integers(n_nodes[0], n_nodes[1] + 1, size=n_fibers).astype(np.int32)
    else:
        lens = np.full(n_fibers, int(n_nodes), dtype=np.int32)
    mu = assign_mus(rng, n_fibers, n_mu, b)
    rates = rng.uniform(rate_lo, rate_hi, size=n_mu)
    offs, times = poisson_trains(rng, rates, t_end_ms)
    junc = centre_junctions(rng, lens, jitter)
    vm0 = None
    if v0_sigma > 0.0:
        total = int(lens.astype(np.int64).sum())
        vm0 = (p["Vrest"] + rng.normal(0.0, v0_sigma, size=total)).astype(np.float32)
    return Workload(name=name, params=p, n_nodes=lens, mu_of_fiber=mu, junction=junc,
                    mu_offsets=offs, fire_times=times, vm0=vm0,
                    n_steps=n_steps_for(t_end_ms, p["dt_split"]), seed=seed)


# --------------------------------------------------------------------------
# The five workloads (sizes as stated for the fiber-bundle benchmarks).
# --------------------------------------------------------------------------

def single_fiber(t_end_ms: float = 10.0, n_nodes: int = 1481) -> Workload:
    """1 fiber of 1481 nodes (14.8 cm at h = 0.01 cm), one stimulus at t = 0 at the centre.

    The stimulus repeats every 100 ms, so within 10 ms it fires once.
    """
    p = dict(DEFAULT_PARAMS)
    period = 100.0
    times = np.arange(0.0, t_end_ms, period, dtype=np.float64)
    lens = np.array([n_nodes], dtype=np.int32)
    return Workload(name=f"single fiber 1x{n_nodes}, {t_end_ms:g} ms", params=p, n_nodes=lens,
                    mu_of_fiber=np.zeros(1, np.int32), junction=centre_junctions(None, lens, 0.0),
                    mu_offsets=np.array([0, times.shape[0]], np.int64), fire_times=times,
                    vm0=None, n_steps=n_steps_for(t_end_ms, p["dt_split"]), seed=0)


def bundle_7744(seed: int = 2, t_end_ms: float = 20.0) -> Workload:
    """7744 (88x88) fibers x 1481 nodes, 100 MUs (b = 1.02), Poisson 10-30 Hz."""
    return bundle("bundle 7744x1481, 100 MUs", 7744, 1481, 100, 1.02, 10.0, 30.0, t_end_ms, seed)


def ragged_20000(seed: int = 3, t_end_ms: float = 50.0) -> Workload:
    """20000 fibers with lengths U{800..2000}, 150 MUs, Poisson 10-40 Hz, V0 = rest + N(0, 0.5)."""
    return bundle("ragged 20000x[800,2000], 150 MUs", 20000, (800, 2000), 150, 10.0 ** (1.0 / 150),
                  10.0, 40.0, t_end_ms, seed, v0_sigma=0.5)


def bundle_67600(seed: int = 5, t_end_ms: float = 100.0) -> Workload:
    """67600 (260x260) fibers x 1481 nodes, 200 MUs, Poisson 10-30 Hz."""
    return bundle("bundle 67600x1481, 200 MUs", 67600, 1481, 200, 10.0 ** (1.0 / 200),
                  10.0, 30.0, t_end_ms, seed)


def small_ragged(seed: int, n_fibers: int, lo: int, hi: int, n_steps: int, n_mu: int = 4,
                 rate_hz: float = 400.0, v0_sigma: float = 0.5) -> Workload:
    """Small ragged case for parity tests: frequent firing so that APs start early."""
    p = dict(DEFAULT_PARAMS)
    t_end = n_steps * p["dt_split"]
    w = bundle(f"small ragged {n_fibers}x[{lo},{hi}]", n_fibers, (lo, hi), n_mu, 1.2,
               rate_hz, rate_hz, t_end, seed, v0_sigma=v0_sigma, params=p)
    w.n_steps = int(n_steps)
    return w


def stratified_by_length(n_nodes: np.ndarray, count: int, seed: int) -> np.ndarray:
    """Fiber indices sampled evenly across the length distribution (seeded)."""
    rng = np.random.default_rng(seed)
    order = np.argsort(n_nodes, kind="stable")
    strata = np.array_split(order, count)
    return np.sort(np.array([s[rng.integers(s.shape[0])] for s in strata if s.shape[0] > 0], dtype=np.int64))


def random_fibers(n_fibers: int, count: int, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return np.sort(rng.choice(n_fibers, size=min(count, n_fibers), replace=False)).astype(np.int64)


def fiber_grid_xy(n_side: int, spacing_cm: float = 0.05) -> np.ndarray:
    """(n_side^2, 2) positions of straight parallel fibers on a square grid in
    the cross-section, fiber f at ((f % n_side) s, (f // n_side) s): the
    synthetic stand-in for a muscle cross-section (the 88 x 88 bundle spans
    4.35 cm, about a biceps belly)."""
    f = np.arange(n_side * n_side)
    return np.stack([(f % n_side) * spacing_cm, (f // n_side) * spacing_cm], axis=1).astype(np.float64)


def box_mesh(fiber_xy: np.ndarray, length_cm: float, n_xy: int, n_z: int) -> dict:
    """A structured 3D mesh spanning the fibers' bounding box and their
    length: n_xy x n_xy x n_z nodes (parameters for fibers_emg_create)."""
    lo = fiber_xy.min(axis=0)
    hi = fiber_xy.max(axis=0)
    return dict(nx=n_xy, ny=n_xy, nz=n_z, origin=(float(lo[0]), float(lo[1]), 0.0),
                spacing=(float(hi[0] - lo[0]) / (n_xy - 1), float(hi[1] - lo[1]) / (n_xy - 1),
                         float(length_cm) / (n_z - 1)))
