"""Data generation and training of the reaction-step surrogate.

Every arithmetic step runs in the library's CUDA kernels (fibers_hh_reaction,
fibers_mlp_train_step, fibers_adam_step, fibers_feature_stats); this module
only orchestrates: it runs plain-method simulations, picks which node states
become samples, shuffles batches, and assembles the blob that
fibers_load_surrogate reads.  Torch provides device memory and index
gathers.

Samples: node states (u, m, h, n) read from trajectories of
the plain FP32 method on seeded bundles, plus the stimulus pattern of the
step; the target is the change of the state over the reaction part of one
split step, computed by the plain HH step.  Nodes away from rest are
over-sampled because most of a bundle sits at rest most of the time.
"""
from __future__ import annotations

import math
from typing import Dict, Iterable, List, Optional, Tuple

import numpy as np

from . import fibers as F
from . import workloads as W

# stimulus substep patterns of one split step with 3 substeps: a pulse of
# 100 substeps covers whole steps except where it starts or ends
STIM_PATTERNS = np.array([1, 3, 7, 6, 4], np.uint8)


def _torch():
    import torch
    return torch


def sample_states(w, n_samples: int, checkpoints: Iterable[int], seed: int, active_fraction: float = 0.85,
                  device: str = "cuda") -> "torch.Tensor":
    """(n, 4) tensor of (u, m, h, n) drawn from the plain-method trajectory of w."""
    torch = _torch()
    cps = sorted(set(int(c) for c in checkpoints))
    per_cp = max(1, n_samples // len(cps))
    gen = torch.Generator(device=device)
    gen.manual_seed(seed)
    total = w.total_nodes
    state = torch.empty(4 * total, dtype=torch.float32, device=device)
    # the library's state holds gates as deviations from rest
    rest = torch.as_tensor(F.fibers_rest_state(w.params), device=device)
    out = []
    with F.Fibers.from_workload(w) as fib:
        done = 0
        for c in cps:
            fib.step(c - done)
            done = c
            F.fibers_read_state(fib.ctx, state)
            s = state.view(4, total)
            u, m, h, n = s[0], s[1] + rest[1], s[2] + rest[2], s[3] + rest[3]
            # activity: distance from rest in voltage and gates
            act = u.abs() + 50.0 * ((m - m.median()).abs() + (h - h.median()).abs() + (n - n.median()).abs())
            active = torch.nonzero(act > 0.05).flatten()
            k_act = min(int(per_cp * active_fraction), active.numel())
            pick = []
            if k_act > 0:
                pick.append(active[torch.randint(active.numel(), (k_act,), generator=gen, device=device)])
            k_rest = per_cp - k_act
            pick.append(torch.randint(total, (k_rest,), generator=gen, device=device))
            idx = torch.cat(pick)
            out.append(torch.stack([u[idx], m[idx], h[idx], n[idx]], dim=1))
    return torch.cat(out)


def make_dataset(params: dict, states: "torch.Tensor", seed: int, stim_fraction: float = 0.15):
    """Inputs X (n x 5: u, m, h, n, s) and targets Y (n x 4: change of u, m, h, n)."""
    torch = _torch()
    dev = states.device
    n = states.shape[0]
    gen = torch.Generator(device=dev)
    gen.manual_seed(seed)
    patterns = torch.as_tensor(STIM_PATTERNS, device=dev)
    on = torch.rand(n, generator=gen, device=dev) < stim_fraction
    mask = torch.where(on, patterns[torch.randint(len(STIM_PATTERNS), (n,), generator=gen, device=dev)],
                       torch.zeros(n, dtype=torch.uint8, device=dev)).to(torch.uint8).contiguous()
    x_in = torch.empty(4, n, dtype=torch.float32, device=dev)
    x_in[0] = states[:, 0] + params["Vrest"]
    x_in[1:] = states[:, 1:].T
    x_out = torch.empty_like(x_in)
    F.fibers_hh_reaction(params, x_in.contiguous(), mask, x_out)
    n_sub = int(round(params["dt_split"] / params["dt_0d"]))
    bits = sum(((mask >> k) & 1).to(torch.float32) for k in range(n_sub))
    X = torch.empty(n, 5, dtype=torch.float32, device=dev)
    X[:, :4] = states
    X[:, 4] = bits / n_sub
    Y = (x_out - x_in).T.contiguous()
    return X.contiguous(), Y


def rest_state(params: dict) -> np.ndarray:
    """(u, m, h, n) at rest as the library initialises it (u = 0, the
    library's resting gates)."""
    r = F.fibers_rest_state(params).astype(np.float64)
    return np.array([0.0, r[1], r[2], r[3]])


def quiet_box(params: dict, du: float = 8.0, dg: float = 0.03):
    """Box of raw inputs around rest that the plain HH step keeps: |u| <= du mV,
    each gate within dg of its rest value, no stimulus."""
    r = rest_state(params)
    lo = np.array([-du, r[1] - dg, r[2] - dg, r[3] - dg, 0.0], np.float32)
    hi = np.array([du, r[1] + dg, r[2] + dg, r[3] + dg, 0.0], np.float32)
    return lo, hi


def trust_box(params: dict, u_hi: float = 10.0, h_hi: float = 0.35):
    """Box of raw inputs where the network replaces the plain HH step: the
    repolarisation tail and the recovery after an action potential (the
    sodium inactivation gate h at most h_hi, depolarisation at most u_hi mV,
    no stimulus).  The upstroke (h still near rest while u rises) and every
    stimulated node stay with the plain step, since errors there move the
    wavefront; errors behind it decay."""
    lo = np.array([-100.0, 0.0, 0.0, 0.0, 0.0], np.float32)
    hi = np.array([u_hi, 1.0, h_hi, 1.0, 0.0], np.float32)
    return lo, hi


def inside_box(X, lo, hi):
    torch = _torch()
    l = torch.as_tensor(lo, device=X.device)
    h = torch.as_tensor(hi, device=X.device)
    return ((X >= l) & (X <= h)).all(dim=1)


def outside_box(X, lo, hi):
    torch = _torch()
    l = torch.as_tensor(lo, device=X.device)
    h = torch.as_tensor(hi, device=X.device)
    return ~((X >= l) & (X <= h)).all(dim=1)


def train(X, Y, epochs: int = 6, batch: int = 8192, lr: float = 2e-3, lr_end: float = 2e-5, seed: int = 0,
          quantize: bool = True, log: Optional[List[float]] = None, quiet=None, trust=None,
          avg_decay: Optional[float] = 0.999) -> np.ndarray:
    """Adam on the normalised data (cosine learning-rate decay); returns the
    blob for fibers_load_surrogate.  Samples inside the quiet box (handled by
    the plain step at run time) are left out, and so are samples outside the
    trust box (None: no restriction); the blob's envelope is the box of the
    samples kept, so the network only sees states like those it learned.

    The blob carries the exponential moving average of the weights over the
    steps (decay avg_decay; None: the last step's weights).  On held-out
    bundles the average's activation times varied far less between training
    seeds than the last weights' did."""
    torch = _torch()
    dev = X.device
    if quiet is None:
        quiet = (np.full(5, 1.0, np.float32), np.full(5, -1.0, np.float32))  # empty box
    keep = outside_box(X, quiet[0], quiet[1])
    if trust is not None:
        keep = keep & inside_box(X, trust[0], trust[1])
    X = X[keep].contiguous()
    Y = Y[keep].contiguous()
    xs = F.fibers_feature_stats(X)
    ys = F.fibers_feature_stats(Y)
    in_mu = xs[:, 0].astype(np.float32)
    in_sigma = np.maximum(xs[:, 1], 1e-6).astype(np.float32)
    in_mu[4], in_sigma[4] = 0.0, 1.0  # stimulus fraction already in [0, 1]
    out_mu = ys[:, 0].astype(np.float32)
    out_sigma = np.maximum(ys[:, 1], 1e-12).astype(np.float32)
    env_lo = xs[:, 2].astype(np.float32)
    env_hi = xs[:, 3].astype(np.float32)
    env_lo[4], env_hi[4] = 0.0, 1.0
    if trust is not None:  # the stimulus column is 0 throughout the trust box
        env_lo[4], env_hi[4] = trust[0][4], trust[1][4]
    Xn = ((X - torch.as_tensor(in_mu, device=dev)) / torch.as_tensor(in_sigma, device=dev)).contiguous()
    Yn = ((Y - torch.as_tensor(out_mu, device=dev)) / torch.as_tensor(out_sigma, device=dev)).contiguous()
    theta = torch.as_tensor(_he_uniform(seed), device=dev).contiguous()
    m = torch.zeros_like(theta)
    v = torch.zeros_like(theta)
    avg = None if avg_decay is None else theta.clone()
    grad = torch.zeros_like(theta)
    loss = torch.zeros(1, dtype=torch.float32, device=dev)
    work = torch.empty(batch * F.SUR_WORK_PER_SAMPLE, dtype=torch.float32, device=dev)
    n = X.shape[0]
    steps_per_epoch = n // batch
    total = max(1, epochs * steps_per_epoch)
    gen = torch.Generator(device=dev)
    gen.manual_seed(seed)
    t = 0
    for _ in range(epochs):
        perm = torch.randperm(n, generator=gen, device=dev)
        for b in range(steps_per_epoch):
            idx = perm[b * batch:(b + 1) * batch]
            xb = Xn[idx].contiguous()
            yb = Yn[idx].contiguous()
            F.fibers_mlp_train_step(theta, quantize, xb, yb, work, grad, loss)
            t += 1
            rate = lr_end + 0.5 * (lr - lr_end) * (1.0 + math.cos(math.pi * t / total))
            F.fibers_adam_step(theta, m, v, grad, rate, t, theta_avg=avg, avg_decay=avg_decay or 0.0)
            if log is not None and (t % 50 == 0 or t == total):
                log.append(float(loss.item()))
    final = theta if avg is None else avg
    return make_blob(final.cpu().numpy(), in_mu, in_sigma, out_mu, out_sigma, env_lo, env_hi, quiet[0], quiet[1])


def make_blob(theta, in_mu, in_sigma, out_mu, out_sigma, env_lo, env_hi, quiet_lo, quiet_hi) -> np.ndarray:
    head = np.array([5, 128, 4], np.float32)
    blob = np.concatenate([head, in_mu, in_sigma, out_mu, out_sigma, env_lo, env_hi, quiet_lo, quiet_hi,
                           np.asarray(theta, np.float32)]).astype(np.float32)
    assert blob.size == F.SUR_BLOB_FLOATS
    return blob


def blob_parts(blob: np.ndarray) -> Dict[str, np.ndarray]:
    b = np.asarray(blob, np.float32)
    k = 3
    parts = {}
    for name, size in (("in_mu", 5), ("in_sigma", 5), ("out_mu", 4), ("out_sigma", 4), ("env_lo", 5),
                       ("env_hi", 5), ("quiet_lo", 5), ("quiet_hi", 5), ("theta", F.SUR_N_PARAMS)):
        parts[name] = b[k:k + size]
        k += size
    return parts


def training_workloads(seed_single: int = 1, seed_bundle: int = 2, bundle_fibers: int = 2048):
    """Trajectories the samples come from: the single fiber (10 ms) and a
    seeded subset of the 7744-fiber bundle (20 ms)."""
    single = W.single_fiber(t_end_ms=10.0)
    bundle = W.bundle_7744(seed=seed_bundle, t_end_ms=20.0)
    sub = bundle.subset(W.random_fibers(bundle.n_fibers, bundle_fibers, seed=seed_bundle + 100))
    return [single, sub]


def build_surrogate(n_samples: int = 16_000_000, epochs: int = 24, seed: int = 0, log: Optional[List[float]] = None,
                    device: str = "cuda", trust: bool = True) -> np.ndarray:
    """Samples from the plain method, trains, and returns the surrogate blob.
    With trust, the network is trained on, and later used in, the trust box
    only (no stimulated samples are drawn then)."""
    torch = _torch()
    ws = training_workloads()
    parts = []
    for i, w in enumerate(ws):
        share = n_samples // len(ws)
        cps = np.linspace(50, w.n_steps, 60).astype(int)
        parts.append(sample_states(w, share, cps, seed=seed + 17 * i, device=device))
    states = torch.cat(parts)
    tb = trust_box(ws[0].params) if trust else None
    X, Y = make_dataset(ws[0].params, states, seed=seed + 1, stim_fraction=0.0 if trust else 0.15)
    return train(X, Y, epochs=epochs, seed=seed, log=log, quiet=quiet_box(ws[0].params), trust=tb)


def _he_uniform(seed: int) -> np.ndarray:
    """Uniform(+-sqrt(6 / fan_in)) weights, zero biases, in the parameter-vector order."""
    rng = np.random.default_rng(seed)
    parts = []
    for shape in ((128, 5), (128,), (128, 128), (128,), (4, 128), (4,)):
        if len(shape) == 2:
            lim = math.sqrt(6.0 / shape[1])
            parts.append(rng.uniform(-lim, lim, size=shape))
        else:
            parts.append(np.zeros(shape))
    return np.concatenate([p.ravel() for p in parts]).astype(np.float32)


BLOB_PATH = __import__("os").path.join(__import__("os").path.dirname(__file__), "data", "hh_surrogate.npy")


def load_blob(path: Optional[str] = None) -> np.ndarray:
    """The committed trained surrogate (written by ``python -m paper_2107_07104_gb300.surrogate``)."""
    return np.load(path or BLOB_PATH).astype(np.float32)


if __name__ == "__main__":
    import argparse
    ap = argparse.ArgumentParser(description="Generate samples with the plain method, train the surrogate on "
                                             "the GPU and write its blob.")
    ap.add_argument("--out", default=BLOB_PATH)
    ap.add_argument("--samples", type=int, default=16_000_000)
    ap.add_argument("--epochs", type=int, default=24)
    ap.add_argument("--seed", type=int, default=0)
    args = ap.parse_args()
    log: List[float] = []
    blob = build_surrogate(args.samples, args.epochs, args.seed, log)
    __import__("os").makedirs(__import__("os").path.dirname(args.out), exist_ok=True)
    np.save(args.out, blob)
    print(f"wrote {args.out}: {blob.size} floats, loss {log[0]:.3e} -> {log[-1]:.3e}")
