"""GPU parity: the CUDA path through the C ABI against the FP64 oracle.

Tolerances (FP32 path vs FP64 oracle over the trajectory): max |dV| <= 0.5 mV
and relative L2 <= 1e-3; activation times within 0.05 ms.
"""
import numpy as np
import pytest

import oracle
from paper_2107_07104_gb300 import fibers as F
from paper_2107_07104_gb300 import workloads as W

from parity import (ACT_TIME_MS, MAX_ABS_MV, REL_L2, activation_times, dense_parity, edge_workload, errors,
                    gpu_checkpoints, oracle_checkpoints, select_fibers)

pytestmark = pytest.mark.gpu


def _report(name, e):
    print(f"[parity] {name}: max|dV| = {e[0]:.3e} mV, rel L2 = {e[1]:.3e}")


# --------------------------------------------------------------------------
# Trajectories
# --------------------------------------------------------------------------

def test_single_fiber_full_trajectory():
    """1 fiber x 1481 nodes, 10 ms (3334 split steps), every 2nd step compared."""
    w = W.single_fiber()
    every = 2
    cps = list(range(every, w.n_steps + 1, every))
    g = gpu_checkpoints(w, cps)
    _, o = oracle.run_workload(w, n_steps=cps[-1], sample_every=every)
    e = errors(g, o)
    _report("single fiber 1x1481, 10 ms", e)
    assert e[0] <= MAX_ABS_MV and e[1] <= REL_L2
    assert o.max() > 0  # an action potential did start and propagate
    tg = activation_times(g, every * w.params["dt_split"])
    to = activation_times(o, every * w.params["dt_split"])
    assert np.array_equal(np.isnan(tg), np.isnan(to))
    fired = ~np.isnan(to)
    assert fired.sum() > 300  # ~1.7 cm each way at ~1.9 m/s in 10 ms
    dt_act = np.max(np.abs(tg[fired] - to[fired]))
    print(f"[parity] activation-time max error {dt_act:.3e} ms over {fired.sum()} nodes")
    assert dt_act <= ACT_TIME_MS


def _edge_workload(n_steps, seed=11, amp=None):
    return edge_workload(n_steps, seed, amp)


@pytest.mark.parametrize("K,Wc", [(4, 0), (8, 0), (8, 8), (12, 0), (16, 0), (16, 2)])
def test_ragged_edge_lengths_every_tuning(K, Wc):
    """Fibers of 1..700 nodes (chunk-aligned and ragged tails, 1-3 node
    fibers, junctions at the ends, unstimulated fibers) in one launch, with
    idle warps (K=8, W=8) and several fibers per CTA."""
    w = _edge_workload(600)
    cps = list(range(30, w.n_steps + 1, 30))
    g = gpu_checkpoints(w, cps, tuning=dict(nodes_per_thread=K, warps_per_cta=Wc, steps_per_launch=45))
    o = oracle_checkpoints(w, cps)
    e = errors(g, o)
    _report(f"edge lengths K={K} W={Wc}", e)
    assert e[0] <= MAX_ABS_MV and e[1] <= REL_L2
    assert o.max() > 0


def _firing_and_random(w, n_firing, n_random, seed):
    firing = [f for f in range(w.n_fibers)
              if w.mu_offsets[w.mu_of_fiber[f] + 1] > w.mu_offsets[w.mu_of_fiber[f]]]
    rng = np.random.default_rng(seed)
    pick = np.concatenate([rng.choice(firing, min(n_firing, len(firing)), replace=False),
                           W.random_fibers(w.n_fibers, n_random, seed=seed + 1)])
    return np.unique(pick)


def _check_dense(name, r):
    print(f"[parity] {name}: every 10 split steps x {r['samples']} samples, max|dV| = {r['max_abs']:.3e} mV, "
          f"rel L2 = {r['rel_l2']:.3e}, activation-time max error {r['act']:.3e} ms over {r['activated']} nodes, "
          f"shape {r['shape']}")
    assert r["max_abs"] <= MAX_ABS_MV and r["rel_l2"] <= REL_L2
    assert r["same_activated"] and r["activated"] > 0
    assert r["act"] <= ACT_TIME_MS


def test_bundle_7744_dense_trajectory():
    """7744 x 1481, 100 MUs, 20 ms (6667 steps), in the benchmark's launch
    shape: 40 seeded fibers (32 of firing motor units) compared with the
    oracle every 10 split steps over the whole run, activation times included."""
    w = W.bundle_7744(seed=2, t_end_ms=20.0)
    fibers = _firing_and_random(w, 32, 8, seed=102)
    _check_dense("bundle 7744x1481", dense_parity(w, fibers, 10, tuning=dict(graph_steps=100)))


def test_ragged_20000_dense_trajectory_autotuned():
    """20000 fibers of 800-2000 nodes, 150 MUs, noisy start, 50 ms (16667
    steps), in the launch shape the autotuner picks for the bundle: 24
    length-stratified fibers every 10 split steps."""
    w = W.ragged_20000(seed=3, t_end_ms=50.0)
    fibers = W.stratified_by_length(w.n_nodes, 24, seed=103)
    _check_dense("ragged 20000", dense_parity(w, fibers, 10, autotune=True))


def test_ragged_20000_graphs_of_1000_steps_autotuned():
    """The same bundle in 1000-step CUDA graphs with the autotuned shape,
    compared at every graph boundary (16 of them)."""
    w = W.ragged_20000(seed=3, t_end_ms=50.0)
    fibers = W.stratified_by_length(w.n_nodes, 24, seed=103)
    r = dense_parity(w, fibers, 1000, tuning=dict(graph_steps=1000), autotune=True)
    print(f"[parity] ragged 20000, graphs of 1000 steps: max|dV| = {r['max_abs']:.3e} mV, rel L2 = {r['rel_l2']:.3e}")
    assert r["max_abs"] <= MAX_ABS_MV and r["rel_l2"] <= REL_L2


def test_bundle_67600_dense_trajectory():
    """67600 x 1481 (1.0e8 nodes), 200 MUs, 100 ms (33334 steps): 24 seeded
    fibers (16 of firing motor units) every 10 split steps."""
    w = W.bundle_67600(seed=5, t_end_ms=100.0)
    fibers = _firing_and_random(w, 16, 8, seed=105)
    _check_dense("bundle 67600x1481", dense_parity(w, fibers, 10))


def test_subthreshold_stimulus_parity():
    """400 uA/cm^2 for 0.1 ms at 3 nodes: below threshold, no action potential."""
    w = W.single_fiber(t_end_ms=5.0)
    w.params["stim_amplitude"] = 400.0
    cps = list(range(10, w.n_steps + 1, 10))
    g = gpu_checkpoints(w, cps)
    o = oracle_checkpoints(w, cps)
    e = errors(g, o)
    _report("sub-threshold stimulus", e)
    assert o.max() < -40.0 and g.max() < -40.0
    assert e[0] <= 0.05 and e[1] <= 1e-4


def test_fp64_thomas_mode_parity():
    w = _edge_workload(400)
    cps = [100, 200, 400]
    g64 = gpu_checkpoints(w, cps, mode=F.FIB_MODE_FP64_THOMAS)
    g32 = gpu_checkpoints(w, cps)
    o = oracle_checkpoints(w, cps)
    e64, e32 = errors(g64, o), errors(g32, o)
    _report("FP64 Thomas", e64)
    assert e64[0] <= MAX_ABS_MV and e64[1] <= REL_L2
    assert np.max(np.abs(g64 - g32)) <= MAX_ABS_MV


# --------------------------------------------------------------------------
# Closed forms and invariants on the GPU (FP32)
# --------------------------------------------------------------------------

def _passive(w):
    w.params.update(gNa=0.0, gK=0.0, gL=0.0, EL=w.params["Vrest"])
    return w


def test_gpu_cn_cosine_mode_closed_form():
    n, m, k = 64, 40, 3
    w = _passive(W.small_ragged(1, 1, n, n, m))
    w.mu_of_fiber[:] = -1
    p = w.params
    c = p["sigma_eff"] / (p["Am"] * p["Cm"])
    v = np.cos(k * np.pi * np.arange(n) / (n - 1))
    w.vm0 = (p["Vrest"] + 10.0 * v).astype(np.float32)
    lam = -(4 * c / p["h"] ** 2) * np.sin(k * np.pi / (2 * (n - 1))) ** 2
    g1 = (1 + lam * p["dt_1d"] / 2) / (1 - lam * p["dt_1d"] / 2)
    g = gpu_checkpoints(w, [m])[0]
    expect = p["Vrest"] + 10.0 * (g1 ** (2 * m)) * v
    assert np.max(np.abs(g - expect)) <= 2e-4


def test_gpu_stimulus_charge_balance():
    w = _passive(W.single_fiber(t_end_ms=0.5, n_nodes=301))
    w.fire_times = np.array([0.0, 0.05, 0.3])
    w.mu_offsets = np.array([0, 3], np.int64)
    g = gpu_checkpoints(w, [w.n_steps])[0]
    wt = np.ones(301)
    wt[0] = wt[-1] = 0.5
    q = wt @ (g - w.params["Vrest"])
    expect = 3 * 250 * w.params["dt_0d"] * w.params["stim_amplitude"]  # substeps [0,150) U [300,400)
    assert abs(q - expect) <= 1e-4 * expect


def test_gpu_rest_stays_at_rest():
    w = W.small_ragged(4, 20, 800, 1600, 2000)
    w.vm0 = None
    w.mu_of_fiber[:] = -1
    g = gpu_checkpoints(w, [2000])[0]
    assert np.max(np.abs(g - w.params["Vrest"])) <= 1e-3


# --------------------------------------------------------------------------
# Execution paths give identical results
# --------------------------------------------------------------------------

def test_graph_eager_and_launch_blocking_are_bitwise_identical():
    w = _edge_workload(2500, seed=5)
    a = gpu_checkpoints(w, [2500], tuning=dict(nodes_per_thread=12, steps_per_launch=100, graph_steps=1000))
    b = gpu_checkpoints(w, [2500], tuning=dict(nodes_per_thread=12, steps_per_launch=100, graph_steps=0))
    c = gpu_checkpoints(w, [2500], tuning=dict(nodes_per_thread=12, steps_per_launch=7, graph_steps=0))
    assert np.array_equal(a, b) and np.array_equal(a, c)


def test_reaction_forms_and_register_budgets_are_bitwise_identical():
    """Packed FP32x2 pairs and the 80- and 64-register builds compute the
    same bits as the scalar 128-register build."""
    w = _edge_workload(700, seed=13)
    for K in (8, 12, 16):
        a = gpu_checkpoints(w, [350, 700], tuning=dict(nodes_per_thread=K, reaction_pairs=1, ctas_per_sm=2))
        for pairs, occ in ((2, 2), (1, 3), (2, 3), (1, 4), (2, 4)):
            b = gpu_checkpoints(w, [350, 700], tuning=dict(nodes_per_thread=K, reaction_pairs=pairs, ctas_per_sm=occ))
            assert np.array_equal(a, b), (K, pairs, occ)


def test_checkpoint_resume_is_bitwise():
    w = _edge_workload(900, seed=6)
    full = gpu_checkpoints(w, [900])[0]
    with F.Fibers.from_workload(w) as f1:
        f1.step(350)
        st = f1.read_state()
        idx, _ = f1.stats()
    assert idx == 350
    with F.Fibers.from_workload(w) as f2:
        f2.write_state(st, idx)
        f2.step(550)
        resumed = f2.read_vm().astype(np.float64)
    assert np.array_equal(full, resumed)


def test_set_tuning_keeps_the_state():
    w = _edge_workload(600, seed=8)
    o = oracle_checkpoints(w, [600])
    with F.Fibers.from_workload(w, tuning=dict(nodes_per_thread=8)) as f:
        f.step(300)
        before = f.read_state()
        f.set_tuning(dict(nodes_per_thread=16))
        assert f.tuning["nodes_per_thread"] == 16
        assert np.array_equal(before, f.read_state())
        f.step(300)
        g = f.read_vm().astype(np.float64)
    e = errors(g[None], o)
    assert e[0] <= MAX_ABS_MV and e[1] <= REL_L2


def test_autotune_restores_state_and_step_index():
    w = _edge_workload(200, seed=9)
    with F.Fibers.from_workload(w) as f:
        f.step(120)
        before = f.read_state()
        best = f.autotune(5)
        assert best["nodes_per_thread"] in (8, 12, 16)
        assert np.array_equal(before, f.read_state())
        assert f.stats()[0] == 120


def test_torch_stream_and_device_buffer():
    import torch
    w = _edge_workload(300, seed=10)
    s = torch.cuda.Stream()
    host = gpu_checkpoints(w, [300])[0]
    with F.Fibers.from_workload(w, stream=s) as f:
        f.step(300)
        out = torch.empty(w.total_nodes, dtype=torch.float32, device="cuda")
        F.read_vm(f.ctx, out)
        dev = out.cpu().numpy().astype(np.float64)
    assert np.array_equal(host, dev)


# --------------------------------------------------------------------------
# Edge cases and errors
# --------------------------------------------------------------------------

def test_zero_fibers_and_zero_steps():
    w = W.small_ragged(1, 1, 5, 5, 10)
    with F.Fibers(w.params, np.zeros(0, np.int32), np.zeros(0, np.int32), np.zeros(0, np.int32),
                  np.array([0], np.int64), []) as f:
        f.step(100)
        assert f.read_vm().shape == (0,)
        assert f.stats()[0] == 100
    with F.Fibers.from_workload(w) as f:
        before = f.read_state()
        f.step(0)
        assert np.array_equal(before, f.read_state())


def _lengths_workload(lengths, seed, n_steps):
    """Fibers of the given lengths, each motor unit firing once early (at
    0.05, 0.3, 0.6 and 0.9 ms), so action potentials run in every fiber."""
    w = W.small_ragged(seed, len(lengths), 5, 5, n_steps)
    rng = np.random.default_rng(seed)
    w.n_nodes = np.array(lengths, np.int32)
    w.junction = W.centre_junctions(rng, w.n_nodes, 0.05)
    w.mu_of_fiber = (np.arange(len(lengths)) % 4).astype(np.int32)
    w.mu_offsets = np.arange(5, dtype=np.int64)
    w.fire_times = np.array([0.05, 0.3, 0.6, 0.9])
    w.vm0 = (w.params["Vrest"] + rng.normal(0, 0.5, size=w.total_nodes)).astype(np.float32)
    return w


@pytest.mark.parametrize("K,lengths", [
    (8, [2048, 2047, 1793, 2048]),      # 8 warps x 32 lanes x 8 nodes: the K = 8 maximum
    (12, [3072, 3071, 2900]),           # the K = 12 maximum
    (16, [4096, 4095, 4081, 3]),        # the library's longest fiber, beside a 3-node one
    (0, [4096, 2048, 1481, 1]),         # the automatic shape picks K for the longest
])
def test_maximum_lengths_match_the_oracle(K, lengths):
    """Fibers at the longest length each launch shape holds, and one below,
    with action potentials running along them."""
    w = _lengths_workload(lengths, seed=70 + K, n_steps=500)
    cps = [125, 250, 375, 500]
    g = gpu_checkpoints(w, cps, tuning=dict(nodes_per_thread=K))
    o = oracle_checkpoints(w, cps)
    e = errors(g, o)
    _report(f"maximum lengths K={K} {lengths}", e)
    assert e[0] <= MAX_ABS_MV and e[1] <= REL_L2
    assert (o[-1] > 0).sum() >= len(lengths) - 1  # depolarised nodes in the last sample (not the 1-3 node fiber)


def test_too_long_fiber_is_rejected():
    w = W.small_ragged(1, 1, 5, 5, 10)
    with pytest.raises(F.FibersError) as ei:
        F.fibers_create(w.params, [5000], [0], [10], tuning=dict(nodes_per_thread=4))
    assert ei.value.status == F.FIB_EINVAL


def test_non_finite_state_is_reported():
    w = W.single_fiber(t_end_ms=1.0, n_nodes=64)
    w.params["stim_amplitude"] = 1e38
    with F.Fibers.from_workload(w) as f:
        f.step(50)
        with pytest.raises(F.FibersError) as ei:
            f.read_vm()
        assert ei.value.status == F.FIB_ENONFINITE


def test_bad_stimulus_tables_are_rejected():
    w = W.small_ragged(1, 3, 5, 9, 10)
    with F.Fibers(w.params, w.n_nodes, w.mu_of_fiber, w.junction) as f:
        with pytest.raises(F.FibersError):
            F.set_stimulus_times(f.ctx, [0, 2], [1.0, 0.5])  # not ascending
        with pytest.raises(F.FibersError):
            F.set_stimulus_times(f.ctx, [0, 1], [-1.0])
        with pytest.raises(F.FibersError):
            F.set_stimulus_times(f.ctx, [1, 1], [0.0])


def test_kernel_launch_count():
    w = _edge_workload(10, seed=12)
    with F.Fibers.from_workload(w, tuning=dict(nodes_per_thread=12, steps_per_launch=100, graph_steps=1000)) as f:
        n0 = f.kernel_launches
        f.step(2350)  # 2 graphs of (10 split-step launches + 1 counter update), then 4 launches + 1 update
        f.synchronize()
        assert f.kernel_launches - n0 == 2 * 11 + 4 + 1
