"""Adaptive computation (sec:adaptive_computation_for_fiber_based): fibers in
equilibrium with no pulse due are skipped, and the result stays within the
FP32 tolerances of the FP64 oracle's full computation."""
import numpy as np
import pytest

from paper_2107_07104_gb300 import fibers as F
from paper_2107_07104_gb300 import workloads as W

from parity import (ACT_TIME_MS, MAX_ABS_MV, REL_L2, activation_times, errors, gpu_checkpoints,
                    oracle_checkpoints)

pytestmark = pytest.mark.gpu


def _adaptive(w):
    w.params["flags"] = F.FIB_FLAG_ADAPTIVE
    return w


def _skipped(w, steps, tuning=None):
    with F.Fibers.from_workload(w, tuning=tuning) as f:
        f.step(steps)
        return F.fibers_adaptive_stats(f.ctx)


def test_adaptive_bundle_matches_the_oracle():
    full = W.bundle_7744(seed=2, t_end_ms=20.0)
    firing = [f for f in range(full.n_fibers)
              if full.mu_offsets[full.mu_of_fiber[f] + 1] > full.mu_offsets[full.mu_of_fiber[f]]]
    rng = np.random.default_rng(21)
    fibers = np.sort(np.concatenate([rng.choice(firing, 12, replace=False),
                                     rng.choice(np.setdiff1d(np.arange(full.n_fibers), firing), 12, replace=False)]))
    w = _adaptive(full.subset(fibers))
    cps = list(range(100, w.n_steps + 1, 100))
    g = gpu_checkpoints(w, cps)
    o = oracle_checkpoints(w, cps)
    e = errors(g, o)
    skipped = _skipped(w, w.n_steps)
    print(f"[adaptive] bundle subset: max|dV| = {e[0]:.3e} mV, rel L2 = {e[1]:.3e}, "
          f"skipped {skipped} of {w.n_fibers * w.n_steps} fiber-steps")
    assert e[0] <= MAX_ABS_MV and e[1] <= REL_L2
    assert skipped >= 0.3 * w.n_fibers * w.n_steps  # the never-stimulated half is skipped


def test_adaptive_ragged_with_noisy_start_matches_the_oracle():
    w = _adaptive(W.small_ragged(seed=22, n_fibers=30, lo=200, hi=1200, n_steps=3000, rate_hz=60.0))
    cps = [500, 1000, 2000, 3000]
    g = gpu_checkpoints(w, cps)
    o = oracle_checkpoints(w, cps)
    e = errors(g, o)
    print(f"[adaptive] ragged noisy start: max|dV| = {e[0]:.3e} mV, rel L2 = {e[1]:.3e}")
    assert e[0] <= MAX_ABS_MV and e[1] <= REL_L2


def test_quiet_fiber_is_woken_by_a_late_pulse():
    w = _adaptive(W.single_fiber(t_end_ms=12.0, n_nodes=601))
    w.fire_times = np.array([6.0])  # after many quiet launches
    every = 5
    cps = list(range(every, w.n_steps + 1, every))
    g = gpu_checkpoints(w, cps)
    o = oracle_checkpoints(w, cps)
    dt = every * w.params["dt_split"]
    tg, to = activation_times(g, dt), activation_times(o, dt)
    assert np.array_equal(np.isnan(tg), np.isnan(to)) and (~np.isnan(to)).sum() > 100
    assert np.nanmax(np.abs(tg - to)) <= ACT_TIME_MS
    assert _skipped(w, w.n_steps) > 0


def test_replacing_the_state_reactivates_fibers():
    w = _adaptive(W.small_ragged(seed=23, n_fibers=8, lo=100, hi=300, n_steps=600, rate_hz=1e-3, v0_sigma=0.0))
    with F.Fibers.from_workload(w) as f:
        f.step(400)
        s0 = F.fibers_adaptive_stats(f.ctx)
        assert s0 > 0  # at rest and never stimulated: skipped after the first launch
        st = f.read_state()
        st[0] += 20.0  # depolarise the first node of fiber 0: it must be computed again
        f.write_state(st, 400)
        f.step(100)
        v = f.read_vm()
    ref = dict(w.params)
    ref["flags"] = 0
    with F.Fibers(ref, w.n_nodes, w.mu_of_fiber, w.junction, w.mu_offsets, w.fire_times, w.vm0) as g:
        g.step(400)
        g.write_state(st, 400)
        g.step(100)
        vp = g.read_vm()
    assert np.max(np.abs(v.astype(np.float64) - vp)) <= MAX_ABS_MV
    assert v[0] != F.make_params(w.params).Vrest + 20.0  # the perturbed node evolved
