"""Scheme variants on the GPU against the FP64 oracle: Godunov splitting
(eq:monodomain_godunov) and the 0D-1D-0D Strang ordering of the splitting
figures, with Crank-Nicolson (eq:lumping_crank_nicolson_2) or implicit-Euler
(eq:lumping_implicit_euler_2) diffusion.  Same tolerances as the default
scheme: max |dV| <= 0.5 mV and relative L2 <= 1e-3 over the trajectory."""
import numpy as np
import pytest

import oracle
from paper_2107_07104_gb300 import fibers as F
from paper_2107_07104_gb300 import workloads as W

from parity import (ACT_TIME_MS, MAX_ABS_MV, REL_L2, activation_times, edge_workload, errors, gpu_checkpoints,
                    oracle_checkpoints)

pytestmark = pytest.mark.gpu

G1, G3 = F.SPLIT_GODUNOV_1D0D, F.SPLIT_GODUNOV_0D1D
S0, S2 = F.SPLIT_STRANG_1D0D1D, F.SPLIT_STRANG_0D1D0D
CN, IE = F.DIFFUSION_CRANK_NICOLSON, F.DIFFUSION_IMPLICIT_EULER

# (name, scheme parameters); dt_split stays 3e-3 ms
SCHEMES = [
    ("godunov 1D-0D, IE, one diffusion step", dict(splitting=G1, diffusion=IE, dt_1d=3e-3)),
    ("godunov 0D-1D, IE, two diffusion steps", dict(splitting=G3, diffusion=IE, dt_1d=1.5e-3)),
    ("godunov 1D-0D, CN", dict(splitting=G1, diffusion=CN, dt_1d=3e-3)),
    ("strang 0D-1D-0D, CN", dict(splitting=S2, diffusion=CN, dt_0d=7.5e-4, dt_1d=3e-3)),
    ("strang 0D-1D-0D, IE", dict(splitting=S2, diffusion=IE, dt_0d=5e-4, dt_1d=1.5e-3)),
    ("strang 1D-0D-1D, IE", dict(splitting=S0, diffusion=IE)),
]


def _with(w, **kw):
    w.params.update(kw)
    return w


def _report(name, e):
    print(f"[schemes] {name}: max|dV| = {e[0]:.3e} mV, rel L2 = {e[1]:.3e}")


@pytest.mark.parametrize("name,scheme", SCHEMES, ids=[s[0] for s in SCHEMES])
def test_scheme_on_ragged_edge_lengths(name, scheme):
    """Fibers of 1..700 nodes with ragged tails, end junctions and
    unstimulated fibers; launches of 45 steps so launch boundaries fall
    inside the trajectory."""
    w = _with(edge_workload(600), **scheme)
    cps = list(range(30, w.n_steps + 1, 30))
    g = gpu_checkpoints(w, cps, tuning=dict(nodes_per_thread=8, steps_per_launch=45))
    o = oracle_checkpoints(w, cps)
    e = errors(g, o)
    _report(name, e)
    assert e[0] <= MAX_ABS_MV and e[1] <= REL_L2
    assert o.max() > 0


@pytest.mark.parametrize("K,Wc,pairs", [(4, 0, 1), (16, 2, 2), (12, 0, 2)])
def test_godunov_implicit_euler_every_tuning(K, Wc, pairs):
    w = _with(edge_workload(400, seed=17), splitting=G3, diffusion=IE, dt_1d=1.5e-3)
    cps = list(range(40, w.n_steps + 1, 40))
    g = gpu_checkpoints(w, cps, tuning=dict(nodes_per_thread=K, warps_per_cta=Wc, reaction_pairs=pairs,
                                            steps_per_launch=25))
    o = oracle_checkpoints(w, cps)
    e = errors(g, o)
    _report(f"godunov 0D-1D IE K={K} W={Wc} pairs={pairs}", e)
    assert e[0] <= MAX_ABS_MV and e[1] <= REL_L2


def test_implicit_euler_fp64_thomas_mode():
    w = _with(edge_workload(300, seed=19), splitting=S2, diffusion=IE, dt_0d=7.5e-4, dt_1d=3e-3)
    cps = list(range(50, w.n_steps + 1, 50))
    g = gpu_checkpoints(w, cps, mode=F.FIB_MODE_FP64_THOMAS)
    o = oracle_checkpoints(w, cps)
    e = errors(g, o)
    _report("strang 0D-1D-0D IE, FP64 tridiagonal solve", e)
    assert e[0] <= MAX_ABS_MV and e[1] <= REL_L2


def test_thesis_scheme_pair_on_a_long_fiber():
    """The two schemes the thesis compares for one fiber: Godunov with
    implicit-Euler diffusion at dt_0D = 1e-4, dt_splitting = dt_1D = 5e-4 ms,
    and Strang 0D-1D-0D with Crank-Nicolson at dt_0D = 2e-3,
    dt_splitting = dt_1D = 4e-3 ms (Heun for the reaction in both)."""
    cases = {
        "godunov IE dt 5e-4": dict(splitting=G3, diffusion=IE, dt_split=5e-4, dt_0d=1e-4, dt_1d=5e-4),
        "strang 0D-1D-0D CN dt 4e-3": dict(splitting=S2, diffusion=CN, dt_split=4e-3, dt_0d=2e-3, dt_1d=4e-3),
    }
    t_end = 3.0
    for name, sc in cases.items():
        w = W.single_fiber(t_end_ms=t_end, n_nodes=701)
        w.params.update(sc)
        dt = sc["dt_split"]
        n = int(round(t_end / dt))
        every = max(1, int(round(0.02 / dt)))
        cps = list(range(every, n + 1, every))
        g = gpu_checkpoints(w, cps)
        state = oracle.init_state(w.params, w.total_nodes, w.vm0)
        o = oracle.run(w.params, w.n_nodes, w.mu_of_fiber, w.junction, w.mu_offsets, w.fire_times, state, 0,
                       cps[-1], sample_every=every)
        e = errors(g, o)
        _report(f"single fiber 701 nodes, {name}", e)
        assert e[0] <= MAX_ABS_MV and e[1] <= REL_L2
        tg = activation_times(g, every * dt)
        to = activation_times(o, every * dt)
        assert np.array_equal(np.isnan(tg), np.isnan(to))
        fired = ~np.isnan(to)
        assert fired.sum() > 60  # about 0.5 cm each way in 3 ms
        assert np.max(np.abs(tg[fired] - to[fired])) <= ACT_TIME_MS


def test_adaptive_godunov_matches_the_oracle():
    w = W.small_ragged(seed=23, n_fibers=24, lo=150, hi=900, n_steps=2000, n_mu=6, rate_hz=150.0, v0_sigma=0.0)
    w.params.update(splitting=G3, diffusion=IE, dt_1d=3e-3, flags=F.FIB_FLAG_ADAPTIVE)
    cps = [400, 800, 1200, 2000]
    g = gpu_checkpoints(w, cps, tuning=dict(steps_per_launch=50))
    o = oracle_checkpoints(w, cps)
    e = errors(g, o)
    with F.Fibers.from_workload(w, tuning=dict(steps_per_launch=50)) as f:
        f.step(w.n_steps)
        skipped = F.fibers_adaptive_stats(f.ctx)
    _report(f"adaptive godunov 0D-1D IE (skipped {skipped} of {w.n_fibers * w.n_steps} fiber-steps)", e)
    assert e[0] <= MAX_ABS_MV and e[1] <= REL_L2
    assert o.max() > 0  # action potentials did start
    assert skipped > 0
