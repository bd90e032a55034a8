"""The split-role step kernels (dedicated reaction and diffusion warps, the
fibers of a CTA in shared memory: two per CTA with warp_roles 2, eight per
1024-thread CTA with warp_roles 3) against the FP64 oracle and against the
fused kernel."""
import numpy as np
import pytest

from paper_2107_07104_gb300 import fibers as F
from paper_2107_07104_gb300 import workloads as W

from parity import (ACT_TIME_MS, MAX_ABS_MV, REL_L2, dense_parity, edge_workload, errors, gpu_checkpoints,
                    oracle_checkpoints)

pytestmark = pytest.mark.gpu

SHAPES = [2, 3]


@pytest.mark.parametrize("roles", SHAPES)
def test_ragged_lengths_and_a_lone_fiber_match_the_oracle(roles):
    # 1..700-node fibers (odd count: the last CTA holds one fiber), junctions
    # at the ends, unstimulated fibers, noisy start; 45-step launches
    w = edge_workload(600)
    if w.n_fibers % 2 == 0:  # drop the last fiber
        keep = w.total_nodes - int(w.n_nodes[-1])
        w.n_nodes, w.junction, w.mu_of_fiber = w.n_nodes[:-1], w.junction[:-1], w.mu_of_fiber[:-1]
        w.vm0 = w.vm0[:keep]
    assert w.n_fibers % 2 == 1
    cps = list(range(30, w.n_steps + 1, 30))
    g = gpu_checkpoints(w, cps, tuning=dict(warp_roles=roles, steps_per_launch=45))
    o = oracle_checkpoints(w, cps)
    e = errors(g, o)
    print(f"[ws{roles}] edge lengths: max|dV| = {e[0]:.3e} mV, rel L2 = {e[1]:.3e}")
    assert e[0] <= MAX_ABS_MV and e[1] <= REL_L2
    assert o.max() > 0


@pytest.mark.parametrize("roles", SHAPES)
def test_the_longest_fibers_fill_the_slot(roles):
    w = W.small_ragged(seed=51, n_fibers=13, lo=1500, hi=1536, n_steps=400)
    cps = [100, 250, 400]
    g = gpu_checkpoints(w, cps, tuning=dict(warp_roles=roles))
    o = oracle_checkpoints(w, cps)
    e = errors(g, o)
    assert e[0] <= MAX_ABS_MV and e[1] <= REL_L2


@pytest.mark.parametrize("roles", SHAPES)
def test_shape_is_reported_and_graphs_match_eager_launches(roles):
    w = W.small_ragged(seed=52, n_fibers=20, lo=900, hi=1481, n_steps=300)
    out = []
    for graph_steps in (0, 100):
        with F.Fibers.from_workload(w, tuning=dict(warp_roles=roles, graph_steps=graph_steps)) as f:
            assert f.tuning["warp_roles"] == roles
            f.step(300)
            out.append(f.read_state())
    assert np.array_equal(out[0], out[1])


@pytest.mark.parametrize("roles", SHAPES)
def test_ineligible_contexts_are_rejected(roles):
    w = W.small_ragged(seed=53, n_fibers=3, lo=1600, hi=1700, n_steps=10)
    with pytest.raises(F.FibersError) as ei:
        F.Fibers.from_workload(w, tuning=dict(warp_roles=roles))
    assert ei.value.status == F.FIB_EINVAL
    w2 = W.small_ragged(seed=53, n_fibers=3, lo=100, hi=200, n_steps=10)
    w2.params["flags"] = F.FIB_FLAG_ADAPTIVE
    with pytest.raises(F.FibersError):
        F.Fibers.from_workload(w2, tuning=dict(warp_roles=roles))


@pytest.mark.parametrize("roles", SHAPES)
def test_bundle_7744_dense_trajectory_split_roles(roles):
    """The 7744-fiber bundle, 20 ms, 40 fibers every 10 split steps."""
    w = W.bundle_7744(seed=2, t_end_ms=20.0)
    firing = [f for f in range(w.n_fibers) if w.mu_offsets[w.mu_of_fiber[f] + 1] > w.mu_offsets[w.mu_of_fiber[f]]]
    rng = np.random.default_rng(102)
    fibers = np.unique(np.concatenate([rng.choice(firing, 32, replace=False), W.random_fibers(w.n_fibers, 8, 103)]))
    r = dense_parity(w, fibers, 10, tuning=dict(warp_roles=roles, graph_steps=100))
    print(f"[ws{roles}] bundle 7744: max|dV| = {r['max_abs']:.3e} mV, rel L2 = {r['rel_l2']:.3e}, act {r['act']:.3e} ms")
    assert r["max_abs"] <= MAX_ABS_MV and r["rel_l2"] <= REL_L2 and r["act"] <= ACT_TIME_MS
    assert r["same_activated"]


@pytest.mark.parametrize("roles", SHAPES)
def test_checkpoint_resume_and_switching_shapes(roles):
    """A split-role run resumed from its checkpoint gives the same bits; a
    re-layout between the fused kernel and a split-role shape keeps the state
    bit for bit, and the mixed run stays on the oracle's trajectory."""
    w = W.small_ragged(seed=54, n_fibers=19, lo=700, hi=1536, n_steps=400)
    t = dict(warp_roles=roles)
    with F.Fibers.from_workload(w, tuning=t) as f:
        f.step(400)
        full = f.read_state()
    with F.Fibers.from_workload(w, tuning=t) as f:
        f.step(150)
        st = f.read_state()
        idx, _ = f.stats()
    with F.Fibers.from_workload(w, tuning=t) as f:
        f.write_state(st, idx)
        f.step(250)
        assert np.array_equal(f.read_state(), full)
    with F.Fibers.from_workload(w, tuning=dict(warp_roles=1)) as f:
        f.step(200)
        before = f.read_state()
        f.set_tuning(t)
        assert f.tuning["warp_roles"] == roles
        assert np.array_equal(f.read_state(), before)
        f.step(200)
        mixed = f.read_vm().astype(np.float64)
    o = oracle_checkpoints(w, [400])[0]
    e = errors(mixed[None, :], o[None, :])
    assert e[0] <= MAX_ABS_MV and e[1] <= REL_L2
