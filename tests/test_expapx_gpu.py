"""The thesis's approximated exponential exp*(x) = (1 + x/1024)^1024
(eq:apx-e-function) on the GPU: parity with the FP64 oracle running the same
approximated model, bitwise agreement of the kernel's reaction forms, and the
size of the approximation's effect against the exact-exponential model."""
import numpy as np
import pytest

import oracle
from paper_2107_07104_gb300 import fibers as F
from paper_2107_07104_gb300 import workloads as W

from parity import (ACT_TIME_MS, MAX_ABS_MV, REL_L2, activation_times, edge_workload, errors, gpu_checkpoints,
                    oracle_checkpoints)

pytestmark = pytest.mark.gpu


def _report(name, e):
    print(f"[exp*] {name}: max|dV| = {e[0]:.3e} mV, rel L2 = {e[1]:.3e}")


@pytest.mark.parametrize("K,pairs", [(8, 2), (8, 1), (16, 2), (4, 1)])
def test_exp_star_path_matches_the_oracle(K, pairs):
    w = edge_workload(600, seed=29)
    w.params["exp_approx"] = 1
    cps = list(range(30, w.n_steps + 1, 30))
    g = gpu_checkpoints(w, cps, tuning=dict(nodes_per_thread=K, reaction_pairs=pairs, steps_per_launch=45))
    o = oracle_checkpoints(w, cps)
    e = errors(g, o)
    _report(f"edge lengths K={K} pairs={pairs}", e)
    assert e[0] <= MAX_ABS_MV and e[1] <= REL_L2
    assert o.max() > 0


def test_exp_star_reaction_forms_are_bitwise_identical():
    w = edge_workload(400, seed=31)
    w.params["exp_approx"] = 1
    a = gpu_checkpoints(w, [200, 400], tuning=dict(nodes_per_thread=8, reaction_pairs=1, ctas_per_sm=2))
    for pairs, occ in ((2, 2), (2, 3), (1, 3), (2, 4)):
        b = gpu_checkpoints(w, [200, 400], tuning=dict(nodes_per_thread=8, reaction_pairs=pairs, ctas_per_sm=occ))
        assert np.array_equal(a, b), (pairs, occ)


def test_exp_star_effect_against_the_exact_model_on_a_fiber():
    """The approximation moves a propagating action potential by well under
    a millivolt and its activation times by microseconds; the GPU exp* path
    shows the same effect against the exact-exponential oracle."""
    w = W.single_fiber(t_end_ms=6.0, n_nodes=801)
    every = 5
    cps = list(range(every, w.n_steps + 1, every))
    wa = w.with_steps(w.n_steps)
    wa.params = dict(w.params, exp_approx=1)
    g = gpu_checkpoints(wa, cps)
    _, o_exact = oracle.run_workload(w, n_steps=cps[-1], sample_every=every)
    _, o_apx = oracle.run_workload(wa, n_steps=cps[-1], sample_every=every)
    e = errors(g, o_apx)
    _report("single fiber 801 nodes vs oracle exp*", e)
    assert e[0] <= MAX_ABS_MV and e[1] <= REL_L2
    d_gpu = errors(g, o_exact)
    d_ref = errors(o_apx, o_exact)
    _report("single fiber, GPU exp* vs exact-exponential oracle", d_gpu)
    _report("single fiber, oracle exp* vs exact-exponential oracle", d_ref)
    assert d_gpu[0] <= 1.5 and abs(d_gpu[0] - d_ref[0]) <= MAX_ABS_MV
    dt = every * w.params["dt_split"]
    tg, tx = activation_times(g, dt), activation_times(o_exact, dt)
    both = ~np.isnan(tg) & ~np.isnan(tx)
    assert both.sum() > 100
    assert np.max(np.abs(tg[both] - tx[both])) <= ACT_TIME_MS
