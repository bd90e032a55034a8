"""The autotuner and its cache on the GPU: a context whose length histogram
and method match an earlier tuned one takes the cached shape without trial
launches, its simulation is unchanged by it, and a cache written to a file
and read back serves a later context the same way."""
import numpy as np
import pytest

from paper_2107_07104_gb300 import fibers as F
from paper_2107_07104_gb300 import workloads as W

pytestmark = pytest.mark.gpu

SHAPE = ("nodes_per_thread", "warps_per_cta", "reaction_pairs", "ctas_per_sm", "warp_roles")


def _launches_of_autotune(f, n=5):
    before = f.kernel_launches
    t = f.autotune(n)
    return f.kernel_launches - before, t


def test_cache_hit_skips_the_trials_and_keeps_the_simulation(tmp_path):
    F.fibers_autotune_cache_clear()
    a = W.small_ragged(seed=61, n_fibers=40, lo=300, hi=900, n_steps=200)
    b = W.small_ragged(seed=62, n_fibers=40, lo=300, hi=900, n_steps=200)  # other junctions, MUs, V0
    b.n_nodes = a.n_nodes.copy()                                          # same length histogram
    b.junction = np.minimum(b.junction, b.n_nodes - 1)
    b.vm0 = None
    with F.Fibers.from_workload(a) as fa:
        fa.step(30)
        miss, ta = _launches_of_autotune(fa)
    assert F.fibers_autotune_cache_size() == 1
    with F.Fibers.from_workload(b) as fb:
        fb.step(30)
        st0 = fb.read_state()
        hit, tb = _launches_of_autotune(fb)
        assert np.array_equal(fb.read_state(), st0)   # the state survives the re-layout
        fb.step(120)
        v_hit = fb.read_vm()
    print(f"[autotune] miss {miss} launches, hit {hit}; shape {ta}")
    assert hit <= 9 < 40 < miss        # a hit: one state gather and scatter; a miss: every candidate twice
    assert all(ta[k] == tb[k] for k in SHAPE)
    assert F.fibers_autotune_cache_size() == 1
    # the same run with the shape set by hand gives the same bits
    with F.Fibers.from_workload(b, tuning={k: ta[k] for k in SHAPE}) as fc:
        fc.step(150)
        assert np.array_equal(fc.read_vm(), v_hit)
    # another histogram misses
    c = W.small_ragged(seed=63, n_fibers=41, lo=300, hi=900, n_steps=200)
    with F.Fibers.from_workload(c) as fd:
        miss2, _ = _launches_of_autotune(fd)
    assert miss2 > 40 and F.fibers_autotune_cache_size() == 2
    # through a file
    path = str(tmp_path / "tune.txt")
    F.fibers_autotune_cache_save(path)
    F.fibers_autotune_cache_clear()
    F.fibers_autotune_cache_load(path)
    assert F.fibers_autotune_cache_size() == 2
    with F.Fibers.from_workload(a) as fe:
        hit2, te = _launches_of_autotune(fe)
    assert hit2 <= 9 and all(te[k] == ta[k] for k in SHAPE)
    F.fibers_autotune_cache_clear()
