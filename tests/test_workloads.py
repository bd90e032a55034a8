"""The seeded workload generator draws inputs of the thesis's shapes."""
import numpy as np

from paper_2107_07104_gb300 import workloads as W


def test_workloads_are_deterministic():
    a = W.small_ragged(7, 30, 10, 200, 100)
    b = W.small_ragged(7, 30, 10, 200, 100)
    for k in ("n_nodes", "mu_of_fiber", "junction", "mu_offsets", "fire_times", "vm0"):
        assert np.array_equal(getattr(a, k), getattr(b, k))


def test_single_fiber_shape():
    w = W.single_fiber()
    assert w.n_fibers == 1 and w.n_nodes[0] == 1481 and w.junction[0] == 740
    assert w.n_steps == 3334  # ceil(10 / 0.003)
    assert list(w.fire_times) == [0.0]


def test_bundle_mu_sizes_follow_the_exponential_progression():
    w = W.bundle_7744(seed=2, t_end_ms=20.0)
    assert w.n_fibers == 7744 and np.all(w.n_nodes == 1481) and w.n_mu == 100
    counts = np.bincount(w.mu_of_fiber, minlength=100)
    assert counts.min() >= 1  # empty MUs repaired
    q = W.mu_size_probabilities(100, 1.02)
    # largest/smallest expected ratio 1.02^99 ~ 7.1; sampled sizes track q
    assert np.corrcoef(counts, q * 7744)[0, 1] > 0.9
    assert np.all(np.abs(w.junction - 740) <= 74)  # centre +- 5% of 1480


def test_poisson_rates_and_ragged_lengths():
    w = W.ragged_20000(seed=3, t_end_ms=50.0)
    assert w.n_nodes.min() >= 800 and w.n_nodes.max() <= 2000
    assert abs(w.vm0.mean() + 75.0) < 0.01 and abs(w.vm0.std() - 0.5) < 0.01
    rng = np.random.default_rng(0)
    offs, times = W.poisson_trains(rng, np.full(2000, 20.0), 1000.0)
    counts = np.diff(offs)
    assert abs(counts.mean() - 20.0) < 0.5  # 20 Hz over 1 s
    for k in range(5):
        t = times[offs[k]:offs[k + 1]]
        assert np.all(np.diff(t) >= 0) and (t.size == 0 or (t[0] >= 0 and t[-1] < 1000.0))


def test_subset_keeps_fibers_and_initial_voltages():
    w = W.small_ragged(3, 12, 10, 50, 20)
    s = w.subset([1, 5, 7])
    off = w.offsets()
    assert np.array_equal(s.n_nodes, w.n_nodes[[1, 5, 7]])
    assert np.array_equal(s.vm0, np.concatenate([w.vm0[off[i]:off[i + 1]] for i in (1, 5, 7)]))


def test_full_scale_bundle_recipe():
    w = W.bundle_67600(seed=5, t_end_ms=100.0)
    assert w.n_fibers == 67600 and np.all(w.n_nodes == 1481) and w.n_mu == 200
    assert w.total_nodes == 100_115_600 and w.n_steps == 33334  # ceil(100 / 0.003)
    counts = np.bincount(w.mu_of_fiber, minlength=200)
    assert counts.min() >= 1
    q = W.mu_size_probabilities(200, 10.0 ** (1.0 / 200))
    assert abs(q[-1] / q[0] - 10.0 ** (199 / 200)) < 1e-9  # largest/smallest MU about 10
    assert np.corrcoef(counts, q * 67600)[0, 1] > 0.95
    # rates uniform in 10-30 Hz: about 2 firings per MU in 100 ms
    assert 1.5 < np.diff(w.mu_offsets).mean() < 2.5
    assert np.all(np.abs(w.junction - 740) <= 74)
