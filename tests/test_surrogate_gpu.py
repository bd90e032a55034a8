"""GPU tests of the reaction-step surrogate: its kernels against the FP64
oracles, and the surrogate path against the plain path and the oracle."""
import numpy as np
import pytest

import oracle
from oracle import mlp as omlp
from paper_2107_07104_gb300 import fibers as F
from paper_2107_07104_gb300 import surrogate as S
from paper_2107_07104_gb300 import workloads as W

from parity import ACT_TIME_MS, MAX_ABS_MV, REL_L2, errors, gpu_checkpoints, oracle_checkpoints, select_fibers

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def test_reaction_kernel_matches_oracle_heun_steps():
    p = dict(W.DEFAULT_PARAMS)
    rng = np.random.default_rng(0)
    n = 4096
    V = rng.uniform(-90, 40, n)
    gates = rng.uniform(0.02, 0.98, (3, n))
    mask = rng.choice(S.STIM_PATTERNS.tolist() + [0, 0, 0], n).astype(np.uint8)
    x_in = torch.tensor(np.concatenate([V, gates.ravel()]), dtype=torch.float32, device="cuda")
    x_out = torch.empty_like(x_in)
    F.fibers_hh_reaction(p, x_in, torch.tensor(mask, device="cuda"), x_out)
    got = x_out.cpu().numpy().reshape(4, n)
    ref = np.zeros((4, n))
    xin = x_in.cpu().numpy().astype(np.float64).reshape(4, n)
    for i in range(n):
        y = xin[:, i].copy()
        for k in range(3):
            on = (mask[i] >> k) & 1
            y = oracle.heun_step(p, y, p["dt_0d"], p["stim_amplitude"] if on else 0.0)
        ref[:, i] = y
    assert np.max(np.abs(got[0] - ref[0])) <= 2e-3  # mV, from FP32 inputs and arithmetic
    assert np.max(np.abs(got[1:] - ref[1:])) <= 2e-5


@pytest.mark.parametrize("quantize,tol", [(False, 2e-4), (True, 2e-2)])
def test_training_kernels_match_the_oracle(quantize, tol):
    rng = np.random.default_rng(1)
    theta = omlp.init_params(3) + rng.normal(0, 0.02, omlp.N_PARAMS)
    B = 96
    x = rng.normal(size=(B, 5))
    t = rng.normal(size=(B, 4))
    th = torch.tensor(theta, dtype=torch.float32, device="cuda")
    xd = torch.tensor(x, dtype=torch.float32, device="cuda")
    td = torch.tensor(t, dtype=torch.float32, device="cuda")
    work = torch.empty(B * F.SUR_WORK_PER_SAMPLE, dtype=torch.float32, device="cuda")
    grad = torch.zeros_like(th)
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    F.fibers_mlp_train_step(th, quantize, xd, td, work, grad, loss)
    # the oracle sees exactly the FP32 values the GPU saw
    th64 = th.cpu().numpy().astype(np.float64)
    x64 = xd.cpu().numpy().astype(np.float64)
    t64 = td.cpu().numpy().astype(np.float64)
    g_ref, l_ref = omlp.backward(th64, x64, t64, quantize=quantize)
    g = grad.cpu().numpy().astype(np.float64)
    assert abs(loss.item() - l_ref) <= tol * l_ref
    assert np.linalg.norm(g - g_ref) <= tol * np.linalg.norm(g_ref)
    out = torch.empty(B, 4, dtype=torch.float32, device="cuda")
    F.fibers_mlp_forward(th, quantize, xd, work, out)
    o_ref, _ = omlp.forward(th64, x64, quantize=quantize)
    assert np.max(np.abs(out.cpu().numpy() - o_ref)) <= tol * max(1.0, np.max(np.abs(o_ref)))


def test_adam_kernel_matches_the_oracle():
    rng = np.random.default_rng(2)
    n = 1000
    th, m, v, g = (rng.normal(size=n) for _ in range(4))
    v = np.abs(v)
    dt = lambda a: torch.tensor(a, dtype=torch.float32, device="cuda")
    T, M, Vv, G = dt(th), dt(m), dt(v), dt(g)
    F.fibers_adam_step(T, M, Vv, G, 1e-3, 7)
    ref, mr, vr = omlp.adam_step(th.astype(np.float32).astype(np.float64), m.astype(np.float32),
                                 v.astype(np.float32), g.astype(np.float32), 7, 1e-3)
    assert np.max(np.abs(T.cpu().numpy() - ref)) <= 1e-6
    assert np.max(np.abs(M.cpu().numpy() - mr)) <= 1e-6


def test_adam_kernel_weight_average_matches_the_oracle():
    rng = np.random.default_rng(5)
    n = 777
    th, m, v, g, avg = (rng.normal(size=n) for _ in range(5))
    v = np.abs(v)
    dt = lambda a: torch.tensor(a, dtype=torch.float32, device="cuda")
    T, M, Vv, G, A = dt(th), dt(m), dt(v), dt(g), dt(avg)
    F.fibers_adam_step(T, M, Vv, G, 1e-3, 3, theta_avg=A, avg_decay=0.99)
    f32 = lambda a: a.astype(np.float32).astype(np.float64)
    ref, _, _ = omlp.adam_step(f32(th), f32(m), f32(v), f32(g), 3, 1e-3)
    ref_avg = omlp.weight_average(f32(avg), ref, 0.99)
    assert np.max(np.abs(A.cpu().numpy() - ref_avg)) <= 1e-6
    with pytest.raises(F.FibersError):
        F.fibers_adam_step(T, M, Vv, G, 1e-3, 4, theta_avg=A, avg_decay=1.5)


def test_feature_stats_kernel():
    rng = np.random.default_rng(3)
    X = rng.normal(size=(10000, 5)) * [1, 2, 3, 4, 5] + [5, 4, 3, 2, 1]
    st = F.fibers_feature_stats(torch.tensor(X, dtype=torch.float32, device="cuda"))
    Xf = X.astype(np.float32).astype(np.float64)
    assert np.allclose(st[:, 0], Xf.mean(0), atol=1e-9)
    assert np.allclose(st[:, 1], Xf.std(0), rtol=1e-6)
    assert np.allclose(st[:, 2], Xf.min(0)) and np.allclose(st[:, 3], Xf.max(0))


def _exclude_all_blob():
    theta = omlp.init_params(5).astype(np.float32)
    lo = np.full(5, 1.0, np.float32)
    hi = np.full(5, -1.0, np.float32)  # empty envelope: every node falls back
    return S.make_blob(theta, np.zeros(5, np.float32), np.ones(5, np.float32), np.zeros(4, np.float32),
                       np.ones(4, np.float32), lo, hi, lo, hi)


@pytest.mark.parametrize("K", [8, 12])
def test_fallback_reproduces_the_plain_path_bit_for_bit(K):
    """With every node outside the envelope the surrogate step is the plain
    step, bit for bit, in the same launch shape (the automatic shapes of the
    two modes differ: K = 8 for the surrogate step, 12 for the plain one)."""
    w = W.small_ragged(seed=31, n_fibers=24, lo=1, hi=700, n_steps=300)
    t = dict(nodes_per_thread=K)
    plain = gpu_checkpoints(w, [150, 300], tuning=t)
    with F.Fibers.from_workload(w, mode=F.FIB_MODE_SURROGATE, tuning=t) as f:
        with pytest.raises(F.FibersError) as ei:
            f.step(1)  # no surrogate loaded yet
        assert ei.value.status == F.FIB_ESTATE
        F.fibers_load_surrogate(f.ctx, _exclude_all_blob())
        f.step(150)
        a = f.read_vm().astype(np.float64)
        f.step(150)
        b = f.read_vm().astype(np.float64)
        _, fallbacks = f.stats()
    assert np.array_equal(a, plain[0]) and np.array_equal(b, plain[1])
    assert fallbacks == 300 * w.total_nodes


@pytest.fixture(scope="module")
def trained_blob():
    """Trained here from scratch: samples from the plain method, GPU training."""
    log = []
    blob = S.build_surrogate(seed=0, log=log)
    assert log[-1] < 0.02 * log[0]  # training reduced the loss by 50x or more
    return blob


def test_surrogate_blob_is_loadable_and_finite(trained_blob):
    assert trained_blob.size == F.SUR_BLOB_FLOATS and np.isfinite(trained_blob).all()
    w = W.small_ragged(seed=1, n_fibers=2, lo=50, hi=60, n_steps=10)
    with F.Fibers.from_workload(w, mode=F.FIB_MODE_SURROGATE) as f:
        F.fibers_load_surrogate(f.ctx, trained_blob)
        f.step(10)
        assert np.isfinite(f.read_vm()).all()


def test_surrogate_on_held_out_bundle(trained_blob):
    """Held-out seed of the 7744-fiber bundle (seed 4), 16 fibers, 20 ms:
    errors against the FP64 oracle, next to the plain FP32 path's."""
    full = W.bundle_7744(seed=4, t_end_ms=20.0)
    firing = [f for f in range(full.n_fibers) if full.mu_offsets[full.mu_of_fiber[f] + 1] > full.mu_offsets[full.mu_of_fiber[f]]]
    fibers = np.sort(np.random.default_rng(4).choice(firing, 16, replace=False))
    w = full.subset(fibers)
    cps = list(range(10, w.n_steps + 1, 10))
    o = oracle_checkpoints(w, cps)
    plain = gpu_checkpoints(w, cps)
    sur = []
    with F.Fibers.from_workload(w, mode=F.FIB_MODE_SURROGATE) as f:
        F.fibers_load_surrogate(f.ctx, trained_blob)
        done = 0
        for c in cps:
            f.step(c - done)
            done = c
            sur.append(f.read_vm().astype(np.float64))
        _, fb = f.stats()
    sur = np.array(sur)
    ep, es = errors(plain, o), errors(sur, o)
    from parity import activation_times
    dt = 10 * w.params["dt_split"]
    to, ts = activation_times(o, dt), activation_times(sur, dt)
    both = ~np.isnan(to) & ~np.isnan(ts)
    act = float(np.max(np.abs(to[both] - ts[both]))) if both.any() else float("nan")
    print(f"[surrogate] plain FP32: max|dV| {ep[0]:.3e} mV rel L2 {ep[1]:.3e}; surrogate: max|dV| {es[0]:.3e} mV "
          f"rel L2 {es[1]:.3e}; activation-time max error {act:.3e} ms over {both.sum()} nodes "
          f"(missed {int((~np.isnan(to) & np.isnan(ts)).sum())}); fallback node-steps {fb}")
    assert np.isfinite(sur).all()
    fired = ~np.isnan(to)
    assert fb < w.n_steps * w.total_nodes             # the network did handle node-steps
    assert both.sum() == fired.sum()                  # every activation the oracle has
    assert (np.isnan(to) & ~np.isnan(ts)).sum() == 0  # no spurious excitation
    assert act <= ACT_TIME_MS                         # activation times within 0.05 ms
    assert es[0] <= MAX_ABS_MV                        # max|dV| <= 0.5 mV over the trajectory
    assert es[1] <= REL_L2                            # relative L2 <= 1e-3 over the trajectory


def test_surrogate_mode_graphs_match_eager_launches():
    """Surrogate split steps replayed as CUDA graphs give the same bits as
    launched one by one, with the committed network handling the firing
    nodes; reloading the weights rebuilds the graph."""
    w = W.small_ragged(seed=33, n_fibers=40, lo=300, hi=1200, n_steps=1600)
    w.mu_offsets = np.arange(5, dtype=np.int64)           # one firing per motor unit
    w.fire_times = np.array([0.05, 0.3, 0.6, 0.9])
    blob = S.load_blob()
    out = []
    # 4.8 ms: the action potentials have passed their peak and repolarise,
    # so nodes enter the network's trust box
    for graph_steps in (0, 200, 200):
        with F.Fibers.from_workload(w, mode=F.FIB_MODE_SURROGATE, tuning=dict(graph_steps=graph_steps)) as f:
            F.fibers_load_surrogate(f.ctx, blob)
            f.step(1400)
            if len(out) == 2:
                F.fibers_load_surrogate(f.ctx, blob)  # invalidates the captured graph
            f.step(200)
            _, fb = f.stats()
            out.append((f.read_state(), fb))
    assert out[0][1] < 1600 * w.total_nodes  # the network did handle nodes
    for st, fb in out[1:]:
        assert np.array_equal(st, out[0][0]) and fb == out[0][1]


def test_surrogate_rewind_matches_a_fresh_context():
    """Rewinding a surrogate context (write_state) empties the network-node
    lists: after 1501 steps (4.5 ms, action potentials repolarising) the list
    of step 1500's parity is full of network nodes; restoring the state of
    step 1000 at step 1000 (the same parity) and stepping on gives the same
    bits as a fresh context started from that state."""
    w = W.small_ragged(seed=34, n_fibers=30, lo=300, hi=1200, n_steps=1600)
    w.mu_offsets = np.arange(5, dtype=np.int64)           # one firing per motor unit
    w.fire_times = np.array([0.0, 0.05, 0.1, 0.15])
    blob = S.load_blob()
    with F.Fibers.from_workload(w, mode=F.FIB_MODE_SURROGATE) as f:
        F.fibers_load_surrogate(f.ctx, blob)
        f.step(1000)
        st = f.read_state()
        _, fb0 = f.stats()
        f.step(501)                 # steps 1000..1500: the last one (even) lists nodes
        _, fb1 = f.stats()
        f.write_state(st, 1000)     # rewind to step 1000 (even)
        f.step(40)
        got = f.read_state()
    with F.Fibers.from_workload(w, mode=F.FIB_MODE_SURROGATE) as g:
        F.fibers_load_surrogate(g.ctx, blob)
        g.write_state(st, 1000)
        g.step(40)
        ref = g.read_state()
    assert fb1 - fb0 < 501 * w.total_nodes  # the network handled nodes before the rewind
    assert np.array_equal(got, ref)


def test_surrogate_gain_over_the_plain_method_at_matched_accuracy():
    """What the trained network gains over the method without it: both paths
    meet the stated tolerances against the FP64 oracle on held-out fibers
    (seed 4 of the 7744-fiber bundle, 20 ms), and both are timed on the
    full 7744-fiber bundle from the same state 4 ms into the run (action
    potentials propagating).  The gain is node-updates/s of the surrogate
    path over the plain FP32 path at that matched accuracy; on GB300 it is
    below 1 (the network's 35 kFLOP and 256 SiLU per node cost more than the
    plain step's 42 special-function and ~240 FP32 operations), and the test
    reports it rather than asserting a speed-up."""
    blob = S.load_blob()
    full = W.bundle_7744(seed=4, t_end_ms=20.0)
    firing = [f for f in range(full.n_fibers)
              if full.mu_offsets[full.mu_of_fiber[f] + 1] > full.mu_offsets[full.mu_of_fiber[f]]]
    w = full.subset(np.sort(np.random.default_rng(4).choice(firing, 16, replace=False)))
    cps = list(range(10, w.n_steps + 1, 10))
    o = oracle_checkpoints(w, cps)
    dt = 10 * w.params["dt_split"]
    from parity import activation_times
    to = activation_times(o, dt)
    acc = {}
    for name, mode in (("plain", F.FIB_MODE_FP32), ("surrogate", F.FIB_MODE_SURROGATE)):
        out = []
        with F.Fibers.from_workload(w, mode=mode) as f:
            if mode == F.FIB_MODE_SURROGATE:
                F.fibers_load_surrogate(f.ctx, blob)
            done = 0
            for c in cps:
                f.step(c - done)
                done = c
                out.append(f.read_vm().astype(np.float64))
        out = np.array(out)
        mx, rel = errors(out, o)
        ts = activation_times(out, dt)
        both = ~np.isnan(to) & ~np.isnan(ts)
        acc[name] = (mx, rel, float(np.max(np.abs(to[both] - ts[both]))))
        assert mx <= MAX_ABS_MV and rel <= REL_L2 and acc[name][2] <= ACT_TIME_MS, (name, acc[name])
    # throughput on the whole bundle from the same mid-run state
    b = W.bundle_7744(seed=2, t_end_ms=20.0)
    stream = torch.cuda.Stream()
    settle, steps = 1334, 300
    with F.Fibers.from_workload(b, stream=stream, tuning=dict(graph_steps=100)) as f:
        f.step(settle)
        state = f.read_state()
    rates = {}
    for name, mode in (("plain", F.FIB_MODE_FP32), ("surrogate", F.FIB_MODE_SURROGATE)):
        with F.Fibers.from_workload(b, stream=stream, mode=mode, tuning=dict(graph_steps=100)) as f:
            if mode == F.FIB_MODE_SURROGATE:
                F.fibers_load_surrogate(f.ctx, blob)
            f.write_state(state, settle)
            f.step(100)
            f.synchronize()
            _, fb0 = f.stats()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            f.step(steps)
            e1.record(stream)
            e1.synchronize()
            _, fb1 = f.stats()
            rates[name] = b.total_nodes * steps / (e0.elapsed_time(e1) * 1e-3)
            if mode == F.FIB_MODE_SURROGATE:
                share = 1.0 - (fb1 - fb0) / (b.total_nodes * steps)
            assert np.isfinite(f.read_vm()).all()
    gain = rates["surrogate"] / rates["plain"]
    print(f"[surrogate gain] plain FP32 {rates['plain']:.3e} node-updates/s (max|dV| {acc['plain'][0]:.3f} mV), "
          f"surrogate {rates['surrogate']:.3e} (max|dV| {acc['surrogate'][0]:.3f} mV, network share "
          f"{share:.4f}): gain {gain:.3f}")
    assert 0.0 < share < 1.0
    assert gain > 0.0
