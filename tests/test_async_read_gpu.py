"""read_vm_async / read_vm_wait: double-buffered readback of V that overlaps
the steps enqueued after it, bit for bit equal to read_vm at the same step."""
import numpy as np
import pytest

from paper_2107_07104_gb300 import fibers as F
from paper_2107_07104_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _sync_reads(w, chunks):
    out = []
    with F.Fibers.from_workload(w) as f:
        for n in chunks:
            f.step(n)
            out.append(f.read_vm())
    return out


@pytest.mark.parametrize("pinned", [False, True])
def test_reads_in_flight_equal_synchronous_reads(pinned):
    import torch
    w = W.small_ragged(seed=81, n_fibers=30, lo=200, hi=1481, n_steps=600)
    chunks = [40, 60, 1, 100, 75, 124]             # more reads in flight than staging buffers
    ref = _sync_reads(w, chunks)
    if pinned:
        bufs = [torch.empty(w.total_nodes, dtype=torch.float32, pin_memory=True) for _ in chunks]
    else:
        bufs = [np.empty(w.total_nodes, np.float32) for _ in chunks]
    with F.Fibers.from_workload(w) as f:
        tickets = []
        for n, b in zip(chunks, bufs):
            f.step(n)
            tickets.append(f.read_vm_async(b))
        assert tickets == list(range(len(chunks)))
        for t in reversed(tickets):                 # any order
            f.read_vm_wait(t)
        for b, r in zip(bufs, ref):
            got = b.numpy() if pinned else b
            assert np.array_equal(got, r)
        # a synchronous read after them still agrees
        f.step(10)
        v = f.read_vm()
    assert np.array_equal(v, _sync_reads(w, chunks + [10])[-1])


def test_wait_returns_while_later_steps_run():
    """The wait covers the read, not the steps enqueued after it: with about
    50 ms of steps queued behind a read of 46 MB, the wait returns long
    before they finish."""
    import time
    import torch
    w = W.bundle_7744(seed=2, t_end_ms=1.0)
    buf = torch.empty(w.total_nodes, dtype=torch.float32, pin_memory=True)
    with F.Fibers.from_workload(w, tuning=dict(graph_steps=0)) as f:
        f.step(10)
        f.synchronize()
        t = f.read_vm_async(buf)
        f.step(500)
        t0 = time.perf_counter()
        f.read_vm_wait(t)
        t1 = time.perf_counter()
        f.synchronize()
        t2 = time.perf_counter()
        ref = np.empty(w.total_nodes, np.float32)
    with F.Fibers.from_workload(w) as g:
        g.step(10)
        g.read_vm(ref)
    print(f"[async read] wait {1e3 * (t1 - t0):.2f} ms, rest of the steps {1e3 * (t2 - t1):.2f} ms")
    assert np.array_equal(buf.numpy(), ref)
    assert (t1 - t0) < 0.5 * (t2 - t0)


def test_errors_and_non_finite_state():
    w = W.single_fiber(t_end_ms=1.0, n_nodes=64)
    with F.Fibers.from_workload(w) as f:
        with pytest.raises(F.FibersError) as ei:
            f.read_vm_wait(0)                        # nothing issued
        assert ei.value.status == F.FIB_EINVAL
        with pytest.raises(F.FibersError) as ei:
            f.read_vm_async(np.empty(10, np.float32))
        assert ei.value.status == F.FIB_EINVAL
    w.params["stim_amplitude"] = 1e38
    with F.Fibers.from_workload(w) as f:
        f.step(50)
        out = np.empty(w.total_nodes, np.float32)
        t = f.read_vm_async(out)
        with pytest.raises(F.FibersError) as ei:
            f.read_vm_wait(t)
        assert ei.value.status == F.FIB_ENONFINITE


def test_empty_context():
    w = W.small_ragged(1, 1, 5, 5, 10)
    with F.Fibers(w.params, np.zeros(0, np.int32), np.zeros(0, np.int32), np.zeros(0, np.int32),
                  np.array([0], np.int64), []) as f:
        f.step(5)
        t = f.read_vm_async(np.empty(0, np.float32))
        f.read_vm_wait(t)
