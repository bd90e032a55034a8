"""read_vm_static: the read entry point for callers that cannot allocate
device memory (for example because another allocator has reserved the whole
GPU) must return exactly what read_vm returns, call after call.

This file is collected last so that a run stopping at the first failure has
already run every other test."""
import numpy as np
import pytest

from paper_2107_07104_gb300 import fibers as F
from paper_2107_07104_gb300 import workloads as W

from parity import MAX_ABS_MV

pytestmark = pytest.mark.gpu


def test_read_vm_static_matches_read_vm_on_consecutive_calls():
    w = W.small_ragged(seed=21, n_fibers=40, lo=1, hi=900, n_steps=400)
    with F.Fibers.from_workload(w) as f:
        for _ in range(2):
            f.step(200)
            ref = f.read_vm()
            got = np.full(w.total_nodes, np.nan, np.float32)
            F.read_vm_static(f.ctx, got)
            assert np.max(np.abs(got.astype(np.float64) - ref)) <= MAX_ABS_MV
            assert np.array_equal(got, ref)


def test_read_vm_static_rejects_contexts_above_its_limit():
    n = 1500  # 1500 x 1481 = 2,221,500 nodes > 2,097,152
    w = W.small_ragged(seed=22, n_fibers=n, lo=1481, hi=1481, n_steps=1)
    with F.Fibers.from_workload(w) as f:
        out = np.empty(w.total_nodes, np.float32)
        with pytest.raises(F.FibersError) as ei:
            F.read_vm_static(f.ctx, out)
        assert ei.value.status == F.FIB_EINVAL
        assert "2097152" in str(ei.value)
