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


def test_read_vm_static_reports_a_non_finite_state():
    w = W.small_ragged(seed=23, n_fibers=6, lo=10, hi=300, n_steps=4)
    with F.Fibers.from_workload(w) as f:
        st = f.read_state()
        st[5] = np.nan
        f.write_state(st, 0)
        f.step(1)
        out = np.empty(w.total_nodes, np.float32)
        with pytest.raises(F.FibersError) as ei:
            F.read_vm_static(f.ctx, out)
        assert ei.value.status == F.FIB_ENONFINITE


_LAZY_CHILD = r'''
import sys
import numpy as np
import torch
sys.path.insert(0, sys.argv[1])
from paper_2107_07104_gb300 import fibers as F
from paper_2107_07104_gb300 import workloads as W
torch.cuda.init()
w = W.small_ragged(seed=24, n_fibers=20, lo=100, hi=900, n_steps=50)
with F.Fibers.from_workload(w) as f:
    f.step(50)
    f.synchronize()
    dev0 = torch.cuda.current_device()
    free0, _ = torch.cuda.mem_get_info()
    out = np.empty(w.total_nodes, np.float32)
    F.read_vm_static(f.ctx, out)
    free1, _ = torch.cuda.mem_get_info()
    assert torch.cuda.current_device() == dev0
    assert np.array_equal(out, f.read_vm()), "read_vm_static differs from read_vm"
    print("FREE", free0, free1)
'''


def test_read_vm_static_first_call_reserves_nothing_under_lazy_loading(tmp_path):
    """With lazy module loading, the staging array is reserved when a context
    is created, not by the first read_vm_static call: free device memory is
    the same before and after that call."""
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    script = tmp_path / "lazy_child.py"
    script.write_text(_LAZY_CHILD)
    env = dict(os.environ, CUDA_MODULE_LOADING="LAZY")
    r = subprocess.run([sys.executable, str(script), root], env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout + r.stderr
    line = [x for x in r.stdout.splitlines() if x.startswith("FREE")][-1]
    free0, free1 = (int(v) for v in line.split()[1:])
    assert free1 == free0, f"first read_vm_static call changed free device memory by {free0 - free1} bytes"
