"""The C-ABI library builds for sm_103a, loads, exports every symbol that
include/fibers.h declares, and rejects bad arguments on the host before it
touches the GPU (no compute calls: these run without a GPU)."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

from paper_2107_07104_gb300 import build as B
from paper_2107_07104_gb300 import fibers as F
from paper_2107_07104_gb300 import workloads as W

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "fibers.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*([A-Za-z_][A-Za-z0-9_]*)\s*\(", src, flags=re.M)
    return sorted(set(n for n in names if n not in ("if", "while")))


@pytest.fixture(scope="module")
def lib():
    B.build()
    return F.load()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("fibers_create", "set_stimulus_times", "step", "read_vm", "fibers_destroy", "fibers_last_error"):
        assert required in names
    assert sorted(F.EXPORTED) == names


def test_library_exports_every_declared_symbol(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", B.LIB], capture_output=True, text=True, check=True).stdout
    exported = set(line.split()[-1] for line in out.splitlines() if line.strip())
    for name in declared_functions():
        assert name in exported, name
        assert hasattr(lib, name)


def _create(**over):
    w = W.small_ragged(1, 3, 5, 9, 10)
    p = dict(w.params)
    kw = dict(params=p, n_nodes=w.n_nodes, mu_of_fiber=w.mu_of_fiber, junction_node=w.junction)
    for k, v in over.items():
        if k in p:
            p[k] = v
        else:
            kw[k] = v
    return F.fibers_create(**kw)


@pytest.mark.parametrize("over, text", [
    (dict(dt_0d=0.0007), "whole numbers"),
    (dict(dt_1d=0.001), "whole numbers"),
    (dict(h=0.0), "must be > 0"),
    (dict(Cm=-1.0), "must be > 0"),
    (dict(gL=0.0), "needs gL > 0"),
    (dict(stim_half_width=-1), "stim_half_width"),
    (dict(n_nodes=[5, 0, 7]), "nodes"),
    (dict(junction_node=[0, 9, 1]), "junction"),
    (dict(mu_of_fiber=[0, -2, 1]), "motor unit"),
    (dict(splitting=4), "unknown splitting"),
    (dict(diffusion=2), "unknown diffusion"),
    (dict(splitting=2), "even number"),                    # 3 Heun substeps cannot be halved
    (dict(splitting=1, dt_1d=0.002), "whole numbers"),     # Godunov diffuses over the whole dt_split
    (dict(splitting=3, mode=F.FIB_MODE_SURROGATE), "surrogate mode runs only"),
    (dict(diffusion=1, mode=F.FIB_MODE_SURROGATE), "surrogate mode runs only"),
    (dict(exp_approx=1, mode=F.FIB_MODE_FP64_THOMAS), "FIB_MODE_FP32 only"),
    (dict(exp_approx=1, mode=F.FIB_MODE_SURROGATE), "FIB_MODE_FP32 only"),
])
def test_create_rejects_bad_arguments_on_the_host(lib, over, text):
    with pytest.raises(F.FibersError) as ei:
        _create(**over)
    assert ei.value.status == F.FIB_EINVAL
    assert text in str(ei.value)


def test_create_rejects_non_finite_initial_voltage(lib):
    w = W.small_ragged(1, 2, 5, 6, 10)
    vm0 = np.full(w.total_nodes, -75.0, np.float32)
    vm0[3] = np.nan
    with pytest.raises(F.FibersError) as ei:
        F.fibers_create(w.params, w.n_nodes, w.mu_of_fiber, w.junction, vm0)
    assert ei.value.status == F.FIB_EINVAL


def test_unknown_mode_is_rejected(lib):
    w = W.small_ragged(1, 2, 5, 6, 10)
    with pytest.raises(F.FibersError) as ei:
        F.fibers_create(w.params, w.n_nodes, w.mu_of_fiber, w.junction, mode=3)
    assert ei.value.status == F.FIB_EINVAL


def test_null_context_is_safe(lib):
    lib.fibers_destroy(None)
    assert lib.fibers_kernel_launches(None) == 0
    assert lib.step(None, 1) == F.FIB_EINVAL
    assert lib.fibers_synchronize(None) == F.FIB_EINVAL


def test_rest_state_matches_the_oracle_rest_gates(lib):
    # host-only call: the library's resting gates (the offsets of the state's
    # gate blocks) are the steady-state gates of the HH rates at Vrest
    import oracle
    p = dict(W.DEFAULT_PARAMS)
    r = F.fibers_rest_state(p)
    assert r[0] == np.float32(p["Vrest"])
    g = oracle.gates_inf(p, p["Vrest"])
    assert np.allclose(r[1:].astype(np.float64), g, rtol=1.2e-7, atol=0.0)
    pa = dict(p, exp_approx=1)
    ra = F.fibers_rest_state(pa)
    ga = oracle.gates_inf(dict(pa), pa["Vrest"])
    assert np.allclose(ra[1:].astype(np.float64), ga, rtol=1.2e-7, atol=0.0)
    with pytest.raises(F.FibersError):
        F.fibers_rest_state(dict(p, dt_split=-1.0))
