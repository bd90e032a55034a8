"""FP64 CPU oracle for the fiber monodomain split step -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path (the CUDA library and
its binding) never imports it, and it imports nothing from the product.

The arithmetic lives in ``fiber_oracle.c`` (plain C, FP64, libm, no fast-math);
this module compiles it with the host C compiler on first use and wraps it with
ctypes.  Every entry point follows a passage of Maier 2021, cited in the C file.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from typing import Optional, Tuple

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fiber_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liborc.so")
_lock = threading.Lock()
_lib = None


class OrcParams(ctypes.Structure):
    _fields_ = [(k, ctypes.c_double) for k in
                ("Cm", "gNa", "gK", "gL", "ENa", "EK", "EL", "Vrest", "sigma_eff", "Am", "h",
                 "dt_split", "dt_0d", "dt_1d", "stim_amplitude", "stim_duration")] + \
               [("stim_half_width", ctypes.c_int32), ("splitting", ctypes.c_int32), ("diffusion", ctypes.c_int32),
                ("exp_approx", ctypes.c_int32)]


def build(force: bool = False) -> str:
    """Compile the oracle into oracle/_build/liborc.so (idempotent)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        cc = os.environ.get("CC", "cc")
        subprocess.check_call([cc, "-O2", "-std=c11", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm", "-lpthread"])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            P = ctypes.POINTER
            d, i32, i64 = ctypes.c_double, ctypes.c_int32, ctypes.c_int64
            pd = P(d)
            L.orc_hh_rates.argtypes = [P(OrcParams), d, pd]
            L.orc_exp_star.argtypes = [d]
            L.orc_exp_star.restype = d
            L.orc_gates_inf.argtypes = [P(OrcParams), d, pd]
            L.orc_leak_reversal_exact.argtypes = [P(OrcParams)]
            L.orc_leak_reversal_exact.restype = d
            L.orc_hh_rhs.argtypes = [P(OrcParams), d, pd, d, pd]
            L.orc_heun_step.argtypes = [P(OrcParams), d, pd, d, d]
            L.orc_thomas.argtypes = [ctypes.c_int, pd, pd, pd, pd, pd, pd]
            L.orc_thomas.restype = ctypes.c_int
            L.orc_cn_system.argtypes = [P(OrcParams), ctypes.c_int, d, pd, pd, pd, pd, pd]
            L.orc_cn_system.restype = ctypes.c_int
            L.orc_cn_step.argtypes = [P(OrcParams), ctypes.c_int, d, pd, pd]
            L.orc_cn_step.restype = ctypes.c_int
            L.orc_ie_step.argtypes = [P(OrcParams), ctypes.c_int, d, pd, pd]
            L.orc_ie_step.restype = ctypes.c_int
            L.orc_init_state.argtypes = [P(OrcParams), i64, P(ctypes.c_float), pd]
            L.orc_init_state.restype = ctypes.c_int
            L.orc_run_fibers.argtypes = [P(OrcParams), i32, P(i32), P(i32), P(i32), i32, P(i64), pd, pd,
                                         i64, i64, i64, pd, i32]
            L.orc_run_fibers.restype = ctypes.c_int
            _lib = L
    return _lib


def params(p: dict) -> OrcParams:
    o = OrcParams()
    for k in ("Cm", "gNa", "gK", "gL", "ENa", "EK", "EL", "Vrest", "sigma_eff", "Am", "h",
              "dt_split", "dt_0d", "dt_1d", "stim_amplitude", "stim_duration"):
        setattr(o, k, float(p[k]))
    o.stim_half_width = int(p.get("stim_half_width", 1))
    o.splitting = int(p.get("splitting", 0))
    o.diffusion = int(p.get("diffusion", 0))
    o.exp_approx = int(p.get("exp_approx", 0))
    return o


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _ip(a: np.ndarray, t):
    return a.ctypes.data_as(ctypes.POINTER(t))


def hh_rates(p: dict, V: float) -> np.ndarray:
    out = np.zeros(6)
    lib().orc_hh_rates(ctypes.byref(params(p)), float(V), _dp(out))
    return out


def exp_star(x: float) -> float:
    return float(lib().orc_exp_star(float(x)))


def gates_inf(p: dict, V: float) -> np.ndarray:
    out = np.zeros(3)
    lib().orc_gates_inf(ctypes.byref(params(p)), float(V), _dp(out))
    return out


def leak_reversal_exact(p: dict) -> float:
    return float(lib().orc_leak_reversal_exact(ctypes.byref(params(p))))


def leak_reversal(p: dict) -> float:
    return leak_reversal_exact(p) if np.isnan(p["EL"]) else float(p["EL"])


def hh_rhs(p: dict, y, istim: float = 0.0) -> np.ndarray:
    y = np.ascontiguousarray(y, dtype=np.float64)
    dy = np.zeros(4)
    lib().orc_hh_rhs(ctypes.byref(params(p)), leak_reversal(p), _dp(y), float(istim), _dp(dy))
    return dy


def heun_step(p: dict, y, dt: float, istim: float = 0.0) -> np.ndarray:
    y = np.array(y, dtype=np.float64)
    lib().orc_heun_step(ctypes.byref(params(p)), leak_reversal(p), _dp(y), float(istim), float(dt))
    return y


def thomas(a, b, c, d) -> np.ndarray:
    a, b, c, d = (np.ascontiguousarray(v, dtype=np.float64) for v in (a, b, c, d))
    n = b.shape[0]
    x = np.zeros(n)
    w = np.zeros(max(n, 1))
    if lib().orc_thomas(n, _dp(a), _dp(b), _dp(c), _dp(d), _dp(x), _dp(w)) != 0:
        raise ZeroDivisionError("zero pivot")
    return x


def cn_system(p: dict, V, dt: float) -> Tuple[np.ndarray, np.ndarray, np.ndarray, np.ndarray]:
    V = np.ascontiguousarray(V, dtype=np.float64)
    n = V.shape[0]
    a, b, c, d = (np.zeros(n) for _ in range(4))
    if lib().orc_cn_system(ctypes.byref(params(p)), n, float(dt), _dp(V), _dp(a), _dp(b), _dp(c), _dp(d)):
        raise ValueError("bad CN system")
    return a, b, c, d


def cn_step(p: dict, V, dt: float) -> np.ndarray:
    V = np.array(V, dtype=np.float64)
    n = V.shape[0]
    work = np.zeros(5 * n)
    if lib().orc_cn_step(ctypes.byref(params(p)), n, float(dt), _dp(V), _dp(work)):
        raise ValueError("CN step failed")
    return V


def ie_step(p: dict, V, dt: float) -> np.ndarray:
    V = np.array(V, dtype=np.float64)
    n = V.shape[0]
    work = np.zeros(5 * n)
    if lib().orc_ie_step(ctypes.byref(params(p)), n, float(dt), _dp(V), _dp(work)):
        raise ValueError("implicit Euler step failed")
    return V


def init_state(p: dict, total: int, vm0: Optional[np.ndarray]) -> np.ndarray:
    st = np.zeros(4 * total)
    v = None
    if vm0 is not None:
        v = np.ascontiguousarray(vm0, dtype=np.float32)
    lib().orc_init_state(ctypes.byref(params(p)), int(total),
                         None if v is None else v.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), _dp(st))
    return st


def run(p: dict, n_nodes, mu_of_fiber, junction, mu_offsets, fire_times, state: np.ndarray,
        step0: int, n_steps: int, sample_every: int = 0, n_threads: Optional[int] = None) -> Optional[np.ndarray]:
    """Advance ``state`` (4*total doubles, ragged V|m|h|n, in place) by n_steps split steps.

    Returns the V samples (rows of ``total``) taken every ``sample_every`` steps, or None.
    """
    n_nodes = np.ascontiguousarray(n_nodes, dtype=np.int32)
    mu = np.ascontiguousarray(mu_of_fiber, dtype=np.int32)
    junc = np.ascontiguousarray(junction, dtype=np.int32)
    offs = np.ascontiguousarray(mu_offsets, dtype=np.int64)
    fire = np.ascontiguousarray(fire_times, dtype=np.float64)
    if fire.shape[0] == 0:
        fire = np.zeros(1)
    total = int(n_nodes.astype(np.int64).sum())
    assert state.dtype == np.float64 and state.flags.c_contiguous and state.shape[0] == 4 * total
    samples = None
    if sample_every and sample_every > 0:
        samples = np.zeros((n_steps // sample_every, total))
    if n_threads is None:
        n_threads = len(os.sched_getaffinity(0))
    st = lib().orc_run_fibers(ctypes.byref(params(p)), n_nodes.shape[0], _ip(n_nodes, ctypes.c_int32),
                              _ip(mu, ctypes.c_int32), _ip(junc, ctypes.c_int32), offs.shape[0] - 1,
                              _ip(offs, ctypes.c_int64), _dp(fire), _dp(state), int(step0), int(n_steps),
                              int(sample_every), None if samples is None else _dp(samples), int(n_threads))
    if st != 0:
        raise ValueError(f"oracle run failed with status {st}")
    return samples


def run_workload(w, n_steps: Optional[int] = None, sample_every: int = 0, state: Optional[np.ndarray] = None,
                 step0: int = 0, n_threads: Optional[int] = None):
    """Convenience: run a workloads.Workload from its initial state (or ``state``)."""
    if state is None:
        state = init_state(w.params, w.total_nodes, w.vm0)
    samples = run(w.params, w.n_nodes, w.mu_of_fiber, w.junction, w.mu_offsets, w.fire_times, state, step0,
                  w.n_steps if n_steps is None else n_steps, sample_every, n_threads)
    return state, samples
