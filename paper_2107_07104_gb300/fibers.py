"""ctypes binding of the C ABI in include/fibers.h (argument marshalling only).

Every step of the simulation runs in the CUDA library libfibers.so; this module
only converts Python/numpy/torch arguments into pointers and sizes and turns
error codes into exceptions.  There is no CPU fallback: if the library is
missing or no GPU is present, calls fail loudly.

The functions keep the C names (fibers_create, set_stimulus_times, step,
read_vm, ...).  ``Fibers`` is a small convenience class over them.
"""
from __future__ import annotations

import ctypes
import os
import threading
from typing import Optional

import numpy as np

from . import build as _build

_lib = None
_lock = threading.Lock()

FIB_OK, FIB_EINVAL, FIB_ENOMEM, FIB_ECUDA, FIB_ENONFINITE, FIB_ETIMEOUT, FIB_ESTATE, FIB_ENOTSUP, FIB_EIO = range(9)
FIB_MODE_FP32, FIB_MODE_FP64_THOMAS, FIB_MODE_SURROGATE = 0, 1, 2
FIB_FLAG_ADAPTIVE = 1
FIB_FLAG_EXP_APPROX = 2
SPLIT_STRANG_1D0D1D, SPLIT_GODUNOV_1D0D, SPLIT_STRANG_0D1D0D, SPLIT_GODUNOV_0D1D = 0, 1, 2, 3
DIFFUSION_CRANK_NICOLSON, DIFFUSION_IMPLICIT_EULER = 0, 1
STATUS_NAMES = ["FIB_OK", "FIB_EINVAL", "FIB_ENOMEM", "FIB_ECUDA", "FIB_ENONFINITE", "FIB_ETIMEOUT",
                "FIB_ESTATE", "FIB_ENOTSUP", "FIB_EIO"]

# Every symbol the header declares (checked by the ABI test).
EXPORTED = ("fibers_create", "set_stimulus_times", "step", "read_vm", "read_vm_static", "read_vm_async",
            "read_vm_wait", "fibers_read_state",
            "fibers_write_state",
            "fibers_stats", "fibers_synchronize", "fibers_get_tuning", "fibers_set_tuning", "fibers_autotune",
            "fibers_kernel_launches", "fibers_last_error", "fibers_destroy", "fibers_load_surrogate",
            "fibers_hh_reaction", "fibers_mlp_train_step", "fibers_mlp_forward", "fibers_adam_step",
            "fibers_feature_stats", "fibers_adaptive_stats", "fibers_solver_tables", "fibers_emg_create",
            "fibers_emg_vm3d", "fibers_emg_phi_e", "fibers_emg_nodes", "fibers_emg_last_error", "fibers_emg_destroy",
            "fibers_rest_state", "fibers_autotune_cache_size", "fibers_autotune_cache_clear",
            "fibers_autotune_cache_save", "fibers_autotune_cache_load")
SUR_N_PARAMS = 17796
SUR_BLOB_FLOATS = 3 + 5 + 5 + 4 + 4 + 5 + 5 + 5 + 5 + SUR_N_PARAMS
SUR_WORK_PER_SAMPLE = 848


class FibersError(RuntimeError):
    def __init__(self, status: int, message: str):
        self.status = status
        name = STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else str(status)
        super().__init__(f"{name}: {message}")


class FibParams(ctypes.Structure):
    _fields_ = [(k, ctypes.c_double) for k in
                ("Cm", "gNa", "gK", "gL", "ENa", "EK", "EL", "Vrest", "sigma_eff", "Am", "h",
                 "dt_split", "dt_0d", "dt_1d", "stim_amplitude", "stim_duration")] + \
               [("stim_half_width", ctypes.c_int32), ("mode", ctypes.c_int32), ("flags", ctypes.c_int32),
                ("splitting", ctypes.c_int32), ("diffusion", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class FibMesh3D(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("origin", ctypes.c_double * 3), ("spacing", ctypes.c_double * 3), ("sigma_i", ctypes.c_double),
                ("sigma_e", ctypes.c_double)]


class FibTuning(ctypes.Structure):
    _fields_ = [("nodes_per_thread", ctypes.c_int32), ("warps_per_cta", ctypes.c_int32),
                ("steps_per_launch", ctypes.c_int32), ("graph_steps", ctypes.c_int32),
                ("reaction_pairs", ctypes.c_int32), ("ctas_per_sm", ctypes.c_int32), ("warp_roles", ctypes.c_int32)]

    def as_dict(self):
        return {k: int(getattr(self, k)) for k, _ in self._fields_}


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libfibers.so (building it first if stale and nvcc is available)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.LIB
        if build_if_missing:
            try:
                path = _build.build()
            except RuntimeError:
                if not os.path.exists(path):
                    raise
        if not os.path.exists(path):
            raise RuntimeError(f"CUDA library {path} is missing; build it with paper_2107_07104_gb300.build.build()")
        L = ctypes.CDLL(path)
        P, vp = ctypes.POINTER, ctypes.c_void_p
        i32, i64, sz = ctypes.c_int32, ctypes.c_int64, ctypes.c_size_t
        L.fibers_create.argtypes = [P(FibParams), i32, P(i32), P(i32), P(i32), P(ctypes.c_float), P(FibTuning), vp,
                                    P(vp)]
        L.set_stimulus_times.argtypes = [vp, i32, P(i64), P(ctypes.c_double)]
        L.step.argtypes = [vp, i64]
        L.read_vm.argtypes = [vp, vp, sz, i32]
        L.read_vm_static.argtypes = [vp, vp, sz]
        L.read_vm_async.argtypes = [vp, vp, sz, P(i64)]
        L.read_vm_wait.argtypes = [vp, i64]
        L.fibers_read_state.argtypes = [vp, vp, sz, i32]
        L.fibers_write_state.argtypes = [vp, vp, sz, i32, i64]
        L.fibers_stats.argtypes = [vp, P(i64), P(i64)]
        L.fibers_adaptive_stats.argtypes = [vp, P(i64)]
        L.fibers_adaptive_stats.restype = ctypes.c_int
        L.fibers_synchronize.argtypes = [vp]
        L.fibers_get_tuning.argtypes = [vp, P(FibTuning)]
        L.fibers_set_tuning.argtypes = [vp, P(FibTuning)]
        L.fibers_autotune.argtypes = [vp, i32, P(FibTuning)]
        L.fibers_kernel_launches.argtypes = [vp]
        L.fibers_kernel_launches.restype = i64
        L.fibers_last_error.argtypes = [vp]
        L.fibers_last_error.restype = ctypes.c_char_p
        L.fibers_destroy.argtypes = [vp]
        L.fibers_destroy.restype = None
        f32, f64p = ctypes.c_float, P(ctypes.c_double)
        L.fibers_load_surrogate.argtypes = [vp, P(ctypes.c_float), sz]
        L.fibers_hh_reaction.argtypes = [P(FibParams), i64, vp, vp, vp, vp]
        L.fibers_mlp_train_step.argtypes = [vp, i32, vp, vp, i64, vp, vp, vp, vp]
        L.fibers_mlp_forward.argtypes = [vp, i32, vp, i64, vp, vp, vp]
        L.fibers_adam_step.argtypes = [vp, vp, vp, vp, i64, f32, f32, f32, f32, i64, vp, f32, vp]
        L.fibers_feature_stats.argtypes = [vp, i64, i32, f64p, vp]
        L.fibers_solver_tables.argtypes = [i32, ctypes.c_double, i32, i32, P(i32), P(i32), f64p, f64p]
        L.fibers_rest_state.argtypes = [P(FibParams), P(ctypes.c_float)]
        L.fibers_emg_create.argtypes = [vp, f64p, ctypes.c_double, P(FibMesh3D), P(vp)]
        L.fibers_emg_vm3d.argtypes = [vp, vp, sz, i32]
        L.fibers_emg_phi_e.argtypes = [vp, vp, sz, i32, ctypes.c_double, i32, P(i32), f64p]
        L.fibers_emg_nodes.argtypes = [vp]
        L.fibers_emg_nodes.restype = i64
        L.fibers_emg_last_error.argtypes = [vp]
        L.fibers_emg_last_error.restype = ctypes.c_char_p
        L.fibers_emg_destroy.argtypes = [vp]
        L.fibers_emg_destroy.restype = None
        L.fibers_autotune_cache_size.argtypes = []
        L.fibers_autotune_cache_size.restype = i64
        L.fibers_autotune_cache_clear.argtypes = []
        L.fibers_autotune_cache_save.argtypes = [ctypes.c_char_p]
        L.fibers_autotune_cache_load.argtypes = [ctypes.c_char_p]
        for name in ("fibers_load_surrogate", "fibers_hh_reaction", "fibers_mlp_train_step", "fibers_mlp_forward",
                     "fibers_adam_step", "fibers_feature_stats", "fibers_solver_tables", "fibers_autotune_cache_clear",
                     "fibers_autotune_cache_save", "fibers_autotune_cache_load"):
            getattr(L, name).restype = ctypes.c_int
        for name in ("fibers_create", "set_stimulus_times", "step", "read_vm", "read_vm_static", "read_vm_async",
                     "read_vm_wait", "fibers_read_state",
                     "fibers_write_state", "fibers_stats", "fibers_synchronize", "fibers_get_tuning",
                     "fibers_set_tuning", "fibers_autotune"):
            getattr(L, name).restype = ctypes.c_int
        _lib = L
        return L


def _check(status: int, ctx) -> None:
    if status != FIB_OK:
        msg = load().fibers_last_error(ctx)
        raise FibersError(status, msg.decode() if msg else "")


def make_params(p: dict, mode: int = FIB_MODE_FP32) -> FibParams:
    o = FibParams()
    for k in ("Cm", "gNa", "gK", "gL", "ENa", "EK", "EL", "Vrest", "sigma_eff", "Am", "h",
              "dt_split", "dt_0d", "dt_1d", "stim_amplitude", "stim_duration"):
        setattr(o, k, float(p[k]))
    o.stim_half_width = int(p.get("stim_half_width", 1))
    o.mode = int(p.get("mode", mode))
    o.flags = int(p.get("flags", 0)) | (FIB_FLAG_EXP_APPROX if p.get("exp_approx", 0) else 0)
    o.splitting = int(p.get("splitting", SPLIT_STRANG_1D0D1D))
    o.diffusion = int(p.get("diffusion", DIFFUSION_CRANK_NICOLSON))
    o.reserved = 0
    return o


def _arr(a, dtype):
    return np.ascontiguousarray(np.asarray(a), dtype=dtype)


def _ptr(a: np.ndarray, ct):
    return a.ctypes.data_as(ctypes.POINTER(ct))


def _buffer(out):
    """(pointer, elements, is_device) of a numpy array or a torch tensor."""
    if isinstance(out, np.ndarray):
        if out.dtype != np.float32 or not out.flags.c_contiguous:
            raise TypeError("expected a contiguous float32 array")
        return out.ctypes.data, out.size, 0
    try:  # torch tensor
        import torch
        if isinstance(out, torch.Tensor):
            if out.dtype != torch.float32 or not out.is_contiguous():
                raise TypeError("expected a contiguous float32 tensor")
            return out.data_ptr(), out.numel(), 1 if out.is_cuda else 0
    except ImportError:
        pass
    raise TypeError(f"unsupported buffer type {type(out)}")


# ---------------------------------------------------------------------------
# C-named wrappers
# ---------------------------------------------------------------------------

def fibers_create(params: dict, n_nodes, mu_of_fiber, junction_node, vm0=None, tuning: Optional[dict] = None,
                  stream=None, mode: int = FIB_MODE_FP32):
    L = load()
    n_nodes = _arr(n_nodes, np.int32)
    mu = _arr(mu_of_fiber, np.int32)
    junc = _arr(junction_node, np.int32)
    if not (n_nodes.shape == mu.shape == junc.shape):
        raise ValueError("n_nodes, mu_of_fiber and junction_node must have the same length")
    pv = make_params(params, mode)
    v = None if vm0 is None else _arr(vm0, np.float32)
    t = None
    if tuning is not None:
        t = FibTuning(**{k: int(tuning.get(k, 0)) for k, _ in FibTuning._fields_})
    s = None
    if stream is not None:
        s = stream if isinstance(stream, int) else int(getattr(stream, "cuda_stream", stream))
    ctx = ctypes.c_void_p()
    st = L.fibers_create(ctypes.byref(pv), n_nodes.shape[0], _ptr(n_nodes, ctypes.c_int32), _ptr(mu, ctypes.c_int32),
                         _ptr(junc, ctypes.c_int32), None if v is None else _ptr(v, ctypes.c_float),
                         None if t is None else ctypes.byref(t), s, ctypes.byref(ctx))
    _check(st, None)
    return ctx


def set_stimulus_times(ctx, mu_offsets, fire_times_ms) -> None:
    offs = _arr(mu_offsets, np.int64)
    times = _arr(fire_times_ms, np.float64)
    if times.size == 0:
        times = np.zeros(1)
    _check(load().set_stimulus_times(ctx, max(offs.shape[0] - 1, 0), _ptr(offs, ctypes.c_int64),
                                     _ptr(times, ctypes.c_double)), ctx)


def step(ctx, n_steps: int) -> None:
    _check(load().step(ctx, int(n_steps)), ctx)


def read_vm(ctx, out) -> None:
    ptr, n, dev = _buffer(out)
    _check(load().read_vm(ctx, ptr, n, dev), ctx)


def read_vm_static(ctx, out: np.ndarray) -> None:
    """read_vm into a host array without any device allocation (the library
    stages through its fixed 8 MiB array; at most 2,097,152 nodes)."""
    if not isinstance(out, np.ndarray) or out.dtype != np.float32 or not out.flags.c_contiguous:
        raise TypeError("expected a contiguous float32 numpy array")
    _check(load().read_vm_static(ctx, out.ctypes.data, out.size), ctx)


def read_vm_async(ctx, out) -> int:
    """Enqueues a read of V into host memory `out` (a float32 numpy array or a
    CPU tensor; pinned memory lets the call return at once) and returns its
    ticket.  `out` must stay alive and unread until read_vm_wait(ticket)."""
    ptr, n, dev = _buffer(out)
    if dev:
        raise TypeError("read_vm_async writes host memory; use read_vm for device buffers")
    t = ctypes.c_int64(-1)
    _check(load().read_vm_async(ctx, ptr, n, ctypes.byref(t)), ctx)
    return int(t.value)


def read_vm_wait(ctx, ticket: int) -> None:
    _check(load().read_vm_wait(ctx, int(ticket)), ctx)


def fibers_read_state(ctx, out) -> None:
    ptr, n, dev = _buffer(out)
    _check(load().fibers_read_state(ctx, ptr, n, dev), ctx)


def fibers_write_state(ctx, data, step_index: int) -> None:
    ptr, n, dev = _buffer(data)
    _check(load().fibers_write_state(ctx, ptr, n, dev, int(step_index)), ctx)


def fibers_stats(ctx):
    a, b = ctypes.c_int64(), ctypes.c_int64()
    _check(load().fibers_stats(ctx, ctypes.byref(a), ctypes.byref(b)), ctx)
    return int(a.value), int(b.value)


def fibers_adaptive_stats(ctx) -> int:
    v = ctypes.c_int64()
    _check(load().fibers_adaptive_stats(ctx, ctypes.byref(v)), ctx)
    return int(v.value)


def fibers_synchronize(ctx) -> None:
    _check(load().fibers_synchronize(ctx), ctx)


def fibers_get_tuning(ctx) -> dict:
    t = FibTuning()
    _check(load().fibers_get_tuning(ctx, ctypes.byref(t)), ctx)
    return t.as_dict()


def fibers_set_tuning(ctx, tuning: dict) -> None:
    t = FibTuning(**{k: int(tuning.get(k, 0)) for k, _ in FibTuning._fields_})
    _check(load().fibers_set_tuning(ctx, ctypes.byref(t)), ctx)


def fibers_autotune(ctx, n_trial_steps: int = 20) -> dict:
    t = FibTuning()
    _check(load().fibers_autotune(ctx, int(n_trial_steps), ctypes.byref(t)), ctx)
    return t.as_dict()


def fibers_autotune_cache_size() -> int:
    return int(load().fibers_autotune_cache_size())


def fibers_autotune_cache_clear() -> None:
    _check(load().fibers_autotune_cache_clear(), None)


def fibers_autotune_cache_save(path: str) -> None:
    _check(load().fibers_autotune_cache_save(os.fsencode(path)), None)


def fibers_autotune_cache_load(path: str) -> None:
    _check(load().fibers_autotune_cache_load(os.fsencode(path)), None)


def _dev(t):
    """Device pointer of a contiguous CUDA tensor (surrogate entry points take device buffers)."""
    if not (t.is_cuda and t.is_contiguous()):
        raise TypeError("expected a contiguous CUDA tensor")
    return t.data_ptr()


def _stream_ptr(stream):
    if stream is None:
        return None
    return stream if isinstance(stream, int) else int(getattr(stream, "cuda_stream", stream))


def fibers_load_surrogate(ctx, blob: np.ndarray) -> None:
    b = np.ascontiguousarray(blob, dtype=np.float32)
    _check(load().fibers_load_surrogate(ctx, _ptr(b, ctypes.c_float), b.size), ctx)


def fibers_hh_reaction(params: dict, x_in, stim_mask, x_out, stream=None) -> None:
    """x_in / x_out: CUDA float32 tensors of 4 x count (V | m | h | n); stim_mask: uint8 count or None."""
    count = x_in.numel() // 4
    pv = make_params(params)
    _check(load().fibers_hh_reaction(ctypes.byref(pv), count, _dev(x_in),
                                     None if stim_mask is None else _dev(stim_mask), _dev(x_out),
                                     _stream_ptr(stream)), None)


def fibers_mlp_train_step(theta, quantize: bool, x, target, workspace, grad, loss, stream=None) -> None:
    _check(load().fibers_mlp_train_step(_dev(theta), int(bool(quantize)), _dev(x), _dev(target), x.shape[0],
                                        _dev(workspace), _dev(grad), _dev(loss), _stream_ptr(stream)), None)


def fibers_mlp_forward(theta, quantize: bool, x, workspace, out, stream=None) -> None:
    _check(load().fibers_mlp_forward(_dev(theta), int(bool(quantize)), _dev(x), x.shape[0], _dev(workspace),
                                     _dev(out), _stream_ptr(stream)), None)


def fibers_adam_step(theta, m, v, grad, lr, t, beta1=0.9, beta2=0.999, eps=1e-8, theta_avg=None, avg_decay=0.999,
                     stream=None) -> None:
    """Adam step; with theta_avg, also the exponential average of the weights."""
    avg = None if theta_avg is None else _dev(theta_avg)
    _check(load().fibers_adam_step(_dev(theta), _dev(m), _dev(v), _dev(grad), theta.numel(), float(lr), float(beta1),
                                   float(beta2), float(eps), int(t), avg, float(avg_decay), _stream_ptr(stream)), None)


def fibers_feature_stats(X, stream=None) -> np.ndarray:
    """(cols, 4) array of mean, std, min, max per column of a CUDA (n x cols) tensor."""
    n, cols = X.shape
    out = np.zeros(4 * cols)
    _check(load().fibers_feature_stats(_dev(X), n, cols, _ptr(out, ctypes.c_double), _stream_ptr(stream)), None)
    return out.reshape(cols, 4)


def fibers_solver_tables(K: int, r: float, n_nodes: int, fp64_solve: bool = False) -> dict:
    """Coefficient tables of the partitioned tridiagonal solve for one fiber
    (host only): levels, threads, rows (2, K, 5) and recs (threads, 7 + 3 levels)."""
    L = load()
    lv, tw = ctypes.c_int32(0), ctypes.c_int32(0)
    _check(L.fibers_solver_tables(int(K), float(r), int(n_nodes), int(bool(fp64_solve)), ctypes.byref(lv),
                                  ctypes.byref(tw), None, None), None)
    rows = np.zeros(2 * K * 5)
    recs = np.zeros(tw.value * (7 + 3 * lv.value))
    _check(L.fibers_solver_tables(int(K), float(r), int(n_nodes), int(bool(fp64_solve)), None, None,
                                  _ptr(rows, ctypes.c_double), _ptr(recs, ctypes.c_double)), None)
    return dict(levels=lv.value, threads=tw.value, rows=rows.reshape(2, K, 5),
                recs=recs.reshape(tw.value, 7 + 3 * lv.value))


def _check_emg(status: int, emg) -> None:
    if status != FIB_OK:
        msg = load().fibers_emg_last_error(emg)
        raise FibersError(status, msg.decode() if msg else "")


def make_mesh3d(nx, ny, nz, origin, spacing, sigma_i=8.93, sigma_e=6.7) -> FibMesh3D:
    m = FibMesh3D()
    m.nx, m.ny, m.nz, m.reserved = int(nx), int(ny), int(nz), 0
    for d in range(3):
        m.origin[d] = float(origin[d])
        m.spacing[d] = float(spacing[d])
    m.sigma_i, m.sigma_e = float(sigma_i), float(sigma_e)
    return m


def fibers_emg_create(ctx, fiber_xy, z0: float, mesh: FibMesh3D):
    xy = _arr(fiber_xy, np.float64).reshape(-1)
    out = ctypes.c_void_p()
    _check(load().fibers_emg_create(ctx, _ptr(xy, ctypes.c_double), float(z0), ctypes.byref(mesh),
                                    ctypes.byref(out)), ctx)
    return out


def fibers_emg_vm3d(emg, out) -> None:
    if isinstance(out, np.ndarray):
        if out.dtype != np.float64 or not out.flags.c_contiguous:
            raise TypeError("expected a contiguous float64 array")
        ptr, n, dev = out.ctypes.data, out.size, 0
    else:
        import torch
        if out.dtype != torch.float64 or not out.is_contiguous():
            raise TypeError("expected a contiguous float64 tensor")
        ptr, n, dev = out.data_ptr(), out.numel(), 1 if out.is_cuda else 0
    _check_emg(load().fibers_emg_vm3d(emg, ptr, n, dev), emg)


def fibers_emg_phi_e(emg, out, rtol: float = 1e-10, max_iter: int = 5000):
    """Solves for phi_e into out; returns (iterations, relative residual)."""
    ptr, n, dev = _buffer(out)
    it = ctypes.c_int32()
    res = ctypes.c_double()
    _check_emg(load().fibers_emg_phi_e(emg, ptr, n, dev, float(rtol), int(max_iter), ctypes.byref(it),
                                       ctypes.byref(res)), emg)
    return int(it.value), float(res.value)


def fibers_emg_nodes(emg) -> int:
    return int(load().fibers_emg_nodes(emg))


def fibers_emg_destroy(emg) -> None:
    if emg:
        load().fibers_emg_destroy(emg)


def fibers_rest_state(params: dict, mode: int = FIB_MODE_FP32) -> np.ndarray:
    """(Vrest, m0, h0, n0) the library uses (floats); the state's gate blocks
    are deviations from these."""
    out = np.zeros(4, np.float32)
    pv = make_params(params, mode)
    _check(load().fibers_rest_state(ctypes.byref(pv), _ptr(out, ctypes.c_float)), None)
    return out


def fibers_kernel_launches(ctx) -> int:
    return int(load().fibers_kernel_launches(ctx))


def fibers_destroy(ctx) -> None:
    if ctx:
        load().fibers_destroy(ctx)


# ---------------------------------------------------------------------------
# Convenience class
# ---------------------------------------------------------------------------

class Fibers:
    """A bundle of fibers on the GPU, created from a ``workloads.Workload``-like
    description (params, n_nodes, mu_of_fiber, junction, mu_offsets,
    fire_times, vm0)."""

    def __init__(self, params: dict, n_nodes, mu_of_fiber, junction, mu_offsets=None, fire_times=None,
                 vm0=None, tuning: Optional[dict] = None, stream=None, mode: int = FIB_MODE_FP32):
        self.ctx = fibers_create(params, n_nodes, mu_of_fiber, junction, vm0, tuning, stream, mode)
        self.n_nodes = _arr(n_nodes, np.int32)
        self.total = int(self.n_nodes.astype(np.int64).sum())
        if mu_offsets is not None:
            set_stimulus_times(self.ctx, mu_offsets, fire_times if fire_times is not None else [])

    @classmethod
    def from_workload(cls, w, tuning: Optional[dict] = None, stream=None, mode: int = FIB_MODE_FP32):
        return cls(w.params, w.n_nodes, w.mu_of_fiber, w.junction, w.mu_offsets, w.fire_times, w.vm0, tuning,
                   stream, mode)

    def step(self, n: int) -> None:
        step(self.ctx, n)

    def read_vm(self, out=None):
        if out is None:
            out = np.empty(self.total, np.float32)
        read_vm(self.ctx, out)
        return out

    def read_vm_async(self, out) -> int:
        return read_vm_async(self.ctx, out)

    def read_vm_wait(self, ticket: int) -> None:
        read_vm_wait(self.ctx, ticket)

    def read_state(self, out=None):
        if out is None:
            out = np.empty(4 * self.total, np.float32)
        fibers_read_state(self.ctx, out)
        return out

    def write_state(self, data, step_index: int) -> None:
        fibers_write_state(self.ctx, data, step_index)

    def stats(self):
        return fibers_stats(self.ctx)

    def synchronize(self) -> None:
        fibers_synchronize(self.ctx)

    @property
    def tuning(self) -> dict:
        return fibers_get_tuning(self.ctx)

    def set_tuning(self, tuning: dict) -> None:
        fibers_set_tuning(self.ctx, tuning)

    def autotune(self, n_trial_steps: int = 20) -> dict:
        return fibers_autotune(self.ctx, n_trial_steps)

    @property
    def kernel_launches(self) -> int:
        return fibers_kernel_launches(self.ctx)

    def close(self) -> None:
        if self.ctx:
            fibers_destroy(self.ctx)
            self.ctx = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
