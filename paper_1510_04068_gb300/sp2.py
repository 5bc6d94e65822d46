"""Thin Python binding of the C ABI in include/sapporo_gb.h.

Functions carry the C names (sp2_open, sp2_set_j, sp2_predict, sp2_compute,
...) and only marshal arguments: torch CUDA tensors are passed as device
pointers (SP2_DEVICE, asynchronous on the context's stream), numpy arrays and
CPU tensors as host pointers (SP2_HOST, synchronous).  Every computation runs
in libsapporo_gb.so; if the library cannot be loaded, every call raises.
``Context`` is a small convenience wrapper over the same calls.
"""
from __future__ import annotations

import ctypes
from ctypes import POINTER, Structure, byref, c_char_p, c_double, c_int, c_int32, c_int64, c_size_t, c_void_p
from pathlib import Path

import numpy as np

SP2_OK = 0
SP2_FP64, SP2_MIXED = 0, 1
SP2_HOST, SP2_DEVICE = 0, 1
STATUS = {0: "SP2_OK", -1: "SP2_ERR_ARG", -2: "SP2_ERR_RANGE", -3: "SP2_ERR_NOMEM", -4: "SP2_ERR_CUDA",
          -5: "SP2_ERR_STATE", -6: "SP2_ERR_TIMEOUT", -7: "SP2_ERR_NONFINITE", -8: "SP2_ERR_UNSUPPORTED"}
(SP2_ERR_ARG, SP2_ERR_RANGE, SP2_ERR_NOMEM, SP2_ERR_CUDA, SP2_ERR_STATE, SP2_ERR_TIMEOUT, SP2_ERR_NONFINITE,
 SP2_ERR_UNSUPPORTED) = range(-1, -9, -1)
STAGES = ("predict", "force", "reduce", "batched", "vjp", "other")

ALLOC_FN = ctypes.CFUNCTYPE(c_void_p, c_size_t, c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, c_void_p, c_void_p)


class sp2_config(Structure):
    _fields_ = [("order", c_int), ("precision", c_int), ("n_max", c_int64), ("eps2", c_double),
                ("with_nn", c_int), ("cuda_stream", c_void_p), ("alloc", ALLOC_FN), ("free", FREE_FN),
                ("alloc_user", c_void_p), ("profile", c_int), ("check_finite", c_int)]


class sp2_launch(Structure):
    _fields_ = [("threads", c_int), ("i_per_thread", c_int), ("j_lanes", c_int), ("j_tile", c_int),
                ("split_j", c_int), ("ctas_per_sm", c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class SP2Error(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


LIB_PATH = Path(__file__).resolve().parent / "_build" / "libsapporo_gb.so"
_lib = None

# (name, argtypes, restype)
_P = c_void_p
_SIGS = [
    ("sp2_config_default", [POINTER(sp2_config)], None),
    ("sp2_open", [POINTER(_P), POINTER(sp2_config)], c_int),
    ("sp2_close", [_P], c_int),
    ("sp2_set_j", [_P, c_int64, c_int64, _P, _P, _P, _P, _P, _P, _P, _P, _P, c_int], c_int),
    ("sp2_predict", [_P, c_double], c_int),
    ("sp2_compute", [_P, c_int64, _P, _P, _P, _P, _P, _P, _P, c_int], c_int),
    ("sp2_compute_range", [_P, c_int64, c_int64, c_int64, _P, _P, _P, _P, _P, _P, _P, c_int], c_int),
    ("sp2_compute_nb", [_P, c_int64, _P, _P, _P, _P, _P, _P, _P, _P, c_int32, _P, _P, c_int], c_int),
    ("sp2_compute_ext", [_P, c_int64, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, c_int], c_int),
    ("sp2_get_j", [_P, c_int64, c_int64, _P, _P, _P, _P, _P, c_int], c_int),
    ("sp2_block_init", [_P, c_double, c_double, c_double], c_int),
    ("sp2_block_run", [_P, c_double, c_double, c_double, _P], c_int),
    ("sp2_block_run_h6", [_P, c_double, c_double, c_double, c_double, _P], c_int),
    ("sp2_batch_plan_create", [_P, c_int64, _P, POINTER(_P)], c_int),
    ("sp2_batch_plan_destroy", [_P], c_int),
    ("sp2_compute_batched", [_P, _P, _P, _P, _P, _P, _P, _P, c_int], c_int),
    ("sp2_forces", [_P, c_int64, _P, _P, _P, _P, _P, _P, c_int], c_int),
    ("sp2_force_vjp", [_P, c_int64, _P, _P, _P, _P, _P, _P, _P, _P, _P, c_int, c_int], c_int),
    ("sp2_hermite4_step", [_P, c_int64, c_double, _P, _P, _P, _P, _P], c_int),
    ("sp2_hermite4_step_vjp", [_P, c_int64, c_double, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P], c_int),
    ("sp2_autotune", [_P, c_int64, POINTER(sp2_launch)], c_int),
    ("sp2_get_launch", [_P, c_int64, POINTER(sp2_launch)], c_int),
    ("sp2_set_launch", [_P, c_int64, POINTER(sp2_launch)], c_int),
    ("sp2_graph_begin", [_P], c_int),
    ("sp2_graph_end", [_P, POINTER(_P)], c_int),
    ("sp2_graph_launch", [_P, _P], c_int),
    ("sp2_graph_destroy", [_P], c_int),
    ("sp2_sync", [_P], c_int),
    ("sp2_profile_reset", [_P], c_int),
    ("sp2_profile_read", [_P, POINTER(c_int64), POINTER(c_double), c_int], c_int),
    ("sp2_kernel_launches", [_P], c_int64),
    ("sp2_measure_pipe_peaks", [_P], c_int),
    ("sp2_info", [_P, POINTER(c_int64), POINTER(c_int64), POINTER(c_int)], c_int),
    ("sp2_step_static", [c_int64, _P, _P, _P, _P, _P, _P, _P, c_double, c_double, c_int64, _P, _P, _P, _P, _P, _P,
                         _P], c_int),
    ("sp2_strerror", [c_int], c_char_p),
    ("sp2_last_error", [_P, c_char_p, c_size_t], c_int),
]
EXPORTED = [s[0] for s in _SIGS]


def load(path: str | Path | None = None):
    """Load libsapporo_gb.so (raises if it is missing: there is no fallback)."""
    global _lib
    if _lib is None or path is not None:
        p = Path(path) if path else LIB_PATH
        if not p.exists():
            raise RuntimeError(f"{p} is not built; run __graft_entry__.build() or paper_1510_04068_gb300.build")
        lib = ctypes.CDLL(str(p))
        for name, args, res in _SIGS:
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = res
        _lib = lib
    return _lib


def _check(status: int, ctx=None):
    if status != SP2_OK:
        msg = ""
        if ctx:
            buf = ctypes.create_string_buffer(512)
            _lib.sp2_last_error(ctx, buf, 512)
            msg = buf.value.decode()
        raise SP2Error(status, msg or (_lib.sp2_strerror(status) or b"").decode())


def _is_torch(a):
    return type(a).__module__.startswith("torch")


def _marshal(arrays, dtypes):
    """Pointers and ptr_kind for a call; all non-None arrays must live together."""
    kinds, ptrs, keep = set(), [], []
    for a, dt in zip(arrays, dtypes):
        if a is None:
            ptrs.append(None)
            continue
        if _is_torch(a):
            import torch
            want = {np.float64: torch.float64, np.int32: torch.int32, np.int64: torch.int64}[dt]
            if a.dtype != want or not a.is_contiguous():
                raise TypeError(f"tensor must be contiguous {want}, got {a.dtype}")
            kinds.add(SP2_DEVICE if a.is_cuda else SP2_HOST)
            ptrs.append(a.data_ptr())
        else:
            if not isinstance(a, np.ndarray) or a.dtype != dt or not a.flags.c_contiguous:
                raise TypeError(f"array must be a C-contiguous numpy {np.dtype(dt).name} array")
            kinds.add(SP2_HOST)
            ptrs.append(a.ctypes.data)
        keep.append(a)
    if len(kinds) > 1:
        raise TypeError("mixing host and device arrays in one call")
    return ptrs, (kinds.pop() if kinds else SP2_HOST), keep


F8, I4, I8 = np.float64, np.int32, np.int64


def sp2_open(order=4, precision=SP2_MIXED, n_max=1, eps2=0.0, with_nn=1, cuda_stream=None,
             profile=0, check_finite=0, alloc=None, free=None):
    """Open a context on the current device; cuda_stream None = torch's current stream."""
    lib = load()
    cfg = sp2_config()
    lib.sp2_config_default(byref(cfg))
    cfg.order, cfg.precision, cfg.n_max, cfg.eps2 = order, precision, n_max, eps2
    cfg.with_nn, cfg.profile, cfg.check_finite = with_nn, profile, check_finite
    if cuda_stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                cuda_stream = torch.cuda.current_stream().cuda_stream
        except Exception:  # pragma: no cover - torch without CUDA
            cuda_stream = None
    cfg.cuda_stream = cuda_stream or None
    if alloc is not None:
        cfg.alloc, cfg.free = alloc, free
    ctx = c_void_p()
    st = lib.sp2_open(byref(ctx), byref(cfg))
    _check(st)
    return ctx


def sp2_close(ctx):
    _check(load().sp2_close(ctx))


def sp2_set_j(ctx, first, id, m, x, v, a, jerk, snap, t, slots=None):
    n = len(id)
    (ps, pid, pm, px, pv, pa, pj, psn, pt), kind, _k = _marshal(
        [slots, id, m, x, v, a, jerk, snap, t], [I4, I4, F8, F8, F8, F8, F8, F8, F8])
    _check(load().sp2_set_j(ctx, first, n, ps, pid, pm, px, pv, pa, pj, psn, pt, kind), ctx)


def sp2_predict(ctx, t):
    _check(load().sp2_predict(ctx, float(t)), ctx)


def sp2_compute(ctx, i_idx, acc=None, jerk=None, snap=None, pot=None, nn_id=None, nn_r2=None, j_range=None):
    ptrs, kind, _k = _marshal([i_idx, acc, jerk, snap, pot, nn_id, nn_r2], [I4, F8, F8, F8, F8, I4, F8])
    if j_range is None:
        _check(load().sp2_compute(ctx, len(i_idx), *ptrs, kind), ctx)
    else:
        _check(load().sp2_compute_range(ctx, int(j_range[0]), int(j_range[1]), len(i_idx), *ptrs, kind), ctx)


def sp2_compute_nb(ctx, i_idx, h2, nb_max, nb_count, nb_ids, acc=None, jerk=None, snap=None, pot=None, nn_id=None,
                   nn_r2=None):
    """Forces plus neighbour lists: nb_count[k] neighbours of sink k within
    sqrt(h2[k]); nb_ids[k, :min(nb_count[k], nb_max)] their ids, ascending."""
    ptrs, kind, _k = _marshal([i_idx, acc, jerk, snap, pot, nn_id, nn_r2, h2, nb_count, nb_ids],
                              [I4, F8, F8, F8, F8, I4, F8, F8, I4, I4])
    pi, pa, pj, ps, pp, pid, pr2, ph2, pcnt, pids = ptrs
    _check(load().sp2_compute_nb(ctx, len(i_idx), pi, pa, pj, ps, pp, pid, pr2, ph2, int(nb_max), pcnt, pids, kind),
           ctx)


def sp2_compute_ext(ctx, xi, vi=None, ai=None, i_slot=None, acc=None, jerk=None, snap=None, pot=None, nn_id=None,
                    nn_r2=None):
    """Forces on explicit sinks (positions xi [n_i x 3], velocities vi, order-6
    accelerations ai); i_slot[k] >= 0 names the loaded slot that is sink k."""
    ptrs, kind, _k = _marshal([i_slot, xi, vi, ai, acc, jerk, snap, pot, nn_id, nn_r2],
                              [I4, F8, F8, F8, F8, F8, F8, F8, I4, F8])
    _check(load().sp2_compute_ext(ctx, len(xi), *ptrs, kind), ctx)


class sp2_pipe_peaks(Structure):
    _fields_ = [("fp32_fma_lane_ops", c_double), ("fp32x2_fma_lane_ops", c_double), ("fp64_fma_ops", c_double),
                ("rsqrt_ops", c_double)]


def measure_pipe_peaks():
    """Measured pipe rates of the current device (operations per second)."""
    pk = sp2_pipe_peaks()
    _check(load().sp2_measure_pipe_peaks(byref(pk)))
    return {name: getattr(pk, name) for name, _ in pk._fields_}


class sp2_block_stats(Structure):
    _fields_ = [("block_steps", c_int64), ("active_sum", c_int64), ("max_active", c_int64), ("min_active", c_int64),
                ("t", c_double)]


def sp2_get_j(ctx, first, n, x=None, v=None, a=None, jerk=None, t=None):
    ptrs, kind, _k = _marshal([x, v, a, jerk, t], [F8, F8, F8, F8, F8])
    _check(load().sp2_get_j(ctx, int(first), int(n), *ptrs, kind), ctx)


def sp2_block_init(ctx, t0, eta_s, dt_max):
    _check(load().sp2_block_init(ctx, float(t0), float(eta_s), float(dt_max)), ctx)


def sp2_block_run(ctx, t_end, eta, dt_max):
    """Advance with block time-steps to t_end; returns the statistics as a dict."""
    st = sp2_block_stats()
    _check(load().sp2_block_run(ctx, float(t_end), float(eta), float(dt_max), byref(st)), ctx)
    return {name: getattr(st, name) for name, _ in st._fields_}


def sp2_block_run_h6(ctx, t_end, eta4, eta6, dt_max):
    """6th-order block time-steps to t_end (averaged criterion); statistics as a dict."""
    st = sp2_block_stats()
    status = load().sp2_block_run_h6(ctx, float(t_end), float(eta4), float(eta6), float(dt_max), byref(st))
    stats = {name: getattr(st, name) for name, _ in st._fields_}
    try:
        _check(status, ctx)
    except SP2Error as e:  # a stopped run (step underflow) still reports how far it got
        e.stats = stats
        raise
    return stats


def sp2_batch_plan_create(ctx, offsets):
    off = np.ascontiguousarray(offsets, dtype=np.int64)
    plan = c_void_p()
    _check(load().sp2_batch_plan_create(ctx, len(off) - 1, off.ctypes.data, byref(plan)), ctx)
    return plan


def sp2_batch_plan_destroy(plan):
    _check(load().sp2_batch_plan_destroy(plan))


def sp2_compute_batched(ctx, plan, acc=None, jerk=None, snap=None, pot=None, nn_id=None, nn_r2=None):
    ptrs, kind, _k = _marshal([acc, jerk, snap, pot, nn_id, nn_r2], [F8, F8, F8, F8, I4, F8])
    _check(load().sp2_compute_batched(ctx, plan, *ptrs, kind), ctx)


def sp2_forces(ctx, m, x, v, acc=None, jerk=None, pot=None):
    ptrs, kind, _k = _marshal([m, x, v, acc, jerk, pot], [F8] * 6)
    _check(load().sp2_forces(ctx, len(m), *ptrs, kind), ctx)


def sp2_force_vjp(ctx, m, x, v, abar, jbar, pbar, xbar, vbar, mbar, accumulate=False):
    ptrs, kind, _k = _marshal([m, x, v, abar, jbar, pbar, xbar, vbar, mbar], [F8] * 9)
    _check(load().sp2_force_vjp(ctx, len(m), *ptrs, int(bool(accumulate)), kind), ctx)


def sp2_hermite4_step(ctx, dt, m, x, v, a, jerk):
    ptrs, kind, _k = _marshal([m, x, v, a, jerk], [F8] * 5)
    if kind != SP2_DEVICE:
        raise TypeError("sp2_hermite4_step takes device tensors")
    _check(load().sp2_hermite4_step(ctx, len(m), float(dt), *ptrs), ctx)


def sp2_hermite4_step_vjp(ctx, dt, m, x, v, a, jerk, gx, gv, ga, gj, gm):
    ptrs, kind, _k = _marshal([m, x, v, a, jerk, gx, gv, ga, gj, gm], [F8] * 10)
    if kind != SP2_DEVICE:
        raise TypeError("sp2_hermite4_step_vjp takes device tensors")
    _check(load().sp2_hermite4_step_vjp(ctx, len(m), float(dt), *ptrs), ctx)


def sp2_autotune(ctx, n_i):
    L = sp2_launch()
    _check(load().sp2_autotune(ctx, int(n_i), byref(L)), ctx)
    return L.as_dict()


def sp2_get_launch(ctx, n_i):
    L = sp2_launch()
    _check(load().sp2_get_launch(ctx, int(n_i), byref(L)), ctx)
    return L.as_dict()


def sp2_set_launch(ctx, n_i, launch: dict):
    L = sp2_launch(**launch)
    _check(load().sp2_set_launch(ctx, int(n_i), byref(L)), ctx)


def sp2_graph_begin(ctx):
    _check(load().sp2_graph_begin(ctx), ctx)


def sp2_graph_end(ctx):
    g = c_void_p()
    _check(load().sp2_graph_end(ctx, byref(g)), ctx)
    return g


def sp2_graph_launch(ctx, graph):
    _check(load().sp2_graph_launch(ctx, graph), ctx)


def sp2_graph_destroy(graph):
    _check(load().sp2_graph_destroy(graph))


def sp2_sync(ctx):
    _check(load().sp2_sync(ctx), ctx)


def sp2_profile_reset(ctx):
    _check(load().sp2_profile_reset(ctx), ctx)


def sp2_profile_read(ctx):
    """{stage: (launches, summed ms)} since the last reset (needs profile=1)."""
    cnt = (c_int64 * len(STAGES))()
    tot = (c_double * len(STAGES))()
    _check(load().sp2_profile_read(ctx, cnt, tot, len(STAGES)), ctx)
    return {STAGES[k]: (int(cnt[k]), float(tot[k])) for k in range(len(STAGES))}


def sp2_step_static(inputs, t, eps2, i_idx, out, cuda_stream=None):
    """Allocation-free mixed Hermite-4 block step on device tensors.

    inputs = [id, m, x, v, a, jerk, t_j] of the sources; out = dict with acc,
    jerk, pot and optionally nn_id, nn_r2.  All work is enqueued on cuda_stream
    (None: the legacy default stream); the library's fixed scratch array is
    shared by every call, so calls must not overlap on the GPU."""
    ids = inputs[0]
    ptrs, kind, _k = _marshal(list(inputs) + [i_idx, out.get("acc"), out.get("jerk"), out.get("pot"),
                                                out.get("nn_id"), out.get("nn_r2")],
                              [I4, F8, F8, F8, F8, F8, F8, I4, F8, F8, F8, I4, F8])
    if kind != SP2_DEVICE:
        raise TypeError("sp2_step_static takes device tensors")
    st = load().sp2_step_static(len(ids), *ptrs[:7], float(t), float(eps2), len(i_idx), *ptrs[7:], cuda_stream)
    _check(st)


def sp2_kernel_launches(ctx) -> int:
    return int(load().sp2_kernel_launches(ctx))


def sp2_info(ctx):
    nl, nm, sm = c_int64(), c_int64(), c_int()
    _check(load().sp2_info(ctx, byref(nl), byref(nm), byref(sm)), ctx)
    return {"n_loaded": nl.value, "n_max": nm.value, "sm_count": sm.value}


class Context:
    """Owning wrapper: ``with Context(order=4, n_max=N, eps2=e) as c: ...``."""

    def __init__(self, **cfg):
        self.order = cfg.get("order", 4)
        self.precision = cfg.get("precision", SP2_MIXED)
        self.ctx = sp2_open(**cfg)

    def close(self):
        if self.ctx:
            sp2_close(self.ctx)
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

    def set_j(self, *a, **k): return sp2_set_j(self.ctx, *a, **k)
    def predict(self, t): return sp2_predict(self.ctx, t)
    def compute(self, *a, **k): return sp2_compute(self.ctx, *a, **k)
    def compute_nb(self, *a, **k): return sp2_compute_nb(self.ctx, *a, **k)
    def compute_ext(self, *a, **k): return sp2_compute_ext(self.ctx, *a, **k)
    def get_j(self, *a, **k): return sp2_get_j(self.ctx, *a, **k)
    def block_init(self, *a): return sp2_block_init(self.ctx, *a)
    def block_run(self, *a): return sp2_block_run(self.ctx, *a)
    def block_run_h6(self, *a): return sp2_block_run_h6(self.ctx, *a)
    def batch_plan(self, offsets): return sp2_batch_plan_create(self.ctx, offsets)
    def compute_batched(self, *a, **k): return sp2_compute_batched(self.ctx, *a, **k)
    def forces(self, *a, **k): return sp2_forces(self.ctx, *a, **k)
    def force_vjp(self, *a, **k): return sp2_force_vjp(self.ctx, *a, **k)
    def hermite4_step(self, *a): return sp2_hermite4_step(self.ctx, *a)
    def hermite4_step_vjp(self, *a): return sp2_hermite4_step_vjp(self.ctx, *a)
    def autotune(self, n_i): return sp2_autotune(self.ctx, n_i)
    def get_launch(self, n_i): return sp2_get_launch(self.ctx, n_i)
    def set_launch(self, n_i, L): return sp2_set_launch(self.ctx, n_i, L)
    def sync(self): return sp2_sync(self.ctx)
    def profile_reset(self): return sp2_profile_reset(self.ctx)
    def profile_read(self): return sp2_profile_read(self.ctx)
    def kernel_launches(self): return sp2_kernel_launches(self.ctx)
    def info(self): return sp2_info(self.ctx)
