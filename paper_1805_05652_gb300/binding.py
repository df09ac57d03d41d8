"""Thin ctypes binding of libfmap (the C ABI in include/fmap.h).

Argument marshalling only: every step of the F-map runs in the library's CUDA
kernels.  Device buffers are torch CUDA tensors passed by ``data_ptr()``;
streams are torch streams passed by their ``cuda_stream`` handle.  There is no
CPU fallback: if ``_lib/libfmap.so`` is missing, every call raises.
"""

from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

from .build import lib_path

c_i32, c_i64, c_u32, c_f32, c_f64 = (ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32,
                                     ctypes.c_float, ctypes.c_double)
c_vp, c_size = ctypes.c_void_p, ctypes.c_size_t

# fmap_status
FMAP_OK, FMAP_PENDING = 0, 1
FMAP_ERR_ARG, FMAP_ERR_NOMEM, FMAP_ERR_CUDA, FMAP_ERR_TIMEOUT = -1, -2, -3, -4
FMAP_ERR_BUSY, FMAP_ERR_DATA, FMAP_ERR_UNSUPPORTED, FMAP_ERR_NONFINITE = -5, -6, -7, -8
# fmap_window / fmap_precision / plan flags
FMAP_RECT, FMAP_EXP, FMAP_TABLE = 0, 1, 2
FMAP_FP64, FMAP_FP32, FMAP_TF32, FMAP_BF16X3 = 0, 1, 2, 3
FMAP_PLAN_PER_TEMPLATE_ANTENNA = 1
FMAP_PLAN_EXP_RECURRENCE = 2
FMAP_PLAN_MAP_BUFFER = 4
FMAP_PLAN_GRAPH = 8
# fmap_summary.flags
FMAP_SUMMARY_REFINED, FMAP_SUMMARY_ARGMAX_EXACT = 1, 2

PRECISIONS = {"fp64": FMAP_FP64, "fp32": FMAP_FP32, "tf32": FMAP_TF32, "bf16x3": FMAP_BF16X3}


class fmap_grid(ctypes.Structure):
    _fields_ = [("t0_min", c_i64), ("dt0", c_i64), ("n_t0", c_i32), ("tau_min", c_i64),
                ("dtau", c_i64), ("n_tau", c_i32), ("t_sft", c_i64), ("window", c_i32),
                ("exp_cut8", c_i32)]


class fmap_atoms(ctypes.Structure):
    _fields_ = [("n_sft", c_i32), ("n_templates", c_i32), ("shared_antenna", c_i32),
                ("t", c_vp), ("antenna", c_vp), ("fafb", c_vp)]


class fmap_summary(ctypes.Structure):
    _fields_ = [("max2F", c_f32), ("m", c_i32), ("n", c_i32), ("flags", c_i32),
                ("logB", c_f64), ("n_valid", c_i64)]


class fmap_batch_item(ctypes.Structure):
    _fields_ = [("grid", fmap_grid), ("atoms", fmap_atoms), ("d_2F", c_vp), ("d_summary", c_vp)]


SUMMARY_DTYPE = np.dtype([("max2F", "<f4"), ("m", "<i4"), ("n", "<i4"), ("flags", "<i4"),
                          ("logB", "<f8"), ("n_valid", "<i8")])
assert SUMMARY_DTYPE.itemsize == ctypes.sizeof(fmap_summary) == 32

EXPORTS = ("fmap_plan", "fmap_plan_destroy", "fmap_workspace_bytes", "fmap_plan_set_log_prior",
           "fmap_compute_rect", "fmap_compute_exp", "fmap_marginalise", "fmap_compute_host",
           "fmap_plan_status", "fmap_count_terms", "fmap_status_string", "fmap_last_error",
           "fmap_plan_enable_timing", "fmap_plan_read_timing", "fmap_marginalise_noalloc",
           "fmap_noalloc_scratch_bytes", "fmap_server_create", "fmap_server_destroy",
           "fmap_submit", "fmap_poll", "fmap_server_stats", "fmap_batch_plan", "fmap_batch_run",
           "fmap_batch_status", "fmap_batch_info", "fmap_batch_profile", "fmap_batch_destroy",
           "fmap_plan_axes", "fmap_plan_count_terms", "fmap_plan_window_table",
           "fmap_compute_table", "fmap_plan_set_refine", "fmap_plan_set_wait_limit",
           "fmap_combine_summaries", "fmap_server_peak")
FMAP_BATCH_AUTOTUNE = 1
N_BATCH_PHASES = 15
FMAP_N_PHASES = 4
FMAP_SUBMIT_MAP = 1
FMAP_SERVER_EXP_FIXED, FMAP_SERVER_EXP_RECURRENCE, FMAP_SERVER_EXP_AUTO = 0, 1, 2
SERVER_EXP_MODES = {"fixed": FMAP_SERVER_EXP_FIXED, "rec": FMAP_SERVER_EXP_RECURRENCE,
                    "auto": FMAP_SERVER_EXP_AUTO}


class fmap_server_config(ctypes.Structure):
    _fields_ = [("device_mem_budget", c_size), ("pinned_bytes", c_size), ("max_inflight", c_i32),
                ("exp_precision", ctypes.c_int), ("rect_precision", ctypes.c_int),
                ("exp_mode", ctypes.c_uint32)]


class FmapError(RuntimeError):
    def __init__(self, status: int, where: str, message: str = ""):
        self.status = status
        super().__init__(f"{where}: {status_string(status)} {message}".strip())


_lib = None


def lib():
    """The loaded libfmap; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    path = lib_path()
    if not os.path.exists(path):
        raise RuntimeError(f"libfmap.so is not built ({path}); run __graft_entry__.build()")
    L = ctypes.CDLL(path)
    P = ctypes.POINTER
    L.fmap_plan.argtypes = [P(c_vp), P(fmap_grid), c_i32, c_i32, ctypes.c_int, c_u32]
    L.fmap_plan_destroy.argtypes = [c_vp]
    L.fmap_plan_destroy.restype = None
    L.fmap_workspace_bytes.argtypes = [P(fmap_grid), c_i32, c_i32, ctypes.c_int]
    L.fmap_workspace_bytes.restype = c_size
    L.fmap_plan_set_log_prior.argtypes = [c_vp, c_f64]
    for f in ("fmap_compute_rect", "fmap_compute_exp", "fmap_compute_table", "fmap_compute_host"):
        getattr(L, f).argtypes = [c_vp, P(fmap_atoms), c_vp, c_vp, c_vp]
    L.fmap_marginalise.argtypes = [c_vp, c_vp, c_vp, c_vp, c_vp]
    L.fmap_plan_status.argtypes = [c_vp]
    L.fmap_count_terms.argtypes = [P(fmap_grid), c_vp, c_i32, P(c_i64), P(c_i64)]
    L.fmap_plan_axes.argtypes = [c_vp, c_vp, c_vp]
    L.fmap_plan_window_table.argtypes = [c_vp, c_vp, c_i32]
    L.fmap_plan_count_terms.argtypes = [c_vp, c_vp, c_i32, P(c_i64), P(c_i64)]
    L.fmap_plan_enable_timing.argtypes = [c_vp, c_i32]
    L.fmap_plan_read_timing.argtypes = [c_vp, c_vp, P(c_i64), P(c_i64)]
    L.fmap_marginalise_noalloc.argtypes = [P(fmap_grid), c_i32, c_vp, c_vp, c_f64, c_vp, c_vp]
    L.fmap_marginalise_noalloc.restype = ctypes.c_int
    L.fmap_noalloc_scratch_bytes.argtypes = []
    L.fmap_noalloc_scratch_bytes.restype = c_size
    L.fmap_server_create.argtypes = [P(c_vp), P(fmap_server_config)]
    L.fmap_server_create.restype = ctypes.c_int
    L.fmap_server_destroy.argtypes = [c_vp]
    L.fmap_server_destroy.restype = None
    L.fmap_submit.argtypes = [c_vp, P(fmap_grid), P(fmap_atoms), c_u32, P(ctypes.c_uint64)]
    L.fmap_submit.restype = ctypes.c_int
    L.fmap_poll.argtypes = [c_vp, ctypes.c_uint64, c_vp, c_vp, c_i64]
    L.fmap_poll.restype = ctypes.c_int
    L.fmap_server_stats.argtypes = [c_vp, P(c_i64), P(c_i64), P(c_i64)]
    L.fmap_server_stats.restype = ctypes.c_int
    L.fmap_server_peak.argtypes = [c_vp, P(c_i64)]
    L.fmap_server_peak.restype = ctypes.c_int
    L.fmap_plan_set_refine.argtypes = [c_vp, c_i32]
    L.fmap_plan_set_wait_limit.argtypes = [c_vp, c_i64]
    L.fmap_combine_summaries.argtypes = [c_vp, c_i32, c_i32, c_vp, c_vp]
    for f in ("fmap_plan_set_refine", "fmap_plan_set_wait_limit", "fmap_combine_summaries"):
        getattr(L, f).restype = ctypes.c_int
    L.fmap_batch_plan.argtypes = [P(c_vp), c_vp, c_i32, c_size, c_u32]
    L.fmap_batch_run.argtypes = [c_vp, c_vp]
    L.fmap_batch_status.argtypes = [c_vp, c_vp]
    L.fmap_batch_info.argtypes = [c_vp, P(c_i32), P(c_i64), P(c_size), c_vp, P(c_i32)]
    L.fmap_batch_profile.argtypes = [c_vp, c_vp, c_vp]
    for f in ("fmap_batch_plan", "fmap_batch_run", "fmap_batch_status", "fmap_batch_info",
              "fmap_batch_profile"):
        getattr(L, f).restype = ctypes.c_int
    L.fmap_batch_destroy.argtypes = [c_vp]
    L.fmap_batch_destroy.restype = None
    L.fmap_status_string.argtypes = [ctypes.c_int]
    L.fmap_status_string.restype = ctypes.c_char_p
    L.fmap_last_error.argtypes = []
    L.fmap_last_error.restype = ctypes.c_char_p
    for f in ("fmap_plan", "fmap_plan_set_log_prior", "fmap_compute_rect", "fmap_compute_exp",
              "fmap_compute_host", "fmap_marginalise", "fmap_plan_status", "fmap_count_terms",
              "fmap_plan_enable_timing", "fmap_plan_read_timing"):
        getattr(L, f).restype = ctypes.c_int
    _lib = L
    return L


def status_string(status: int) -> str:
    return lib().fmap_status_string(int(status)).decode()


def last_error() -> str:
    return lib().fmap_last_error().decode()


def _check(status: int, where: str):
    if status != FMAP_OK:
        raise FmapError(status, where, last_error())


def make_grid(grid) -> fmap_grid:
    """``grid``: an object with t0_min, dt0, n_t0, tau_min, dtau, n_tau, window,
    t_sft attributes, or the tuple (t0_min, dt0, n_t0, tau_min, dtau, n_tau,
    t_sft, window)."""
    if isinstance(grid, fmap_grid):
        return grid
    if isinstance(grid, (tuple, list)):
        t0_min, dt0, n_t0, tau_min, dtau, n_tau, t_sft, window = grid[:8]
        exp_cut8 = grid[8] if len(grid) > 8 else 0
    else:
        t0_min, dt0, n_t0 = grid.t0_min, grid.dt0, grid.n_t0
        tau_min, dtau, n_tau = grid.tau_min, grid.dtau, grid.n_tau
        t_sft, window = grid.t_sft, grid.window
        exp_cut8 = getattr(grid, "exp_cut8", 0)
    return fmap_grid(int(t0_min), int(dt0), int(n_t0), int(tau_min), int(dtau), int(n_tau),
                     int(t_sft), int(window), int(exp_cut8))


def _ptr(x) -> int:
    if x is None:
        return 0
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return int(x.data_ptr())
    if isinstance(x, np.ndarray):
        return int(x.ctypes.data)
    raise TypeError(f"cannot take the address of {type(x)}")


def _stream(stream) -> int:
    if stream is None:
        import torch
        return int(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)


def make_atoms(n_sft, n_templates, shared_antenna, t, antenna, fafb) -> fmap_atoms:
    return fmap_atoms(int(n_sft), int(n_templates), int(bool(shared_antenna)), _ptr(t),
                      _ptr(antenna), _ptr(fafb))


# ---- the C ABI under its own names ----------------------------------------

def fmap_plan(grid, n_sft: int, n_templates: int, precision=FMAP_FP64, flags: int = 0) -> int:
    if isinstance(precision, str):
        precision = PRECISIONS[precision]
    h = c_vp()
    g = make_grid(grid)
    _check(lib().fmap_plan(ctypes.byref(h), ctypes.byref(g), int(n_sft), int(n_templates),
                           int(precision), int(flags)), "fmap_plan")
    return h.value


def fmap_plan_destroy(plan: int):
    if plan:
        lib().fmap_plan_destroy(c_vp(plan))


def fmap_workspace_bytes(grid, n_sft, n_templates, precision=FMAP_FP64) -> int:
    g = make_grid(grid)
    return int(lib().fmap_workspace_bytes(ctypes.byref(g), int(n_sft), int(n_templates),
                                          int(precision)))


def fmap_plan_set_log_prior(plan: int, c: float):
    _check(lib().fmap_plan_set_log_prior(c_vp(plan), float(c)), "fmap_plan_set_log_prior")


def fmap_compute_rect(plan: int, atoms: fmap_atoms, d_2F, d_summary, stream=None):
    _check(lib().fmap_compute_rect(c_vp(plan), ctypes.byref(atoms), _ptr(d_2F), _ptr(d_summary),
                                   _stream(stream)), "fmap_compute_rect")


def fmap_compute_exp(plan: int, atoms: fmap_atoms, d_2F, d_summary, stream=None):
    _check(lib().fmap_compute_exp(c_vp(plan), ctypes.byref(atoms), _ptr(d_2F), _ptr(d_summary),
                                  _stream(stream)), "fmap_compute_exp")


def fmap_compute_table(plan: int, atoms: fmap_atoms, d_2F, d_summary, stream=None):
    _check(lib().fmap_compute_table(c_vp(plan), ctypes.byref(atoms), _ptr(d_2F),
                                    _ptr(d_summary), _stream(stream)), "fmap_compute_table")


def fmap_plan_window_table(handle, w):
    """Samples of a generic window (FMAP_TABLE plans), host float32."""
    a = np.ascontiguousarray(w, dtype=np.float32)
    _check(lib().fmap_plan_window_table(handle, _ptr(a), int(a.shape[0])), "fmap_plan_window_table")


def fmap_compute_host(plan: int, atoms: fmap_atoms, h_2F, h_summary, stream=None):
    _check(lib().fmap_compute_host(c_vp(plan), ctypes.byref(atoms), _ptr(h_2F), _ptr(h_summary),
                                   _stream(stream)), "fmap_compute_host")


def fmap_marginalise(plan: int, d_2F, d_valid, d_summary, stream=None):
    _check(lib().fmap_marginalise(c_vp(plan), _ptr(d_2F), _ptr(d_valid), _ptr(d_summary),
                                  _stream(stream)), "fmap_marginalise")


def fmap_marginalise_noalloc(grid, n_templates: int, d_2F, d_valid, log_prior_const: float,
                             d_summary, stream=None):
    """Marginalisation without a plan or any device allocation (fixed 8 MiB
    library scratch; serialise calls that could overlap on the GPU)."""
    g = make_grid(grid)
    _check(lib().fmap_marginalise_noalloc(ctypes.byref(g), int(n_templates), _ptr(d_2F),
                                          _ptr(d_valid), float(log_prior_const), _ptr(d_summary),
                                          _stream(stream)), "fmap_marginalise_noalloc")


def fmap_noalloc_scratch_bytes() -> int:
    return int(lib().fmap_noalloc_scratch_bytes())


def fmap_plan_status(plan: int) -> int:
    return int(lib().fmap_plan_status(c_vp(plan)))


def fmap_plan_set_refine(plan: int, max_cells: int):
    """FP64 refinement of the cells nearest each template's maximum (0: off,
    < 0: the precision's default)."""
    _check(lib().fmap_plan_set_refine(c_vp(plan), int(max_cells)), "fmap_plan_set_refine")


def fmap_plan_set_wait_limit(plan: int, limit_ns: int):
    """Limit of the plan kernels' bounded waits (ns; < 0: the default 2 s)."""
    _check(lib().fmap_plan_set_wait_limit(c_vp(plan), int(limit_ns)), "fmap_plan_set_wait_limit")


def fmap_combine_summaries(shards, m_offsets) -> np.ndarray:
    """Combine row-shard summaries: ``shards`` [n_shards][T] records
    (SUMMARY_DTYPE), ``m_offsets`` the first global t0 row of each shard."""
    arr = np.ascontiguousarray(np.asarray(shards, dtype=SUMMARY_DTYPE))
    if arr.ndim == 1:
        arr = arr[None]
    n_shards, T = int(arr.shape[0]), int(arr.shape[1]) if arr.ndim == 2 else 0
    offs = np.ascontiguousarray(m_offsets, dtype=np.int32)
    if offs.shape != (n_shards,):
        raise ValueError("one row offset per shard")
    out = np.zeros(T, dtype=SUMMARY_DTYPE)
    _check(lib().fmap_combine_summaries(_ptr(arr), n_shards, T, _ptr(offs), _ptr(out)),
           "fmap_combine_summaries")
    return out


def fmap_plan_enable_timing(plan: int, enable: bool = True):
    _check(lib().fmap_plan_enable_timing(c_vp(plan), int(bool(enable))), "fmap_plan_enable_timing")


def fmap_plan_read_timing(plan: int):
    """(ms per phase [4], timed calls, kernels launched)."""
    ms = np.zeros(FMAP_N_PHASES, dtype=np.float64)
    calls, launches = c_i64(), c_i64()
    _check(lib().fmap_plan_read_timing(c_vp(plan), _ptr(ms), ctypes.byref(calls),
                                       ctypes.byref(launches)), "fmap_plan_read_timing")
    return ms, int(calls.value), int(launches.value)


def fmap_plan_axes(handle, t0_values, tau_values):
    """Explicit (t0, tau) axes for a plan (host int64 arrays), or None, None
    for the uniform grid."""
    if t0_values is None:
        _check(lib().fmap_plan_axes(handle, None, None), "fmap_plan_axes")
        return
    a = np.ascontiguousarray(t0_values, dtype=np.int64)
    b = np.ascontiguousarray(tau_values, dtype=np.int64)
    _check(lib().fmap_plan_axes(handle, _ptr(a), _ptr(b)), "fmap_plan_axes")


def fmap_plan_count_terms(handle, t_host: np.ndarray):
    t = np.ascontiguousarray(t_host, dtype=np.int64)
    a, b = c_i64(), c_i64()
    _check(lib().fmap_plan_count_terms(handle, _ptr(t), int(t.shape[0]), ctypes.byref(a),
                                       ctypes.byref(b)), "fmap_plan_count_terms")
    return int(a.value), int(b.value)


def fmap_count_terms(grid, t_host: np.ndarray):
    g = make_grid(grid)
    t = np.ascontiguousarray(t_host, dtype=np.int64)
    a, b = c_i64(), c_i64()
    _check(lib().fmap_count_terms(ctypes.byref(g), _ptr(t), int(t.shape[0]), ctypes.byref(a),
                                  ctypes.byref(b)), "fmap_count_terms")
    return int(a.value), int(b.value)


def fmap_server_create(device_mem_budget: int, pinned_bytes: int, max_inflight: int,
                       exp_precision=FMAP_BF16X3, rect_precision=FMAP_FP64,
                       exp_mode=FMAP_SERVER_EXP_FIXED) -> int:
    if isinstance(exp_precision, str):
        exp_precision = PRECISIONS[exp_precision]
    if isinstance(rect_precision, str):
        rect_precision = PRECISIONS[rect_precision]
    if isinstance(exp_mode, str):
        exp_mode = SERVER_EXP_MODES[exp_mode]
    cfg = fmap_server_config(int(device_mem_budget), int(pinned_bytes), int(max_inflight),
                             int(exp_precision), int(rect_precision), int(exp_mode))
    h = c_vp()
    _check(lib().fmap_server_create(ctypes.byref(h), ctypes.byref(cfg)), "fmap_server_create")
    return h.value


def fmap_server_destroy(server: int):
    if server:
        lib().fmap_server_destroy(c_vp(server))


def fmap_submit(server: int, grid, atoms: fmap_atoms, flags: int = 0) -> int:
    g = make_grid(grid)
    t = ctypes.c_uint64()
    _check(lib().fmap_submit(c_vp(server), ctypes.byref(g), ctypes.byref(atoms), int(flags),
                             ctypes.byref(t)), "fmap_submit")
    return int(t.value)


def fmap_poll(server: int, ticket: int, h_summary=None, h_2F=None, wait_us: int = -1) -> int:
    """FMAP_OK (results copied) or FMAP_PENDING; raises on a failed request."""
    st = int(lib().fmap_poll(c_vp(server), ctypes.c_uint64(ticket), _ptr(h_summary), _ptr(h_2F),
                             int(wait_us)))
    if st not in (FMAP_OK, FMAP_PENDING):
        raise FmapError(st, "fmap_poll", last_error())
    return st


def fmap_server_stats(server: int):
    q, r, c = c_i64(), c_i64(), c_i64()
    _check(lib().fmap_server_stats(c_vp(server), ctypes.byref(q), ctypes.byref(r),
                                   ctypes.byref(c)), "fmap_server_stats")
    return int(q.value), int(r.value), int(c.value)


def fmap_server_peak(server: int) -> int:
    """Most requests running at once since the server was created."""
    p = c_i64()
    _check(lib().fmap_server_peak(c_vp(server), ctypes.byref(p)), "fmap_server_peak")
    return int(p.value)


def fmap_batch_plan(items, workspace_budget: int = 0, flags: int = 0) -> int:
    """items: sequence of fmap_batch_item (device pointers)."""
    arr = (fmap_batch_item * len(items))(*items)
    h = c_vp()
    _check(lib().fmap_batch_plan(ctypes.byref(h), ctypes.cast(arr, c_vp), len(items),
                                 int(workspace_budget), int(flags)), "fmap_batch_plan")
    return h.value


def fmap_batch_run(batch: int, stream=None):
    _check(lib().fmap_batch_run(c_vp(batch), _stream(stream)), "fmap_batch_run")


def fmap_batch_status(batch: int, stream=None) -> int:
    return int(lib().fmap_batch_status(c_vp(batch), _stream(stream)))


def fmap_batch_info(batch: int):
    w, l, b, t = c_i32(), c_i64(), c_size(), c_i32()
    occ = np.zeros(N_BATCH_PHASES, dtype=np.int32)
    _check(lib().fmap_batch_info(c_vp(batch), ctypes.byref(w), ctypes.byref(l), ctypes.byref(b),
                                 _ptr(occ), ctypes.byref(t)), "fmap_batch_info")
    return dict(waves=int(w.value), launches_per_run=int(l.value), workspace_bytes=int(b.value),
                occupancy=occ.tolist(), rec_templates_per_block=int(t.value))


def fmap_batch_profile(batch: int, stream=None):
    ms = np.zeros(N_BATCH_PHASES, dtype=np.float32)
    _check(lib().fmap_batch_profile(c_vp(batch), _stream(stream), _ptr(ms)), "fmap_batch_profile")
    return ms


BATCH_PHASES = ("prep", "index", "exp_copy", "rect_antenna", "exp_antenna", "rect_coef", "rect_data",
                "exp_recurrence", "rect_cells", "flag_count", "flag_scan", "flag_write", "fixup",
                "reduce_groups", "reduce_final")


def fmap_batch_destroy(batch: int):
    if batch:
        lib().fmap_batch_destroy(c_vp(batch))


class Batch:
    """Owns a batch plan over torch CUDA tensors (kept alive here)."""

    def __init__(self, instances, want_map=True, workspace_budget=0, autotune=True):
        import torch

        self.keep = []
        self.maps, self.sums = [], []
        items = []
        for (grid, t, antenna, fafb) in instances:
            g = make_grid(grid)
            T = int(fafb.shape[0])
            m = (torch.empty((T, g.n_t0, g.n_tau), dtype=torch.float32, device=t.device)
                 if want_map else None)
            s = torch.empty((max(T, 1), 32), dtype=torch.uint8, device=t.device)
            a = make_atoms(int(t.shape[0]), T, antenna.dim() == 2, t, antenna, fafb)
            items.append(fmap_batch_item(g, a, _ptr(m), _ptr(s)))
            self.keep += [t, antenna, fafb]
            self.maps.append(m)
            self.sums.append(s)
        self.handle = fmap_batch_plan(items, workspace_budget,
                                      FMAP_BATCH_AUTOTUNE if autotune else 0)

    def run(self, stream=None):
        fmap_batch_run(self.handle, stream)

    def status(self, stream=None) -> int:
        return fmap_batch_status(self.handle, stream)

    def info(self):
        return fmap_batch_info(self.handle)

    def profile(self, stream=None):
        """Per-phase device milliseconds of one run (summed over waves)."""
        return dict(zip(BATCH_PHASES, fmap_batch_profile(self.handle, stream).tolist()))

    def close(self):
        if getattr(self, "handle", None):
            fmap_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Owns one fmap server; submit() takes host numpy atoms."""

    def __init__(self, device_mem_budget=8 << 30, pinned_bytes=512 << 20, max_inflight=8,
                 exp_precision="bf16x3", rect_precision="fp64", exp_mode="fixed"):
        self.handle = fmap_server_create(device_mem_budget, pinned_bytes, max_inflight,
                                         exp_precision, rect_precision, exp_mode)
        self.meta = {}

    def submit(self, grid, t, antenna, fafb, want_map=False) -> int:
        t = np.ascontiguousarray(t, dtype=np.int64)
        antenna = np.ascontiguousarray(antenna, dtype=np.float32)
        fafb = np.ascontiguousarray(fafb, dtype=np.float32)
        a = make_atoms(t.shape[0], fafb.shape[0], antenna.ndim == 2, t, antenna, fafb)
        g = make_grid(grid)
        tk = fmap_submit(self.handle, g, a, FMAP_SUBMIT_MAP if want_map else 0)
        self.meta[tk] = (fafb.shape[0], g.n_t0, g.n_tau, want_map)
        return tk

    def poll(self, ticket: int, wait_us: int = -1):
        """(status, summary records, map or None)."""
        T, n_t0, n_tau, want_map = self.meta[ticket]
        hs = np.zeros(T, dtype=SUMMARY_DTYPE)
        hm = np.zeros((T, n_t0, n_tau), dtype=np.float32) if want_map else None
        st = fmap_poll(self.handle, ticket, hs, hm, wait_us)
        if st == FMAP_OK:
            del self.meta[ticket]
        return st, hs, hm

    def stats(self):
        return fmap_server_stats(self.handle)

    def peak(self) -> int:
        return fmap_server_peak(self.handle)

    def close(self):
        if getattr(self, "handle", None):
            fmap_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---- convenience wrapper on torch tensors ---------------------------------

def summary_to_numpy(buf) -> np.ndarray:
    """Device or host summary buffer (uint8 [T, 32] tensor or ndarray) -> records."""
    if hasattr(buf, "cpu"):
        buf = buf.cpu().numpy()
    return np.frombuffer(np.ascontiguousarray(buf).tobytes(), dtype=SUMMARY_DTYPE)


@dataclass
class Plan:
    """Owns one fmap plan; ``compute`` takes torch CUDA tensors."""

    grid: object
    n_sft: int
    n_templates: int
    precision: int = FMAP_FP64
    flags: int = 0

    def __post_init__(self):
        if isinstance(self.precision, str):
            self.precision = PRECISIONS[self.precision]
        self.g = make_grid(self.grid)
        self.handle = fmap_plan(self.g, self.n_sft, self.n_templates, self.precision, self.flags)
        if getattr(self.grid, "t0_values", None) is not None:   # explicit axes
            self.set_axes(self.grid.t0_values, self.grid.tau_values)
        if getattr(self.grid, "window_table", None) is not None:   # generic window
            fmap_plan_window_table(self.handle, self.grid.window_table)

    def set_axes(self, t0_values, tau_values):
        fmap_plan_axes(self.handle, t0_values, tau_values)

    def count_terms(self, t_host):
        return fmap_plan_count_terms(self.handle, t_host)

    def close(self):
        if getattr(self, "handle", None):
            fmap_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def atoms(self, t, antenna, fafb) -> fmap_atoms:
        shared = antenna.dim() == 2
        return make_atoms(self.n_sft, self.n_templates, shared, t, antenna, fafb)

    def compute(self, t, antenna, fafb, want_map=True, want_summary=True, out_map=None,
                out_summary=None, stream=None):
        """Run the plan's window; returns (map [T, n_t0, n_tau] or None,
        summary uint8 [T, 32] or None) as device tensors."""
        import torch

        dev = t.device
        T = self.n_templates
        m = out_map
        if m is None and want_map:
            m = torch.empty((T, self.g.n_t0, self.g.n_tau), dtype=torch.float32, device=dev)
        s = out_summary
        if s is None and want_summary:
            s = torch.empty((T, 32), dtype=torch.uint8, device=dev)
        a = self.atoms(t, antenna, fafb)
        if self.g.window == FMAP_TABLE:
            fmap_compute_table(self.handle, a, m, s, stream)
        elif self.g.window == FMAP_RECT:
            fmap_compute_rect(self.handle, a, m, s, stream)
        else:
            fmap_compute_exp(self.handle, a, m, s, stream)
        return m, s

    def compute_host(self, t, antenna, fafb, h_map=None, h_summary=None, stream=None):
        """End-to-end call with host (numpy or pinned torch) buffers."""
        shared = antenna.ndim == 2 if hasattr(antenna, "ndim") else antenna.dim() == 2
        a = make_atoms(self.n_sft, self.n_templates, shared, t, antenna, fafb)
        fmap_compute_host(self.handle, a, h_map, h_summary, stream)
        return h_map, h_summary

    def marginalise(self, d_map, d_valid=None, out_summary=None, stream=None):
        import torch

        s = out_summary
        if s is None:
            s = torch.empty((self.n_templates, 32), dtype=torch.uint8, device=d_map.device)
        fmap_marginalise(self.handle, d_map, d_valid, s, stream)
        return s

    def status(self) -> int:
        return fmap_plan_status(self.handle)

    def set_log_prior(self, c: float):
        fmap_plan_set_log_prior(self.handle, c)

    def set_refine(self, max_cells: int):
        fmap_plan_set_refine(self.handle, max_cells)

    def set_wait_limit(self, limit_ns: int):
        fmap_plan_set_wait_limit(self.handle, limit_ns)
