"""CPU oracle of the transient F-statistic map (plain C, FP64, OpenMP).

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the CPU-baseline leg
of the benchmark use it; the library under ``paper_1805_05652_gb300`` never
imports it.  It shares no code with the CUDA path.

All functions take plain numpy arrays (atoms are promoted to float64), so the
caller decides which inputs the oracle sees.  Grid tuples are
``(t0_min, dt0, n_t0, tau_min, dtau, n_tau, t_sft, window)``; ``window`` is 0
for rectangular and 1 for exponential windows (Sec. 2, Eq. winrect/winexp).
"""

from __future__ import annotations

import ctypes
import os

import numpy as np

from .build import build, lib_path  # noqa: F401

_lib = None


def _load():
    global _lib
    if _lib is not None:
        return _lib
    path = lib_path()
    if not os.path.exists(path):
        build()
    lib = ctypes.CDLL(path)
    P = ctypes.c_void_p
    i32, i64, f64 = ctypes.c_int, ctypes.c_int64, ctypes.c_double
    lib.oracle_max_threads.restype = i32
    lib.oracle_twoF_from_sums.restype = f64
    lib.oracle_twoF_from_sums.argtypes = [f64] * 7 + [ctypes.c_int32, P]
    lib.oracle_sums.argtypes = [P, i32, P, i32, i32, P, P, P, P, i32]
    lib.oracle_fmap.argtypes = [i32, P, i32, P, i32, i32, P, P, P, P, P, i32]
    lib.oracle_cells.argtypes = [P, i32, P, i32, i32, P, P, i64, P, P, P, P, P, i32]
    lib.oracle_summary.argtypes = [i32, i64, i64, P, P, f64, P, P, P, P, P]
    for f in ("oracle_sums", "oracle_fmap", "oracle_cells", "oracle_summary"):
        getattr(lib, f).restype = i32
    _lib = lib
    return lib


def _p(a):
    return ctypes.c_void_p(a.ctypes.data) if a is not None else ctypes.c_void_p(0)


def _grid_array(grid, inclusive=False):
    """int64 grid array of the C oracle.  ``grid``: (t0_min, dt0, n_t0,
    tau_min, dtau, n_tau, t_sft, window[, exp_cut8[, t0_values, tau_values[,
    window_table]]]); explicit axes (or None) replace the uniform t0 and tau
    steps, a window table (float32 samples) defines window 2."""
    g = list(grid)
    axes, table = None, None
    if len(g) == 12:
        table = g[11]
        g = g[:11]
    if len(g) == 11:
        if g[9] is not None:
            axes = (np.asarray(g[9], dtype=np.int64), np.asarray(g[10], dtype=np.int64))
        g = g[:9]
    if len(g) == 8:
        g.append(0)
    if len(g) != 9:
        raise ValueError("grid must be (t0_min, dt0, n_t0, tau_min, dtau, n_tau, t_sft, window"
                         "[, exp_cut8[, t0_values, tau_values[, window_table]]])")
    tab = None if table is None else np.ascontiguousarray(table, dtype=np.float32)
    head = [int(v) for v in g[:8]] + [1 if inclusive else 0, int(g[8]), 1 if axes else 0,
                                      0 if tab is None else int(tab.shape[0])]
    parts = [np.array(head, dtype=np.int64)]
    if axes is not None:
        if axes[0].shape != (head[2],) or axes[1].shape != (head[5],):
            raise ValueError("axes must hold n_t0 t0 values and n_tau tau values")
        parts += [axes[0], axes[1]]
    if tab is not None:
        parts.append(tab.view(np.uint32).astype(np.int64))
    return np.concatenate(parts)


def _atoms(t, antenna, fafb):
    t = np.ascontiguousarray(t, dtype=np.int64)
    antenna = np.ascontiguousarray(antenna, dtype=np.float64)
    fafb = np.ascontiguousarray(fafb, dtype=np.float64)
    n = t.shape[0]
    if fafb.ndim != 3 or fafb.shape[1:] != (4, n):
        raise ValueError("fafb must be [T][4][N]")
    shared = antenna.ndim == 2
    if shared and antenna.shape != (3, n):
        raise ValueError("antenna must be [3][N] or [T][3][N]")
    if not shared and antenna.shape != (fafb.shape[0], 3, n):
        raise ValueError("antenna must be [3][N] or [T][3][N]")
    return t, antenna, fafb, shared


def max_threads() -> int:
    return int(_load().oracle_max_threads())


def twoF_from_sums(A, B, C, fa_re, fa_im, fb_re, fb_im, count):
    """2F of Eq. (F_FaFb) for one set of sums; returns (2F, valid)."""
    v = ctypes.c_int32(0)
    r = _load().oracle_twoF_from_sums(float(A), float(B), float(C), float(fa_re), float(fa_im),
                                      float(fb_re), float(fb_im), int(count), ctypes.byref(v))
    return float(r), bool(v.value)


def sums(t, antenna, fafb, grid, inclusive=False, threads=0):
    """Windowed sums by direct definition: ``[T][n_t0][n_tau][7]`` with
    (A, B, C, Re Fa, Im Fa, Re Fb, Im Fb), and atom counts ``[n_t0][n_tau]``."""
    t, antenna, fafb, shared = _atoms(t, antenna, fafb)
    g = _grid_array(grid, inclusive)
    T = fafb.shape[0]
    out = np.zeros((T, int(g[2]), int(g[5]), 7))
    cnt = np.zeros((int(g[2]), int(g[5])), dtype=np.int32)
    rc = _load().oracle_sums(_p(g), t.shape[0], _p(t), T, int(shared), _p(antenna), _p(fafb),
                             _p(out), _p(cnt), int(threads))
    if rc:
        raise RuntimeError(f"oracle_sums failed: {rc}")
    return out, cnt


def fmap(t, antenna, fafb, grid, mode="direct", inclusive=False, threads=0):
    """The 2F map ``[T][n_t0][n_tau]`` (float64), the validity mask and the
    per-cell atom counts.  ``mode='direct'`` visits every atom for every cell;
    ``mode='fast'`` runs the paper's per-row algorithms (Sec. 3)."""
    t, antenna, fafb, shared = _atoms(t, antenna, fafb)
    g = _grid_array(grid, inclusive)
    T = fafb.shape[0]
    shape = (T, int(g[2]), int(g[5]))
    m2 = np.zeros(shape)
    val = np.zeros(shape, dtype=np.uint8)
    cnt = np.zeros(shape[1:], dtype=np.int32)
    rc = _load().oracle_fmap(0 if mode == "direct" else 1, _p(g), t.shape[0], _p(t), T,
                             int(shared), _p(antenna), _p(fafb), _p(m2), _p(val), _p(cnt),
                             int(threads))
    if rc:
        raise RuntimeError(f"oracle_fmap failed: {rc}")
    return m2, val.astype(bool), cnt


def cells(t, antenna, fafb, grid, cell_idx, inclusive=False, threads=0, want_sums=False):
    """Direct-definition 2F of listed cells ``cell_idx[k] = (template, m, n)``."""
    t, antenna, fafb, shared = _atoms(t, antenna, fafb)
    g = _grid_array(grid, inclusive)
    idx = np.ascontiguousarray(cell_idx, dtype=np.int64).reshape(-1, 3)
    k = idx.shape[0]
    out = np.zeros(k)
    val = np.zeros(k, dtype=np.uint8)
    cnt = np.zeros(k, dtype=np.int32)
    sm = np.zeros((k, 7)) if want_sums else None
    rc = _load().oracle_cells(_p(g), t.shape[0], _p(t), fafb.shape[0], int(shared), _p(antenna),
                              _p(fafb), k, _p(idx), _p(out), _p(val), _p(cnt), _p(sm),
                              int(threads))
    if rc:
        raise RuntimeError(f"oracle_cells failed: {rc}")
    if want_sums:
        return out, val.astype(bool), cnt, sm
    return out, val.astype(bool), cnt


def summary(map2F, valid, log_prior_const=0.0):
    """Per-template max 2F, argmax (m, n), log Bayes factor, N_valid."""
    m2 = np.ascontiguousarray(map2F, dtype=np.float64)
    if m2.ndim == 2:
        m2 = m2[None]
    v = np.ascontiguousarray(valid, dtype=np.uint8).reshape(m2.shape)
    T, n_t0, n_tau = m2.shape
    mx = np.zeros(T)
    am = np.zeros(T, dtype=np.int32)
    an = np.zeros(T, dtype=np.int32)
    lb = np.zeros(T)
    nv = np.zeros(T, dtype=np.int64)
    _load().oracle_summary(T, n_t0, n_tau, _p(m2), _p(v), float(log_prior_const), _p(mx),
                           _p(am), _p(an), _p(lb), _p(nv))
    return dict(max2F=mx, m=am, n=an, logB=lb, n_valid=nv)
