"""The C-ABI library without a GPU: it loads, exports every symbol declared in
include/fmap.h, and its host-only entry points (validation, workspace sizing,
window bookkeeping) behave."""

import ctypes
import os
import re

import numpy as np
import pytest

import paper_1805_05652_gb300 as fm
import synth
from synth import EXP, RECT, T_SFT, Grid

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    fm.build()
    return fm.lib()


def _declared_functions():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            src = open(os.path.join(ROOT, "include", h)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            for m in re.finditer(r"\b(fmap_\w+)\s*\(", src):
                names.add(m.group(1))
    return names


def test_exports_every_declared_symbol(L):
    declared = _declared_functions()
    assert "fmap_plan" in declared and "fmap_compute_exp" in declared
    for name in sorted(declared):
        assert hasattr(L, name), f"libfmap.so does not export {name}"
    for name in fm.binding.EXPORTS:
        assert name in declared


def test_struct_sizes_match_header(L):
    assert ctypes.sizeof(fm.binding.fmap_summary) == 32
    assert ctypes.sizeof(fm.binding.fmap_grid) == 64
    assert ctypes.sizeof(fm.binding.fmap_atoms) == 40
    assert ctypes.sizeof(fm.binding.fmap_batch_item) == 120
    assert ctypes.sizeof(fm.binding.fmap_server_config) == 32


@pytest.mark.parametrize("bad", [dict(max_inflight=0), dict(max_inflight=65),
                                 dict(exp_mode=3), dict(pinned_bytes=1024)])
def test_server_rejects_bad_config(L, bad):
    """The configuration is checked before any device memory is touched."""
    cfg = dict(device_mem_budget=1 << 30, pinned_bytes=1 << 24, max_inflight=4,
               exp_precision=fm.FMAP_BF16X3, rect_precision=fm.FMAP_FP64,
               exp_mode=fm.FMAP_SERVER_EXP_AUTO)
    cfg.update(bad)
    with pytest.raises(fm.FmapError) as e:
        fm.fmap_server_create(cfg["device_mem_budget"], cfg["pinned_bytes"], cfg["max_inflight"],
                              cfg["exp_precision"], cfg["rect_precision"], cfg["exp_mode"])
    assert e.value.status == fm.FMAP_ERR_ARG
    assert "exp_mode" in fm.last_error() or "max_inflight" in fm.last_error()


def test_status_strings(L):
    assert fm.status_string(0) == "FMAP_OK"
    assert fm.status_string(fm.FMAP_ERR_DATA) == "FMAP_ERR_DATA"
    assert fm.status_string(fm.FMAP_ERR_UNSUPPORTED) == "FMAP_ERR_UNSUPPORTED"


@pytest.mark.parametrize("bad", [
    dict(n_t0=-1), dict(tau_min=0), dict(t_sft=0), dict(dtau=0), dict(dt0=-5), dict(window=7),
    dict(n_t0=70000, n_tau=70000), dict(tau_min=2_200_000_000),
    dict(window=EXP, tau_min=800_000_000), dict(window=EXP, exp_cut8=8, tau_min=2_200_000_000),
    dict(window=EXP, exp_cut8=-1), dict(window=EXP, exp_cut8=1025),
])
def test_plan_rejects_bad_grids(L, bad):
    """Grid checks, including the window length L(tau_max) < 2^31 s (rect
    L = tau, exp L = exp_cut8 tau / 8, default 3 tau) and the cut's range."""
    g = dict(t0_min=0, dt0=T_SFT, n_t0=10, tau_min=T_SFT, dtau=T_SFT, n_tau=10, t_sft=T_SFT,
             window=RECT, exp_cut8=0)
    g.update(bad)
    grid = (g["t0_min"], g["dt0"], g["n_t0"], g["tau_min"], g["dtau"], g["n_tau"], g["t_sft"],
            g["window"], g["exp_cut8"])
    with pytest.raises(fm.FmapError) as e:
        fm.fmap_plan(grid, 100, 1, fm.FMAP_FP64)
    assert e.value.status == fm.FMAP_ERR_ARG
    assert fm.last_error()


def test_plan_rejects_tensor_precision_for_rect(L):
    grid = (0, T_SFT, 10, T_SFT, T_SFT, 10, T_SFT, RECT)
    for prec in (fm.FMAP_TF32, fm.FMAP_BF16X3):
        with pytest.raises(fm.FmapError) as e:
            fm.fmap_plan(grid, 100, 1, prec)
        assert e.value.status == fm.FMAP_ERR_UNSUPPORTED


def test_plan_rejects_bad_sizes_and_flags(L):
    grid = (0, T_SFT, 10, T_SFT, T_SFT, 10, T_SFT, EXP)
    for args in ((-1, 1, 0, 0), (10, -1, 0, 0), (10, 70000, 0, 0), (10, 1, 9, 0), (10, 1, 0, 16),
                 (10, 1, 0, 1 << 16)):
        with pytest.raises(fm.FmapError) as e:
            fm.fmap_plan(grid, *args)
        assert e.value.status == fm.FMAP_ERR_ARG


def test_workspace_bytes_grows_with_problem(L):
    g1 = (0, T_SFT, 100, T_SFT, T_SFT, 100, T_SFT, EXP)
    g2 = (0, T_SFT, 200, T_SFT, T_SFT, 200, T_SFT, EXP)
    assert 0 < fm.fmap_workspace_bytes(g1, 500, 4) < fm.fmap_workspace_bytes(g2, 500, 4)
    assert fm.fmap_workspace_bytes((0, 1, -1, 1, 1, 1, 1, 0), 5, 1) == 0


@pytest.mark.parametrize("window", [RECT, EXP])
def test_count_terms_matches_window_counts(L, window):
    """The library's host-side term count equals the oracle's per-cell atom
    counts summed over cells with >= 2 atoms."""
    import oracle

    grid = Grid(-4000, 1300, 50, 900, 2100, 60, window)
    inst = synth.make_instance(3, n_det=2, presence=0.8, n_merged=90, grid=grid,
                               dtype=np.float64)
    _, cnt = oracle.sums(inst.t, inst.antenna, inst.fafb, grid.as_tuple())
    terms, cells2 = fm.fmap_count_terms(grid, inst.t)
    assert cells2 == int((cnt >= 2).sum())
    assert terms == int(cnt[cnt >= 2].sum())


def test_compute_rejects_null_plan(L):
    a = fm.make_atoms(0, 0, 1, 0, 0, 0)
    assert L.fmap_compute_exp(None, ctypes.byref(a), None, None, None) == fm.FMAP_ERR_ARG
    assert L.fmap_plan_status(None) == fm.FMAP_ERR_ARG
