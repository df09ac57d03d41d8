"""Host logic of bench.py that needs no GPU: the clock sampler keeps the
nvidia-smi samples whose own timestamps fall inside the timed regions (and
says so when it has to fall back to the whole run), nvidia-smi's timestamp
format parses, and the oracle arm's term count (numpy, no library code)
equals a brute-force count of the window rule."""

import importlib.util
import os

import numpy as np
import pytest

import synth
from synth import EXP, RECT, T_SFT, Grid

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _row(uuid, mhz, power_cap="Not Active", hw="Not Active"):
    # uuid, clocks.sm, clocks.max.sm, power.draw, reasons.active, hw_slowdown,
    # hw_thermal_slowdown, sw_thermal_slowdown, sw_power_cap
    return [uuid, str(mhz), "2070", "900.0", "0x0", hw, "Not Active", "Not Active", power_cap]


def test_samples_inside_the_timed_regions(bench):
    cs = bench.ClockSampler("GPU-a")
    cs.rows = [(0.00, _row("GPU-a", 1000)), (1.00, _row("GPU-a", 2070)),
               (1.01, _row("GPU-a", 2050, power_cap="Active")), (1.50, _row("GPU-a", 900)),
               (3.00, _row("GPU-a", 1990)), (1.00, _row("GPU-b", 300))]
    cs.spans = [(0.99, 1.02), (2.9, 3.1)]
    s = cs.summary()
    assert s["scope"] == "timed regions"
    assert s["samples"] == 3 and s["samples_total"] == 5   # the other GPU's row is dropped
    assert s["sm_mhz"] == 2050.0 and s["sm_max_mhz"] == 2070.0
    assert s["reasons"] == ["sw_power_cap"]


def test_region_shorter_than_a_sample_falls_back_and_says_so(bench):
    cs = bench.ClockSampler("GPU-a")
    cs.rows = [(0.0, _row("GPU-a", 2070, hw="Active")), (1.0, _row("GPU-a", 2070))]
    cs.spans = [(5.0, 5.001)]
    s = cs.summary()
    assert s["scope"].startswith("whole run")
    assert s["samples"] == 2 and s["reasons"] == ["hw_slowdown"]


def test_no_samples_is_an_error(bench):
    cs = bench.ClockSampler("GPU-a")
    assert "error" in cs.summary()


def test_nvidia_smi_timestamps(bench):
    a = bench.ClockSampler._stamp("2026/12/04 06:12:33.125")
    b = bench.ClockSampler._stamp("2026/12/04 06:12:34.000")
    assert abs((b - a) - 0.875) < 1e-6
    assert bench.ClockSampler._stamp("garbage") is None


@pytest.mark.parametrize("window", [RECT, EXP])
def test_term_count_matches_brute_force(bench, window):
    g = Grid(-3 * T_SFT, 1300, 23, 2 * T_SFT if window == RECT else 700, 900, 31, window)
    inst = synth.make_instance(5, n_det=2, presence=0.8, n_merged=90, grid=g)
    t = inst.t
    terms = cells2 = 0
    for t0 in g.t0():
        for tau in g.tau():
            c = int(((t >= t0) & (t + T_SFT <= t0 + g.window_len(int(tau)))).sum())
            if c >= 2:
                terms += c
                cells2 += 1
    assert bench.count_terms_np(g, t) == (terms, cells2)
