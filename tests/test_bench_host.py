"""Host logic of bench.py that needs no GPU: the clock sampler keeps the
nvidia-smi samples that arrived inside the timed region, and says so when it
has to fall back to the whole run."""

import importlib.util
import os

import pytest

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


def test_samples_inside_the_timed_region(bench):
    cs = bench.ClockSampler("GPU-a")
    cs.rows = [(0.00, _row("GPU-a", 1000)), (1.00, _row("GPU-a", 2070)),
               (1.01, _row("GPU-a", 2050, power_cap="Active")), (1.50, _row("GPU-a", 900)),
               (1.00, _row("GPU-b", 300))]
    cs.t_begin, cs.t_end = 0.99, 1.02
    s = cs.summary()
    assert s["scope"] == "timed region"
    assert s["samples"] == 2 and s["samples_total"] == 4   # the other GPU's row is dropped
    assert s["sm_mhz"] == 2060.0 and s["sm_max_mhz"] == 2070.0
    assert s["reasons"] == ["sw_power_cap"]


def test_region_shorter_than_a_sample_falls_back_and_says_so(bench):
    cs = bench.ClockSampler("GPU-a")
    cs.rows = [(0.0, _row("GPU-a", 2070, hw="Active")), (1.0, _row("GPU-a", 2070))]
    cs.t_begin, cs.t_end = 5.0, 5.001
    s = cs.summary()
    assert s["scope"].startswith("whole run")
    assert s["samples"] == 2 and s["reasons"] == ["hw_slowdown"]


def test_no_samples_is_an_error(bench):
    cs = bench.ClockSampler("GPU-a")
    assert "error" in cs.summary()


def test_default_steps_cover_every_workload(bench):
    assert set(bench.DEFAULT_STEPS) == set(bench.WORKLOADS)
    assert all(k >= 3 for k in bench.DEFAULT_STEPS.values())
