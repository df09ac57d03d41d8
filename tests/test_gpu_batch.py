"""Uneven batches in one captured graph of persistent launches: every
instance's map and summary must equal what the single-plan path computes with
the same algorithm (bit for bit) and match the oracle; waves, autotuning and
edge-case instances included."""

import numpy as np
import pytest

import oracle
import synth
from synth import EXP, RECT, T_SFT, Grid
from tests.parity_util import LOGB_TOL, TOL, check_map, check_summary

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1805_05652_gb300 as fm  # noqa: E402


def _instances(k, seed=2024):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(k):
        window = EXP if i % 2 else RECT
        n = int(rng.integers(30, 700))
        n_t0, n_tau = int(rng.integers(3, 140)), int(rng.integers(3, 300))
        T = int(rng.integers(1, 6))
        dt0 = int(rng.integers(600, 3 * T_SFT))
        dtau = int(rng.integers(600, 3 * T_SFT))
        g = Grid(-int(rng.integers(0, 5000)), dt0, n_t0, 2 * T_SFT if window == RECT else T_SFT,
                 dtau, n_tau, window)
        inst = synth.make_instance(seed + i, n_det=1 + (i % 3 == 0), presence=0.9, n_merged=n,
                                   n_templates=T, grid=g, shared_antenna=(i % 7 != 3),
                                   injections=[(0, window, 10 * T_SFT, 30 * T_SFT, 150.0)])
        out.append(inst)
    # many templates over shared antenna rows (the template-major cells
    # kernel): T_sft steps (staged prefixes) and coarse t0 steps (global path)
    g3 = Grid(-2 * T_SFT, T_SFT, 21, 2 * T_SFT, T_SFT, 90, RECT)
    out.append(synth.make_instance(seed + 502, n_det=2, presence=0.9, n_merged=260,
                                   n_templates=40, grid=g3,
                                   injections=[(35, RECT, 5 * T_SFT, 40 * T_SFT, 150.0)]))
    g4 = Grid(0, 30 * T_SFT, 17, 2 * T_SFT, 2 * T_SFT, 70, RECT)
    out.append(synth.make_instance(seed + 503, n_merged=600, n_templates=33, grid=g4))
    # edge cases: a single SFT, an empty grid
    g1 = Grid(0, T_SFT, 10, T_SFT, T_SFT, 10, EXP)
    out.append(synth.make_instance(seed + 500, n_slots=1, n_templates=2, grid=g1))
    g2 = Grid(0, T_SFT, 0, 2 * T_SFT, T_SFT, 10, RECT)
    out.append(synth.make_instance(seed + 501, n_slots=50, n_templates=1, grid=g2))
    return out


def _dev(inst):
    dev = torch.device("cuda:0")
    return (inst.grid, torch.from_numpy(inst.t).to(dev), torch.from_numpy(inst.antenna).to(dev),
            torch.from_numpy(inst.fafb).to(dev))


def _single(inst, d):
    grid, t, a, x = d
    flags = 0 if inst.shared_antenna else fm.FMAP_PLAN_PER_TEMPLATE_ANTENNA
    if grid.window == EXP:
        flags |= fm.FMAP_PLAN_EXP_RECURRENCE
    plan = fm.Plan(grid, inst.n_sft, inst.n_templates, "fp64", flags)
    plan.set_refine(0)      # batches do not refine: compare the same computation
    m, s = plan.compute(t, a, x)
    torch.cuda.synchronize()
    plan.close()
    return m.cpu().numpy(), fm.summary_to_numpy(s)


@pytest.fixture(scope="module")
def insts():
    fm.build()
    return _instances(40)


@pytest.mark.parametrize("budget,autotune", [(0, True), (3 << 20, False)])
def test_batch_equals_single_plans_and_oracle(insts, budget, autotune):
    devs = [_dev(i) for i in insts]
    b = fm.Batch(devs, want_map=True, workspace_budget=budget, autotune=autotune)
    info = b.info()
    if budget:
        assert info["waves"] > 1
    # one persistent launch per phase and wave
    assert info["launches_per_run"] <= fm.binding.N_BATCH_PHASES * info["waves"]
    first = None
    for rep in range(2):                        # graph replays give the same bits
        b.run()
        assert b.status() == fm.FMAP_OK
        torch.cuda.synchronize()
        out = [(b.maps[k].cpu().numpy(), fm.summary_to_numpy(b.sums[k][: inst.n_templates]))
               for k, inst in enumerate(insts)]
        if first is None:
            first = out
            continue
        for (m0, s0), (m1, s1) in zip(first, out):
            assert np.array_equal(m0, m1) and s0.tobytes() == s1.tobytes()
    # Single plans give the same maps and summaries up to rounding: a batch
    # scans short exponential data sets with fewer threads per tau, which
    # changes only the order of the additions.
    for k, inst in enumerate(insts):
        got, gs = first[k]
        ref_m, ref_s = _single(inst, devs[k])
        if inst.grid.window == RECT:
            assert np.array_equal(got, ref_m) and gs.tobytes() == ref_s.tobytes(), k
            continue
        assert np.allclose(got, ref_m, rtol=1e-5, atol=1e-5), k
        assert np.array_equal(gs["n_valid"], ref_s["n_valid"]), k
        assert np.allclose(gs["max2F"], ref_s["max2F"], rtol=1e-5, atol=1e-5), k
        assert np.allclose(gs["logB"], ref_s["logB"], rtol=0, atol=1e-5, equal_nan=True), k
    for k in range(len(insts) - 1):   # every instance but the empty grid, against the oracle
        inst = insts[k]
        ref, valid, _ = oracle.fmap(inst.t, inst.antenna, inst.fafb, inst.grid.as_tuple(),
                                    mode="fast")
        got = b.maps[k].cpu().numpy().astype(np.float64)
        check_map(got, ref, valid, TOL["fp64"])
        check_summary(fm.summary_to_numpy(b.sums[k][: inst.n_templates]), ref, valid,
                      TOL["fp64"], LOGB_TOL, refined=False)
    b.close()


def test_batch_profile_times_phases_and_matches_run(insts):
    devs = [_dev(i) for i in insts[:12]]
    b = fm.Batch(devs, want_map=True, workspace_budget=3 << 20, autotune=False)
    b.run()
    assert b.status() == fm.FMAP_OK
    ref = [m.cpu().numpy().copy() for m in b.maps]
    launches = b.info()["launches_per_run"]
    for m in b.maps:
        m.fill_(-7.0)
    ph = b.profile()
    torch.cuda.synchronize()
    assert b.status() == fm.FMAP_OK
    assert set(ph) == set(fm.binding.BATCH_PHASES)
    assert all(v >= 0.0 for v in ph.values()) and ph["index"] > 0.0
    assert b.info()["launches_per_run"] == launches
    for k, m in enumerate(b.maps):
        assert np.array_equal(m.cpu().numpy(), ref[k]), k
    b.close()


def test_batch_reports_bad_timestamps(insts):
    inst = insts[1]
    grid, t, a, x = _dev(inst)
    t = t.clone()
    t[5] = t[4]
    b = fm.Batch([_dev(insts[0]), (grid, t, a, x)], autotune=False)
    b.run()
    assert b.status() == fm.FMAP_ERR_DATA
    b.close()
