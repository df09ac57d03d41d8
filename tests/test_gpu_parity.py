"""GPU parity: the CUDA path through the C ABI against the CPU oracle on the
same seeded inputs, element by element, plus the reductions, edge cases and
the device-side data checks."""

import numpy as np
import pytest

import oracle
import synth
from synth import EXP, RECT, T_SFT, Grid
from tests.parity_util import (LOGB_TOL, TOL, check_map, check_summary, oracle_map,
                               rel_err, run_gpu)

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - CPU container
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1805_05652_gb300 as fm  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _built():
    fm.build()
    oracle.build()


def _parity(inst, prec, mode="fast"):
    ref, valid, _ = oracle_map(inst, mode)
    got, gs = run_gpu(inst, prec)
    worst = check_map(got, ref, valid, TOL[prec])
    near, ties, dlogb = check_summary(gs, ref, valid, TOL[prec], LOGB_TOL)
    print(f"{prec}: max rel 2F err {worst:.2e}, max |dlogB| {dlogb:.2e}, "
          f"near ties {near}, FP64 ties {ties} of {inst.n_templates}")
    return worst


# ---------------------------------------------------------------- rect --------

@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_rect_small_config(prec):
    """200 single-detector SFTs with 10% gaps, 200 x 200 cells, one injection."""
    inst = synth.config_small_rect()
    _parity(inst, prec, mode="direct")


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_rect_ragged_tiles_offgrid_per_template_antenna(prec):
    """n_tau spanning two 256-cell tiles and a ragged tail, t0 before the data
    and windows past its end, off-grid steps, per-template antenna rows."""
    grid = Grid(-7000, 1000, 37, 700, 1900, 600, RECT)
    inst = synth.make_instance(41, n_det=2, presence=0.85, n_merged=700, n_templates=3,
                               grid=grid, shared_antenna=False,
                               injections=[(1, RECT, 30000, 200000, 150.0)])
    _parity(inst, prec)


@pytest.mark.parametrize("shared", [True, False])
@pytest.mark.parametrize("dt0_sfts", [1, 25])
@pytest.mark.parametrize("n_templates", [2, 5, 37])
def test_rect_template_chunks(shared, dt0_sfts, n_templates):
    """2, 5 and 37 templates (one, two or four template lanes per tile; 37
    spans a full 32-template chunk and a ragged one) over 2 detectors with
    gaps; t0 steps of one SFT keep a group's prefix entries in shared memory,
    steps of 25 SFTs spread its rows too far apart and take the global
    float-pair path; ragged tiles in both directions."""
    grid = Grid(-3 * T_SFT, dt0_sfts * T_SFT, 45, 2 * T_SFT, T_SFT, 150, RECT)
    inj = [(1, RECT, 10 * T_SFT, 40 * T_SFT, 120.0)]
    if n_templates > 33:
        inj.append((33, RECT, 2 * T_SFT, 90 * T_SFT, 200.0))
    inst = synth.make_instance(43 + dt0_sfts, n_det=2, presence=0.9, n_merged=420,
                               n_templates=n_templates, grid=grid, shared_antenna=shared,
                               injections=inj)
    _parity(inst, "fp64")


# ----------------------------------------------------------------- exp --------

@pytest.mark.parametrize("prec", ["fp64", "fp32", "tf32", "bf16x3", "rec"])
def test_exp_ragged(prec):
    """Exp windows: 11 templates (ragged template chunks), n_tau = 300 (two
    128-cell tiles and a tail), off-grid t0 and tau steps, 2 detectors."""
    grid = Grid(-2500, 1000, 29, 900, 1300, 300, EXP)
    inst = synth.make_instance(43, n_det=2, presence=0.9, n_merged=400, n_templates=11,
                               grid=grid, injections=[(0, EXP, 20000, 60000, 200.0)])
    try:
        _parity(inst, prec)
    except fm.FmapError as e:
        if e.status == fm.FMAP_ERR_UNSUPPORTED:
            pytest.skip(f"{prec} not built")
        raise


@pytest.mark.parametrize("cut8", [1, 8, 20, 40])
@pytest.mark.parametrize("prec", ["fp64", "bf16x3", "rec"])
def test_exp_window_cut(cut8, prec):
    """Exp windows cut at L = cut8 tau / 8 instead of 3 tau (tau / 8, tau,
    2.5 tau, 5 tau): every path against the oracle's definition with the same
    cut; short cuts leave many cells with < 2 SFTs."""
    grid = Grid(-2500, 1000, 29, 900, 1300, 150, EXP, T_SFT, cut8)
    inst = synth.make_instance(44, n_det=2, presence=0.9, n_merged=300, n_templates=5,
                               grid=grid, injections=[(1, EXP, 20000, 60000, 200.0)])
    try:
        _parity(inst, prec)
    except fm.FmapError as e:
        if e.status == fm.FMAP_ERR_UNSUPPORTED:
            pytest.skip(f"{prec} not built")
        raise


def _axes_instance(window, seed):
    """A non-uniform (t0, tau) grid: sorted random values with uneven steps,
    t0 from before the data to past its end, 48 x 160 cells (several tiles
    and ragged tails)."""
    rng = np.random.default_rng(seed)
    t0 = np.sort(rng.choice(np.arange(-4 * T_SFT, 300 * T_SFT, 211), size=48, replace=False))
    lo = 2 * T_SFT if window == RECT else T_SFT // 2
    tau = np.sort(rng.choice(np.arange(lo, 200 * T_SFT, 173), size=160, replace=False))
    grid = Grid(0, 1, len(t0), 1, 1, len(tau), window, T_SFT, 0,
                tuple(int(v) for v in t0), tuple(int(v) for v in tau))
    return synth.make_instance(seed, n_det=2, presence=0.9, n_merged=300, n_templates=5,
                               grid=grid, injections=[(2, window, 40 * T_SFT, 60 * T_SFT, 200.0)])


@pytest.mark.parametrize("window,prec", [(RECT, "fp64"), (RECT, "fp32"), (EXP, "fp64"),
                                         (EXP, "tf32"), (EXP, "bf16x3"), (EXP, "rec")])
def test_explicit_axes(window, prec):
    """Non-uniform grids through fmap_plan_axes: every path against the
    oracle on the same axes."""
    inst = _axes_instance(window, 61 + window)
    try:
        _parity(inst, prec)
    except fm.FmapError as e:
        if e.status == fm.FMAP_ERR_UNSUPPORTED:
            pytest.skip(f"{prec} not built")
        raise


def test_explicit_axes_checks_count_and_reset():
    """fmap_plan_axes rejects unsorted or non-positive values and a missing
    axis; fmap_plan_count_terms counts the axes' windows; (NULL, NULL)
    restores the uniform grid."""
    import torch

    inst = _axes_instance(EXP, 70)
    g = inst.grid
    plan = fm.Plan(g, inst.n_sft, inst.n_templates, "fp64")
    t0, tau = np.array(g.t0_values), np.array(g.tau_values)
    for bad_t0, bad_tau in ((t0[::-1], tau), (t0, tau[::-1]), (t0, np.r_[0, tau[1:]])):
        with pytest.raises(fm.FmapError) as e:
            plan.set_axes(bad_t0, bad_tau)
        assert e.value.status == fm.FMAP_ERR_ARG
    tau64 = np.ascontiguousarray(tau, dtype=np.int64)
    assert fm.binding.lib().fmap_plan_axes(plan.handle, None, tau64.ctypes.data) == fm.FMAP_ERR_ARG
    plan.set_axes(t0, tau)
    _, cnt = oracle.sums(inst.t, inst.antenna, inst.fafb, g.as_tuple())
    assert plan.count_terms(inst.t) == (int(cnt[cnt >= 2].sum()), int((cnt >= 2).sum()))
    # back to the uniform grid of the struct fields
    plan.set_axes(None, None)
    uni = Grid(-T_SFT, 2 * T_SFT, g.n_t0, T_SFT, 3 * T_SFT, g.n_tau, EXP)
    plan.close()
    plan = fm.Plan(uni, inst.n_sft, inst.n_templates, "fp64")
    dev = torch.device("cuda", 0)
    args = (torch.from_numpy(inst.t).to(dev), torch.from_numpy(inst.antenna).to(dev),
            torch.from_numpy(inst.fafb).to(dev))
    m_uni, _ = plan.compute(*args)
    plan.set_axes(uni.t0(), uni.tau())
    m_ax, _ = plan.compute(*args)
    plan.set_axes(None, None)
    m_back, _ = plan.compute(*args)
    torch.cuda.synchronize()
    assert torch.equal(m_uni, m_ax) and torch.equal(m_uni, m_back)
    plan.close()


def _table_instance(seed, shared=True, cut8=0, n_points=64):
    """A generic window: a smooth bump times a decay, sampled on [0, X] (rising
    then falling, with a kink), on a grid spanning several tiles."""
    X = (cut8 or 24) / 8.0
    x = np.linspace(0.0, X, n_points)
    w = (np.sin(np.pi * np.minimum(x / 0.4, 1.0) / 2) ** 2) * np.exp(-0.7 * x) + 0.05
    grid = Grid(-2500, 1000, 29, 900, 1300, 300, synth.TABLE, T_SFT, cut8, None, None,
                tuple(float(v) for v in w.astype(np.float32)))
    return synth.make_instance(seed, n_det=2, presence=0.9, n_merged=400, n_templates=6,
                               grid=grid, shared_antenna=shared,
                               injections=[(1, EXP, 20000, 60000, 200.0)])


@pytest.mark.parametrize("prec", ["fp64", "fp32", "tf32", "bf16x3"])
def test_table_window(prec):
    """Generic (table) windows: every precision against the oracle's
    definition (linear interpolation of the same samples)."""
    try:
        _parity(_table_instance(81), prec)
    except fm.FmapError as e:
        if e.status == fm.FMAP_ERR_UNSUPPORTED:
            pytest.skip(f"{prec} not built")
        raise


@pytest.mark.parametrize("prec", ["fp64", "bf16x3"])
def test_table_window_per_template_antenna_and_cut(prec):
    """Table windows with per-template antenna rows and a 2 tau support."""
    try:
        _parity(_table_instance(82, shared=False, cut8=16, n_points=1024), prec)
    except fm.FmapError as e:
        if e.status == fm.FMAP_ERR_UNSUPPORTED:
            pytest.skip(f"{prec} not built")
        raise


def test_table_window_api_checks():
    """A table plan needs its samples before computing; samples are refused
    for other windows and outside 2..1024."""
    import torch

    inst = _table_instance(83)
    g = inst.grid
    bare = Grid(g.t0_min, g.dt0, g.n_t0, g.tau_min, g.dtau, g.n_tau, synth.TABLE)
    plan = fm.Plan(bare, inst.n_sft, inst.n_templates, "fp64")
    dev = torch.device("cuda", 0)
    args = (torch.from_numpy(inst.t).to(dev), torch.from_numpy(inst.antenna).to(dev),
            torch.from_numpy(inst.fafb).to(dev))
    with pytest.raises(fm.FmapError) as e:
        plan.compute(*args)
    assert e.value.status == fm.FMAP_ERR_ARG
    for bad in (np.ones(1), np.ones(1025), np.array([1.0, np.nan])):
        with pytest.raises(fm.FmapError) as e:
            fm.binding.fmap_plan_window_table(plan.handle, bad)
        assert e.value.status == fm.FMAP_ERR_ARG
    plan.close()
    ex = fm.Plan(Grid(0, T_SFT, 4, T_SFT, T_SFT, 4, EXP), inst.n_sft, 1, "fp64")
    with pytest.raises(fm.FmapError) as e:
        fm.binding.fmap_plan_window_table(ex.handle, np.ones(4))
    assert e.value.status == fm.FMAP_ERR_ARG
    ex.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32", "rec", "tf32", "bf16x3"])
def test_exp_per_template_antenna(prec):
    grid = Grid(0, T_SFT, 20, T_SFT, T_SFT, 140, EXP)
    inst = synth.make_instance(44, n_det=1, presence=0.9, n_merged=200, n_templates=3,
                               grid=grid, shared_antenna=False)
    _parity(inst, prec)


@pytest.mark.parametrize("shared", [True, False])
@pytest.mark.parametrize("n_templates", [25, 70])
@pytest.mark.parametrize("prec", ["tf32", "bf16x3"])
def test_exp_tensor_core_template_chunks(prec, n_templates, shared):
    """25 templates: one chunk of N = 128 data columns (100 used); 70: two
    full 32-template chunks of N = 128 and a ragged third of 6 templates; over
    2 x 128-cell tiles and a tail of tau."""
    grid = Grid(0, 2 * T_SFT, 9, T_SFT, T_SFT, 290, EXP)
    inst = synth.make_instance(46, n_det=2, presence=0.9, n_merged=260,
                               n_templates=n_templates, grid=grid, shared_antenna=shared,
                               injections=[(n_templates - 1, EXP, 4 * T_SFT, 40 * T_SFT, 150.0)])
    _parity(inst, prec)


def test_exp_recurrence_cells_not_staged():
    """6000 SFTs and 2500 t0 rows: the recurrence's per-cell window records of
    one tau no longer fit shared memory beside the suffix sums
    (24 n_sft + 32 n_t0 > 220 KB) and are recomputed per template."""
    grid = Grid(-5 * T_SFT, 2 * T_SFT, 2500, T_SFT, 2 * T_SFT, 12, EXP)
    inst = synth.make_instance(45, n_det=1, presence=0.95, n_merged=6000, n_templates=2,
                               grid=grid, injections=[(1, EXP, 900 * T_SFT, 9 * T_SFT, 150.0)])
    _parity(inst, "rec")


# ------------------------------------------------------- reductions, API ------

def test_marginalise_matches_oracle():
    rng = np.random.default_rng(5)
    T, n_t0, n_tau = 3, 70, 130
    m = (rng.chisquare(4, size=(T, n_t0, n_tau)) * 2).astype(np.float32)
    m[1, 10, 20] = m[1, 30, 40] = 77.0          # tie: lowest index wins
    v = rng.random(m.shape) > 0.2
    v[2] = False                                  # a template with no valid cell
    grid = (0, T_SFT, n_t0, T_SFT, T_SFT, n_tau, T_SFT, RECT)
    plan = fm.Plan(grid, 10, T, "fp64")
    dm = torch.from_numpy(m).cuda()
    dv = torch.from_numpy(v.astype(np.uint8)).cuda()
    gs = fm.summary_to_numpy(plan.marginalise(dm, dv))
    rs = oracle.summary(m.astype(np.float64), v)
    assert np.array_equal(gs["n_valid"], rs["n_valid"])
    for j in range(2):
        assert (gs["m"][j], gs["n"][j]) == (rs["m"][j], rs["n"][j])
        assert gs["max2F"][j] == np.float32(rs["max2F"][j])
        assert abs(gs["logB"][j] - rs["logB"][j]) < 1e-6
    assert gs["m"][2] == -1 and np.isnan(gs["logB"][2])
    gs2 = fm.summary_to_numpy(plan.marginalise(dm, None))
    rs2 = oracle.summary(m.astype(np.float64), np.ones_like(v))
    assert np.allclose(gs2["logB"], rs2["logB"], atol=1e-6, rtol=0)
    plan.close()


def test_log_prior_constant_shifts_logB():
    inst = synth.config_small_rect()
    _, gs0 = run_gpu(inst, "fp64")
    import paper_1805_05652_gb300 as fm2
    t = torch.from_numpy(inst.t).cuda()
    a = torch.from_numpy(inst.antenna).cuda()
    x = torch.from_numpy(inst.fafb).cuda()
    plan = fm2.Plan(inst.grid, inst.n_sft, 1, "fp64")
    plan.set_log_prior(-2.5)
    _, s = plan.compute(t, a, x)
    gs = fm2.summary_to_numpy(s)
    assert abs(gs["logB"][0] - (gs0["logB"][0] - 2.5)) < 1e-12
    plan.close()


@pytest.mark.parametrize("window,prec", [(RECT, "fp64"), (EXP, "fp32")])
def test_host_api_equals_device_api(window, prec):
    """fmap_compute_host (host buffers, copies inside) gives the same bits as
    the device entry point."""
    grid = Grid(0, T_SFT, 30, 2 * T_SFT, T_SFT, 90, window)
    inst = synth.make_instance(9, n_slots=150, n_templates=4, grid=grid)
    got, gs = run_gpu(inst, prec)
    plan = fm.Plan(grid, inst.n_sft, inst.n_templates, prec)
    hm = np.zeros((4, 30, 90), dtype=np.float32)
    hs = np.zeros(4, dtype=fm.SUMMARY_DTYPE)
    plan.compute_host(inst.t, inst.antenna, inst.fafb, hm, hs)
    assert np.array_equal(hm.astype(np.float64), got)
    assert hs.tobytes() == gs.tobytes()
    plan.close()


@pytest.mark.parametrize("window,prec", [(RECT, "fp64"), (EXP, "fp64"), (EXP, "fp32")])
def test_deterministic(window, prec):
    grid = Grid(0, T_SFT, 25, T_SFT, T_SFT, 140, window)
    inst = synth.make_instance(12, n_slots=120, n_templates=5, grid=grid)
    a, sa = run_gpu(inst, prec)
    b, sb = run_gpu(inst, prec)
    assert np.array_equal(a, b) and sa.tobytes() == sb.tobytes()


# ----------------------------------------------------------------- edges -----

@pytest.mark.parametrize("window", [RECT, EXP])
@pytest.mark.parametrize("case", ["one_sft", "grid_after_data", "too_short", "empty_grid",
                                  "no_sft"])
def test_degenerate_inputs(window, case):
    n = {"one_sft": 1, "no_sft": 0}.get(case, 40)
    grid = Grid(0, T_SFT, 12, T_SFT if window == EXP else 2 * T_SFT, T_SFT, 9, window)
    if case == "grid_after_data":
        grid = Grid(10**6, T_SFT, 12, T_SFT, T_SFT, 9, window)
    if case == "too_short":
        grid = Grid(0, T_SFT, 12, 100, 50, 9, window)        # windows shorter than an SFT
    if case == "empty_grid":
        grid = Grid(0, T_SFT, 0, T_SFT, T_SFT, 9, window)
    if n > 0:
        inst = synth.make_instance(13, n_slots=n, n_templates=2, grid=grid)
    else:
        inst = synth.Instance(np.zeros(0, np.int64), np.zeros((3, 0), np.float32),
                              np.zeros((2, 4, 0), np.float32), grid)
    for prec in ("fp64", "fp32"):
        got, gs = run_gpu(inst, prec)
        assert np.all(got == 0.0)
        assert np.all(gs["n_valid"] == 0) and np.all(gs["m"] == -1)
        assert np.all(np.isnan(gs["logB"]))


def test_nonincreasing_timestamps_reported():
    grid = Grid(0, T_SFT, 5, T_SFT, T_SFT, 5, EXP)
    inst = synth.make_instance(14, n_slots=30, grid=grid)
    t = inst.t.copy()
    t[10] = t[9]
    plan = fm.Plan(grid, inst.n_sft, 1, "fp32")
    plan.compute(torch.from_numpy(t).cuda(), torch.from_numpy(inst.antenna).cuda(),
                 torch.from_numpy(inst.fafb).cuda())
    assert plan.status() == fm.FMAP_ERR_DATA
    assert plan.status() == fm.FMAP_OK            # latched error was cleared
    plan.close()


def test_recurrence_flag_validation():
    grid = Grid(0, T_SFT, 5, T_SFT, T_SFT, 5, EXP)
    for args, status in (((grid.with_window(RECT), 10, 1, "fp64"), fm.FMAP_ERR_ARG),
                         ((grid, 10, 1, "bf16x3"), fm.FMAP_ERR_ARG),
                         ((grid, 20000, 1, "fp64"), fm.FMAP_ERR_UNSUPPORTED)):
        with pytest.raises(fm.FmapError) as e:
            fm.fmap_plan(*args, flags=fm.FMAP_PLAN_EXP_RECURRENCE)
        assert e.value.status == status


def test_mismatched_calls_rejected():
    grid = Grid(0, T_SFT, 5, T_SFT, T_SFT, 5, RECT)
    inst = synth.make_instance(15, n_slots=30, grid=grid)
    plan = fm.Plan(grid, inst.n_sft, 1, "fp64")
    t = torch.from_numpy(inst.t).cuda()
    a = torch.from_numpy(inst.antenna).cuda()
    x = torch.from_numpy(inst.fafb).cuda()
    atoms = plan.atoms(t, a, x)
    out = torch.empty(25, device="cuda")
    with pytest.raises(fm.FmapError) as e:
        fm.fmap_compute_exp(plan.handle, atoms, out, None)
    assert e.value.status == fm.FMAP_ERR_ARG
    bad = fm.make_atoms(inst.n_sft + 1, 1, 1, t, a, x)
    with pytest.raises(fm.FmapError):
        fm.fmap_compute_rect(plan.handle, bad, out, None)
    plan.close()


# ------------------------------------------------------------- refinement -----

@pytest.mark.parametrize("window,prec", [(RECT, "fp32"), (EXP, "bf16x3"), (EXP, "fp64")])
def test_refinement_summary_only_and_off(window, prec):
    """Summaries with the map given, summary-only with the plan's own map
    buffer (bit-identical), summary-only without it (unrefined: flags 0,
    within the fast path's tolerances), and refinement turned off."""
    grid = Grid(-3000, 1500, 40, 2 * T_SFT if window == RECT else T_SFT, T_SFT, 260, window)
    inst = synth.make_instance(81, n_det=2, presence=0.9, n_merged=500, n_templates=6,
                               grid=grid, injections=[(2, window, 30000, 90000, 220.0)])
    ref, valid, _ = oracle_map(inst)
    dev = torch.device("cuda:0")
    t = torch.from_numpy(inst.t).to(dev)
    a = torch.from_numpy(inst.antenna).to(dev)
    x = torch.from_numpy(inst.fafb).to(dev)
    with_map = fm.Plan(inst.grid, inst.n_sft, inst.n_templates, prec)
    m, s = with_map.compute(t, a, x)
    own = fm.Plan(inst.grid, inst.n_sft, inst.n_templates, prec, fm.FMAP_PLAN_MAP_BUFFER)
    _, s_own = own.compute(t, a, x, want_map=False)
    bare = fm.Plan(inst.grid, inst.n_sft, inst.n_templates, prec)
    _, s_bare = bare.compute(t, a, x, want_map=False)
    off = fm.Plan(inst.grid, inst.n_sft, inst.n_templates, prec)
    off.set_refine(0)
    m_off, s_off = off.compute(t, a, x)
    torch.cuda.synchronize()
    for p in (with_map, own, bare, off):
        assert p.status() == fm.FMAP_OK
        p.close()
    gs = fm.summary_to_numpy(s)
    check_map(m.cpu().numpy().astype(np.float64), ref, valid, TOL[prec])
    check_summary(gs, ref, valid, TOL[prec], LOGB_TOL)
    assert fm.summary_to_numpy(s_own).tobytes() == gs.tobytes()
    for raw in (s_bare, s_off):
        g2 = fm.summary_to_numpy(raw)
        assert np.all(g2["flags"] == 0)
        assert np.array_equal(g2["n_valid"], gs["n_valid"])
        rs = oracle.summary(ref, valid)
        assert np.all(np.abs(g2["max2F"] - rs["max2F"]) <= TOL[prec] * np.maximum(rs["max2F"], 1))
    # refinement rewrites only the collected cells of the map, with FP64 values
    got, got_off = m.cpu().numpy(), m_off.cpu().numpy()
    changed = got != got_off
    assert changed.sum() <= inst.n_templates * 512
    err = np.abs(got[changed] - ref[changed]) / np.maximum(np.abs(ref[changed]), 1.0)
    assert err.size == 0 or err.max() <= 1e-6


@pytest.mark.parametrize("window,prec", [(RECT, "fp64"), (EXP, "rec")])
def test_refinement_flat_maximum(window, prec):
    """Windows that run past the data's end hold the same atoms for every
    longer tau: more cells than the cap (64 for the FP64 class) lie within
    1/16 of the maximum, and the refinement takes that whole top bin (up to
    4096 cells), so every template is still refined with an exact argmax."""
    # (exponential: tau far beyond the data span, so that the weights, and
    # 2F, barely change along tau)
    grid = Grid(0, T_SFT, 12, 2 * T_SFT if window == RECT else 2000 * T_SFT, T_SFT, 400, window)
    inst = synth.make_instance(83, n_det=1, presence=1.0, n_merged=60, n_templates=3,
                               grid=grid, injections=[(1, RECT, 0, 60 * T_SFT, 400.0)])
    ref, valid, _ = oracle_map(inst)
    rs = oracle.summary(ref, valid)
    top = [(valid[j] & (ref[j] >= rs["max2F"][j] - 1.0 / 16)).sum() for j in range(3)]
    assert max(top) > 64   # the case this test is for
    got, gs = run_gpu(inst, prec)
    check_map(got, ref, valid, TOL[prec])
    check_summary(gs, ref, valid, TOL[prec], LOGB_TOL)


@pytest.mark.parametrize("window,prec", [(RECT, "fp64"), (EXP, "rec")])
@pytest.mark.parametrize("cap", [64, 4096])
def test_refinement_kept_cells_overflow(window, prec, cap):
    """The histogram pass keeps the cells of the bins the cut may take (at
    most 8192 per template) and the cut is applied to them; a template that
    kept more is collected by a second scan of its tiles.  With a cap of 4096
    the bound covers the whole window below the maximum, so the noise
    template (maximum ~20: nearly every cell within 16 of it) overflows while
    the injected one keeps a few cells: both paths in one call, each against
    the oracle."""
    import torch

    g = Grid(0, T_SFT, 300, 2 * T_SFT if window == RECT else T_SFT, T_SFT, 300, window)
    inst = synth.make_instance(77, n_det=1, presence=1.0, n_merged=350, n_templates=2, grid=g,
                               injections=[(0, window, 20 * T_SFT, 100 * T_SFT, 3000.0)])
    ref, valid, _ = oracle_map(inst)
    rs = oracle.summary(ref, valid)
    within = [int((valid[j] & (ref[j] >= rs["max2F"][j] - 16.0)).sum()) for j in range(2)]
    assert within[1] > 8192 and within[0] < 8192, within   # the case this test is for
    dev = torch.device("cuda:0")
    flags = fm.FMAP_PLAN_EXP_RECURRENCE if prec == "rec" else 0
    plan = fm.Plan(g, inst.n_sft, 2, "fp64", flags)
    plan.set_refine(cap)
    m, s = plan.compute(torch.from_numpy(inst.t).to(dev), torch.from_numpy(inst.antenna).to(dev),
                        torch.from_numpy(inst.fafb).to(dev))
    torch.cuda.synchronize()
    assert plan.status() == fm.FMAP_OK
    plan.close()
    gs = fm.summary_to_numpy(s)
    assert np.all(gs["flags"] & fm.FMAP_SUMMARY_REFINED), gs["flags"]
    check_map(m.cpu().numpy().astype(np.float64), ref, valid, TOL[prec])
    check_summary(gs, ref, valid, TOL[prec], LOGB_TOL)


@pytest.mark.parametrize("window,prec", [(RECT, "fp64"), (EXP, "rec"), (EXP, "bf16x3")])
def test_graph_replay(window, prec):
    """FMAP_PLAN_GRAPH: the first call captures its launches, later calls with
    the same pointers replay them (bit-identical to direct launches, reading
    the atoms as they are at each call), other pointers capture anew."""
    import torch

    g = Grid(-2000, T_SFT, 60, 2 * T_SFT if window == RECT else T_SFT, T_SFT, 150, window)
    insts = [synth.make_instance(90 + k, n_det=2, presence=0.9, n_merged=300, n_templates=5,
                                 grid=g, injections=[(1, window, 10 * T_SFT, 40 * T_SFT, 150.0)])
             for k in range(2)]
    dev = torch.device("cuda:0")
    flags = fm.FMAP_PLAN_EXP_RECURRENCE if prec == "rec" else 0
    p_prec = "fp64" if prec == "rec" else prec
    direct = fm.Plan(g, insts[0].n_sft, 5, p_prec, flags)
    graph = fm.Plan(g, insts[0].n_sft, 5, p_prec, flags | fm.FMAP_PLAN_GRAPH)
    t = torch.from_numpy(insts[0].t).to(dev)
    a = torch.from_numpy(np.ascontiguousarray(insts[0].antenna)).to(dev)
    x = torch.from_numpy(np.ascontiguousarray(insts[0].fafb)).to(dev)
    m = torch.empty((5, g.n_t0, g.n_tau), device=dev)
    s = torch.empty((5, 32), dtype=torch.uint8, device=dev)
    for inst in insts + insts[:1]:   # the same buffers, the data replaced in place
        t.copy_(torch.from_numpy(inst.t))
        a.copy_(torch.from_numpy(np.ascontiguousarray(inst.antenna)))
        x.copy_(torch.from_numpy(np.ascontiguousarray(inst.fafb)))
        m_ref, s_ref = direct.compute(t, a, x)
        graph.compute(t, a, x, out_map=m, out_summary=s)
        torch.cuda.synchronize()
        assert graph.status() == fm.FMAP_OK and direct.status() == fm.FMAP_OK
        assert torch.equal(m, m_ref) and torch.equal(s, s_ref)
    # another output buffer: captured again, same results
    m2 = torch.empty_like(m)
    graph.compute(t, a, x, out_map=m2, out_summary=s)
    torch.cuda.synchronize()
    assert torch.equal(m2, m)
    # a setting changed after the capture: the next call captures anew
    logb = fm.summary_to_numpy(s)["logB"].copy()
    graph.set_log_prior(1.5)
    graph.compute(t, a, x, out_map=m2, out_summary=s)
    torch.cuda.synchronize()
    assert np.allclose(fm.summary_to_numpy(s)["logB"], logb + 1.5, rtol=0, atol=1e-12,
                       equal_nan=True)
    graph.set_log_prior(0.0)
    graph.compute(t, a, x, out_map=m2, out_summary=s)
    torch.cuda.synchronize()
    ref, valid, _ = oracle_map(insts[0])
    check_map(m2.cpu().numpy().astype(np.float64), ref, valid, TOL[prec])
    check_summary(fm.summary_to_numpy(s), ref, valid, TOL[prec], LOGB_TOL)
    direct.close()
    graph.close()
