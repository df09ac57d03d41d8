"""Pins of the CPU oracle against what the paper and the mathematics fix.

Every check here is independent of the oracle's own code path: closed forms
(geometric series of the exponential window, the paper's summation counts of
App. A), an independent linear solve of Eq. (F_xMx), the chi^2_4 law of 2F in
Gaussian noise, the exact noise-free value of an injected signal, a different
algorithm (the decayed-suffix recurrence) for exponential sums, scipy's
logsumexp, and the multi-detector form of the sums.
"""

import json
import math
import os

import numpy as np
import pytest

import oracle
import synth
from synth import EXP, RECT, T_SFT, Grid

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_printed.json")


def _gapfree(n, n_templates=1, dtype=np.float64, seed=11, grid=None):
    grid = grid or Grid(0, T_SFT, 1, 2 * T_SFT, T_SFT, 1, RECT)
    return synth.make_instance(seed, n_slots=n, n_templates=n_templates, grid=grid, dtype=dtype)


def _linsolve_F(s):
    """F from Eq. (F_xMx): 0.5 x^T M^{-1} x with the 4x4 antenna matrix
    M = 0.5 diag(M2, M2), M2 = [[A, C], [C, B]], x = (Re Fa, Re Fb, Im Fa, Im Fb)."""
    A, B, C, far, fai, fbr, fbi = s
    M2 = np.array([[A, C], [C, B]])
    M = 0.5 * np.block([[M2, np.zeros((2, 2))], [np.zeros((2, 2)), M2]])
    x = np.array([far, fbr, fai, fbi])
    return 0.5 * x @ np.linalg.solve(M, x)


def test_golden_facts_present():
    g = json.load(open(GOLDEN))
    assert g["t_sft_seconds"]["value"] == T_SFT
    assert g["min_sfts_per_cell"]["value"] == 2
    assert g["exp_cutoff_efolds"]["value"] == 3


@pytest.mark.parametrize("window", [RECT, EXP])
def test_counts_match_appendix_formulas(window):
    """Per-cell atom counts are the summands of Eq. (Nsums-rect)/(Nsums-exp):
    floor(min(T_data - t0, L) / T_sft), L = tau or 3 tau, gap-free data,
    including windows that run past the data end (App. A convention)."""
    n = 40
    g = json.load(open(GOLDEN))
    efolds = g["exp_cutoff_efolds"]["value"]
    grid = Grid(0, 900, 90, 500, 1300, 70, window)
    inst = _gapfree(n, grid=grid)
    _, cnt = oracle.sums(inst.t, inst.antenna, inst.fafb, grid.as_tuple())
    t_data = n * T_SFT
    t0 = grid.t0()[:, None]
    L = grid.tau()[None, :] * (1 if window == RECT else efolds)
    # atoms start on multiples of T_sft: the first one inside is ceil(t0/T_sft)
    first = -(-t0 // T_SFT) * T_SFT
    expect = np.clip(np.minimum(t_data - first, (t0 + L) - first) // T_SFT, 0, None)
    expect = np.where(first < t_data, expect, 0)
    assert np.array_equal(cnt, expect)


@pytest.mark.parametrize("cut8", [1, 8, 20, 40])
def test_counts_with_other_exp_cuts(cut8):
    """The exp window cut as a parameter: L(tau) = floor(cut8 tau / 8) in
    place of 3 tau in the per-cell count floor(min(T_data - t0, L) / T_sft)
    of App. A (gap-free data, windows past the data end included)."""
    n = 40
    grid = Grid(0, 900, 90, 500, 1300, 70, EXP, T_SFT, cut8)
    inst = _gapfree(n, grid=grid)
    _, cnt = oracle.sums(inst.t, inst.antenna, inst.fafb, grid.as_tuple())
    t_data = n * T_SFT
    t0 = grid.t0()[:, None]
    L = cut8 * grid.tau()[None, :] // 8
    first = -(-t0 // T_SFT) * T_SFT
    expect = np.clip(np.minimum(t_data - first, (t0 + L) - first) // T_SFT, 0, None)
    expect = np.where(first < t_data, expect, 0)
    assert np.array_equal(cnt, expect)
    # the default (0) is the 3 tau cut of Eq. winexp
    _, c3 = oracle.sums(inst.t, inst.antenna, inst.fafb, Grid(0, 900, 90, 500, 1300, 70, EXP).as_tuple())
    _, c24 = oracle.sums(inst.t, inst.antenna, inst.fafb,
                         Grid(0, 900, 90, 500, 1300, 70, EXP, T_SFT, 24).as_tuple())
    assert np.array_equal(c3, c24)


def test_host_count_terms_follow_the_cut():
    """fmap_count_terms (host code of the library) counts the same windows as
    the oracle for several cuts."""
    fm = pytest.importorskip("paper_1805_05652_gb300")
    fm.build()
    inst = synth.make_instance(12, n_det=2, presence=0.8, n_merged=90,
                               grid=Grid(0, 1, 1, 1, 1, 1, EXP), dtype=np.float64)
    for cut8 in (0, 3, 8, 17, 64):
        grid = Grid(-4000, 1500, 40, 900, 2100, 33, EXP, T_SFT, cut8)
        _, cnt = oracle.sums(inst.t, inst.antenna, inst.fafb, grid.as_tuple())
        terms, cells2 = fm.fmap_count_terms(grid, inst.t)
        assert terms == int(cnt[cnt >= 2].sum()) and cells2 == int((cnt >= 2).sum())


def test_counts_on_grid_equal_paper_sum():
    """On the paper's T_sft-step grids the total count equals Eq. (Nsums-exp)
    and its embedded-case closed form 3 N_t0 N_tau (tau_min + Delta_tau/2)/T_sft."""
    n = 300
    grid = Grid(0, T_SFT, 20, T_SFT, T_SFT, 30, EXP)           # embedded: 20 + 90 < 300
    inst = _gapfree(n, grid=grid)
    _, cnt = oracle.sums(inst.t, inst.antenna, inst.fafb, grid.as_tuple())
    t_data = n * T_SFT
    nsums = sum(min(t_data - t0, 3 * tau) // T_SFT for t0 in grid.t0() for tau in grid.tau())
    assert cnt.sum() == nsums
    dtau_span = grid.tau()[-1] - grid.tau()[0]
    closed = 3 * grid.n_t0 * grid.n_tau * (grid.tau_min + 0.5 * dtau_span) / T_SFT
    assert cnt.sum() == pytest.approx(closed, rel=0, abs=1e-9)


def test_rect_timing_layout_ratio():
    """App. A: in the timing layout (t0 in [T0, T_data - 2 T_sft],
    tau in [2 T_sft, T_data], steps T_sft) the per-row running-sum steps
    sum to ~0.5 N_t0 tau_max / T_sft."""
    n = 400
    g = json.load(open(GOLDEN))
    grid = Grid(0, T_SFT, n - 1, 2 * T_SFT, T_SFT, n - 1, RECT)
    inst = _gapfree(n, grid=grid)
    _, cnt = oracle.sums(inst.t, inst.antenna, inst.fafb, grid.as_tuple())
    steps = cnt[:, -1].sum()                          # longest window per row
    ratio = steps / (grid.n_t0 * grid.tau()[-1] / T_SFT)
    assert ratio == pytest.approx(g["nsums_rect_timing_layout_ratio"]["value"], abs=2.0 / n)


def test_two_sft_minimum():
    """Sec. 4.1: tau = 2 T_sft holds exactly 2 SFTs and is a valid cell; one SFT
    is not; the last row t0 = T_obs - 2 T_sft still holds 2 SFTs."""
    n = 30
    grid = Grid(0, T_SFT, n, T_SFT, T_SFT, 3, RECT)
    inst = _gapfree(n, grid=grid, seed=3)
    m2, val, cnt = oracle.fmap(inst.t, inst.antenna, inst.fafb, grid.as_tuple())
    assert (cnt[: n - 1, 0] == 1).all() and not val[0, :, 0].any()
    assert (m2[0, :, 0] == 0).all()
    assert (cnt[: n - 2, 1] == 2).all() and val[0, : n - 2, 1].all()
    assert cnt[n - 2, 1] == 2 and cnt[n - 1, 1] == 1


def test_inclusive_reading_adds_one_atom():
    """The literal reading t in [t0, t0 + tau] of Eq. (winrect) counts one more
    SFT than the end-of-SFT reading for on-grid windows inside the data."""
    n = 50
    grid = Grid(0, T_SFT, 10, 2 * T_SFT, T_SFT, 10, RECT)
    inst = _gapfree(n, grid=grid)
    _, c0 = oracle.sums(inst.t, inst.antenna, inst.fafb, grid.as_tuple())
    _, c1 = oracle.sums(inst.t, inst.antenna, inst.fafb, grid.as_tuple(), inclusive=True)
    assert np.array_equal(c1, c0 + 1)


@pytest.mark.parametrize("offset", [0, 600])
@pytest.mark.parametrize("tau_sft", [0.5, 1, 3.25, 40])
def test_exp_window_geometric_series(offset, tau_sft):
    """Constant atoms turn the exponential window sums into geometric series:
    Fa = q sum_k r^k with r = e^{-T_sft/tau}, q = e^{-offset/tau} (window
    weight, Eq. winexp) and A = q^2 sum_k r^{2k} (squared weight)."""
    n = 200
    tau = int(tau_sft * T_SFT)
    t = np.arange(n, dtype=np.int64) * T_SFT
    ant = np.stack([np.ones(n), 2 * np.ones(n), 0.5 * np.ones(n)])
    x = np.zeros((1, 4, n))
    x[0, 0] = 1.0
    x[0, 3] = -2.0
    t0 = 10 * T_SFT - offset
    grid = (t0, 1, 1, tau, 1, 1, T_SFT, EXP)
    s, cnt = oracle.sums(t, ant, x, grid)
    K = int(cnt[0, 0])
    assert K == (t0 + 3 * tau - 10 * T_SFT) // T_SFT
    r = math.exp(-T_SFT / tau)
    q = math.exp(-offset / tau)
    geo1 = q * (1 - r ** K) / (1 - r)
    geo2 = q * q * (1 - r ** (2 * K)) / (1 - r * r)
    A, B, C, far, fai, fbr, fbi = s[0, 0, 0]
    assert A == pytest.approx(geo2, rel=1e-12)
    assert B == pytest.approx(2 * geo2, rel=1e-12)
    assert C == pytest.approx(0.5 * geo2, rel=1e-12)
    assert far == pytest.approx(geo1, rel=1e-12)
    assert fbi == pytest.approx(-2 * geo1, rel=1e-12)
    assert fai == 0 and fbr == 0


def test_rect_window_constant_atoms():
    t = np.arange(100, dtype=np.int64) * T_SFT
    ant = np.ones((3, 100))
    x = np.ones((1, 4, 100))
    s, cnt = oracle.sums(t, ant, x, (5 * T_SFT, 1, 1, 7 * T_SFT, 1, 1, T_SFT, RECT))
    assert cnt[0, 0] == 7
    assert np.allclose(s[0, 0, 0], 7.0, rtol=0, atol=0)


def test_F_closed_form_matches_linear_solve():
    """Eq. (F_FaFb) equals the 4-dimensional form Eq. (F_xMx) solved as a
    linear system, for random positive-definite antenna matrices."""
    rng = np.random.default_rng(0)
    for _ in range(200):
        a, b = rng.random(6) + 0.1, rng.random(6) + 0.1
        A, B, C = (a * a).sum(), (b * b).sum(), (a * b).sum()
        fa = rng.normal(size=2)
        fb = rng.normal(size=2)
        s = (A, B, C, fa[0], fa[1], fb[0], fb[1])
        twoF, valid = oracle.twoF_from_sums(*s, count=6)
        assert valid
        assert twoF == pytest.approx(2 * _linsolve_F(s), rel=1e-11)


def test_cells_linear_solve_and_full_span():
    """A rectangular window over all data is the ordinary full-span
    F-statistic (Sec. 2, after Eq. F_FaFb), computed here from plain column
    sums of the atoms and the linear-solve form of Eq. (F_xMx)."""
    inst = synth.make_instance(5, n_det=2, presence=0.8, n_merged=120, n_templates=3,
                               grid=Grid(0, T_SFT, 1, 1, 1, 1, RECT), dtype=np.float64)
    t_data = int(inst.t[-1]) + T_SFT
    grid = (int(inst.t[0]), 1, 1, t_data - int(inst.t[0]), 1, 1, T_SFT, RECT)
    for j in range(3):
        out, val, cnt, sm = oracle.cells(inst.t, inst.antenna, inst.fafb, grid, [[j, 0, 0]],
                                         want_sums=True)
        full = np.concatenate([inst.antenna.sum(axis=1), inst.fafb[j].sum(axis=1)])
        assert cnt[0] == inst.n_sft and val[0]
        assert np.allclose(sm[0], full, rtol=1e-13)
        assert out[0] == pytest.approx(2 * _linsolve_F(full), rel=1e-11)


@pytest.mark.parametrize("window,tau_sft", [(RECT, 3), (RECT, 25), (EXP, 2), (EXP, 12)])
def test_noise_is_chi2_4(window, tau_sft):
    """In Gaussian noise 2F of a fixed window follows chi^2 with 4 degrees of
    freedom (F is a log-likelihood ratio over 4 amplitudes, Sec. 2, Eq.
    F_OSG): mean 4, variance 8.  This pins the squared window weight of the
    antenna sums and the factor 2 of 2F."""
    from scipy import stats

    T = 12000
    grid = Grid(0, T_SFT, 1, T_SFT, T_SFT, 1, window)
    inst = synth.make_instance(21, n_det=2, presence=0.85, n_merged=60, n_templates=T,
                               grid=grid, dtype=np.float64)
    g = (int(inst.t[5]), 1, 1, int(tau_sft * T_SFT), 1, 1, T_SFT, window)
    idx = np.stack([np.arange(T), np.zeros(T, int), np.zeros(T, int)], axis=1)
    v2F, val, cnt = oracle.cells(inst.t, inst.antenna, inst.fafb, g, idx)
    assert val.all() and cnt[0] >= 2
    sem = math.sqrt(8.0 / T)
    assert abs(v2F.mean() - 4.0) < 5 * sem
    assert abs(v2F.var() - 8.0) < 0.6
    assert stats.kstest(v2F, stats.chi2(4).cdf).pvalue > 1e-4


@pytest.mark.parametrize("window", [RECT, EXP])
def test_noise_free_injection_exact(window):
    """Noise-free data with an injected transient: at the true (t0, tau) the
    oracle returns 2F = rho^2 = 2 u^H M u exactly (the synthesis scales the
    signal energy sum w^2 |a A + b B|^2 to rho^2 / 2), and that cell is the
    unique argmax of the map."""
    n = 160
    grid = Grid(0, T_SFT, 60, 2 * T_SFT, T_SFT, 70, window)
    m_true, n_true = 23, 31
    t0, tau = m_true * T_SFT, grid.tau()[n_true]
    inst = synth.make_instance(8, n_det=2, presence=1.0, n_slots=n, grid=grid,
                               injections=[(0, window, t0, int(tau), 150.0)],
                               dtype=np.float64, noise_scale=0.0)
    m2, val, _ = oracle.fmap(inst.t, inst.antenna, inst.fafb, grid.as_tuple())
    assert m2[0, m_true, n_true] == pytest.approx(150.0, rel=1e-12)
    s = oracle.summary(m2, val)
    assert (s["m"][0], s["n"][0]) == (m_true, n_true)
    others = np.delete(m2[0].ravel(), m_true * grid.n_tau + n_true)
    assert others.max() < 150.0 * (1 - 1e-9)


def test_injection_recovered_in_noise():
    inst = synth.config_small_rect(dtype=np.float64)
    m2, val, _ = oracle.fmap(inst.t, inst.antenna, inst.fafb, inst.grid.as_tuple())
    s = oracle.summary(m2, val)
    assert abs(int(s["m"][0]) - 40) <= 6 and abs(int(s["n"][0]) - 58) <= 8
    assert s["max2F"][0] > 60


@pytest.mark.parametrize("cut8", [0, 8, 40])
def test_exp_sums_match_decayed_suffix_recurrence(cut8):
    """A different algorithm for the exponential sums: the backward
    recurrence E[i] = x_i + e^{-(t_{i+1} - t_i)/s} E[i+1] gives
    sum_{i0 <= a < j} e^{-(t_a - t0)/s} x_a
      = e^{-(t_{i0} - t0)/s} (E[i0] - e^{-(t_j - t_{i0})/s} E[j]),
    with s = tau for Fa, Fb and tau / 2 for the squared weights."""
    inst = synth.make_instance(31, n_det=2, presence=0.7, n_merged=150, n_templates=2,
                               grid=Grid(0, 1, 1, 1, 1, 1, EXP), dtype=np.float64)
    grid = Grid(-3000, 2500, 30, 700, 4100, 25, EXP, T_SFT, cut8)
    s, cnt = oracle.sums(inst.t, inst.antenna, inst.fafb, grid.as_tuple())
    t = inst.t.astype(np.float64)
    n = inst.n_sft
    L8 = cut8 or 24

    def suffix(x, scale):
        E = np.zeros(n + 1)
        for i in range(n - 1, -1, -1):
            decay = math.exp(-(t[i + 1] - t[i]) / scale) if i + 1 < n else 0.0
            E[i] = x[i] + decay * E[i + 1]
        return E

    for ni, tau in enumerate(grid.tau()):
        Es = [suffix(inst.antenna[k], tau / 2) for k in range(3)]
        Ex = [[suffix(inst.fafb[j, k], tau) for k in range(4)] for j in range(2)]
        for mi, t0 in enumerate(grid.t0()):
            i0 = int(np.searchsorted(inst.t, t0, side="left"))
            j = i0
            while j < n and 8 * (inst.t[j] + T_SFT - t0) <= L8 * tau:
                j += 1
            assert cnt[mi, ni] == j - i0
            if j == i0:
                continue
            tj = t[j] if j < n else 0.0

            def win(E, scale):
                tail = math.exp(-(tj - t[i0]) / scale) * E[j] if j < n else 0.0
                return math.exp(-(t[i0] - t0) / scale) * (E[i0] - tail)

            for jj in range(2):
                ref = [win(Es[k], tau / 2) for k in range(3)] + [win(Ex[jj][k], tau) for k in range(4)]
                assert np.allclose(s[jj, mi, ni], ref, rtol=1e-10, atol=1e-12)


def test_multidetector_atoms_sum_per_detector():
    """Merged atoms (sums over detectors at a timestamp) give the same windowed
    sums as summing every per-detector atom directly: the window depends on
    time only."""
    grid = Grid(-2000, 3100, 25, 900, 2900, 20, EXP)
    inst = synth.make_instance(17, n_det=3, presence=0.6, n_merged=90, n_templates=2,
                               grid=grid, dtype=np.float64, keep_detectors=True)
    d = inst.detectors
    pres = d["present"]
    ts, ant, x = [], [], [[] for _ in range(2)]
    for k in range(pres.shape[0]):
        for a in np.nonzero(pres[k])[0]:
            ts.append(inst.t[a])
            ant.append([d["a"][k, a] ** 2, d["b"][k, a] ** 2, d["a"][k, a] * d["b"][k, a]])
            for j in range(2):
                fa, fb = d["fa"][j, k, a], d["fb"][j, k, a]
                x[j].append([fa.real, fa.imag, fb.real, fb.imag])
    ts = np.array(ts, dtype=np.int64)
    ant = np.array(ant).T.copy()
    x = np.array([np.array(xx).T for xx in x])
    for window in (RECT, EXP):
        g = grid.with_window(window).as_tuple()
        s_merged, _ = oracle.sums(inst.t, inst.antenna, inst.fafb, g)
        s_det, _ = oracle.sums(ts, ant, x, g)
        assert np.allclose(s_merged, s_det, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("window", [RECT, EXP])
def test_fast_mode_equals_direct(window):
    """The paper's per-row algorithms (Sec. 3) agree with the direct
    definition, with gaps, off-grid steps, windows before the data and past
    its end, and per-template antenna rows."""
    grid = Grid(-5000, 1700, 40, 900, 2300, 45, window)
    inst = synth.make_instance(4, n_det=2, presence=0.75, n_merged=70, n_templates=3,
                               grid=grid, shared_antenna=False, dtype=np.float64)
    a = oracle.fmap(inst.t, inst.antenna, inst.fafb, grid.as_tuple(), mode="direct")
    b = oracle.fmap(inst.t, inst.antenna, inst.fafb, grid.as_tuple(), mode="fast")
    assert np.array_equal(a[1], b[1]) and np.array_equal(a[2], b[2])
    assert np.allclose(a[0], b[0], rtol=1e-11, atol=1e-11)
    shared = synth.make_instance(4, n_det=2, presence=0.75, n_merged=70, n_templates=3,
                                 grid=grid, dtype=np.float64)
    a = oracle.fmap(shared.t, shared.antenna, shared.fafb, grid.as_tuple(), mode="direct")
    b = oracle.fmap(shared.t, shared.antenna, shared.fafb, grid.as_tuple(), mode="fast")
    assert np.allclose(a[0], b[0], rtol=1e-11, atol=1e-11)


def test_cells_equal_map():
    inst = synth.config_small_rect(dtype=np.float64)
    m2, val, cnt = oracle.fmap(inst.t, inst.antenna, inst.fafb, inst.grid.as_tuple())
    rng = np.random.default_rng(2)
    idx = np.stack([np.zeros(300, int), rng.integers(0, 200, 300), rng.integers(0, 200, 300)], 1)
    v, ok, c = oracle.cells(inst.t, inst.antenna, inst.fafb, inst.grid.as_tuple(), idx)
    assert np.array_equal(v, m2[0, idx[:, 1], idx[:, 2]])
    assert np.array_equal(ok, val[0, idx[:, 1], idx[:, 2]])


def test_logB_special_cases_and_logsumexp():
    """logB = ln((1/N_valid) sum_valid e^{F}): a constant map F = c gives c; one
    valid cell gives its F; invalid cells are ignored; it equals scipy's
    logsumexp(F) - ln N_valid; ties in max 2F go to the lowest m N_tau + n."""
    from scipy.special import logsumexp

    c = 7.25
    m = np.full((1, 5, 6), 2 * c)
    v = np.ones_like(m, dtype=bool)
    s = oracle.summary(m, v)
    assert s["logB"][0] == pytest.approx(c, abs=1e-13)
    assert (s["m"][0], s["n"][0]) == (0, 0)
    v2 = np.zeros_like(v)
    v2[0, 3, 4] = True
    m2 = m.copy()
    m2[0, 3, 4] = 31.0
    m2[0, 1, 1] = 99.0                       # invalid cell: ignored
    s = oracle.summary(m2, v2)
    assert s["logB"][0] == pytest.approx(15.5, abs=1e-13)
    assert (s["m"][0], s["n"][0], s["n_valid"][0]) == (3, 4, 1)
    assert s["max2F"][0] == 31.0
    s = oracle.summary(m2, np.zeros_like(v))
    assert np.isnan(s["logB"][0]) and s["m"][0] == -1 and s["n_valid"][0] == 0
    rng = np.random.default_rng(3)
    mm = rng.chisquare(4, size=(3, 40, 50)) * 3
    vv = rng.random(mm.shape) > 0.1
    s = oracle.summary(mm, vv)
    for j in range(3):
        F = 0.5 * mm[j][vv[j]]
        assert s["logB"][j] == pytest.approx(logsumexp(F) - math.log(F.size), abs=1e-12)
    mt = np.zeros((1, 4, 4))
    mt[0, 2, 1] = mt[0, 1, 3] = 5.0
    s = oracle.summary(mt, np.ones_like(mt, dtype=bool))
    assert (s["m"][0], s["n"][0]) == (1, 3)
    s = oracle.summary(m, v, log_prior_const=-1.5)
    assert s["logB"][0] == pytest.approx(c - 1.5, abs=1e-13)


def _axes_grid(window, cut8=0):
    """A non-uniform grid: sorted random t0 values (some before the data,
    some past its end) and tau values with uneven steps."""
    rng = np.random.default_rng(5 + window)
    t0 = np.sort(rng.choice(np.arange(-3 * T_SFT, 40 * T_SFT, 97), size=23, replace=False))
    tau = np.sort(rng.choice(np.arange(T_SFT // 2, 30 * T_SFT, 113), size=17, replace=False))
    return Grid(0, 1, len(t0), 1, 1, len(tau), window, T_SFT, cut8,
                tuple(int(v) for v in t0), tuple(int(v) for v in tau))


@pytest.mark.parametrize("window", [RECT, EXP])
def test_explicit_axes_equal_uniform_grid(window):
    """Explicit axes holding a uniform grid's own values give that grid's
    sums and maps exactly (direct and per-row modes)."""
    grid = Grid(-2000, 1700, 30, 900, 2300, 25, window)
    inst = synth.make_instance(8, n_det=2, presence=0.8, n_merged=120, n_templates=2,
                               grid=grid, dtype=np.float64)
    ax = Grid(7, 3, grid.n_t0, 11, 5, grid.n_tau, window, T_SFT, 0,
              tuple(int(v) for v in grid.t0()), tuple(int(v) for v in grid.tau()))
    s_u, c_u = oracle.sums(inst.t, inst.antenna, inst.fafb, grid.as_tuple())
    s_a, c_a = oracle.sums(inst.t, inst.antenna, inst.fafb, ax.as_tuple())
    assert np.array_equal(c_u, c_a) and np.array_equal(s_u, s_a)
    for mode in ("direct", "fast"):
        m_u, v_u, _ = oracle.fmap(inst.t, inst.antenna, inst.fafb, grid.as_tuple(), mode=mode)
        m_a, v_a, _ = oracle.fmap(inst.t, inst.antenna, inst.fafb, ax.as_tuple(), mode=mode)
        assert np.array_equal(v_u, v_a) and np.array_equal(m_u, m_a)


@pytest.mark.parametrize("window,cut8", [(RECT, 0), (EXP, 0), (EXP, 12)])
def test_explicit_axes_brute_force(window, cut8):
    """Window sums on a non-uniform grid against a plain double loop over the
    atoms with the membership rule t0 <= t, t + T_sft <= t0 + L(tau) and the
    weights of Eq. winrect / winexp (w for Fa, Fb; w^2 for A, B, C); the
    per-row fast mode agrees with the direct one."""
    grid = _axes_grid(window, cut8)
    inst = synth.make_instance(9, n_det=2, presence=0.7, n_merged=30, n_templates=2,
                               grid=Grid(0, 1, 1, 1, 1, 1, window), dtype=np.float64)
    s, cnt = oracle.sums(inst.t, inst.antenna, inst.fafb, grid.as_tuple())
    L8 = 8 if window == RECT else (cut8 or 24)
    for mi, t0 in enumerate(grid.t0()):
        for ni, tau in enumerate(grid.tau()):
            ref = np.zeros((2, 7))
            c = 0
            for a, t in enumerate(inst.t):
                if t < t0 or 8 * (t + T_SFT - t0) > L8 * tau:
                    continue
                w = 1.0 if window == RECT else math.exp(-(t - t0) / tau)
                c += 1
                for j in range(2):
                    ref[j, :3] += w * w * inst.antenna[:, a]
                    ref[j, 3:] += w * inst.fafb[j, :, a]
            assert cnt[mi, ni] == c
            assert np.allclose(s[:, mi, ni], ref, rtol=1e-12, atol=1e-13)
    m_d, v_d, _ = oracle.fmap(inst.t, inst.antenna, inst.fafb, grid.as_tuple(), mode="direct")
    m_f, v_f, _ = oracle.fmap(inst.t, inst.antenna, inst.fafb, grid.as_tuple(), mode="fast")
    assert np.array_equal(v_d, v_f)
    assert np.allclose(m_d, m_f, rtol=1e-10, atol=1e-10)


def _table_grid(table, cut8=0, window=synth.TABLE):
    return Grid(-2000, 1700, 30, 900, 2300, 25, window, T_SFT, cut8, None, None,
                tuple(float(v) for v in table))


@pytest.mark.parametrize("mode", ["direct", "fast"])
def test_table_window_constant_is_rect(mode):
    """A table window w = 1 on [0, 1] (cut 8 eighths: support [t0, t0 + tau])
    is the rectangular window of Eq. winrect: identical sums and maps."""
    inst = synth.make_instance(21, n_det=2, presence=0.8, n_merged=120, n_templates=2,
                               grid=Grid(0, 1, 1, 1, 1, 1, RECT), dtype=np.float64)
    rect = Grid(-2000, 1700, 30, 900, 2300, 25, RECT)
    tab = _table_grid(np.ones(7), cut8=8)
    s_r, c_r = oracle.sums(inst.t, inst.antenna, inst.fafb, rect.as_tuple())
    s_t, c_t = oracle.sums(inst.t, inst.antenna, inst.fafb, tab.as_tuple())
    assert np.array_equal(c_r, c_t) and np.array_equal(s_r, s_t)
    m_r, v_r, _ = oracle.fmap(inst.t, inst.antenna, inst.fafb, rect.as_tuple(), mode=mode)
    m_t, v_t, _ = oracle.fmap(inst.t, inst.antenna, inst.fafb, tab.as_tuple(), mode=mode)
    assert np.array_equal(v_r, v_t) and np.array_equal(m_r, m_t)


def test_table_window_sampled_exponential_within_interpolation_bound():
    """Samples of e^{-x} on [0, 3] joined linearly reproduce the exponential
    window of Eq. winexp to within the linear-interpolation bound h^2/8 max|w''|
    (h the sample step) on every weight, plus the float32 rounding of the
    samples: |S_table - S_exp| <= (bound) sum |x| per cell and row."""
    n = 301
    h = 3.0 / (n - 1)
    w = np.exp(-np.linspace(0.0, 3.0, n))
    inst = synth.make_instance(22, n_det=2, presence=0.85, n_merged=150, n_templates=2,
                               grid=Grid(0, 1, 1, 1, 1, 1, EXP), dtype=np.float64)
    ex = Grid(-2000, 1700, 30, 900, 2300, 25, EXP)
    tab = _table_grid(w)
    s_e, c_e = oracle.sums(inst.t, inst.antenna, inst.fafb, ex.as_tuple())
    s_t, c_t = oracle.sums(inst.t, inst.antenna, inst.fafb, tab.as_tuple())
    assert np.array_equal(c_e, c_t)
    dw = h * h / 8.0 + 1.2e-7                       # per weight (w <= 1, w'' <= 1)
    absx = np.abs(np.concatenate([inst.antenna, inst.fafb.reshape(-1, inst.n_sft)]))
    # sum of |x| over each cell's window, by the oracle itself on |x| rows with w = 1
    flat = Grid(-2000, 1700, 30, 900, 2300, 25, synth.TABLE, T_SFT, 0, None, None, (1.0, 1.0))
    s_abs, _ = oracle.sums(inst.t, absx[:3], absx[3:].reshape(2, 4, -1), flat.as_tuple())
    bound = np.concatenate([2 * dw * s_abs[..., :3], dw * s_abs[..., 3:]], axis=-1) + 1e-12
    assert np.all(np.abs(s_t - s_e) <= bound)


@pytest.mark.parametrize("cut8", [0, 12])
def test_table_window_brute_force(cut8):
    """Window sums of a random table window against a plain loop over the
    atoms with numpy's linear interpolation of the samples (w for Fa, Fb;
    w^2 for A, B, C; 0 past the support)."""
    rng = np.random.default_rng(3)
    table = rng.uniform(0.0, 2.0, size=17).astype(np.float32)
    grid = Grid(-2500, 1300, 20, 700, 1900, 18, synth.TABLE, T_SFT, cut8, None, None,
                tuple(float(v) for v in table))
    inst = synth.make_instance(23, n_det=1, presence=0.8, n_merged=40, n_templates=2,
                               grid=Grid(0, 1, 1, 1, 1, 1, EXP), dtype=np.float64)
    s, cnt = oracle.sums(inst.t, inst.antenna, inst.fafb, grid.as_tuple())
    X = (cut8 or 24) / 8.0
    xs = np.linspace(0.0, X, len(table))
    for mi, t0 in enumerate(grid.t0()):
        for ni, tau in enumerate(grid.tau()):
            ref = np.zeros((2, 7))
            c = 0
            for a, t in enumerate(inst.t):
                if t < t0 or 8 * (t + T_SFT - t0) > (cut8 or 24) * tau:
                    continue
                w = float(np.interp((t - t0) / tau, xs, table.astype(np.float64)))
                c += 1
                for j in range(2):
                    ref[j, :3] += w * w * inst.antenna[:, a]
                    ref[j, 3:] += w * inst.fafb[j, :, a]
            assert cnt[mi, ni] == c
            assert np.allclose(s[:, mi, ni], ref, rtol=1e-10, atol=1e-12)
