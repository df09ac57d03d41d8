"""Synthetic atoms and (t0, tau) grids for the workloads of the F-map.

Data model (Sec. 2, Sec. 3 and Sec. 4.1 of arXiv:1805.05652):

* SFTs of length ``T_SFT = 1800`` s start at integer-second timestamps
  ``t = k * T_SFT`` (slot ``k``); a detector may miss a slot (a gap).
* Each detector ``d`` has the antenna-pattern coefficients
  ``a_d(t) = 0.4 + 0.3 cos(Omega t + phi_a)`` and
  ``b_d(t) = 0.2 + 0.3 sin(Omega t + phi_b)`` (sidereal ``Omega``, seeded
  phases), an illustrative stand-in for the real detector response.
* Noise: one complex Gaussian ``z ~ CN(0, 1)`` per detector and SFT
  (real and imaginary parts each of variance 1/2), entering both projections
  as ``Fa = a z`` and ``Fb = b z``.  Drawing ``Fa`` and ``Fb`` independently
  would give them the wrong covariance; with one shared ``z`` the matched
  filter outputs have covariance equal to the antenna matrix, which is what
  the F-statistic assumes.
* Signal: ``z -> z + w(t) (a A + b B)`` with complex amplitudes ``(A, B)`` and
  the transient envelope ``w`` of Eq. (winrect) / (winexp).  The amplitude is
  scaled so that the signal energy ``sum_{d,SFT} w^2 |a A + b B|^2`` equals
  ``rho2 / 2``.
* Atoms of a timestamp sum over the detectors present there ("merged atoms"):
  ``a2 = sum a_d^2``, ``b2 = sum b_d^2``, ``ab = sum a_d b_d``,
  ``Fa = sum a_d (z_d + s_d)``, ``Fb = sum b_d (z_d + s_d)``; they are stored
  as real32 like the paper's atoms.

Window membership (used here only for the signal envelope): an SFT starting
at ``t`` lies inside the window of ``(t0, tau)`` when ``t0 <= t`` and the SFT
ends no later than ``t0 + tau`` (rectangular) or ``t0 + 3 tau`` (exponential,
weight ``exp(-(t - t0)/tau)``).  This is the reading that reproduces the
paper's summation counts (App. A, Eq. Nsums-rect / Nsums-exp) and its
two-SFT minimum (Sec. 4.1).

Layouts (shared with the library's C interface): timestamps int64 ``[N]``;
antenna rows ``[3][N]`` (a2, b2, ab) when shared by all templates, else
``[T][3][N]``; data rows ``[T][4][N]`` (Re Fa, Im Fa, Re Fb, Im Fb).
"""

from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

T_SFT = 1800
OMEGA_SID = 2.0 * math.pi / 86164.0
RECT = 0
EXP = 1
TABLE = 2   # generic window function given by samples
BASE_SEED = 20180515


def philox(*key: int) -> np.random.Generator:
    """Counter-based generator keyed by up to two integers."""
    k = list(key) + [0] * (2 - len(key))
    return np.random.Generator(np.random.Philox(key=np.array(k[:2], dtype=np.uint64)))


def rect(t, t0, tau, t_sft=T_SFT):
    """Envelope of a rectangular transient (Eq. winrect), SFT-start convention."""
    t = np.asarray(t, dtype=np.int64)
    inside = (t >= t0) & (t + t_sft <= t0 + tau)
    return inside.astype(np.float64)


def exp_(t, t0, tau, t_sft=T_SFT):
    """Envelope of an exponential transient cut after 3 tau (Eq. winexp)."""
    t = np.asarray(t, dtype=np.int64)
    inside = (t >= t0) & (t + t_sft <= t0 + 3 * tau)
    dt = (t - t0).astype(np.float64)
    return np.where(inside, np.exp(-np.where(inside, dt, 0.0) / float(tau)), 0.0)


def envelope(window, t, t0, tau, t_sft=T_SFT):
    return rect(t, t0, tau, t_sft) if window == RECT else exp_(t, t0, tau, t_sft)


@dataclass
class Grid:
    """Uniform (t0, tau) grid: t0_m = t0_min + m dt0, tau_n = tau_min + n dtau
    (integer seconds, Eq. Fmn).  exp_cut8: exponential window length in
    eighths of tau (0: Eq. winexp's 3 tau)."""

    t0_min: int
    dt0: int
    n_t0: int
    tau_min: int
    dtau: int
    n_tau: int
    window: int = RECT
    t_sft: int = T_SFT
    exp_cut8: int = 0
    # explicit axes (a non-uniform grid): strictly increasing t0 and tau
    # values replacing t0_min + m dt0 and tau_min + n dtau
    t0_values: tuple | None = None
    tau_values: tuple | None = None
    # TABLE windows: samples of w on [0, exp_cut8 / 8] (x = (t - t0) / tau)
    window_table: tuple | None = None

    def t0(self) -> np.ndarray:
        if self.t0_values is not None:
            return np.asarray(self.t0_values, dtype=np.int64)
        return self.t0_min + self.dt0 * np.arange(self.n_t0, dtype=np.int64)

    def tau(self) -> np.ndarray:
        if self.tau_values is not None:
            return np.asarray(self.tau_values, dtype=np.int64)
        return self.tau_min + self.dtau * np.arange(self.n_tau, dtype=np.int64)

    @property
    def has_axes(self) -> bool:
        return self.t0_values is not None

    @property
    def n_cells(self) -> int:
        return self.n_t0 * self.n_tau

    def with_window(self, window: int) -> "Grid":
        return Grid(self.t0_min, self.dt0, self.n_t0, self.tau_min, self.dtau,
                    self.n_tau, window, self.t_sft, self.exp_cut8, self.t0_values,
                    self.tau_values, self.window_table)

    def window_len(self, tau):
        """L(tau) in seconds: tau (rect) or floor(exp_cut8 tau / 8) (exp)."""
        if self.window == RECT:
            return tau
        return (self.exp_cut8 or 24) * tau // 8

    def as_tuple(self):
        base = (self.t0_min, self.dt0, self.n_t0, self.tau_min, self.dtau,
                self.n_tau, self.t_sft, self.window, self.exp_cut8)
        if self.window_table is not None:
            axes = ((tuple(int(v) for v in self.t0_values), tuple(int(v) for v in self.tau_values))
                    if self.has_axes else (None, None))
            return base + axes + (tuple(float(v) for v in self.window_table),)
        if self.has_axes:
            return base + (tuple(int(v) for v in self.t0_values),
                           tuple(int(v) for v in self.tau_values))
        return base


@dataclass
class Injection:
    template: int
    window: int
    t0: int
    tau: int
    rho2: float
    amp: tuple = (0j, 0j)  # (A, B) after scaling


@dataclass
class Instance:
    t: np.ndarray            # int64 [N]
    antenna: np.ndarray      # [3][N] or [T][3][N]
    fafb: np.ndarray         # [T][4][N]
    grid: Grid
    shared_antenna: bool = True
    injections: list = field(default_factory=list)
    detectors: dict | None = None   # per-detector atoms, when requested

    @property
    def n_sft(self) -> int:
        return int(self.t.shape[0])

    @property
    def n_templates(self) -> int:
        return int(self.fafb.shape[0])

    def antenna_of(self, template: int) -> np.ndarray:
        return self.antenna if self.shared_antenna else self.antenna[template]

    def templates(self, idx) -> "Instance":
        """Sub-instance made of the listed templates (same timestamps, grid)."""
        idx = np.atleast_1d(np.asarray(idx, dtype=np.int64))
        ant = self.antenna if self.shared_antenna else self.antenna[idx]
        inj = [Injection(int(np.nonzero(idx == j.template)[0][0]), j.window, j.t0,
                         j.tau, j.rho2, j.amp)
               for j in self.injections if j.template in set(idx.tolist())]
        return Instance(self.t, ant, np.ascontiguousarray(self.fafb[idx]), self.grid,
                        self.shared_antenna, inj, None)


def _slots_presence(rng, n_det, presence, n_merged=None, n_slots=None, n_drop=0):
    """Boolean presence [n_slots][n_det] of each detector in each SFT slot."""
    if n_slots is not None:
        pres = np.ones((n_slots, n_det), dtype=bool)
        if n_drop:
            drop = rng.choice(n_slots, size=n_drop, replace=False)
            pres[drop, :] = False
        if presence < 1.0:
            pres &= rng.random((n_slots, n_det)) < presence
        return pres
    rows = []
    merged = 0
    while merged < n_merged:
        p = rng.random(n_det) < presence
        rows.append(p)
        merged += bool(p.any())
    return np.array(rows, dtype=bool)


def make_instance(seed: int, *, n_det: int = 1, presence: float = 1.0,
                  n_merged: int | None = None, n_slots: int | None = None,
                  n_drop: int = 0, n_templates: int = 1, grid: Grid,
                  shared_antenna: bool = True, injections=(),
                  dtype=np.float32, keep_detectors: bool = False,
                  t_first: int = 0, noise_scale: float = 1.0) -> Instance:
    """Build one seeded instance.

    ``injections`` lists ``(template, window, t0, tau, rho2)``;
    ``noise_scale = 0`` gives noise-free data.
    Streams: ``philox(seed, 0)`` slot layout, ``philox(seed, 1)`` phases,
    ``philox(seed, 2 + 2 j)`` noise of template ``j`` and
    ``philox(seed, 3 + 2 j)`` its signal direction.
    """
    t_sft = grid.t_sft
    pres = _slots_presence(philox(seed, 0), n_det, presence, n_merged, n_slots, n_drop)
    keep = pres.any(axis=1)
    slots = np.nonzero(keep)[0]
    pres = pres[keep]
    t = (t_first + slots.astype(np.int64) * t_sft).astype(np.int64)
    n = t.shape[0]
    ph = philox(seed, 1).random((n_det, 2)) * 2.0 * math.pi
    ts = t.astype(np.float64)
    a = np.stack([0.4 + 0.3 * np.cos(OMEGA_SID * ts + ph[d, 0]) for d in range(n_det)])
    b = np.stack([0.2 + 0.3 * np.sin(OMEGA_SID * ts + ph[d, 1]) for d in range(n_det)])
    m = pres.T.astype(np.float64)                       # [n_det][N]
    a2 = (m * a * a).sum(0)
    b2 = (m * b * b).sum(0)
    ab = (m * a * b).sum(0)
    antenna64 = np.stack([a2, b2, ab])
    inj_by_t = {}
    for (tmpl, win, it0, itau, rho2) in injections:
        inj_by_t[int(tmpl)] = (int(win), int(it0), int(itau), float(rho2))
    fafb = np.empty((n_templates, 4, n), dtype=dtype)
    det_fa = np.empty((n_templates, n_det, n), dtype=np.complex128) if keep_detectors else None
    det_fb = np.empty_like(det_fa) if keep_detectors else None
    inj_out = []
    for j in range(n_templates):
        g = philox(seed, 2 + 2 * j)
        z = (g.standard_normal((n_det, n)) + 1j * g.standard_normal((n_det, n))) * math.sqrt(0.5)
        z = z * m * noise_scale
        if j in inj_by_t:
            win, it0, itau, rho2 = inj_by_t[j]
            env = envelope(win, t, it0, itau, t_sft)
            gs = philox(seed, 3 + 2 * j)
            u = gs.standard_normal(4)
            amp_a, amp_b = complex(u[0], u[1]), complex(u[2], u[3])
            h = env[None, :] * (a * amp_a + b * amp_b) * m
            energy = float((np.abs(h) ** 2).sum())
            scale = math.sqrt(rho2 / (2.0 * energy)) if energy > 0 else 0.0
            z = z + scale * h
            inj_out.append(Injection(j, win, it0, itau, rho2, (amp_a * scale, amp_b * scale)))
        fa = (a * z).sum(0)
        fb = (b * z).sum(0)
        fafb[j, 0] = fa.real
        fafb[j, 1] = fa.imag
        fafb[j, 2] = fb.real
        fafb[j, 3] = fb.imag
        if keep_detectors:
            det_fa[j] = a * z
            det_fb[j] = b * z
    if shared_antenna:
        antenna = antenna64.astype(dtype)
    else:
        antenna = np.broadcast_to(antenna64.astype(dtype), (n_templates, 3, n)).copy()
    detectors = None
    if keep_detectors:
        detectors = dict(present=pres.T.copy(), a=a, b=b, fa=det_fa, fb=det_fb)
    return Instance(t, antenna, fafb, grid, shared_antenna, inj_out, detectors)


# --------------------------------------------------------------------------
# Workloads.  Sizes follow the five workload definitions of the F-map
# deliverable; each is synthetic (the paper's data came from LALSuite
# simulations that are not reproducible here).
# --------------------------------------------------------------------------

def config_small_rect(dtype=np.float32, seed=BASE_SEED + 0) -> Instance:
    """Rectangular F-map, 1 template: 200 single-detector SFTs (223 slots,
    23 dropped: 10% gaps), t0_m = m T_sft, tau_n = (n + 2) T_sft,
    200 x 200 cells, one rectangular injection at t0 = 40 T_sft,
    tau = 60 T_sft, rho^2 = 100."""
    grid = Grid(0, T_SFT, 200, 2 * T_SFT, T_SFT, 200, RECT)
    return make_instance(seed, n_det=1, n_slots=223, n_drop=23, grid=grid,
                         injections=[(0, RECT, 40 * T_SFT, 60 * T_SFT, 100.0)],
                         dtype=dtype)


def config_exp16(dtype=np.float32, seed=BASE_SEED + 1, n_templates=16) -> Instance:
    """Exponential F-map: 2 detectors each present per slot with p = 0.9,
    2000 merged SFTs, t0_m = m T_sft (m < 1000), tau_n = (n + 1) T_sft
    (n < 1000), 16 templates, template 0 carries an exponential injection at
    t0 = 200 T_sft, tau = 100 T_sft, rho^2 = 250."""
    grid = Grid(0, T_SFT, 1000, T_SFT, T_SFT, 1000, EXP)
    return make_instance(seed, n_det=2, presence=0.9, n_merged=2000,
                         n_templates=n_templates, grid=grid,
                         injections=[(0, EXP, 200 * T_SFT, 100 * T_SFT, 250.0)],
                         dtype=dtype)


def config_batched(window=RECT, n_templates=1024, dtype=np.float32,
                   seed=BASE_SEED + 2, n_sft=5000, n_t0=2000, n_tau=2000) -> Instance:
    """Batched templates: 1 detector, gap-free, 5000 SFTs, 2000 x 2000 cells
    at steps T_sft, tau_min = 2 T_sft (rect) or T_sft (exp), 1024 templates
    sharing the antenna rows, 8 of them injected (alternating windows)."""
    tau_min = 2 * T_SFT if window == RECT else T_SFT
    grid = Grid(0, T_SFT, n_t0, tau_min, T_SFT, n_tau, window)
    g = philox(seed, 99)
    inj = []
    step = max(1, n_templates // 8)
    for k, tmpl in enumerate(range(0, n_templates, step)):
        if len(inj) == 8:
            break
        m = int(g.integers(0, n_t0 // 2))
        nn = int(g.integers(n_tau // 20, n_tau // 4))
        w = RECT if k % 2 == 0 else EXP
        inj.append((tmpl, w, m * T_SFT, tau_min + nn * T_SFT, float(g.uniform(100, 260))))
    return make_instance(seed, n_det=1, n_slots=n_sft, n_templates=n_templates,
                         grid=grid, injections=inj, dtype=dtype)


def uneven_spec(i: int, seed=BASE_SEED + 3, t_range=(1, 1)):
    """Size draw of instance ``i`` of the uneven batch: N_SFT log-uniform in
    [100, 8000], N_t0 and N_tau uniform in {50..2000}, window fair coin,
    5% with an injection of the instance's own window; ``t_range`` bounds
    the (uniform) template count."""
    g = philox(seed, 1_000_000 + i)
    n_sft = int(math.floor(math.exp(g.uniform(math.log(100), math.log(8000)))))
    n_t0 = int(g.integers(50, 2001))
    n_tau = int(g.integers(50, 2001))
    window = int(g.integers(0, 2))
    injected = bool(g.random() < 0.05)
    n_templates = int(g.integers(t_range[0], t_range[1] + 1))
    return dict(n_sft=n_sft, n_t0=n_t0, n_tau=n_tau, window=window,
                injected=injected, n_templates=n_templates,
                inst_seed=int(g.integers(0, 2**62)))


def instance_from_spec(spec, dtype=np.float32) -> Instance:
    """Instance for an uneven-batch draw: 1 detector, slots present with
    p = 0.9, t0 grid spanning [0, T_data - 2 T_sft] and tau grid spanning
    [2 T_sft, T_data], both with integer-second steps (Sec. 4.1 layout)."""
    seed = spec["inst_seed"]
    n_sft = spec["n_sft"]
    pres = _slots_presence(philox(seed, 0), 1, 0.9, n_merged=n_sft)
    t_data = pres.shape[0] * T_SFT
    n_t0, n_tau = spec["n_t0"], spec["n_tau"]
    dt0 = max(1, int(round((t_data - 2 * T_SFT) / max(1, n_t0 - 1))))
    dtau = max(1, int(round((t_data - 2 * T_SFT) / max(1, n_tau - 1))))
    grid = Grid(0, dt0, n_t0, 2 * T_SFT, dtau, n_tau, spec["window"])
    inj = []
    if spec["injected"]:
        g = philox(seed, 77)
        m = int(g.integers(0, max(1, n_t0 // 2)))
        nn = int(g.integers(max(1, n_tau // 10), max(2, n_tau // 2)))
        inj.append((0, spec["window"], m * dt0, 2 * T_SFT + nn * dtau, float(g.uniform(100, 260))))
    return make_instance(seed, n_det=1, presence=0.9, n_merged=n_sft,
                         n_templates=spec["n_templates"], grid=grid,
                         injections=inj, dtype=dtype)


def config_uneven(n_instances=4096, seed=BASE_SEED + 3):
    """Specs of the uneven batch (instances are built on demand)."""
    return [uneven_spec(i, seed) for i in range(n_instances)]


def config_serving_stream(n_requests=10_000, rate_hz=200.0, seed=BASE_SEED + 4):
    """Poisson arrival times (s) and size draws of the serving workload:
    sizes as the uneven batch, 1 to 64 templates per request."""
    g = philox(seed, 0)
    gaps = g.exponential(1.0 / rate_hz, size=n_requests)
    arrivals = np.cumsum(gaps)
    specs = [uneven_spec(i, seed, t_range=(1, 64)) for i in range(n_requests)]
    return arrivals, specs
