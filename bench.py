#!/usr/bin/env python3
"""Throughput and accuracy of the transient F-statistic map on one GB300.

Metric: F-map (t0, tau)-SFT terms per second: over all templates and all
cells with >= 2 SFTs in their window, the number of SFTs inside the window
(App. A, Eq. Nsums-exp for the exponential window), per second of device
time, with the inputs resident in HBM and the map and summaries written.

Default run (no --workload): one JSON line whose headline is the largest
single-GPU workload, the batched exponential F-map (1024 templates x 5000
SFTs x 2000 x 2000 (t0, tau) cells) computed by the FP64-class decayed-suffix
recurrence; beside it (``also``) the tensor-core forms (BF16x3, 3xTF32) and
the plain FP32 contraction on the same workload, and (``configs``) the other
four workloads: the small rectangular map, the 16-template exponential map
(FP32 against FP64), the 1024-template rectangular batch, the uneven batch
of 4096 instances (one captured graph) and the serving loop (Poisson
arrivals).  Every result carries its accuracy against the FP64 oracle on
sampled templates (computed outside the timed regions).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
    python bench.py --workload exp16|batch_exp|batch_rect|small_rect|uneven
                    [--precision P] [--templates T] ...   (one workload only)

For N > 1 run under torch.distributed.run: every rank computes its own
workload (independent replicas with different seeds; weak scaling), timing is
max over ranks.
"""

from __future__ import annotations

import argparse
import datetime
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import synth  # noqa: E402

WORKLOADS = {
    "batch_exp": "exp-window F-map, 1024 templates x 5000 SFTs (1 detector, gap-free), "
                 "2000 x 2000 (t0, tau) cells at T_sft steps, tau in [T_sft, 2000 T_sft], cut at "
                 "3 tau, 8 templates injected",
    "exp16": "exp-window F-map, 16 templates, 2000 merged SFTs (2 detectors, 10% gaps each), "
             "1000 x 1000 (t0, tau) cells at T_sft steps, tau in [T_sft, 1000 T_sft], cut at 3 tau",
    "small_rect": "rect-window F-map, 1 template, 200 SFTs (10% gaps), 200 x 200 cells",
    "batch_rect": "rect-window F-map, 1024 templates x 5000 SFTs, 2000 x 2000 (t0, tau) cells",
    "uneven": "uneven batch: 4096 single-template instances, N_SFT log-uniform in [100, 8000], "
              "N_t0, N_tau uniform in {50..2000}, rect/exp 50/50, 5% injected; one captured "
              "graph of persistent per-phase launches (fmap_batch_run), autotuned",
    "serving": "Poisson arrivals (200/s) of F-map requests with the uneven batch's size mix and "
               "1-64 templates each, through fmap_submit / fmap_poll",
}
L2_FLUSH_BYTES = 256 << 20
# templates of the batched workloads whose maps are checked against the oracle:
# two injected (rectangular and exponential envelopes) and two noise-only
SAMPLE_TEMPLATES = (0, 128, 511, 1023)
DTYPE = {"fp64": "f64", "fp32": "f32", "tf32": "tf32x3", "bf16x3": "bf16x3", "rec": "f32x2"}


def log(*a):
    print(*a, file=sys.stderr, flush=True)


# ------------------------------------------------------------------ inputs --

def jitter_axes(grid, seed):
    """Explicit axes for a uniform grid: every t0 and tau moved later by a
    seeded offset in [0, step / 2), so the values stay strictly increasing
    but the steps are no longer uniform."""
    g = synth.philox(seed, 5)
    t0 = grid.t0() + g.integers(0, max(1, grid.dt0 // 2), size=grid.n_t0)
    tau = grid.tau() + g.integers(0, max(1, grid.dtau // 2), size=grid.n_tau)
    grid.t0_values = tuple(int(v) for v in t0)
    grid.tau_values = tuple(int(v) for v in tau)


def window_table(shape, cut8=0, n=1024):
    """Samples of a generic window on [0, X], X = cut8 / 8 (default 3): "exp"
    is e^{-x} (the exponential window through the generic path), "bump" a
    rise over 0.4 then a decay."""
    x = np.linspace(0.0, (cut8 or 24) / 8.0, n)
    if shape == "exp":
        w = np.exp(-x)
    elif shape == "bump":
        w = np.sin(np.pi * np.minimum(x / 0.4, 1.0) / 2) ** 2 * np.exp(-0.7 * x)
    else:
        raise SystemExit(f"unknown window table {shape}")
    return tuple(float(v) for v in w.astype(np.float32))


def make_workload(name, rank, templates=None, exp_cut8=0, axes=False, table=None):
    kw = {} if templates is None else {"n_templates": templates}
    if name == "exp16":
        inst = synth.config_exp16(seed=synth.BASE_SEED + 1 + 1000 * rank, **kw)
        inst.grid.exp_cut8 = exp_cut8   # window length exp_cut8 tau / 8 (0: 3 tau)
        if axes:
            jitter_axes(inst.grid, synth.BASE_SEED + 1 + 1000 * rank)
        if table:
            inst.grid.window = synth.TABLE
            inst.grid.window_table = window_table(table, exp_cut8)
        return inst
    if name == "batch_rect":
        return synth.config_batched(window=synth.RECT, seed=synth.BASE_SEED + 2 + 1000 * rank, **kw)
    if name == "batch_exp":
        return synth.config_batched(window=synth.EXP, seed=synth.BASE_SEED + 2 + 1000 * rank, **kw)
    if name == "small_rect":
        return synth.config_small_rect(seed=synth.BASE_SEED + 1000 * rank)
    raise SystemExit(f"unknown workload {name}")


def count_terms_np(grid, t):
    """(terms, cells with >= 2 SFTs) of a grid by the window rule (an SFT at t
    is inside (t0, tau) iff t0 <= t and t + T_sft <= t0 + L(tau)), with numpy
    searches; no library code."""
    t0 = grid.t0()
    L = np.array([grid.window_len(int(v)) for v in grid.tau()], dtype=np.int64)
    i0 = np.searchsorted(t, t0, side="left")
    terms, cells2 = 0, 0
    for a in range(0, len(t0), 256):
        lim = t0[a:a + 256, None] + L[None, :] - grid.t_sft
        j = np.maximum(np.searchsorted(t, lim, side="right"), i0[a:a + 256, None])
        c = j - i0[a:a + 256, None]
        terms += int(c[c >= 2].sum())
        cells2 += int((c >= 2).sum())
    return terms, cells2


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
                "sm_max_mhz": 2070.0}, "fallback"


# DRAM bytes (read + written) per launch of a dominant kernel, from one ncu
# capture of the unchanged kernel (profiles/): a 64-template cut of the rect
# batch, scaled to its 1024 templates (the traffic grows with them).
NCU_TRAFFIC = {("batch_rect", "fp64"): 1078.0e6 * 16}


# ------------------------------------------------------------------ clocks --

class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons (every 20 ms),
    each stamped with nvidia-smi's own sample time.  begin() / end() mark the
    timed region on the wall clock; the summary keeps the samples taken
    inside it (all samples, and says so, when it is shorter than a period)."""

    PERIOD_MS = 20

    FIELDS = ("timestamp,uuid,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid):
        self.uuid = uuid
        self.rows = []
        self.proc = None
        self.thread = None
        self.error = None
        self.spans = []
        self._t0 = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", str(self.PERIOD_MS)], stdout=subprocess.PIPE,
                stderr=subprocess.DEVNULL, text=True)
        except OSError as e:
            self.error = str(e)
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    @staticmethod
    def _stamp(s):
        """nvidia-smi's 'YYYY/MM/DD HH:MM:SS.mmm' (local time) as epoch seconds."""
        try:
            return datetime.datetime.strptime(s.strip(), "%Y/%m/%d %H:%M:%S.%f").timestamp()
        except ValueError:
            return None

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 10:
                ts = self._stamp(parts[0])
                if ts is not None:
                    self.rows.append((ts, parts[1:]))

    def begin(self):
        self._t0 = time.time()

    def end(self):
        if self._t0 is not None:
            self.spans.append((self._t0, time.time()))
        self._t0 = None

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        if self.thread:
            self.thread.join(timeout=5)

    def summary(self):
        if self.error:
            return {"error": self.error}
        rows = [(t, r) for t, r in self.rows if not self.uuid or self.uuid in r[0]] or self.rows
        if not rows:
            return {"error": "no nvidia-smi samples"}
        inside = [(t, r) for t, r in rows if any(a <= t <= b for a, b in self.spans)]
        scope = "timed regions" if inside else "whole run (timed regions shorter than a sample)"
        n_total = len(rows)
        rows = [r for _, r in (inside or rows)]

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None

        sm = [num(r[1]) for r in rows if num(r[1]) is not None]
        mx = [num(r[2]) for r in rows if num(r[2]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({n for r in rows for n, v in zip(names, r[5:9]) if "Active" in v and
                          "Not" not in v})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows), "samples_total": n_total, "scope": scope,
                "period_ms": self.PERIOD_MS, "stamp": "nvidia-smi timestamp field"}


# ---------------------------------------------------------------- accuracy --

def accuracy(fm, oracle, got_map, summ, ref, valid, templates=None):
    """Per-result accuracy against the FP64 oracle: max relative 2F error
    (floor 1) over the checked maps, max |dlogB|, argmax matches (exact cell)
    and near ties (oracle top-2 gap within 2e-3 of the maximum)."""
    rs = oracle.summary(ref, valid)
    err = np.abs(got_map - ref) / np.maximum(np.abs(ref), 1.0)
    worst = float(err[valid].max()) if valid.any() else 0.0
    dlogb, match, near, flagged = 0.0, 0, 0, 0
    want = fm.FMAP_SUMMARY_REFINED | fm.FMAP_SUMMARY_ARGMAX_EXACT
    n = ref.shape[0]
    for j in range(n):
        if rs["n_valid"][j] == 0:
            match += int(summ["m"][j] == -1)
            continue
        dlogb = max(dlogb, abs(float(summ["logB"][j]) - float(rs["logB"][j])))
        match += int((int(summ["m"][j]), int(summ["n"][j])) == (int(rs["m"][j]), int(rs["n"][j])))
        flat = np.where(valid[j], ref[j], -np.inf).ravel()
        top2 = np.partition(flat, -2)[-2:] if flat.size > 1 else np.array([-np.inf, 0.0])
        near += int(rs["max2F"][j] - top2.min() <= 2e-3 * max(rs["max2F"][j], 1.0))
        flagged += int((int(summ["flags"][j]) & want) == want)
    out = {"max_rel_2F_err": worst, "max_abs_dlogB": dlogb, "argmax_match": f"{match}/{n}",
           "near_ties": near, "refined_exact_argmax": f"{flagged}/{n}"}
    if templates is not None:
        out["templates"] = list(templates)
    return out


# ------------------------------------------------------------ cpu baseline --

def sample_grid(g, rows):
    stride = max(1, g.n_t0 // rows)
    sg = synth.Grid(g.t0_min + stride // 2 * g.dt0, g.dt0 * stride, min(rows, g.n_t0),
                    g.tau_min, g.dtau, g.n_tau, g.window, g.t_sft, g.exp_cut8)
    if g.has_axes:   # every stride-th t0 of the explicit axes
        sg.t0_values = tuple(g.t0_values[stride // 2::stride][:sg.n_t0])
        sg.n_t0 = len(sg.t0_values)
        sg.tau_values = g.tau_values
    sg.window_table = g.window_table
    return sg


def cpu_baseline(inst, target_s=12.0):
    """The CPU oracle (fast mode, FP64, OpenMP over t0 rows on all host
    cores) on a bounded sample of the workload: at least as many t0 rows as
    cores (every k-th row), all tau, the first templates, sized from a
    one-row probe to about target_s of work."""
    import oracle

    oracle.build()
    g = inst.grid
    cores = oracle.max_threads()

    def run(rows, n_t):
        sg = sample_grid(g, rows)
        sub = inst if n_t >= inst.n_templates else inst.templates(list(range(n_t)))
        t0 = time.perf_counter()
        oracle.fmap(sub.t, sub.antenna, sub.fafb, sg.as_tuple(), mode="fast")
        return time.perf_counter() - t0, sg

    probe_t = min(inst.n_templates, 4)
    dt1, _ = run(1, probe_t)
    per = dt1 / probe_t                    # seconds per (t0 row, template) on one core
    rows = min(g.n_t0, max(1, cores))
    n_t = int(min(inst.n_templates, max(1, target_s * cores / max(per * rows, 1e-9))))
    if n_t == inst.n_templates:
        rows = int(min(g.n_t0, max(rows, target_s * cores / max(per * n_t, 1e-9))))
    dt, sg = run(rows, n_t)
    terms = count_terms_np(sg, inst.t)[0] * n_t
    return {"value": terms / dt, "unit": "terms/s", "cores": cores, "kind": "oracle",
            "sample": f"{sg.n_t0} of {g.n_t0} t0 rows (every {g.n_t0 // max(1, sg.n_t0)}th), "
                      f"all {g.n_tau} tau, {n_t} of {inst.n_templates} templates; "
                      f"{terms:.3e} terms in {dt:.2f} s"}, sg, terms, n_t


# ------------------------------------------------------------ one workload --

class Runner:
    """Times plans of one workload on resident inputs (map and summaries
    written), L2 flushed between timed steps."""

    def __init__(self, fm, torch, dev, inst, dist, clocks):
        self.fm, self.torch, self.dev, self.inst, self.dist, self.clocks = \
            fm, torch, dev, inst, dist, clocks
        self.stream = torch.cuda.current_stream(dev)
        self.t = torch.from_numpy(inst.t).to(dev)
        self.ant = torch.from_numpy(inst.antenna).to(dev)
        self.x = torch.from_numpy(inst.fafb).to(dev)
        g = inst.grid
        T = inst.n_templates
        self.map = torch.empty((T, g.n_t0, g.n_tau), dtype=torch.float32, device=dev)
        self.sum = torch.empty((T, 32), dtype=torch.uint8, device=dev)
        self.flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    def plan(self, prec, extra_flags=0):
        fm, inst = self.fm, self.inst
        flags = extra_flags | (0 if inst.shared_antenna else fm.FMAP_PLAN_PER_TEMPLATE_ANTENNA)
        if prec == "rec":
            return fm.Plan(inst.grid, inst.n_sft, inst.n_templates, "fp64",
                           flags | fm.FMAP_PLAN_EXP_RECURRENCE)
        return fm.Plan(inst.grid, inst.n_sft, inst.n_templates, prec, flags)

    def step(self, p):
        p.compute(self.t, self.ant, self.x, out_map=self.map, out_summary=self.sum,
                  stream=self.stream)

    def time(self, p, steps, warmup):
        """(per-step ms list, per-phase ms of one call, kernels launched)."""
        torch, fm = self.torch, self.fm
        for _ in range(warmup):
            self.step(p)
        torch.cuda.synchronize()
        if self.dist:
            self.dist.barrier()
        torch.cuda.synchronize()
        fm.fmap_plan_enable_timing(p.handle, True)
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(steps)]
        if self.clocks:
            self.clocks.begin()
        for k in range(steps):
            self.flush.fill_(float(k))                     # untimed: evict the L2
            evs[k][0].record(self.stream)
            self.step(p)
            evs[k][1].record(self.stream)
        torch.cuda.synchronize()
        if self.clocks:
            self.clocks.end()
        if self.dist:
            self.dist.barrier()
        per = [a.elapsed_time(b) for a, b in evs]
        ph, calls, launches = fm.fmap_plan_read_timing(p.handle)
        fm.fmap_plan_enable_timing(p.handle, False)
        st = p.status()
        if st != fm.FMAP_OK:
            raise SystemExit(f"device status {fm.status_string(st)}")
        return per, ph / max(calls, 1), launches

    def time_graph(self, prec, steps, warmup):
        """ms per step of a plan replaying one captured CUDA graph per call
        (FMAP_PLAN_GRAPH; the plan's phase timing is off, so no phases)."""
        torch, fm = self.torch, self.fm
        p = self.plan(prec, fm.FMAP_PLAN_GRAPH)
        for _ in range(warmup):
            self.step(p)
        torch.cuda.synchronize()
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(steps)]
        for k in range(steps):
            self.flush.fill_(float(k))
            evs[k][0].record(self.stream)
            self.step(p)
            evs[k][1].record(self.stream)
        torch.cuda.synchronize()
        st = p.status()
        p.close()
        if st != fm.FMAP_OK:
            raise SystemExit(f"device status {fm.status_string(st)}")
        per = [a.elapsed_time(b) for a, b in evs]
        return {"ms_per_step": sum(per) / steps, "steps": steps,
                "note": "the same step replayed as one CUDA graph (FMAP_PLAN_GRAPH)"}

    def sampled(self, templates):
        """Host copies of the map rows and summaries of some templates."""
        idx = self.torch.tensor(list(templates), device=self.dev)
        m = self.map.index_select(0, idx).cpu().numpy().astype(np.float64)
        s = self.fm.summary_to_numpy(self.sum.index_select(0, idx))
        return m, s


def oracle_of(inst, templates=None, mode="fast"):
    import oracle

    oracle.build()
    sub = inst if templates is None else inst.templates(list(templates))
    ref, valid, _ = oracle.fmap(sub.t, sub.antenna, sub.fafb, sub.grid.as_tuple(), mode=mode)
    return ref, valid


def roofline_exp(peaks, peak_src, prec, terms, dom_ms, n_tau, n_sft, T, cells):
    """Roofline of the exp path's dominant kernel (phase 2).  Tensor forms:
    8 flops per (cell, SFT, template) term (multiply + add on 4 data
    columns) against the kind's tensor peak.  FP32 plain: the same flops
    against the FP32 FMA peak.  Recurrence: 4 flops per (tau, data column,
    template, SFT) -- the recurrence's multiply-add and the one forming E from
    the chunk-local sum -- plus 24 per (cell, template), against the FP32 FMA
    peak."""
    sm_mhz = peaks.get("sm_max_mhz", 2070.0)
    if prec in ("bf16x3", "tf32"):
        flops = 8.0 * terms
        if prec == "bf16x3":
            peak, src = peaks["bf16_tflops"], f"bf16 dense, {peak_src}"
        else:
            peak = peaks["bf16_tflops"] * (1.1 / 2.25)
            src = f"tf32 = bf16 x 1.1/2.25 nominal, {peak_src}"
        ach = flops / (dom_ms / 1e3) / 1e12
        return {"bound": "tensor", "achieved": ach, "peak": peak, "unit": "TFLOP/s",
                "frac": ach / peak, "traffic": None, "kernel": "exp contraction (phase 2)",
                "peak_source": src, "work": "8 flops per (cell, SFT, template) term"}
    if prec == "rec":
        flops = 4.0 * 4 * n_tau * n_sft * T + 24.0 * cells * T
        peak = 152 * 128 * 2 * sm_mhz * 1e6 / 1e12
        ach = flops / (dom_ms / 1e3) / 1e12
        return {"bound": "alu", "achieved": ach, "peak": peak, "unit": "TFLOP/s",
                "frac": ach / peak, "traffic": None, "kernel": "exp recurrence (phase 2)",
                "peak_source": "FP32 FMA: 152 SM x 128 lanes x 2 x max SM clock",
                "work": "4 flops per (tau, data column, template, SFT): the recurrence's FMA "
                        "and the FMA forming E; 24 per (cell, template): two window "
                        "differences on 4 columns and the 2F form"}
    flops = 8.0 * terms
    peak = 152 * 128 * 2 * sm_mhz * 1e6 / 1e12
    ach = flops / (dom_ms / 1e3) / 1e12
    return {"bound": "alu", "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak,
            "traffic": None, "kernel": "exp contraction (phase 2)",
            "peak_source": "FP32 FMA: 152 SM x 128 lanes x 2 x max SM clock",
            "work": "8 flops per (cell, SFT, template) term"}


def time_forms(run, forms, steps, warmup, terms, acc_templates=None, ref=None, valid=None,
               roof=None):
    """Times each precision form of a workload and checks its accuracy."""
    import oracle

    fm = run.fm
    out = {}
    for prec in forms:
        try:
            p = run.plan(prec)
        except fm.FmapError as e:
            out[prec] = {"error": str(e)}
            continue
        per, ph, launches = run.time(p, steps, warmup)
        p.close()
        ms = statistics.mean(per)
        rec = {"value": terms / (ms / 1e3), "unit": "terms/s", "ms_per_step": ms,
               "dtype": DTYPE[prec], "phases_ms": [float(v) for v in ph], "steps": steps,
               "kernel_launches_per_step": launches / max(steps, 1)}
        if roof:
            rec["roofline"] = roof(prec, float(ph[2]))
        if ref is not None:
            if acc_templates is None:
                m = run.map.cpu().numpy().astype(np.float64)
                s = fm.summary_to_numpy(run.sum)
            else:
                m, s = run.sampled(acc_templates)
            rec["accuracy"] = accuracy(fm, oracle, m, s, ref, valid, acc_templates)
        out[prec] = rec
        log(f"  {prec}: {ms:.3f} ms/step, {rec['value']:.3e} terms/s",
            rec.get("accuracy", {}).get("max_abs_dlogB", ""))
    return out


# -------------------------------------------------------------------- main --

def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None,
                    help="timed steps of the headline (default 20; single workloads about a "
                         "second of work; the reference arm 5)")
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=None, choices=sorted(WORKLOADS),
                    help="time one workload only (profiling runs)")
    ap.add_argument("--precision", default=None)
    ap.add_argument("--exp-cut8", type=int, default=0,
                    help="exp16: window length in eighths of tau (0: 3 tau, Eq. winexp)")
    ap.add_argument("--grid-axes", action="store_true",
                    help="exp16: explicit non-uniform (t0, tau) axes (seeded jitter of the steps)")
    ap.add_argument("--window-table", default=None, choices=["exp", "bump"],
                    help="exp16: a generic (table) window of 1024 samples instead of exp")
    ap.add_argument("--templates", type=int, default=None,
                    help="override the workload's template count (profiling runs)")
    ap.add_argument("--instances", type=int, default=4096,
                    help="instances of the uneven workload")
    ap.add_argument("--uneven-window", default="both", choices=["rect", "exp", "both"],
                    help="uneven workload: keep only instances of one window (profiling runs)")
    ap.add_argument("--uneven-nsft", type=int, nargs=2, default=(0, 1 << 30),
                    metavar=("MIN", "MAX"), help="uneven workload: keep MIN <= N_SFT <= MAX")
    ap.add_argument("--profile-phases", action="store_true",
                    help="uneven workload: run the batch once phase by phase (no graph) and "
                         "print the per-phase milliseconds (profiling runs)")
    ap.add_argument("--budget-gb", type=float, default=24.0,
                    help="uneven workload: batch workspace budget (GB)")
    ap.add_argument("--serving-requests", type=int, default=10_000)
    ap.add_argument("--serving-warmup-s", type=float, default=5.0)
    ap.add_argument("--quick", action="store_true",
                    help="default run with smaller sub-records (development runs)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        if args.steps is None:
            args.steps = 5
        return reference_arm(args, rank, world)

    import torch

    import paper_1805_05652_gb300 as fm

    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    dist = None
    if world > 1:
        import torch.distributed as dist  # noqa: F811
        dist.init_process_group("nccl", device_id=dev)
    fm.build()
    uuid = None
    try:
        uuid = str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:
        pass
    clocks = ClockSampler(uuid)
    clocks.start()
    try:
        if args.workload is None:
            result = run_default(args, fm, torch, dev, dist, rank, world, clocks)
        elif args.workload == "uneven":
            result = run_uneven(args, fm, torch, dev, dist, rank, world, clocks)
        elif args.workload == "serving":
            result = {"metric": "serving", **serving(fm, args.serving_requests,
                                                     warmup_s=args.serving_warmup_s)}
        else:
            result = run_single(args, fm, torch, dev, dist, rank, world, clocks)
    finally:
        clocks.stop()
    if result is not None and rank == 0:
        if "clocks" in result:
            result["clocks"] = clocks.summary()
        print(json.dumps(result), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


def headline_line(args, world, value, ms, per, inst, terms, cells2, prec, roof, launches,
                  workload):
    g = inst.grid
    srt = sorted(per)
    return {
        "metric": "F-map (t0,tau)-SFT terms/s",
        "value": value, "unit": "terms/s", "n_gpus": world, "steps": len(per),
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": DTYPE[prec], "data": "synthetic",
        "config": {"workload": workload, "description": WORKLOADS[workload], "precision": prec,
                   "templates": inst.n_templates, "n_sft": inst.n_sft, "n_t0": g.n_t0,
                   "n_tau": g.n_tau, "terms_per_step": terms, "cells_with_2plus_sft": cells2,
                   "l2": "flushed between timed steps (256 MiB write, untimed); the map "
                         "written each step is far larger than L2",
                   "parallelism": f"replicas x{world} (an independent workload per rank)"},
        "latency_ms": {"p50": srt[len(srt) // 2],
                       "p99": srt[min(len(srt) - 1, int(math.ceil(0.99 * len(srt))) - 1)],
                       "max": srt[-1]},
        "roofline": roof,
        "gpu_launches": int(launches),
        "clocks": None,
    }


def run_default(args, fm, torch, dev, dist, rank, world, clocks):
    """The headline (batched exp, recurrence) and every other workload."""
    peaks, peak_src = load_peaks()
    steps = args.steps or 20
    t_start = time.perf_counter()
    # ---- headline: batched exponential map, FP64-class recurrence ----
    inst = make_workload("batch_exp", rank)
    g = inst.grid
    T = inst.n_templates
    terms_t, cells2 = count_terms_np(g, inst.t)
    terms = terms_t * T
    run = Runner(fm, torch, dev, inst, dist, clocks)
    p = run.plan("rec")
    per, ph, launches = run.time(p, steps, args.warmup)
    total_ms = sum(per)
    if dist:
        tt = torch.tensor([total_ms], device=dev, dtype=torch.float64)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        total_ms = float(tt.item())
    ms = total_ms / steps
    value = terms * world / (ms / 1e3)
    roof_of = lambda prec, dom: roofline_exp(peaks, peak_src, prec, terms, dom, g.n_tau,  # noqa: E731
                                             inst.n_sft, T, g.n_t0 * g.n_tau)
    res = headline_line(args, world, value, ms, per, inst, terms, cells2, "rec",
                        roof_of("rec", float(ph[2])), launches, "batch_exp")
    res["phases_ms"] = {"checks_index": float(ph[0]), "antenna": float(ph[1]),
                        "recurrence": float(ph[2]), "fixup_reduce_refine": float(ph[3])}
    log(f"headline: {ms:.2f} ms/step, {value:.3e} terms/s")
    if rank != 0 or world > 1:
        # several GPUs: the headline only (the other workloads are 1-GPU records)
        p.close()
        if rank == 0:
            res["clocks"] = None
            return res
        return None
    # accuracy of the headline on sampled templates (outside the timed region)
    ref, valid = oracle_of(inst, SAMPLE_TEMPLATES)
    m, s = run.sampled(SAMPLE_TEMPLATES)
    import oracle

    res["accuracy"] = accuracy(fm, oracle, m, s, ref, valid, SAMPLE_TEMPLATES)
    # end to end: host atoms in, summaries out, through fmap_compute_host
    if not args.no_e2e:
        res["e2e"] = end_to_end(fm, inst, "rec", terms, max(3, steps // 4))
    p.close()
    # ---- the tensor-core forms and the plain FP32 path, same workload ----
    few = 2 if args.quick else 3
    res["also"] = time_forms(run, ["bf16x3", "tf32", "fp32"], few, 1, terms, SAMPLE_TEMPLATES,
                             ref, valid, roof_of)
    for prec in ("bf16x3", "tf32"):
        r = res["also"].get(prec, {})
        if "ms_per_step" in r and "ms_per_step" in res["also"].get("fp32", {}):
            r["speedup_vs_fp32_plain"] = res["also"]["fp32"]["ms_per_step"] / r["ms_per_step"]
    del run
    torch.cuda.empty_cache()
    # ---- the CPU oracle on a sample of the headline workload ----
    if world == 1 and not args.no_cpu_baseline:
        res["cpu_baseline"] = cpu_baseline(inst, target_s=6.0 if args.quick else 8.0)[0]
    del inst
    configs = {}
    # ---- small rect (1 template, 200 SFTs) ----
    sr = make_workload("small_rect", rank)
    run = Runner(fm, torch, dev, sr, dist, clocks)
    ref, valid = oracle_of(sr, mode="direct")
    tt_ = count_terms_np(sr.grid, sr.t)[0]
    configs["small_rect"] = {"description": WORKLOADS["small_rect"],
                             "forms": time_forms(run, ["fp64", "fp32"], 200, 5, tt_, None, ref,
                                                 valid),
                             "fp64_graph": run.time_graph("fp64", 200, 5)}
    del run
    # ---- exp16: FP32 against FP64 (and the other forms) ----
    e16 = make_workload("exp16", rank)
    run = Runner(fm, torch, dev, e16, dist, clocks)
    ref, valid = oracle_of(e16)
    tt_ = count_terms_np(e16.grid, e16.t)[0] * e16.n_templates
    roof16 = lambda prec, dom: roofline_exp(peaks, peak_src, prec, tt_, dom, e16.grid.n_tau,  # noqa: E731
                                            e16.n_sft, e16.n_templates,
                                            e16.grid.n_t0 * e16.grid.n_tau)
    forms16 = time_forms(run, ["fp64"], 3, 1, tt_, None, ref, valid, roof16)
    forms16.update(time_forms(run, ["fp32", "rec", "bf16x3", "tf32"], 50, 5, tt_, None, ref,
                              valid, roof16))
    configs["exp16"] = {"description": WORKLOADS["exp16"], "forms": forms16,
                        "rec_graph": run.time_graph("rec", 50, 5)}
    f = configs["exp16"]["forms"]
    if "fp32" in f and "fp64" in f and "ms_per_step" in f["fp64"]:
        configs["exp16"]["fp32_vs_fp64_speedup"] = f["fp64"]["ms_per_step"] / f["fp32"]["ms_per_step"]
    del run
    # ---- rect batch: 1024 templates ----
    br = make_workload("batch_rect", rank)
    run = Runner(fm, torch, dev, br, dist, clocks)
    ref, valid = oracle_of(br, SAMPLE_TEMPLATES)
    tt_ = count_terms_np(br.grid, br.t)[0] * br.n_templates

    def roof_rect(prec, dom):
        byts = br.n_templates * br.grid.n_t0 * br.grid.n_tau * 4.0
        ach = byts / (dom / 1e3) / 1e9
        r = {"bound": "hbm", "achieved": ach, "peak": peaks["hbm_gbs"], "unit": "GB/s",
             "frac": ach / peaks["hbm_gbs"], "traffic": NCU_TRAFFIC.get(("batch_rect", prec)),
             "kernel": "rect cells (phase 2)", "peak_source": peak_src,
             "work": "4 bytes of map written per (cell, template)"}
        return r

    configs["batch_rect"] = {"description": WORKLOADS["batch_rect"],
                             "forms": time_forms(run, ["fp64"], 20 if args.quick else 60, 3, tt_,
                                                 SAMPLE_TEMPLATES, ref, valid, roof_rect)}
    del run
    torch.cuda.empty_cache()
    # ---- uneven batch ----
    try:
        configs["uneven"] = run_uneven(args, fm, torch, dev, None, 0, 1, clocks, sub=True)
    except Exception as e:   # reported, never fatal to the headline
        configs["uneven"] = {"error": repr(e)}
    torch.cuda.empty_cache()
    # ---- serving ----
    try:
        n_req = 2000 if args.quick else args.serving_requests
        configs["serving"] = serving(fm, n_req, warmup_s=1.0 if args.quick else
                                     args.serving_warmup_s)
    except Exception as e:
        configs["serving"] = {"error": repr(e)}
    res["configs"] = configs
    res["clocks"] = None
    res["wall_s"] = time.perf_counter() - t_start
    return res


def run_single(args, fm, torch, dev, dist, rank, world, clocks):
    """One workload, one precision (profiling and development runs)."""
    name = args.workload
    inst = make_workload(name, rank, args.templates, args.exp_cut8, args.grid_axes,
                         args.window_table)
    g = inst.grid
    prec = args.precision or ("fp64" if g.window == synth.RECT else "rec")
    run = Runner(fm, torch, dev, inst, dist, clocks)
    if g.has_axes or g.window_table is not None:
        p = run.plan(prec)
        terms_t, cells2 = p.count_terms(inst.t)
        p.close()
    else:
        terms_t, cells2 = count_terms_np(g, inst.t)
    terms = terms_t * inst.n_templates
    steps = args.steps or {"exp16": 500, "small_rect": 1000}.get(name, 20)
    p = run.plan(prec)
    per, ph, launches = run.time(p, steps, args.warmup)
    p.close()
    total_ms = sum(per)
    if dist:
        tt = torch.tensor([total_ms], device=dev, dtype=torch.float64)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        total_ms = float(tt.item())
    ms = total_ms / steps
    if rank != 0:
        return None
    peaks, peak_src = load_peaks()
    if g.window == synth.RECT:
        byts = inst.n_templates * g.n_t0 * g.n_tau * 4.0
        ach = byts / (float(ph[2]) / 1e3) / 1e9
        roof = {"bound": "hbm", "achieved": ach, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": ach / peaks["hbm_gbs"], "traffic": None, "kernel": "rect cells (phase 2)",
                "peak_source": peak_src}
    else:
        roof = roofline_exp(peaks, peak_src, prec, terms, float(ph[2]), g.n_tau, inst.n_sft,
                            inst.n_templates, g.n_t0 * g.n_tau)
    res = headline_line(args, world, terms * world / (ms / 1e3), ms, per, inst, terms, cells2,
                        prec, roof, launches, name)
    res["phases_ms"] = [float(v) for v in ph]
    return res


# ------------------------------------------------------------------ uneven --

def uneven_instances(args, rank):
    keep = {"rect": (synth.RECT,), "exp": (synth.EXP,), "both": (synth.RECT, synth.EXP)}
    specs = synth.config_uneven(n_instances=args.instances, seed=synth.BASE_SEED + 3 + 1000 * rank)
    lo, hi = args.uneven_nsft
    specs = [s for s in specs if s["window"] in keep[args.uneven_window] and lo <= s["n_sft"] <= hi]
    return [synth.instance_from_spec(sp) for sp in specs]


def run_uneven(args, fm, torch, dev, dist, rank, world, clocks, sub=False):
    """The uneven batch through fmap_batch_plan / fmap_batch_run: all
    instances' atoms resident, maps and summaries written, one graph launch
    per step."""
    from concurrent.futures import ThreadPoolExecutor

    t_build = time.perf_counter()
    insts = uneven_instances(args, rank)
    with ThreadPoolExecutor(max(1, os.cpu_count() or 1)) as ex:
        counts = list(ex.map(lambda i: fm.fmap_count_terms(i.grid, i.t), insts))
    terms = sum(c[0] * i.n_templates for c, i in zip(counts, insts))
    cells = sum(i.grid.n_t0 * i.grid.n_tau * i.n_templates for i in insts)
    items = [(i.grid, torch.from_numpy(i.t).to(dev), torch.from_numpy(i.antenna).to(dev),
              torch.from_numpy(i.fafb).to(dev)) for i in insts]
    t_plan = time.perf_counter()
    batch = fm.Batch(items, want_map=True, workspace_budget=int(args.budget_gb * (1 << 30)),
                     autotune=not args.profile_phases)
    torch.cuda.synchronize()
    plan_s = time.perf_counter() - t_plan
    info = batch.info()
    log(f"uneven: {len(insts)} instances built in {t_plan - t_build:.1f} s, planned+tuned in "
        f"{plan_s:.1f} s; {info}")
    stream = torch.cuda.current_stream(dev)
    if args.profile_phases:
        phases = batch.profile(stream)
        st = batch.status(stream)
        batch.close()
        return {"workload": "uneven", "instances": len(insts), "status": fm.status_string(st),
                "info": info, "phases_ms": {k: round(v, 3) for k, v in phases.items()}}
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    for _ in range(args.warmup):
        batch.run(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    steps = 5 if sub else (args.steps or 5)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(steps)]
    clocks.begin()
    for k in range(steps):
        flush.fill_(float(k))
        evs[k][0].record(stream)
        batch.run(stream)
        evs[k][1].record(stream)
    torch.cuda.synchronize()
    clocks.end()
    if dist:
        dist.barrier()
    st = batch.status(stream)
    if st != fm.FMAP_OK:
        raise SystemExit(f"batch status {fm.status_string(st)}")
    per = [a.elapsed_time(b) for a, b in evs]
    phases = batch.profile(stream)          # untimed: one extra run, phase by phase
    total_ms = sum(per)
    if dist:
        tt = torch.tensor([total_ms], device=dev, dtype=torch.float64)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        total_ms = float(tt.item())
    ms_per_step = total_ms / steps
    value = terms * world * steps / (total_ms / 1e3)
    result = None
    if rank == 0:
        peaks, peak_src = load_peaks()
        map_bytes = cells * 4.0
        ach = map_bytes / (ms_per_step / 1e3) / 1e9
        roof = {"bound": "hbm", "achieved": ach, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": ach / peaks["hbm_gbs"], "traffic": None,
                "kernel": "whole batch step (all phases; map bytes / step time)",
                "peak_source": peak_src}
        acc = uneven_accuracy(fm, batch, insts, counts)
        n_rect = sum(1 for i in insts if i.grid.window == synth.RECT)
        result = {
            "metric": "F-map (t0,tau)-SFT terms/s",
            "value": value, "unit": "terms/s", "n_gpus": world, "steps": steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64/f32x2",
            "data": "synthetic",
            "config": {"workload": "uneven", "description": WORKLOADS["uneven"],
                       "instances": len(insts), "rect_instances": n_rect,
                       "terms_per_step": terms, "cells_per_step": cells,
                       "precision": "rect fp64 prefix sums; exp decayed-suffix recurrence",
                       "waves": info["waves"], "launches_per_run": info["launches_per_run"],
                       "workspace_bytes": info["workspace_bytes"],
                       "autotune_occupancy": info["occupancy"],
                       "rec_templates_per_block": info["rec_templates_per_block"],
                       "plan_and_tune_s": plan_s,
                       "l2": "flushed between timed steps (256 MiB write, untimed)",
                       "parallelism": f"replicas x{world}"},
            "latency_ms": {"p50": sorted(per)[len(per) // 2], "max": max(per)},
            "phases_ms": {k: v for k, v in phases.items() if v > 0},
            "roofline": roof,
            "accuracy": acc,
            "gpu_launches": int(info["launches_per_run"]) * steps,
        }
        if not sub:
            result["clocks"] = None
            if world == 1 and not args.no_cpu_baseline:
                result["cpu_baseline"] = uneven_cpu_baseline(insts, counts)
    batch.close()
    return result


def uneven_accuracy(fm, batch, insts, counts, per_class=2, max_terms=3e8):
    """Oracle parity of sampled instances of every (window, N_SFT decade)
    class: maps and (unrefined batch) summaries."""
    import oracle

    oracle.build()
    picked, seen = [], {}
    for k, (inst, c) in enumerate(zip(insts, counts)):
        key = (inst.grid.window, int(math.log10(max(inst.n_sft, 1))))
        if c[0] * inst.n_templates > max_terms or seen.get(key, 0) >= per_class:
            continue
        seen[key] = seen.get(key, 0) + 1
        picked.append(k)
    worst, dlogb, match = 0.0, 0.0, 0
    for k in picked:
        inst = insts[k]
        ref, valid, _ = oracle.fmap(inst.t, inst.antenna, inst.fafb, inst.grid.as_tuple(),
                                    mode="fast")
        got = batch.maps[k].cpu().numpy().astype(np.float64)
        gs = fm.summary_to_numpy(batch.sums[k][: inst.n_templates])
        a = accuracy(fm, oracle, got, gs, ref, valid)
        worst = max(worst, a["max_rel_2F_err"])
        dlogb = max(dlogb, a["max_abs_dlogB"])
        match += int(a["argmax_match"].split("/")[0] == a["argmax_match"].split("/")[1])
    return {"instances_checked": len(picked), "classes": sorted(f"{'rect' if w == 0 else 'exp'}"
                                                                f" 1e{d}" for w, d in seen),
            "max_rel_2F_err": worst, "max_abs_dlogB": dlogb,
            "argmax_match": f"{match}/{len(picked)}",
            "note": "batch summaries are not refined"}


def uneven_cpu_baseline(insts, counts, target_s=12.0):
    """The oracle (fast mode, all host cores) over the first instances of the
    uneven batch until about target_s of CPU work."""
    import oracle

    oracle.build()
    done, terms, t_all = 0, 0, 0.0
    for inst, c in zip(insts, counts):
        t0 = time.perf_counter()
        oracle.fmap(inst.t, inst.antenna, inst.fafb, inst.grid.as_tuple(), mode="fast")
        t_all += time.perf_counter() - t0
        terms += c[0] * inst.n_templates
        done += 1
        if t_all > target_s:
            break
    return {"value": terms / t_all, "unit": "terms/s", "cores": oracle.max_threads(),
            "kind": "oracle",
            "sample": f"first {done} of {len(insts)} instances, {terms:.3e} terms in {t_all:.2f} s"}


# ----------------------------------------------------------------- end to end

def end_to_end(fm, inst, precision, terms, steps):
    """Same metric through fmap_compute_host: pinned host atoms in, the
    per-template summaries out (the search result), copies inside the timed
    region (host wall clock).  The plan keeps its own map (refinement)."""
    import torch

    g = inst.grid
    T = inst.n_templates
    flags = fm.FMAP_PLAN_MAP_BUFFER
    if precision == "rec":
        plan = fm.Plan(g, inst.n_sft, T, "fp64", flags | fm.FMAP_PLAN_EXP_RECURRENCE)
    else:
        plan = fm.Plan(g, inst.n_sft, T, precision, flags)
    h_t = torch.from_numpy(inst.t).pin_memory()
    h_a = torch.from_numpy(inst.antenna).pin_memory()
    h_x = torch.from_numpy(inst.fafb).pin_memory()
    h_s = torch.empty((T, 32), dtype=torch.uint8).pin_memory()
    stream = torch.cuda.current_stream()
    atoms = fm.make_atoms(inst.n_sft, T, inst.shared_antenna, h_t, h_a, h_x)
    for _ in range(2):
        fm.fmap_compute_host(plan.handle, atoms, None, h_s, stream)
    t0 = time.perf_counter()
    for _ in range(steps):
        fm.fmap_compute_host(plan.handle, atoms, None, h_s, stream)
    dt = (time.perf_counter() - t0) / steps
    plan.close()
    h2d = h_t.numel() * 8 + h_a.numel() * 4 + h_x.numel() * 4
    d2h = h_s.numel()
    return {"value": terms / dt, "unit": "terms/s", "h2d_bytes_per_step": int(h2d),
            "d2h_bytes_per_step": int(d2h), "ms_per_step": dt * 1e3, "steps": steps,
            "api": "fmap_compute_host (pinned host buffers; summaries returned, map kept on "
                   "the device)"}


# ----------------------------------------------------------------- serving --

def serving(fm, n_requests=10_000, rate_hz=200.0, max_inflight=8, pool_size=64, seed=None,
            saturated_hz=2000.0, warmup_s=5.0, exp_mode="auto"):
    """Serving workload: Poisson arrivals of F-map requests with the uneven
    batch's size mix and 1-64 templates each, through fmap_submit/fmap_poll,
    after warmup_s seconds of the same stream (untimed).  Latency = scheduled
    arrival -> the poller sees the request finished.  Continuous batching (up
    to 8 requests in flight) against one-at-a-time launches; accuracy of the
    summaries of sampled requests against the oracle."""
    import threading as th

    import oracle

    kw = {} if seed is None else {"seed": seed}
    n_warm = int(warmup_s * rate_hz)
    arrivals, specs = synth.config_serving_stream(n_requests=n_requests + n_warm,
                                                  rate_hz=rate_hz, **kw)
    pool = [synth.instance_from_spec(sp) for sp in specs[:pool_size]]
    terms = [fm.fmap_count_terms(inst.grid, inst.t)[0] * inst.n_templates for inst in pool]

    def run(inflight, arrivals, n_total, n_skip, mode=exp_mode):
        srv = fm.Server(device_mem_budget=24 << 30, pinned_bytes=2 << 30, max_inflight=inflight,
                        exp_mode=mode)
        tickets = [None] * n_total
        done = [0.0] * n_total
        sums = {}
        lock = th.Lock()
        t0 = time.perf_counter() + 0.05

        def submitter():
            for i in range(n_total):
                dt = t0 + arrivals[i] - time.perf_counter()
                if dt > 0:
                    time.sleep(dt)
                inst = pool[i % pool_size]
                while True:
                    try:
                        tk = srv.submit(inst.grid, inst.t, inst.antenna, inst.fafb)
                        break
                    except fm.FmapError as e:
                        if e.status != fm.FMAP_ERR_BUSY:
                            raise
                        time.sleep(1e-4)
                with lock:
                    tickets[i] = tk

        sub = th.Thread(target=submitter)
        sub.start()
        pending = set(range(n_total))
        while pending:
            progressed = False
            for i in list(pending):
                with lock:
                    tk = tickets[i]
                if tk is None:
                    continue
                st, s, _ = srv.poll(tk, wait_us=0)
                if st == fm.FMAP_OK:
                    done[i] = time.perf_counter()
                    if i % pool_size == i:
                        sums[i] = s
                    pending.discard(i)
                    progressed = True
            if not progressed:
                time.sleep(5e-5)
        sub.join()
        peak = srv.peak()
        srv.close()
        idx = range(n_skip, n_total)
        lat = np.array([done[i] - (t0 + arrivals[i]) for i in idx]) * 1e3
        span = max(done[i] for i in idx) - (t0 + arrivals[n_skip])
        tot = sum(terms[i % pool_size] for i in idx)
        return {"p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                "mean_ms": float(lat.mean()), "throughput_terms_per_s": tot / span,
                "requests_per_s": len(lat) / span, "max_inflight": inflight,
                "peak_running": peak}, sums

    n_total = n_requests + n_warm
    cont, sums = run(max_inflight, arrivals, n_total, n_warm)
    serial, _ = run(1, arrivals, n_total, n_warm)
    # every exponential request by BF16x3 (no per-request choice), a shorter stream
    n_fix = min(2000, n_requests)
    fixed, _ = run(max_inflight, arrivals[:n_fix + n_warm], n_fix + n_warm, n_warm, "fixed")
    # The same request sequence arriving 10x faster than the one-at-a-time
    # server can drain it: continuous batching's overlap shows in throughput
    # and tail latency.
    n_sat = min(500, n_requests)
    sat_arr = arrivals[:n_sat] * (rate_hz / saturated_hz)
    sat = {"rate_hz": saturated_hz, "requests": n_sat,
           "continuous_batching": run(max_inflight, sat_arr, n_sat, 0)[0],
           "one_at_a_time": run(1, sat_arr, n_sat, 0)[0]}
    # accuracy of the summaries of the pool's smaller requests
    oracle.build()
    worst, match, ties, unref, checked, ntmpl = 0.0, 0, 0, 0, 0, 0
    for i, inst in enumerate(pool):
        if i not in sums or terms[i] > 1e9 or checked >= 12:
            continue
        ref, valid, _ = oracle.fmap(inst.t, inst.antenna, inst.fafb, inst.grid.as_tuple(),
                                    mode="fast")
        rs = oracle.summary(ref, valid)
        s = sums[i]
        for j in range(inst.n_templates):
            if rs["n_valid"][j]:
                ntmpl += 1
                worst = max(worst, abs(float(s["logB"][j]) - float(rs["logB"][j])))
                gm, gn = int(s["m"][j]), int(s["n"][j])
                if (gm, gn) == (int(rs["m"][j]), int(rs["n"][j])):
                    match += 1
                elif rs["max2F"][j] - ref[j, gm, gn] <= 1e-9 * max(rs["max2F"][j], 1.0):
                    ties += 1   # another cell of the FP64 maximum (tied windows)
                unref += int(not int(s["flags"][j]) & 1)
        checked += 1
    return {"description": WORKLOADS["serving"], "requests": n_requests,
            "warmup_requests": n_warm, "warmup_s": warmup_s, "rate_hz": rate_hz,
            "distinct_request_shapes": pool_size, "continuous_batching": cont,
            "one_at_a_time": serial, "saturated": sat,
            "continuous_batching_exp_bf16x3_only": dict(fixed, requests=n_fix),
            "precision": {"exp": f"server exp_mode '{exp_mode}': per request the recurrence "
                                 "(FP64 class) or BF16x3, whichever the cost model estimates "
                                 "faster", "rect": "fp64"},
            "priority": "requests estimated below 1 ms run on high-priority streams",
            "accuracy": {"requests_checked": checked, "max_abs_dlogB": worst,
                         "argmax_match": f"{match}/{ntmpl}",
                         "argmax_other_cell_of_fp64_tie": ties,
                         "templates_unrefined": unref}}


# --------------------------------------------------------------- reference --

def reference_arm(args, rank, world):
    """The CPU oracle as the reference implementation, on the host cores, on
    a bounded sample of the headline workload (no library code runs here)."""
    if rank != 0:
        return
    name = args.workload or "batch_exp"
    inst = make_workload(name, 0, None, args.exp_cut8, args.grid_axes, args.window_table)
    info, sg, terms, n_t = cpu_baseline(inst, target_s=min(4.0, 150.0 / (args.steps + args.warmup)))
    import oracle

    sub = inst if n_t >= inst.n_templates else inst.templates(list(range(n_t)))
    times = []
    for k in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        oracle.fmap(sub.t, sub.antenna, sub.fafb, sg.as_tuple(), mode="fast")
        if k >= args.warmup:
            times.append(time.perf_counter() - t0)
    mean = statistics.mean(times)
    value = terms / mean
    info["value"] = value
    res = {"impl": "reference", "metric": "F-map (t0,tau)-SFT terms/s", "value": value,
           "unit": "terms/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": mean * 1e3, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": name, "description": WORKLOADS[name],
                      "sample": info["sample"]},
           "cpu_baseline": info,
           "e2e": {"value": value, "unit": "terms/s", "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}}
    print(json.dumps(res), flush=True)


if __name__ == "__main__":
    main()
