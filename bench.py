#!/usr/bin/env python3
"""Throughput of the transient F-statistic map on GB300.

Metric: F-map (t0, tau)-SFT terms per second: over all templates and all
cells with >= 2 SFTs in their window, the number of SFTs inside the window
(App. A, Eq. Nsums-exp for the exponential window), per second of device
time.  One step = one fmap_compute_* call over the whole workload with the
inputs resident in HBM (map and summaries written).  Default workload: the
16-template exponential F-map (2000 merged SFTs of 2 detectors, 1000 x 1000
(t0, tau) cells, 1 injected template); see synth.config_exp16.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                       [--precision bf16x3|tf32|fp32|fp64] [--workload exp16|batch_rect|uneven]
For N > 1 run under torch.distributed.run: every rank computes its own
workload (different seeds; weak scaling), timing is max over ranks.
"""

from __future__ import annotations

import argparse
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
    "exp16": "exp-window F-map, 16 templates, 2000 merged SFTs (2 detectors, 10% gaps each), "
             "1000 x 1000 (t0, tau) cells at T_sft steps, tau in [T_sft, 1000 T_sft], cut at 3 tau",
    "batch_rect": "rect-window F-map, 1024 templates x 5000 SFTs, 2000 x 2000 (t0, tau) cells",
    "uneven": "uneven batch: 4096 single-template instances, N_SFT log-uniform in [100, 8000], "
              "N_t0, N_tau uniform in {50..2000}, rect/exp 50/50, 5% injected; one captured "
              "graph of persistent per-phase launches (fmap_batch_run), autotuned",
}
L2_FLUSH_BYTES = 256 << 20


def log(*a):
    print(*a, file=sys.stderr, flush=True)


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
    if name == "exp16":
        kw = {} if templates is None else {"n_templates": templates}
        inst = synth.config_exp16(seed=synth.BASE_SEED + 1 + 1000 * rank, **kw)
        inst.grid.exp_cut8 = exp_cut8   # window length exp_cut8 tau / 8 (0: 3 tau)
        if axes:
            jitter_axes(inst.grid, synth.BASE_SEED + 1 + 1000 * rank)
        if table:
            inst.grid.window = synth.TABLE
            inst.grid.window_table = window_table(table, exp_cut8)
        return inst
    if name == "batch_rect":
        kw = {} if templates is None else {"n_templates": templates}
        return synth.config_batched(window=synth.RECT, seed=synth.BASE_SEED + 2 + 1000 * rank, **kw)
    raise SystemExit(f"unknown workload {name}")


def count_terms(grid, t):
    """(terms, cells with >= 2 SFTs) of a grid: the library's host count for
    uniform grids; for explicit axes the same rule with numpy searches."""
    if not grid.has_axes:
        import paper_1805_05652_gb300 as fm
        return fm.fmap_count_terms(grid, t)
    t0 = grid.t0()
    i0 = np.searchsorted(t, t0, side="left")
    lim = t0[:, None] + np.array([grid.window_len(int(v)) for v in grid.tau()])[None, :] - grid.t_sft
    j = np.maximum(np.searchsorted(t, lim, side="right"), i0[:, None])
    c = j - i0[:, None]
    return int(c[c >= 2].sum()), int((c >= 2).sum())


# DRAM bytes (read + written) per launch of the dominant kernel, from one ncu
# capture of the unchanged kernel on the workload (a 64-template cut of the
# rect batch, scaled to its 1024 templates: the traffic grows with them).
NCU_TRAFFIC = {("exp16", "bf16x3"): 31.5e6,
               ("batch_rect", "fp64"): 1078.0e6 * 16}


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
                "sm_max_mhz": 2070.0}, "fallback"


# ------------------------------------------------------------------ clocks --

# default timed steps: about a second of device work, so that the clock
# samples (every 20 ms) fall inside the timed region
DEFAULT_STEPS = {"exp16": 1000, "batch_rect": 100, "uneven": 5}


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons (every 20 ms).
    begin() / end() mark the timed region on the host clock; the summary
    keeps the samples that arrived inside it (falling back to all samples,
    and saying so, when the region is shorter than the sampling period)."""

    PERIOD_MS = 20

    FIELDS = ("uuid,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid):
        self.uuid = uuid
        self.rows = []
        self.proc = None
        self.thread = None
        self.error = None
        self.t_begin = None
        self.t_end = None

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

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                self.rows.append((time.monotonic(), parts))

    def begin(self):
        self.t_begin = time.monotonic()

    def end(self):
        self.t_end = time.monotonic()

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
        # a line arrives a few ms after its sample: allow one period of lag
        lag = self.PERIOD_MS / 1e3
        inside = [(t, r) for t, r in rows if self.t_begin is not None and self.t_end is not None
                  and self.t_begin <= t <= self.t_end + lag]
        scope = "timed region" if inside else "whole run (timed region shorter than a sample)"
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
                "period_ms": self.PERIOD_MS}


# ------------------------------------------------------------ cpu baseline --

def cpu_baseline(inst, target_s=12.0):
    """The CPU oracle (fast mode, FP64, OpenMP on all host cores) on a bounded
    sample of the workload: every k-th t0 row, all tau, all templates."""
    import oracle

    oracle.build()
    g = inst.grid

    def sample_grid(rows):
        stride = max(1, g.n_t0 // rows)
        sg = synth.Grid(g.t0_min + stride // 2 * g.dt0, g.dt0 * stride,
                        min(rows, g.n_t0), g.tau_min, g.dtau, g.n_tau, g.window, g.t_sft,
                        g.exp_cut8)
        if g.has_axes:   # every stride-th t0 of the explicit axes
            sg.t0_values = tuple(g.t0_values[stride // 2::stride][:sg.n_t0])
            sg.n_t0 = len(sg.t0_values)
            sg.tau_values = g.tau_values
        sg.window_table = g.window_table
        return sg

    def run(rows):
        sg = sample_grid(rows)
        t0 = time.perf_counter()
        oracle.fmap(inst.t, inst.antenna, inst.fafb, sg.as_tuple(), mode="fast")
        return time.perf_counter() - t0, sg

    import paper_1805_05652_gb300 as fm

    rows = 2
    dt, sg = run(rows)
    while dt < 0.5 and rows < g.n_t0:
        rows = min(g.n_t0, rows * 4)
        dt, sg = run(rows)
    per_row = dt / sg.n_t0
    rows = int(min(g.n_t0, max(1, target_s / max(per_row, 1e-9))))
    dt, sg = run(rows)
    terms = count_terms(sg, inst.t)[0] * inst.n_templates
    return {"value": terms / dt, "unit": "terms/s", "cores": oracle.max_threads(),
            "kind": "oracle",
            "sample": f"{sg.n_t0} of {g.n_t0} t0 rows (every {g.n_t0 // max(1, sg.n_t0)}th), "
                      f"all {g.n_tau} tau, all {inst.n_templates} templates; "
                      f"{terms:.3e} terms in {dt:.2f} s"}, sg, terms


# -------------------------------------------------------------------- main --

def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None,
                    help="timed steps (default: about a second of work: exp16 1000, "
                         "batch_rect 100, uneven 5; the reference arm 5)")
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default=None)
    ap.add_argument("--workload", default="exp16", choices=sorted(WORKLOADS))
    ap.add_argument("--exp-cut8", type=int, default=0,
                    help="exp16: window length in eighths of tau (0: 3 tau, Eq. winexp)")
    ap.add_argument("--grid-axes", action="store_true",
                    help="exp16: explicit non-uniform (t0, tau) axes (seeded jitter of the steps)")
    ap.add_argument("--window-table", default=None, choices=["exp", "bump"],
                    help="exp16: a generic (table) window of 1024 samples instead of exp")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--also", default="fp32,tf32,rec",
                    help="comma list of extra precisions timed beside the headline")
    ap.add_argument("--templates", type=int, default=None,
                    help="override the workload's template count (profiling runs)")
    ap.add_argument("--serving-requests", type=int, default=1000,
                    help="requests of the serving measurement added to the line (0: skip)")
    ap.add_argument("--instances", type=int, default=4096,
                    help="instances of the uneven workload")
    ap.add_argument("--budget-gb", type=float, default=24.0,
                    help="uneven workload: batch workspace budget (GB)")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)
    if args.steps is None:
        args.steps = 5 if args.impl == "reference" else DEFAULT_STEPS.get(args.workload, 30)

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
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

    if args.workload == "uneven":
        result = run_uneven(args, fm, torch, dev, dist, rank, world)
        if dist:
            dist.barrier()
            dist.destroy_process_group()
        if result is not None:
            print(json.dumps(result), flush=True)
        return

    inst = make_workload(args.workload, rank, args.templates, args.exp_cut8, args.grid_axes,
                         args.window_table)
    g = inst.grid
    window = g.window
    precision = args.precision
    if precision is None:
        precision = "fp64" if window == synth.RECT else "bf16x3"
    def make_plan(prec):
        if prec == "rec":
            return fm.Plan(g, inst.n_sft, inst.n_templates, "fp64", fm.FMAP_PLAN_EXP_RECURRENCE)
        return fm.Plan(g, inst.n_sft, inst.n_templates, prec)

    try:
        plan = make_plan(precision)
    except fm.FmapError as e:
        if e.status != fm.FMAP_ERR_UNSUPPORTED or args.precision is not None:
            raise
        precision = "fp32"
        plan = make_plan(precision)

    stream = torch.cuda.current_stream(dev)
    t = torch.from_numpy(inst.t).to(dev)
    ant = torch.from_numpy(inst.antenna).to(dev)
    x = torch.from_numpy(inst.fafb).to(dev)
    T = inst.n_templates
    out_map = torch.empty((T, g.n_t0, g.n_tau), dtype=torch.float32, device=dev)
    out_sum = torch.empty((T, 32), dtype=torch.uint8, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    terms_per_tmpl, cells2 = plan.count_terms(inst.t)
    terms = terms_per_tmpl * T

    def step(p):
        p.compute(t, ant, x, out_map=out_map, out_summary=out_sum, stream=stream)

    def timed(p, steps, warmup, sampler=None):
        for _ in range(warmup):
            step(p)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        fm.fmap_plan_enable_timing(p.handle, True)
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(steps)]
        if sampler:
            sampler.begin()
        for k in range(steps):
            flush.fill_(float(k))                     # untimed: evict the L2
            evs[k][0].record(stream)
            step(p)
            evs[k][1].record(stream)
        torch.cuda.synchronize()
        if sampler:
            sampler.end()
        if dist:
            dist.barrier()
        per = [a.elapsed_time(b) for a, b in evs]
        ph, calls, launches = fm.fmap_plan_read_timing(p.handle)
        fm.fmap_plan_enable_timing(p.handle, False)
        return per, ph / max(calls, 1), launches

    uuid = None
    try:
        uuid = str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:
        pass
    clocks = ClockSampler(uuid)
    clocks.start()
    per, phase_ms, launches = timed(plan, args.steps, args.warmup, clocks)
    clocks.stop()
    torch.cuda.synchronize()
    st = plan.status()
    if st != fm.FMAP_OK:
        raise SystemExit(f"device status {fm.status_string(st)}")

    total_ms = sum(per)
    if dist:
        tt = torch.tensor([total_ms], device=dev, dtype=torch.float64)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        total_ms = float(tt.item())
    ms_per_step = total_ms / args.steps
    value = terms * world * args.steps / (total_ms / 1e3)

    extra = {}
    for alt in [a for a in args.also.split(",") if a and a != precision]:
        try:
            p2 = make_plan(alt)
        except fm.FmapError:
            continue
        per2, ph2, _ = timed(p2, max(3, args.steps // 3), 3)
        extra[alt] = {"value": terms * world / (statistics.mean(per2) / 1e3),
                      "ms_per_step": statistics.mean(per2),
                      "contraction_ms": float(ph2[2])}
        p2.close()

    result = None
    if rank == 0:
        peaks, peak_src = load_peaks()
        dom_ms = float(phase_ms[2])
        flops = 2.0 * terms * 4            # multiply + add per (cell, SFT, data column) x 4 columns
        wname = "table" if window == synth.TABLE else "exp"
        if window != synth.RECT and precision in ("bf16x3", "tf32"):
            if precision == "bf16x3":
                peak, unit_peak = peaks["bf16_tflops"], "TFLOP/s (bf16, %s)" % peak_src
            else:
                peak = peaks["bf16_tflops"] * (1.1 / 2.25)
                unit_peak = "TFLOP/s (tf32 = bf16 x 1.1/2.25 nominal, %s)" % peak_src
            ach = flops / (dom_ms / 1e3) / 1e12
            roof = {"bound": "tensor", "achieved": ach, "peak": peak, "unit": "TFLOP/s",
                    "frac": ach / peak, "traffic": None, "kernel": f"{wname} contraction (phase 2)",
                    "peak_source": unit_peak}
        elif window != synth.RECT:
            sm_mhz = peaks.get("sm_max_mhz", 2070.0)
            peak = 152 * 128 * 2 * sm_mhz * 1e6 / 1e12
            ach = flops / (dom_ms / 1e3) / 1e12
            roof = {"bound": "alu", "achieved": ach, "peak": peak, "unit": "TFLOP/s",
                    "frac": ach / peak, "traffic": None, "kernel": f"{wname} contraction (phase 2)",
                    "peak_source": "FP32 FMA: 152 SM x 128 lanes x 2 x max SM clock"}
        else:
            byts = T * g.n_t0 * g.n_tau * 4.0
            ach = byts / (dom_ms / 1e3) / 1e9
            peak = peaks["hbm_gbs"]
            roof = {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s",
                    "frac": ach / peak, "traffic": None, "kernel": "rect cells (phase 2)",
                    "peak_source": peak_src}
        key = (args.workload, precision)
        plain_workload = not (args.exp_cut8 or args.grid_axes or args.templates or args.window_table)
        if plain_workload and key in NCU_TRAFFIC:
            roof["traffic"] = NCU_TRAFFIC[key]
            roof["traffic_source"] = "ncu dram__bytes_read.sum + dram__bytes_write.sum per launch"
        cpu = None
        if world == 1 and not args.no_cpu_baseline:
            cpu, _, _ = cpu_baseline(inst)
        e2e = None
        if not args.no_e2e:
            e2e = end_to_end(fm, inst, precision, terms, args)
        serve = None
        if world == 1 and args.serving_requests > 0:
            try:
                serve = serving(fm, n_requests=args.serving_requests)
            except Exception as e:  # reported, never fatal to the headline
                serve = {"error": repr(e)}
        srt = sorted(per)
        result = {
            "metric": "F-map (t0,tau)-SFT terms/s",
            "value": value, "unit": "terms/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": {"fp64": "f64", "fp32": "f32", "tf32": "tf32x3", "bf16x3": "bf16x3",
                      "rec": "f32x2"}[precision],
            "data": "synthetic",
            "config": {"workload": args.workload, "description": WORKLOADS[args.workload],
                       "precision": precision, "templates": T, "n_sft": inst.n_sft,
                       "n_t0": g.n_t0, "n_tau": g.n_tau, "terms_per_step": terms,
                       "cells_with_2plus_sft": cells2,
                       **({"exp_window_len": f"{g.exp_cut8}/8 tau" if g.exp_cut8 else "3 tau"}
                          if g.window != synth.RECT else {}),
                       **({"window": f"table ({args.window_table}, 1024 samples)"}
                          if g.window == synth.TABLE else {}),
                       **({"grid": "explicit axes (steps jittered by [0, step/2))"}
                          if g.has_axes else {}),
                       "l2": "flushed between timed steps (256 MiB write, untimed)",
                       "parallelism": f"replicas x{world} (templates sharded by rank)"},
            "latency_ms": {"p50": srt[len(srt) // 2], "p99": srt[min(len(srt) - 1,
                                                                  int(math.ceil(0.99 * len(srt))) - 1)],
                           "max": srt[-1]},
            "phases_ms": {"index": float(phase_ms[0]), "antenna": float(phase_ms[1]),
                          "contraction": float(phase_ms[2]), "reduce": float(phase_ms[3])},
            "roofline": roof,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": int(launches),
            "clocks": clocks.summary(),
            "also": extra,
            "serving": serve,
        }
    plan.close()
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    if result is not None:
        print(json.dumps(result), flush=True)


def uneven_instances(n, rank):
    specs = synth.config_uneven(n_instances=n, seed=synth.BASE_SEED + 3 + 1000 * rank)
    return [synth.instance_from_spec(sp) for sp in specs]


def run_uneven(args, fm, torch, dev, dist, rank, world):
    """The uneven batch through fmap_batch_plan / fmap_batch_run: all
    instances' atoms resident, maps and summaries written, one graph launch
    per step."""
    from concurrent.futures import ThreadPoolExecutor

    t_build = time.perf_counter()
    insts = uneven_instances(args.instances, rank)
    with ThreadPoolExecutor(max(1, os.cpu_count() or 1)) as ex:
        counts = list(ex.map(lambda i: fm.fmap_count_terms(i.grid, i.t), insts))
    terms = sum(c[0] * i.n_templates for c, i in zip(counts, insts))
    cells = sum(i.grid.n_t0 * i.grid.n_tau * i.n_templates for i in insts)
    items = [(i.grid, torch.from_numpy(i.t).to(dev), torch.from_numpy(i.antenna).to(dev),
              torch.from_numpy(i.fafb).to(dev)) for i in insts]
    t_plan = time.perf_counter()
    batch = fm.Batch(items, want_map=True, workspace_budget=int(args.budget_gb * (1 << 30)),
                     autotune=True)
    torch.cuda.synchronize()
    plan_s = time.perf_counter() - t_plan
    info = batch.info()
    log(f"uneven: {len(insts)} instances built in {t_plan - t_build:.1f} s, planned+tuned in "
        f"{plan_s:.1f} s; {info}")
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    for _ in range(args.warmup):
        batch.run(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    uuid = None
    try:
        uuid = str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:
        pass
    clocks = ClockSampler(uuid)
    clocks.start()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    clocks.begin()
    for k in range(args.steps):
        flush.fill_(float(k))
        evs[k][0].record(stream)
        batch.run(stream)
        evs[k][1].record(stream)
    torch.cuda.synchronize()
    clocks.end()
    clocks.stop()
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
    ms_per_step = total_ms / args.steps
    value = terms * world * args.steps / (total_ms / 1e3)
    result = None
    if rank == 0:
        peaks, peak_src = load_peaks()
        map_bytes = cells * 4.0
        ach = map_bytes / (ms_per_step / 1e3) / 1e9
        roof = {"bound": "hbm", "achieved": ach, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": ach / peaks["hbm_gbs"], "traffic": None,
                "kernel": "whole batch step (all phases; map bytes / step time)",
                "peak_source": peak_src}
        cpu = None
        if world == 1 and not args.no_cpu_baseline:
            cpu = uneven_cpu_baseline(fm, insts, counts)
        srt = sorted(per)
        n_rect = sum(1 for i in insts if i.grid.window == synth.RECT)
        result = {
            "metric": "F-map (t0,tau)-SFT terms/s",
            "value": value, "unit": "terms/s", "n_gpus": world, "steps": args.steps,
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
            "latency_ms": {"p50": srt[len(srt) // 2], "max": srt[-1]},
            "phases_ms": {k: v for k, v in phases.items() if v > 0},
            "roofline": roof,
            "cpu_baseline": cpu,
            "e2e": None,
            "gpu_launches": int(info["launches_per_run"]) * args.steps,
            "clocks": clocks.summary(),
        }
    batch.close()
    return result


def uneven_cpu_baseline(fm, insts, counts, target_s=12.0):
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


def end_to_end(fm, inst, precision, terms, args):
    """Same metric through fmap_compute_host: pinned host atoms in, map and
    summaries out, copies inside the timed region (host wall clock)."""
    import torch

    g = inst.grid
    T = inst.n_templates
    if precision == "rec":
        plan = fm.Plan(g, inst.n_sft, T, "fp64", fm.FMAP_PLAN_EXP_RECURRENCE)
    else:
        plan = fm.Plan(g, inst.n_sft, T, precision)
    h_t = torch.from_numpy(inst.t).pin_memory()
    h_a = torch.from_numpy(inst.antenna).pin_memory()
    h_x = torch.from_numpy(inst.fafb).pin_memory()
    h_m = torch.empty((T, g.n_t0, g.n_tau), dtype=torch.float32).pin_memory()
    h_s = torch.empty((T, 32), dtype=torch.uint8).pin_memory()
    stream = torch.cuda.current_stream()
    atoms = fm.make_atoms(inst.n_sft, T, True, h_t, h_a, h_x)
    for _ in range(3):
        fm.fmap_compute_host(plan.handle, atoms, h_m, h_s, stream)
    n = max(3, args.steps // 2)
    t0 = time.perf_counter()
    for _ in range(n):
        fm.fmap_compute_host(plan.handle, atoms, h_m, h_s, stream)
    dt = (time.perf_counter() - t0) / n
    plan.close()
    h2d = h_t.numel() * 8 + h_a.numel() * 4 + h_x.numel() * 4
    d2h = h_m.numel() * 4 + h_s.numel()
    return {"value": terms / dt, "unit": "terms/s", "h2d_bytes_per_step": int(h2d),
            "d2h_bytes_per_step": int(d2h), "ms_per_step": dt * 1e3,
            "api": "fmap_compute_host (pinned host buffers)"}


def serving(fm, n_requests=1000, rate_hz=200.0, max_inflight=8, pool_size=64, seed=None,
            saturated_hz=2000.0):
    """Serving workload: Poisson arrivals of F-map requests with the uneven
    batch's size mix and 1-64 templates each, through fmap_submit/fmap_poll.
    Latency = scheduled arrival -> the poller sees the request finished."""
    import threading as th

    kw = {} if seed is None else {"seed": seed}
    arrivals, specs = synth.config_serving_stream(n_requests=n_requests, rate_hz=rate_hz, **kw)
    pool = [synth.instance_from_spec(sp) for sp in specs[:pool_size]]
    terms = [fm.fmap_count_terms(inst.grid, inst.t)[0] * inst.n_templates for inst in pool]

    def run(inflight, arrivals=arrivals, n_requests=n_requests):
        srv = fm.Server(device_mem_budget=24 << 30, pinned_bytes=2 << 30, max_inflight=inflight)
        tickets = [None] * n_requests
        done = [0.0] * n_requests
        lock = th.Lock()
        t0 = time.perf_counter() + 0.05

        def submitter():
            for i in range(n_requests):
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
        pending = set(range(n_requests))
        while pending:
            progressed = False
            for i in list(pending):
                with lock:
                    tk = tickets[i]
                if tk is None:
                    continue
                st, _, _ = srv.poll(tk, wait_us=0)
                if st == fm.FMAP_OK:
                    done[i] = time.perf_counter()
                    pending.discard(i)
                    progressed = True
            if not progressed:
                time.sleep(5e-5)
        sub.join()
        srv.close()
        lat = np.array([done[i] - (t0 + arrivals[i]) for i in range(n_requests)]) * 1e3
        span = max(done) - t0
        tot = sum(terms[i % pool_size] for i in range(n_requests))
        return {"p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                "mean_ms": float(lat.mean()), "throughput_terms_per_s": tot / span,
                "requests_per_s": n_requests / span, "max_inflight": inflight}

    cont = run(max_inflight)
    serial = run(1)
    # The same request sequence arriving 10x faster than the one-at-a-time
    # server can drain it: continuous batching's overlap shows in throughput
    # and tail latency.
    n_sat = max(1, n_requests // 2)
    sat_arr = arrivals[:n_sat] * (rate_hz / saturated_hz)
    sat = {"rate_hz": saturated_hz, "requests": n_sat,
           "continuous_batching": run(max_inflight, sat_arr, n_sat),
           "one_at_a_time": run(1, sat_arr, n_sat)}
    return {"requests": n_requests, "rate_hz": rate_hz, "distinct_request_shapes": pool_size,
            "continuous_batching": cont, "one_at_a_time": serial, "saturated": sat,
            "precision": {"exp": "bf16x3", "rect": "fp64"}}


def reference_arm(args, rank, world):
    """The CPU oracle as the reference implementation, on the host cores."""
    if rank != 0:
        return
    inst = make_workload(args.workload, 0, None, args.exp_cut8, args.grid_axes, args.window_table)
    info, sg, terms = cpu_baseline(inst, target_s=min(4.0, 150.0 / (args.steps + args.warmup)))
    import oracle

    times = []
    for k in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        oracle.fmap(inst.t, inst.antenna, inst.fafb, sg.as_tuple(), mode="fast")
        if k >= args.warmup:
            times.append(time.perf_counter() - t0)
    mean = statistics.mean(times)
    value = terms / mean
    info["value"] = value
    res = {"impl": "reference", "metric": "F-map (t0,tau)-SFT terms/s", "value": value,
           "unit": "terms/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": mean * 1e3, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": args.workload, "description": WORKLOADS[args.workload],
                      "exp_window_len": (f"{args.exp_cut8}/8 tau" if args.exp_cut8 else "3 tau"),
                      "sample": info["sample"]},
           "cpu_baseline": info,
           "e2e": {"value": value, "unit": "terms/s", "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}}
    print(json.dumps(res), flush=True)


if __name__ == "__main__":
    main()
