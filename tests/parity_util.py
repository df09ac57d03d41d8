"""Shared helpers of the GPU parity tests: run the CUDA path through the C ABI
and compare it with the oracle under the stated tolerances."""

import numpy as np

import oracle

# Relative 2F tolerance, |d2F| / max(|2F_oracle|, 1): 1e-5 for the FP64-assisted
# path, 1e-3 for the FP32 sums and the tensor-core forms.
TOL = {"fp64": 1e-5, "rec": 1e-5, "fp32": 1e-3, "tf32": 1e-3, "bf16x3": 1e-3}
FP64_CLASS = ("fp64", "rec")
# Every form: absolute log-Bayes error, and the argmax cell identical to the
# oracle's unless the oracle's two best cells tie at FP64 level (relative gap
# below FP64_TIE; the GPU's refined cells and the oracle sum the same atoms
# in different orders).
LOGB_TOL = 1e-4
FP64_TIE = 1e-9
# Refined maxima are FP64 values rounded to float.
MAX_TOL_REFINED = 1e-6


def run_gpu(inst, precision, want_map=True, plan_flags=0, stream=None):
    import torch

    import paper_1805_05652_gb300 as fm

    dev = torch.device("cuda:0")
    t = torch.from_numpy(np.ascontiguousarray(inst.t)).to(dev)
    ant = torch.from_numpy(np.ascontiguousarray(inst.antenna, dtype=np.float32)).to(dev)
    x = torch.from_numpy(np.ascontiguousarray(inst.fafb, dtype=np.float32)).to(dev)
    flags = plan_flags | (0 if inst.shared_antenna else fm.FMAP_PLAN_PER_TEMPLATE_ANTENNA)
    if precision == "rec":          # decayed-suffix recurrence for exponential windows
        precision, flags = "fp64", flags | fm.FMAP_PLAN_EXP_RECURRENCE
    plan = fm.Plan(inst.grid, inst.n_sft, inst.n_templates, precision, flags)
    m, s = plan.compute(t, ant, x, want_map=want_map, stream=stream)
    torch.cuda.synchronize()
    st = plan.status()
    plan.close()
    assert st == fm.FMAP_OK, fm.status_string(st)
    got = m.cpu().numpy().astype(np.float64) if m is not None else None
    return got, fm.summary_to_numpy(s)


def oracle_map(inst, mode="fast"):
    return oracle.fmap(inst.t, inst.antenna, inst.fafb, inst.grid.as_tuple(), mode=mode)


def rel_err(got, ref):
    return np.abs(got - ref) / np.maximum(np.abs(ref), 1.0)


def check_map(got, ref, valid, tol):
    """Element-wise: invalid cells are exactly 0, valid cells within tol."""
    assert got.shape == ref.shape
    assert np.all(got[~valid] == 0.0)
    err = rel_err(got, ref)
    worst = float(err.max()) if err.size else 0.0
    assert worst <= tol, f"max relative 2F error {worst:.3g} > {tol:g}"
    return worst


def check_summary(gs, ref_map, valid, tol, logb_tol=LOGB_TOL, refined=True, report=None):
    """Summary vs the oracle's reductions of its own map.

    n_valid exact; |logB - logB_oracle| <= logb_tol; the argmax equal to the
    oracle's unless its two best cells tie at FP64 level, where the GPU's cell
    must be one of the tied ones.  With refinement on, every template must be
    refined with a verified argmax (summary flags) and max2F is the FP64
    value to float rounding; unrefined summaries (batches) may pick another
    cell among those within 2 tol max(2F, 1) of the maximum.  Returns (near_ties, fp64_ties, worst |dlogB|):
    near ties are templates whose top-2 gap lies within the fast path's own
    error bound (2 tol max(2F, 1)), where an unrefined argmax could differ.
    ``report`` (a list) collects one line per template for the test log."""
    import paper_1805_05652_gb300 as fm

    rs = oracle.summary(ref_map, valid)
    T = ref_map.shape[0]
    near_ties = fp64_ties = 0
    worst = 0.0
    for j in range(T):
        assert gs["n_valid"][j] == rs["n_valid"][j]
        if rs["n_valid"][j] == 0:
            assert gs["m"][j] == -1 and gs["n"][j] == -1 and np.isnan(gs["logB"][j])
            continue
        mx = rs["max2F"][j]
        scale = max(abs(mx), 1.0)
        if refined:
            want = fm.FMAP_SUMMARY_REFINED | fm.FMAP_SUMMARY_ARGMAX_EXACT
            assert int(gs["flags"][j]) & want == want, (j, int(gs["flags"][j]))
            assert abs(gs["max2F"][j] - mx) <= MAX_TOL_REFINED * scale, (j, gs["max2F"][j], mx)
        else:
            assert abs(gs["max2F"][j] - mx) <= tol * scale
        flat = np.where(valid[j], ref_map[j], -np.inf).ravel()
        top2 = np.partition(flat, -2)[-2:] if flat.size > 1 else np.array([-np.inf, mx])
        gap = mx - top2.min()
        near_ties += int(gap <= 2 * tol * scale)
        gm, gn = int(gs["m"][j]), int(gs["n"][j])
        # unrefined summaries (batches) decide the argmax on their fast values
        tie = FP64_TIE if refined else 2 * tol
        if gap > tie * scale:
            assert (gm, gn) == (rs["m"][j], rs["n"][j]), (j, (gm, gn), (rs["m"][j], rs["n"][j]))
        else:
            fp64_ties += 1
            assert valid[j, gm, gn]
            assert mx - ref_map[j, gm, gn] <= tie * scale
        d = abs(gs["logB"][j] - rs["logB"][j])
        worst = max(worst, d)
        if report is not None:
            report.append(f"T{j}: 2Fmax {mx:.4f} dlogB {d:.2e} top-2 gap {gap:.3e}")
        assert d <= logb_tol, (j, gs["logB"][j], rs["logB"][j])
    return near_ties, fp64_ties, worst
