"""Shared helpers of the GPU parity tests: run the CUDA path through the C ABI
and compare it with the oracle under the stated tolerances."""

import numpy as np

import oracle

# Relative 2F tolerance, |d2F| / max(|2F_oracle|, 1): 1e-5 for the FP64-assisted
# path, 1e-3 for the FP32 sums and the tensor-core forms.
TOL = {"fp64": 1e-5, "rec": 1e-5, "fp32": 1e-3, "tf32": 1e-3, "bf16x3": 1e-3}
# precision forms held to the FP64 bar (strict logB tolerance)
FP64_CLASS = ("fp64", "rec")
LOGB_TOL = 1e-4


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


def check_summary(gs, ref_map, valid, tol, logb_tol=LOGB_TOL, f_err=0.0):
    """Summary vs the oracle's reductions of its own map (P10 argmax rule:
    exact when the oracle's top-2 gap exceeds the tolerance, else the GPU's
    argmax must be a near-maximum of the oracle map)."""
    rs = oracle.summary(ref_map, valid)
    T = ref_map.shape[0]
    near_ties = 0
    for j in range(T):
        assert gs["n_valid"][j] == rs["n_valid"][j]
        if rs["n_valid"][j] == 0:
            assert gs["m"][j] == -1 and gs["n"][j] == -1 and np.isnan(gs["logB"][j])
            continue
        mx = rs["max2F"][j]
        assert abs(gs["max2F"][j] - mx) <= tol * max(abs(mx), 1.0)
        flat = np.where(valid[j], ref_map[j], -np.inf).ravel()
        top2 = np.partition(flat, -2)[-2:] if flat.size > 1 else np.array([-np.inf, mx])
        gap = mx - top2.min()
        gm, gn = int(gs["m"][j]), int(gs["n"][j])
        if gap > 2 * tol * max(abs(mx), 1.0):
            assert (gm, gn) == (rs["m"][j], rs["n"][j]), (j, (gm, gn), (rs["m"][j], rs["n"][j]))
        else:
            near_ties += 1
            assert valid[j, gm, gn]
            assert mx - ref_map[j, gm, gn] <= 2 * tol * max(abs(mx), 1.0)
        assert abs(gs["logB"][j] - rs["logB"][j]) <= logb_tol + f_err, \
            (j, gs["logB"][j], rs["logB"][j])
    return near_ties
