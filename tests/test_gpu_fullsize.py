"""Parity at the full workload sizes, in the launch configuration the
benchmark times.

* 16-template exponential F-map (2000 merged SFTs, 1000 x 1000 cells): the
  whole map against the oracle's per-cell brute force, every precision.
* 1024-template batch (5000 SFTs, 2000 x 2000 cells), rectangular: the full
  maps of sampled templates against the oracle's running sums, the
  summaries of those templates.
* 1024-template batch, exponential: sampled cells of every template by the
  oracle's direct definition, and the full map of the injected template.
"""

import numpy as np
import pytest

import oracle
import synth
from synth import EXP, RECT
from tests.parity_util import (LOGB_TOL, TOL, check_map, check_summary, rel_err,
                               run_gpu)

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1805_05652_gb300 as fm  # noqa: E402


@pytest.fixture(scope="module")
def exp16():
    fm.build()
    inst = synth.config_exp16()
    ref, valid, _ = oracle.fmap(inst.t, inst.antenna, inst.fafb, inst.grid.as_tuple(), mode="fast")
    return inst, ref, valid


@pytest.mark.parametrize("prec", ["fp32", "tf32", "bf16x3", "fp64", "rec"])
def test_exp16_full_map(exp16, prec):
    inst, ref, valid = exp16
    try:
        got, gs = run_gpu(inst, prec)
    except fm.FmapError as e:
        if e.status == fm.FMAP_ERR_UNSUPPORTED:
            pytest.skip(f"{prec} not built")
        raise
    worst = check_map(got, ref, valid, TOL[prec])
    rep = []
    near, ties, dlogb = check_summary(gs, ref, valid, TOL[prec], LOGB_TOL, report=rep)
    print("\n".join(rep))
    inj = inst.injections[0]
    # the injected template peaks near its true (t0, tau)
    m_true = inj.t0 // inst.grid.dt0
    n_true = (inj.tau - inst.grid.tau_min) // inst.grid.dtau
    assert abs(int(gs["m"][0]) - m_true) <= 15 and abs(int(gs["n"][0]) - n_true) <= 40
    print(f"exp16 {prec}: max rel 2F err {worst:.3g}, max |dlogB| {dlogb:.2e}, near ties {near}, "
          f"FP64 ties {ties}")


@pytest.fixture(scope="module")
def batch_rect():
    fm.build()
    return synth.config_batched(window=RECT)


def test_batched_rect_sampled_templates(batch_rect):
    inst = batch_rect
    dev = torch.device("cuda:0")
    t = torch.from_numpy(inst.t).to(dev)
    a = torch.from_numpy(inst.antenna).to(dev)
    x = torch.from_numpy(inst.fafb).to(dev)
    plan = fm.Plan(inst.grid, inst.n_sft, inst.n_templates, "fp64")
    m, s = plan.compute(t, a, x)
    torch.cuda.synchronize()
    assert plan.status() == fm.FMAP_OK
    gs = fm.summary_to_numpy(s)
    pick = np.array([0, 1, 513, inst.n_templates - 1])
    sub = inst.templates(pick)
    ref, valid, _ = oracle.fmap(sub.t, sub.antenna, sub.fafb, sub.grid.as_tuple(), mode="fast")
    got = m[torch.from_numpy(pick).to(dev)].cpu().numpy().astype(np.float64)
    check_map(got, ref, valid, TOL["fp64"])
    check_summary(gs[pick], ref, valid, TOL["fp64"], LOGB_TOL)
    del m
    plan.close()


@pytest.fixture(scope="module")
def batch_exp():
    fm.build()
    return synth.config_batched(window=EXP)


@pytest.mark.parametrize("prec", ["fp32", "tf32", "bf16x3", "rec"])
def test_batched_exp_sampled_cells(batch_exp, prec):
    inst = batch_exp
    dev = torch.device("cuda:0")
    t = torch.from_numpy(inst.t).to(dev)
    a = torch.from_numpy(inst.antenna).to(dev)
    x = torch.from_numpy(inst.fafb).to(dev)
    flags = 0
    if prec == "rec":
        prec, flags = "fp64", fm.FMAP_PLAN_EXP_RECURRENCE
    try:
        plan = fm.Plan(inst.grid, inst.n_sft, inst.n_templates, prec, flags)
    except fm.FmapError as e:
        if e.status == fm.FMAP_ERR_UNSUPPORTED:
            pytest.skip(f"{prec} not built")
        raise
    m, s = plan.compute(t, a, x)
    torch.cuda.synchronize()
    assert plan.status() == fm.FMAP_OK
    g = inst.grid
    rng = np.random.default_rng(77)
    k = 6000
    idx = np.stack([rng.integers(0, inst.n_templates, k), rng.integers(0, g.n_t0, k),
                    rng.integers(0, g.n_tau, k)], axis=1)
    ref, valid, _ = oracle.cells(inst.t, inst.antenna, inst.fafb, g.as_tuple(), idx)
    ti = torch.from_numpy(idx).to(dev)
    got = m[ti[:, 0], ti[:, 1], ti[:, 2]].cpu().numpy().astype(np.float64)
    assert np.all(got[~valid] == 0.0)
    assert rel_err(got, ref).max() <= TOL[prec]
    gs = fm.summary_to_numpy(s)
    # the injected template's full map and summary
    sub = inst.templates([0])
    ref0, valid0, _ = oracle.fmap(sub.t, sub.antenna, sub.fafb, g.as_tuple(), mode="fast")
    got0 = m[0:1].cpu().numpy().astype(np.float64)
    check_map(got0, ref0, valid0, TOL[prec])
    near, ties, dlogb = check_summary(gs[:1], ref0, valid0, TOL[prec], LOGB_TOL)
    print(f"batched exp {prec}: injected template |dlogB| {dlogb:.2e}")
    del m
    plan.close()
