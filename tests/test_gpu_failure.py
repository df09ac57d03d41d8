"""Failure detection on the GPU without faulting it.

* A bounded device wait that runs out: a plan whose wait limit is 0 makes
  the rectangular cells kernel give up at its first bulk-copy wait (one
  non-blocking poll right after the copy is issued); the kernel lets that
  copy land, issues nothing more, and the plan reports FMAP_ERR_TIMEOUT.
  The same plan, with the default limit back, then computes the map
  correctly: the context stayed usable.
* Non-finite atoms (a NaN or an infinity in a data or antenna row) are
  reported as FMAP_ERR_NONFINITE by single plans and by batches, and the
  next call with clean atoms succeeds.
"""

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


@pytest.fixture(scope="module", autouse=True)
def _built():
    fm.build()
    oracle.build()


def _dev(inst):
    dev = torch.device("cuda:0")
    return (torch.from_numpy(inst.t).to(dev), torch.from_numpy(inst.antenna).to(dev),
            torch.from_numpy(inst.fafb).to(dev))


def test_rect_wait_limit_zero_times_out_then_recovers():
    inst = synth.config_small_rect()
    t, a, x = _dev(inst)
    plan = fm.Plan(inst.grid, inst.n_sft, inst.n_templates, "fp64")
    plan.set_wait_limit(0)
    plan.compute(t, a, x)
    torch.cuda.synchronize()
    assert plan.status() == fm.FMAP_ERR_TIMEOUT
    assert "wait gave up" in fm.last_error()
    plan.set_wait_limit(-1)
    m, s = plan.compute(t, a, x)
    torch.cuda.synchronize()
    assert plan.status() == fm.FMAP_OK
    ref, valid, _ = oracle.fmap(inst.t, inst.antenna, inst.fafb, inst.grid.as_tuple(), mode="fast")
    check_map(m.cpu().numpy().astype(np.float64), ref, valid, TOL["fp64"])
    check_summary(fm.summary_to_numpy(s), ref, valid, TOL["fp64"], LOGB_TOL)
    plan.close()


def _small(window, seed=61):
    g = Grid(0, T_SFT, 30, 2 * T_SFT if window == RECT else T_SFT, T_SFT, 90, window)
    return synth.make_instance(seed, n_det=2, presence=0.9, n_merged=160, n_templates=3, grid=g)


@pytest.mark.parametrize("window,prec", [(RECT, "fp64"), (EXP, "fp64"), (EXP, "bf16x3")])
@pytest.mark.parametrize("where", ["data", "antenna"])
def test_nonfinite_atoms(window, prec, where):
    inst = _small(window)
    t, a, x = _dev(inst)
    plan = fm.Plan(inst.grid, inst.n_sft, inst.n_templates, prec)
    bad_a, bad_x = a.clone(), x.clone()
    if where == "data":
        bad_x[1, 2, 40] = float("nan")
    else:
        bad_a[1, 77] = float("inf")
    plan.compute(t, bad_a, bad_x)
    torch.cuda.synchronize()
    assert plan.status() == fm.FMAP_ERR_NONFINITE
    assert "NaN or infinite" in fm.last_error()
    m, s = plan.compute(t, a, x)
    torch.cuda.synchronize()
    assert plan.status() == fm.FMAP_OK
    ref, valid, _ = oracle.fmap(inst.t, inst.antenna, inst.fafb, inst.grid.as_tuple(), mode="fast")
    check_map(m.cpu().numpy().astype(np.float64), ref, valid, TOL[prec])
    plan.close()


def test_nonfinite_atoms_in_a_batch():
    insts = [_small(RECT, 70), _small(EXP, 71)]
    dev = torch.device("cuda:0")
    items = []
    for i in insts:
        t, a, x = _dev(i)
        items.append((i.grid, t, a, x))
    items[1][3][0, 0, 5] = float("nan")
    b = fm.Batch(items, want_map=True, autotune=False)
    b.run()
    assert b.status() == fm.FMAP_ERR_NONFINITE
    items[1][3][0, 0, 5] = float(insts[1].fafb[0, 0, 5])   # atoms fixed in place
    b.run()
    assert b.status() == fm.FMAP_OK
    b.close()
    del dev
