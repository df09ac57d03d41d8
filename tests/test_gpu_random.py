"""Seeded random instances through single plans, every form, every cell
against the oracle: data sizes, t0 and tau steps off the SFT lattice, gaps,
one or two detectors, shared or per-template antenna rows, exponential cuts
other than 3 tau.  Sizes stay small (the oracle's direct sums take well
under a second each) but span several tiles of every kernel and ragged
edges."""

import numpy as np
import pytest

import oracle
import synth
from synth import EXP, RECT, T_SFT, Grid
from tests.parity_util import LOGB_TOL, TOL, check_map, check_summary, run_gpu

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - CPU container
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1805_05652_gb300 as fm  # noqa: E402

N_CASES = 24


@pytest.fixture(scope="module", autouse=True)
def _built():
    fm.build()
    oracle.build()


def _case(k):
    rng = np.random.default_rng(7000 + k)
    window = EXP if k % 2 else RECT
    n = int(rng.integers(40, 900))
    n_t0, n_tau = int(rng.integers(5, 160)), int(rng.integers(5, 260))
    T = int(rng.integers(1, 12))
    dt0 = int(rng.integers(300, 4 * T_SFT))
    dtau = int(rng.integers(300, 4 * T_SFT))
    cut8 = 0 if window == RECT or k % 4 != 3 else int(rng.integers(8, 40))
    tau_min = 2 * T_SFT if window == RECT else int(rng.integers(T_SFT // 2, 3 * T_SFT))
    g = Grid(-int(rng.integers(0, 8000)), dt0, n_t0, tau_min, dtau, n_tau, window, exp_cut8=cut8)
    inj = [(int(rng.integers(0, T)), window, int(rng.integers(0, 40)) * T_SFT,
            int(rng.integers(5, 60)) * T_SFT, float(rng.uniform(60, 300)))]
    return synth.make_instance(7000 + k, n_det=1 + (k % 3 == 0), presence=float(rng.uniform(0.7, 1.0)),
                               n_merged=n, n_templates=T, grid=g, shared_antenna=(k % 5 != 2),
                               injections=inj)


FORMS = {RECT: ["fp64", "fp32"], EXP: ["fp64", "rec", "bf16x3", "tf32", "fp32"]}


@pytest.mark.parametrize("k", range(N_CASES))
def test_random_instance_every_form(k):
    inst = _case(k)
    ref, valid, _ = oracle.fmap(inst.t, inst.antenna, inst.fafb, inst.grid.as_tuple(), mode="fast")
    for prec in FORMS[inst.grid.window]:
        got, gs = run_gpu(inst, prec)
        worst = check_map(got, ref, valid, TOL[prec])
        near, ties, dlogb = check_summary(gs, ref, valid, TOL[prec], LOGB_TOL)
        print(f"case {k} {prec}: max rel 2F err {worst:.2e}, max |dlogB| {dlogb:.2e}")
