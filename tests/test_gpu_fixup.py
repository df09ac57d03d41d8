"""The ill-conditioned cells at their worst: one detector whose antenna
pattern turns slowly (3e-4 rad per SFT), so that the 2x2 antenna matrix of a
window of a few SFTs is nearly singular (A B / D up to ~1e7) and every such
cell is recomputed by the fix-up kernels (Sec. 2: windowed sums, Eq. F_FaFb).
Fa and Fb follow the antenna pattern plus a small component along the weak
direction, so both D and the numerator of 2F cancel to ~1e-7 of their
terms.  Single plans (one thread per entry below 8 templates, one per
template above), per-template antenna rows, and uneven batches."""

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

COND_FIXUP = 100.0     # cells above this A B / D go to the fix-up


@pytest.fixture(scope="module", autouse=True)
def _built():
    fm.build()
    oracle.build()


def _ill_instance(seed, window, T, shared, eps=3e-4, n_merged=260):
    tau_min = T_SFT if window == EXP else 2 * T_SFT
    g = Grid(-700, 1300, 150, tau_min, T_SFT // 2, 14, window)   # t0 off the SFT lattice
    base = synth.make_instance(seed, presence=0.9, n_merged=n_merged, n_templates=T, grid=g)
    k = (base.t - base.t[0]).astype(np.float64) / T_SFT
    rng = np.random.default_rng(seed)
    n = base.n_sft
    ants, fafb = [], np.empty((T, 4, n), dtype=np.float32)
    for j in range(T if not shared else 1):
        phi = 0.3 + eps * (1 + j) * k
        r = 0.5 + 0.05 * np.sin(k / 40.0 + j)
        ants.append((r * np.cos(phi), r * np.sin(phi)))
    for j in range(T):
        a, b = ants[0 if shared else j]
        z = (rng.standard_normal(n) + 1j * rng.standard_normal(n)) * np.sqrt(0.5)
        weak = (rng.standard_normal(n) + 1j * rng.standard_normal(n)) * 1e-4
        fa = a * z - b * weak
        fb = b * z + a * weak
        fafb[j] = np.stack([fa.real, fa.imag, fb.real, fb.imag])
    rows = [np.stack([a * a, b * b, a * b]).astype(np.float32) for a, b in ants]
    antenna = rows[0] if shared else np.ascontiguousarray(np.stack(rows))
    return synth.Instance(base.t, antenna, fafb, g, shared)


def _conditioning(inst):
    s, cnt = oracle.sums(inst.t, inst.antenna, inst.fafb, inst.grid.as_tuple())
    A, B, C = s[..., 0], s[..., 1], s[..., 2]
    D = A * B - C * C
    ok = (cnt[None] >= 2) & (D > 0)
    cond = np.where(ok, A * B / np.where(ok, D, 1.0), 0.0)
    return cond


@pytest.mark.parametrize("window,prec,T,shared", [
    (RECT, "fp64", 1, True), (RECT, "fp64", 9, True), (RECT, "fp64", 3, False),
    (EXP, "fp64", 1, True), (EXP, "rec", 1, True), (EXP, "rec", 9, True),
    (EXP, "rec", 3, False), (EXP, "bf16x3", 2, True), (EXP, "fp64", 9, False),
])
def test_fixup_worst_conditioning(window, prec, T, shared):
    inst = _ill_instance(11 + T + 7 * window, window, T, shared)
    cond = _conditioning(inst)
    n_fix = int((cond > COND_FIXUP).sum())
    assert n_fix > 100 and cond.max() > 1e6, (n_fix, cond.max())
    ref, valid, _ = oracle.fmap(inst.t, inst.antenna, inst.fafb, inst.grid.as_tuple(), mode="fast")
    got, gs = run_gpu(inst, prec)
    worst = check_map(got, ref, valid, TOL[prec])
    fix = cond > COND_FIXUP
    err_fix = float((np.abs(got - ref) / np.maximum(np.abs(ref), 1.0))[fix].max())
    check_summary(gs, ref, valid, TOL[prec], LOGB_TOL)
    print(f"{prec} T={T}: {n_fix} fix-up cells, max A B / D {cond.max():.2e}, "
          f"max rel 2F err {worst:.2e} (fix-up cells {err_fix:.2e})")


def test_fixup_in_uneven_batch():
    insts = [_ill_instance(40 + i, EXP if i % 2 else RECT, 1 + (i % 3) * 4, i % 4 != 3,
                           n_merged=120 + 40 * i)
             for i in range(6)]
    dev = torch.device("cuda:0")
    devs = [(i.grid, torch.from_numpy(i.t).to(dev), torch.from_numpy(i.antenna).to(dev),
             torch.from_numpy(i.fafb).to(dev)) for i in insts]
    b = fm.Batch(devs, want_map=True)
    b.run()
    torch.cuda.synchronize()
    assert b.status() == fm.FMAP_OK
    for k, inst in enumerate(insts):
        cond = _conditioning(inst)
        assert (cond > COND_FIXUP).sum() > 50
        ref, valid, _ = oracle.fmap(inst.t, inst.antenna, inst.fafb, inst.grid.as_tuple(),
                                    mode="fast")
        got = b.maps[k].cpu().numpy().astype(np.float64)
        check_map(got, ref, valid, TOL["fp64"])
        check_summary(fm.summary_to_numpy(b.sums[k][: inst.n_templates]), ref, valid,
                      TOL["fp64"], LOGB_TOL, refined=False)
    b.close()
