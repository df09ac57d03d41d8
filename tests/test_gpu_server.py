"""The serving loop: continuous batching of F-map requests of mixed sizes,
windows and template counts.  Each result must be the same whether the
request ran alone or among others (bit-identical here: a request's plan,
tiling and reduction order depend only on its own sizes), and must match the
oracle; admission by device memory, pinned-arena back-pressure and error
reporting are checked too."""

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


def _requests(k, seed=900):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(k):
        window = RECT if i % 2 == 0 else EXP
        n = int(rng.integers(60, 400))
        n_t0, n_tau = int(rng.integers(10, 90)), int(rng.integers(20, 300))
        T = int(rng.integers(1, 20))
        g = Grid(0, T_SFT, n_t0, 2 * T_SFT if window == RECT else T_SFT, T_SFT, n_tau, window)
        inst = synth.make_instance(seed + i, n_det=1 + (i % 3 == 0), presence=0.9, n_merged=n,
                                   n_templates=T, grid=g,
                                   injections=[(0, window, 5 * T_SFT, 20 * T_SFT, 150.0)])
        out.append(inst)
    return out


def _run(server, inst, want_map=True):
    tk = server.submit(inst.grid, inst.t, inst.antenna, inst.fafb, want_map=want_map)
    return tk


@pytest.fixture(scope="module")
def reqs():
    fm.build()
    return _requests(24)


@pytest.mark.parametrize("exp_mode", ["fixed", "rec", "auto"])
def test_alone_equals_mixed_and_matches_oracle(reqs, exp_mode):
    """exp_mode: exponential requests by BF16x3 (fixed), by the recurrence,
    or per request by the server's cost model (auto); mixes of high- and
    normal-priority streams in the burst."""
    kw = dict(device_mem_budget=1 << 30, pinned_bytes=256 << 20, exp_mode=exp_mode)
    alone = fm.Server(max_inflight=1, **kw)
    solo = []
    for inst in reqs:
        tk = _run(alone, inst)
        st, s, m = alone.poll(tk, wait_us=-1)
        assert st == fm.FMAP_OK
        solo.append((s, m))
    alone.close()
    mixed = fm.Server(max_inflight=6, **kw)
    tickets = [_run(mixed, inst) for inst in reqs]
    for k, tk in enumerate(tickets):
        st, s, m = mixed.poll(tk, wait_us=-1)
        assert st == fm.FMAP_OK
        assert s.tobytes() == solo[k][0].tobytes()
        assert np.array_equal(m, solo[k][1])
    q, r, c = mixed.stats()
    assert q == 0 and r == 0 and c == len(reqs)
    # the burst really overlapped on the device
    assert mixed.peak() > 1
    mixed.close()
    for k, inst in enumerate(reqs):
        ref, valid, _ = oracle.fmap(inst.t, inst.antenna, inst.fafb, inst.grid.as_tuple(),
                                    mode="fast")
        prec = "fp64" if inst.grid.window == RECT else ("rec" if exp_mode == "rec" else "bf16x3")
        check_map(solo[k][1].astype(np.float64), ref, valid, TOL[prec])
        check_summary(solo[k][0], ref, valid, TOL[prec], LOGB_TOL)


def test_nonfinite_atoms_are_reported(reqs):
    """A request whose atoms hold a NaN (or an infinity) fails with
    FMAP_ERR_NONFINITE; the server keeps serving."""
    srv = fm.Server(device_mem_budget=1 << 30, pinned_bytes=64 << 20, max_inflight=2)
    inst = reqs[2]
    bad = inst.fafb.copy()
    bad[0, 1, 7] = np.nan
    tk = srv.submit(inst.grid, inst.t, inst.antenna, bad)
    with pytest.raises(fm.FmapError) as e:
        srv.poll(tk, wait_us=-1)
    assert e.value.status == fm.FMAP_ERR_NONFINITE
    ant = inst.antenna.copy()
    ant[..., 3] = np.inf
    tk = srv.submit(inst.grid, inst.t, ant, inst.fafb)
    with pytest.raises(fm.FmapError) as e:
        srv.poll(tk, wait_us=-1)
    assert e.value.status == fm.FMAP_ERR_NONFINITE
    tk = srv.submit(inst.grid, inst.t, inst.antenna, inst.fafb)
    assert srv.poll(tk, wait_us=-1)[0] == fm.FMAP_OK
    srv.close()


def test_admission_waits_for_memory(reqs):
    """A pool that holds only a few requests at once still completes a burst
    (admission waits for memory to free up); a request larger than the pool
    is refused at submission."""
    big = reqs[3]
    need = fm.fmap_workspace_bytes(big.grid, big.n_sft, big.n_templates,
                                   fm.FMAP_BF16X3 if big.grid.window == EXP else fm.FMAP_FP64)
    # plus its atoms and outputs (the device always holds the request's map)
    need += (4 * big.grid.n_t0 * big.grid.n_tau + 32 + 16 * big.n_sft + 12) * big.n_templates + \
        8 * big.n_sft + 12 * big.n_sft + 8192
    srv = fm.Server(device_mem_budget=max(need * 3, 2 << 20), pinned_bytes=256 << 20,
                    max_inflight=8)
    tickets = [_run(srv, reqs[3], want_map=False) for _ in range(10)]
    outs = [srv.poll(tk, wait_us=-1) for tk in tickets]
    assert all(st == fm.FMAP_OK for st, _, _ in outs)
    assert all(o[1].tobytes() == outs[0][1].tobytes() for o in outs)
    srv.close()
    tiny = fm.Server(device_mem_budget=1 << 20, pinned_bytes=64 << 20, max_inflight=2)
    with pytest.raises(fm.FmapError) as e:
        _run(tiny, reqs[3])
    assert e.value.status == fm.FMAP_ERR_NOMEM
    tiny.close()


def test_pinned_backpressure_and_errors(reqs):
    srv = fm.Server(device_mem_budget=1 << 30, pinned_bytes=1 << 20, max_inflight=2)
    inst = reqs[1]
    tickets = []
    with pytest.raises(fm.FmapError) as e:
        for _ in range(1000):
            tickets.append(_run(srv, inst, want_map=False))
    assert e.value.status == fm.FMAP_ERR_BUSY and len(tickets) >= 1
    for tk in tickets:
        assert srv.poll(tk, wait_us=-1)[0] == fm.FMAP_OK
    tk = _run(srv, inst, want_map=False)     # room again after polling
    assert srv.poll(tk, wait_us=-1)[0] == fm.FMAP_OK
    bad_t = inst.t.copy()
    bad_t[3] = bad_t[2]
    tk = srv.submit(inst.grid, bad_t, inst.antenna, inst.fafb)
    with pytest.raises(fm.FmapError) as e:
        srv.poll(tk, wait_us=-1)
    assert e.value.status == fm.FMAP_ERR_DATA
    with pytest.raises(fm.FmapError) as e:
        fm.fmap_poll(srv.handle, 987654321, None, None, 0)
    assert e.value.status == fm.FMAP_ERR_BUSY
    srv.close()
