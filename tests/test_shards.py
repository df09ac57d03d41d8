"""Host logic of a split F-map: per-shard summaries (t0-row shards) combine
into the summary of the whole map through the library's
fmap_combine_summaries (a host function of the C ABI, no GPU needed),
directly and over a 2-rank gloo process group on CPU.  The shard summaries
here come from the oracle, so the test exercises only the combination rule;
shards without valid cells follow the library's empty-summary convention
(max2F = 0, m = n = -1, logB = NaN)."""

import math
import os
import socket
import tempfile

import numpy as np
import pytest

import oracle
import synth
from synth import EXP, RECT, T_SFT, Grid

import paper_1805_05652_gb300.shards as shards
from paper_1805_05652_gb300 import SUMMARY_DTYPE


def _records(s, log_prior=0.0):
    T = len(s["n_valid"])
    r = np.zeros(T, dtype=SUMMARY_DTYPE)
    for j in range(T):
        nv = int(s["n_valid"][j])
        r[j]["n_valid"] = nv
        r[j]["max2F"] = np.float32(s["max2F"][j]) if nv else 0.0
        r[j]["m"] = s["m"][j] if nv else -1
        r[j]["n"] = s["n"][j] if nv else -1
        r[j]["logB"] = s["logB"][j] if nv else float("nan")
    return r


def _map(window, seed=7):
    grid = Grid(-2 * T_SFT, T_SFT, 37, T_SFT if window == EXP else 2 * T_SFT, T_SFT, 50, window)
    inst = synth.make_instance(seed, n_det=2, presence=0.85, n_merged=160, n_templates=3,
                               grid=grid, injections=[(2, window, 9 * T_SFT, 20 * T_SFT, 120.0)])
    m, valid, _ = oracle.fmap(inst.t, inst.antenna, inst.fafb, grid.as_tuple(), mode="fast")
    return m, valid


def _shard_summary(m, valid, lo, hi, log_prior=0.0):
    return _records(oracle.summary(m[:, lo:hi], valid[:, lo:hi], log_prior))


@pytest.fixture(scope="module", autouse=True)
def _built():
    oracle.build()


@pytest.mark.parametrize("window", [RECT, EXP])
@pytest.mark.parametrize("cuts", [(0, 37), (0, 5, 37), (0, 12, 13, 30, 37)])
def test_combine_equals_whole_map(window, cuts):
    m, valid = _map(window)
    whole = _records(oracle.summary(m, valid, 1.5))
    parts = [_shard_summary(m, valid, a, b, 1.5) for a, b in zip(cuts[:-1], cuts[1:])]
    got = shards.combine(parts, list(cuts[:-1]))
    assert np.array_equal(got["n_valid"], whole["n_valid"])
    assert np.array_equal(got["max2F"], whole["max2F"])
    assert np.array_equal(got["m"], whole["m"]) and np.array_equal(got["n"], whole["n"])
    assert np.allclose(got["logB"], whole["logB"], rtol=0, atol=1e-12)


def test_combine_ties_empty_shards_and_all_invalid():
    rng = np.random.default_rng(3)
    m = rng.chisquare(4, size=(2, 20, 9))
    valid = rng.random(m.shape) > 0.3
    m[0, 3, 4] = m[0, 15, 1] = 99.0          # tie across shards: the lower row wins
    valid[0, 3, 4] = valid[0, 15, 1] = True
    valid[0, 8:14] = False                    # one shard with no valid cell
    valid[1] = False                          # a template with no valid cell at all
    whole = _records(oracle.summary(m, valid))
    cuts = (0, 8, 14, 20)
    parts = [_shard_summary(m, valid, a, b) for a, b in zip(cuts[:-1], cuts[1:])]
    got = shards.combine(parts, list(cuts[:-1]))
    assert (got[0]["m"], got[0]["n"]) == (3, 4)
    assert got[0]["n_valid"] == whole[0]["n_valid"]
    assert math.isclose(got[0]["logB"], whole[0]["logB"], rel_tol=0, abs_tol=1e-12)
    assert got[1]["n_valid"] == 0 and got[1]["m"] == -1 and math.isnan(got[1]["logB"])
    assert got[1]["max2F"] == 0.0 and got[1]["n"] == -1


def test_combine_flags_are_common_to_nonempty_shards():
    from paper_1805_05652_gb300 import FMAP_SUMMARY_ARGMAX_EXACT, FMAP_SUMMARY_REFINED

    a = np.zeros(1, dtype=SUMMARY_DTYPE)
    b = np.zeros(1, dtype=SUMMARY_DTYPE)
    e = np.zeros(1, dtype=SUMMARY_DTYPE)
    a[0] = (5.0, 1, 2, FMAP_SUMMARY_REFINED | FMAP_SUMMARY_ARGMAX_EXACT, 0.5, 10)
    b[0] = (7.0, 0, 3, FMAP_SUMMARY_REFINED, 1.5, 30)
    e[0] = (0.0, -1, -1, 0, float("nan"), 0)          # empty shard: ignored
    got = shards.combine([a, e, b], [0, 4, 9])[0]
    assert got["flags"] == FMAP_SUMMARY_REFINED
    assert (got["m"], got["n"]) == (9, 3) and got["max2F"] == np.float32(7.0)
    assert got["n_valid"] == 40
    want = math.log((10 * math.exp(0.5) + 30 * math.exp(1.5)) / 40)
    assert math.isclose(got["logB"], want, rel_tol=0, abs_tol=1e-12)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, cuts, window, out_dir):
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    m, valid = _map(window)
    lo, hi = cuts[rank], cuts[rank + 1]
    comb = shards.allgather_combine(_shard_summary(m, valid, lo, hi), lo)
    np.save(os.path.join(out_dir, f"r{rank}.npy"), comb.view(np.uint8))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("window", [RECT, EXP])
def test_gloo_two_ranks(window):
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp

    m, valid = _map(window)
    whole = _records(oracle.summary(m, valid))
    cuts = (0, 19, 37)
    with tempfile.TemporaryDirectory() as d:
        mp.start_processes(_rank_main, args=(2, _free_port(), cuts, window, d), nprocs=2,
                           join=True, start_method="spawn")
        for r in range(2):
            got = np.load(os.path.join(d, f"r{r}.npy")).view(SUMMARY_DTYPE)
            assert np.array_equal(got["n_valid"], whole["n_valid"])
            assert np.array_equal(got["max2F"], whole["max2F"])
            assert np.array_equal(got["m"], whole["m"]) and np.array_equal(got["n"], whole["n"])
            assert np.allclose(got["logB"], whole["logB"], rtol=0, atol=1e-12)
    del torch
