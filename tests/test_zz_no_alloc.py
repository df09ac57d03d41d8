"""fmap_marginalise_noalloc against fmap_marginalise.

The no-allocation entry point serves callers that cannot allocate device
memory while running (a latency-bound serving loop, or a host application
whose allocator owns all device memory); it keeps its reduction scratch in a
fixed array inside the library.  This file checks, through the C ABI, that it
returns what the plan-based entry point returns, on two calls in a row (the
second call reuses the scratch the first one left behind), and that it
refuses a map too large for its scratch.  The file is named to be collected
last.
"""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1805_05652_gb300 as fm  # noqa: E402


def test_noalloc_marginalise_matches_plan_entry_point():
    fm.build()
    rng = np.random.default_rng(11)
    T, n_t0, n_tau = 5, 90, 230
    grid = (0, 1800, n_t0, 1800, 1800, n_tau, 1800, 1)
    plan = fm.Plan(grid, 10, T, "fp32")
    for call in range(2):
        m = (rng.chisquare(4, size=(T, n_t0, n_tau)) * (1.0 + call)).astype(np.float32)
        m[call, 7, 9] = 250.0
        v = rng.random(m.shape) > 0.15
        v[call, 7, 9] = True
        dm = torch.from_numpy(m).cuda()
        dv = torch.from_numpy(v.astype(np.uint8)).cuda()
        ref = fm.summary_to_numpy(plan.marginalise(dm, dv))
        out = torch.full((T, 32), 0xAB, dtype=torch.uint8, device="cuda")
        fm.fmap_marginalise_noalloc(grid, T, dm, dv, 0.0, out)
        got = fm.summary_to_numpy(out)
        assert np.array_equal(got["n_valid"], ref["n_valid"])
        assert np.array_equal(got["m"], ref["m"]) and np.array_equal(got["n"], ref["n"])
        assert np.array_equal(got["max2F"], ref["max2F"])
        assert np.allclose(got["logB"], ref["logB"], rtol=0, atol=1e-4)
        assert (got["m"][call], got["n"][call]) == (7, 9)
    plan.close()


def test_noalloc_rejects_map_beyond_scratch():
    cap = fm.fmap_noalloc_scratch_bytes() // 16
    grid = (0, 1, 2000, 1, 1, 2048, 1800, 1)          # 2000 slots per template
    T = cap // 2000 + 1
    out = torch.empty((T, 32), dtype=torch.uint8, device="cuda")
    dm = torch.empty(1, device="cuda")
    with pytest.raises(fm.FmapError) as e:
        fm.fmap_marginalise_noalloc(grid, T, dm, None, 0.0, out)
    assert e.value.status == fm.FMAP_ERR_ARG
    assert "scratch" in fm.last_error()
