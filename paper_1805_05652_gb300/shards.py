"""Combining the summaries of an F-map split across processes.

Templates and t0 rows are independent pieces of the F-map (Sec. 3: the
detection statistic is evaluated cell by cell, and the paper notes the
search splits further over templates).  A rank that computed the rows
[m_offset, m_offset + n_t0_shard) of a template holds that shard's
summary: max 2F, the argmax in shard rows, log B over its valid cells and
their count.  The shard summaries combine exactly:

* n_valid adds;
* max 2F is the maximum over shards with valid cells; the argmax is the
  lowest global cell index (m n_tau + n) among the shards attaining it,
  which with contiguous row shards is the lowest (m, n);
* log B = ln(1/N sum e^F) + c: with S_r = sum over shard r of e^F,
  ln S_r = log B_r - c + ln N_r, so
  log B = logsumexp_r(log B_r + ln N_r) - ln N (the prior constant c rides
  along).

No collective runs on the data path: ranks exchange only these 32-byte
records (all_gather of a small tensor), on any torch.distributed backend.
"""

from __future__ import annotations

import math

import numpy as np

from .binding import SUMMARY_DTYPE


def combine(shards, m_offsets):
    """Combine per-shard summaries.

    ``shards``: sequence of structured arrays of SUMMARY_DTYPE, one per
    shard, each of length T (one record per template); ``m_offsets``: the
    first global t0 row of each shard.  Returns an array of T records.
    """
    shards = [np.asarray(s, dtype=SUMMARY_DTYPE) for s in shards]
    if not shards:
        raise ValueError("no shards")
    T = shards[0].shape[0]
    if any(s.shape != (T,) for s in shards) or len(m_offsets) != len(shards):
        raise ValueError("shards must be [T] summaries with one row offset each")
    out = np.zeros(T, dtype=SUMMARY_DTYPE)
    for j in range(T):
        n_tot = 0
        best = None            # (max2F, m, n)
        lse_terms = []
        for s, off in zip(shards, m_offsets):
            r = s[j]
            nv = int(r["n_valid"])
            if nv <= 0:
                continue
            n_tot += nv
            gm, gn = int(r["m"]) + int(off), int(r["n"])
            cand = (float(r["max2F"]), gm, gn)
            if best is None or cand[0] > best[0] or (cand[0] == best[0] and (gm, gn) < best[1:]):
                best = cand
            lse_terms.append(float(r["logB"]) + math.log(nv))
        out[j]["n_valid"] = n_tot
        if n_tot == 0:
            out[j]["max2F"] = -1.0
            out[j]["m"] = out[j]["n"] = -1
            out[j]["logB"] = float("nan")
            continue
        out[j]["max2F"] = best[0]
        out[j]["m"], out[j]["n"] = best[1], best[2]
        hi = max(lse_terms)
        out[j]["logB"] = hi + math.log(sum(math.exp(v - hi) for v in lse_terms)) - math.log(n_tot)
    return out


def allgather_combine(summary, m_offset, group=None):
    """All-gather this rank's shard summary ([T] records) and row offset over
    a torch.distributed process group and return the combined [T] summary
    (the same on every rank)."""
    import torch
    import torch.distributed as dist

    rec = np.ascontiguousarray(np.asarray(summary, dtype=SUMMARY_DTYPE))
    raw = torch.from_numpy(rec.view(np.uint8).copy())
    off = torch.tensor([int(m_offset)], dtype=torch.int64)
    world = dist.get_world_size(group)
    raws = [torch.empty_like(raw) for _ in range(world)]
    offs = [torch.empty_like(off) for _ in range(world)]
    dist.all_gather(raws, raw, group=group)
    dist.all_gather(offs, off, group=group)
    shards = [r.numpy().view(SUMMARY_DTYPE) for r in raws]
    return combine(shards, [int(o.item()) for o in offs])
