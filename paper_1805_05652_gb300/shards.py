"""Combining the summaries of an F-map split across processes.

Templates and t0 rows are independent pieces of the F-map (Sec. 3: the
detection statistic is evaluated cell by cell, and the search splits further
over templates).  A rank that computed the rows [m_offset, m_offset +
n_t0_shard) of every template holds that shard's summaries.  The combine
itself is the library's ``fmap_combine_summaries`` (n_valid adds, the
maximum with the lowest global argmax, logB = logsumexp_r(logB_r + ln N_r) -
ln N); this module only moves the 32-byte records.

No collective runs on the data path: ranks exchange only these records
(all_gather of a small tensor), on any torch.distributed backend.
"""

from __future__ import annotations

import numpy as np

from .binding import SUMMARY_DTYPE, fmap_combine_summaries


def combine(shards, m_offsets):
    """Combine per-shard summaries: ``shards`` is a sequence of [T] record
    arrays (SUMMARY_DTYPE), one per shard; ``m_offsets`` the first global t0
    row of each shard.  Returns the [T] combined records."""
    shards = [np.asarray(s, dtype=SUMMARY_DTYPE) for s in shards]
    if not shards:
        raise ValueError("no shards")
    T = shards[0].shape[0]
    if any(s.shape != (T,) for s in shards) or len(m_offsets) != len(shards):
        raise ValueError("shards must be [T] summaries with one row offset each")
    return fmap_combine_summaries(np.stack(shards), np.asarray(m_offsets, dtype=np.int32))


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
