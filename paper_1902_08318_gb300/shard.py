"""Sharding a batch of documents over ranks (one process per GPU).

Documents are independent, so a batch shards with no exchange on the data
path: each rank takes a contiguous range of documents holding about the same
number of bytes, parses it with its own parser, and the per-document results
are gathered to rank 0 at the end.  A single large document is not sharded:
its stage-1 and stage-2 carries would need an exchange between ranks; with one
GPU per process that is done by replicas instead.

Host logic only; the parse itself is a callable (the CUDA library's
Parser.parse_batch in practice), so the partition and the gather run on any
torch.distributed backend (gloo on CPU in the tests).
"""
from __future__ import annotations

import numpy as np


def partition(offsets: np.ndarray, world: int) -> list[tuple[int, int]]:
    """Contiguous document ranges [lo, hi) per rank with near-equal byte sums.

    offsets: n+1 non-decreasing byte offsets.  Every rank gets a range (it may
    be empty when there are fewer documents than ranks)."""
    off = np.asarray(offsets, dtype=np.int64)
    n = off.size - 1
    if world <= 0:
        raise ValueError("world must be positive")
    total = int(off[-1] - off[0])
    cuts = [0]
    for r in range(1, world):
        target = off[0] + (total * r) // world
        # first document whose start is at or past the target byte
        k = int(np.searchsorted(off[:-1], target, side="left"))
        cuts.append(min(max(k, cuts[-1]), n))
    cuts.append(n)
    return [(cuts[r], cuts[r + 1]) for r in range(world)]


def parse_shard(parse_batch, buf: np.ndarray, offsets: np.ndarray, rank: int, world: int):
    """Parse this rank's share.  parse_batch(buf_slice, local_offsets) must return
    an array of int32 error codes (one per document).  Returns (lo, hi, errors)."""
    lo, hi = partition(offsets, world)[rank]
    off = np.asarray(offsets, dtype=np.uint64)
    if hi <= lo:
        return lo, hi, np.zeros(0, dtype=np.int32)
    base = int(off[lo])
    local = off[lo: hi + 1] - np.uint64(base)
    errs = parse_batch(buf[base: int(off[hi])], local)
    return lo, hi, np.asarray(errs, dtype=np.int32)


def gather_errors(dist, lo: int, hi: int, errs: np.ndarray, n_docs: int):
    """Gather per-document error codes to rank 0 (None elsewhere)."""
    parts = [None] * dist.get_world_size() if dist.get_rank() == 0 else None
    dist.gather_object((lo, hi, errs.tolist()), parts, dst=0)
    if dist.get_rank() != 0:
        return None
    out = np.full(n_docs, -1, dtype=np.int32)
    for plo, phi, perr in parts:
        out[plo:phi] = perr
    return out
