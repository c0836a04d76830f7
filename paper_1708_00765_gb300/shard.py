"""Sharding CLS histories over processes (one per GPU).

Histories are independent and keyed by id (Philox counter), so N ranks walk
disjoint id ranges of one seed with no exchange during the walk.  The only
exchange is at the end: a sum of raw tallies (cls_raw_tallies), checked for
coverage -- a rank that dropped or repeated its range changes the merged
history count -- and normalised once with cls_finalize_raw.
"""
from __future__ import annotations

import numpy as np

COUNT_KEYS = ("n_histories", "nR", "nT", "nA", "n_coll", "n_interface", "n_reflect", "n_events", "n_capped")


class CoverageError(RuntimeError):
    """The merged tallies do not cover the expected histories exactly once."""


def shard_range(rank: int, world: int, n_total: int, first: int = 0) -> tuple[int, int]:
    """(first history, count) of `rank`'s contiguous share of [first, first + n_total)."""
    if not (0 <= rank < world):
        raise ValueError("rank out of range")
    base, extra = divmod(n_total, world)
    start = rank * base + min(rank, extra)
    return first + start, base + (1 if rank < extra else 0)


def allreduce_raw(raw: dict, group=None, expected_histories: int | None = None) -> dict:
    """Sum raw tallies over the ranks of `group` (torch.distributed): counts and
    sums add, max_events takes the maximum.  If expected_histories is given the
    merged count must equal it (every history walked exactly once)."""
    import torch
    import torch.distributed as dist
    counts = torch.tensor([int(raw[k]) for k in COUNT_KEYS], dtype=torch.int64)
    sums = torch.tensor([raw["sum_t"], raw["sum_t2"], raw["track"][0], raw["track"][1]], dtype=torch.float64)
    flux = torch.from_numpy(np.ascontiguousarray(raw["flux"], dtype=np.float64)).clone()
    bh = torch.from_numpy(np.ascontiguousarray(raw["batch_histories"]).astype(np.int64))
    mx = torch.tensor([int(raw["max_events"])], dtype=torch.int64)
    for t in (counts, sums, flux, bh):
        dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    dist.all_reduce(mx, op=dist.ReduceOp.MAX, group=group)
    out = {k: int(v) for k, v in zip(COUNT_KEYS, counts.tolist())}
    out["sum_t"], out["sum_t2"], t0, t1 = sums.tolist()
    out["track"] = (t0, t1)
    out["flux"] = flux.numpy()
    out["batch_histories"] = bh.numpy().astype(np.uint64)
    out["max_events"] = int(mx.item())
    if expected_histories is not None and out["n_histories"] != expected_histories:
        raise CoverageError(f"merged tallies cover {out['n_histories']} histories, expected {expected_histories}")
    if out["nR"] + out["nT"] + out["nA"] + out["n_capped"] != out["n_histories"]:
        raise CoverageError("merged outcomes do not add up to the merged history count")
    return out
