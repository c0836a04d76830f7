"""Sharding CLS histories over processes (one per GPU).

Histories are independent and keyed by id (Philox counter), so N ranks walk
disjoint id ranges of one seed with no exchange during the walk.  The only
exchange is at the end: a sum of raw tallies (cls_raw_tallies), checked for
coverage -- every rank states the id range it walked, and the ranges must tile
the expected range exactly, without gap or overlap -- and normalised once with
cls_finalize_raw.
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


def check_cover(ranges, expected: tuple[int, int]) -> None:
    """The (first, count) ranges the ranks walked must tile [first, first + count) of
    `expected` exactly once: no gap, no overlap (ranges of count 0 are ignored)."""
    lo, n = expected
    pos = lo
    for first, count in sorted((int(f), int(c)) for f, c in ranges if int(c) > 0):
        if first < pos:
            raise CoverageError(f"history ids [{first}, {pos}) were walked more than once")
        if first > pos:
            raise CoverageError(f"history ids [{pos}, {first}) were not walked")
        pos = first + count
    if pos != lo + n:
        raise CoverageError(f"history ids [{min(pos, lo + n)}, {max(pos, lo + n)}) "
                            + ("were not walked" if pos < lo + n else "lie beyond the expected range"))


def allreduce_raw(raw: dict, group=None, expected_histories: int | None = None,
                  history_range: tuple[int, int] | None = None,
                  expected_range: tuple[int, int] | None = None) -> dict:
    """Sum raw tallies over the ranks of `group` (torch.distributed): counts and
    sums add, max_events takes the maximum.

    Coverage checks: with `history_range` = (first, count), the ids this rank
    walked, and `expected_range` = (first, count) of the whole job, the ranks'
    ranges are gathered and must tile the expected range exactly once, and each
    rank's tallies must hold `count` histories; with `expected_histories`, the
    merged count must equal it."""
    import torch
    import torch.distributed as dist
    if history_range is not None and int(raw["n_histories"]) != int(history_range[1]):
        raise CoverageError(f"this rank's tallies hold {raw['n_histories']} histories, "
                            f"its range {history_range[1]}")
    counts = torch.tensor([int(raw[k]) for k in COUNT_KEYS], dtype=torch.int64)
    sums = torch.tensor([raw["sum_t"], raw["sum_t2"], raw["track"][0], raw["track"][1]], dtype=torch.float64)
    flux = torch.from_numpy(np.ascontiguousarray(raw["flux"], dtype=np.float64)).clone()
    bh = torch.from_numpy(np.ascontiguousarray(raw["batch_histories"]).astype(np.int64))
    mx = torch.tensor([int(raw["max_events"])], dtype=torch.int64)
    for t in (counts, sums, flux, bh):
        dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    dist.all_reduce(mx, op=dist.ReduceOp.MAX, group=group)
    ranges = None
    if expected_range is not None:
        mine = torch.tensor(list(history_range) if history_range is not None else [0, -1], dtype=torch.int64)
        gathered = [torch.zeros(2, dtype=torch.int64) for _ in range(dist.get_world_size(group))]
        dist.all_gather(gathered, mine, group=group)
        ranges = [tuple(int(v) for v in g.tolist()) for g in gathered]
    out = {k: int(v) for k, v in zip(COUNT_KEYS, counts.tolist())}
    out["sum_t"], out["sum_t2"], t0, t1 = sums.tolist()
    out["track"] = (t0, t1)
    out["flux"] = flux.numpy()
    out["batch_histories"] = bh.numpy().astype(np.uint64)
    out["max_events"] = int(mx.item())
    if ranges is not None:
        if any(c < 0 for _, c in ranges):
            raise CoverageError("a rank did not state the history range it walked")
        check_cover(ranges, expected_range)
        out["ranges"] = ranges
        if out["n_histories"] != int(expected_range[1]):
            raise CoverageError(f"merged tallies cover {out['n_histories']} histories, expected {expected_range[1]}")
    if expected_histories is not None and out["n_histories"] != expected_histories:
        raise CoverageError(f"merged tallies cover {out['n_histories']} histories, expected {expected_histories}")
    if out["nR"] + out["nT"] + out["nA"] + out["n_capped"] != out["n_histories"]:
        raise CoverageError("merged outcomes do not add up to the merged history count")
    return out
