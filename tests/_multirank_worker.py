"""Rank body for the multi-process tests (spawned; gloo on the CPU).

Each rank walks its shard of the history ids -- with the oracle, since the
test has no GPU -- and the ranks then merge raw tallies with the library's
host-side path (shard.allreduce_raw, then cls_finalize_raw)."""
import os

import numpy as np


def oracle_raw(case, seed, first, n):
    import oracle
    if n == 0:
        return {"n_histories": 0, "nR": 0, "nT": 0, "nA": 0, "n_coll": 0, "n_interface": 0, "n_reflect": 0,
                "n_events": 0, "n_capped": 0, "max_events": 0, "sum_t": 0.0, "sum_t2": 0.0, "track": (0.0, 0.0),
                "flux": np.zeros((oracle.DEFAULT_NBATCH, case.nbins)),
                "batch_histories": np.zeros(oracle.DEFAULT_NBATCH, dtype=np.uint64)}
    return oracle_raw_from(oracle.run(case, seed, first, n), n)


def oracle_raw_from(r, n):
    """The library's raw-tally layout (cls_raw_t fields, flux[nbatch][nbins] and the
    histories per batch) of an oracle run of n histories."""
    bl = r["batch_len"]
    bh = np.array([max(0, min(bl, n - b * bl)) for b in range(r["nbatch"])], dtype=np.uint64)
    return {"n_histories": r["n_histories"], "nR": r["nR"], "nT": r["nT"], "nA": r["nA"], "n_coll": r["n_coll"],
            "n_interface": r["n_int"], "n_reflect": r["n_refl"], "n_events": r["n_events"],
            "n_capped": r["n_capped"], "max_events": r["max_events"], "sum_t": r["sum_t"], "sum_t2": r["sum_t2"],
            "track": r["track"], "flux": r["flux"], "batch_histories": bh}


def run(rank, world, port, case_tuple, seed, n_total, fault, out_q):
    """`fault`: None, ("drop", r) -- rank r lost its shard -- or ("repeat", r) --
    rank r walked its neighbour r - 1's range instead of its own."""
    import torch.distributed as dist

    import oracle
    from paper_1708_00765_gb300 import _native, shard
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        case = oracle.Case(*case_tuple)
        first, n = shard.shard_range(rank, world, n_total)
        if fault and fault[1] == rank:
            if fault[0] == "drop":
                n = 0  # this rank lost its shard
            else:
                first, n = shard.shard_range(rank - 1, world, n_total)  # walked its neighbour's ids
        raw = oracle_raw(case, seed, first, n)
        try:
            merged = shard.allreduce_raw(raw, history_range=(first, n), expected_range=(0, n_total))
        except shard.CoverageError as e:
            out_q.put((rank, "coverage", str(e)))
            return
        res = _native.finalize_raw(merged, case.L)
        out_q.put((rank, "ok", {k: merged[k] for k in shard.COUNT_KEYS} | {
            "max_events": merged["max_events"], "sum_t": merged["sum_t"], "flux_total": merged["flux"].sum(0),
            "R": res["R"], "total_flux": res["total_flux"]}))
    finally:
        dist.destroy_process_group()
