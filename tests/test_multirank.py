"""Multi-process path on the CPU: world_size 2 over gloo.

Ranks walk disjoint history ranges and exchange nothing but a final sum of raw
tallies; the merge must equal one run over the whole range (counts bit-exact,
flux to summation order), and a rank that lost its shard must be detected."""
import multiprocessing as mp
import socket

import numpy as np
import pytest

import oracle
from paper_1708_00765_gb300 import _native, shard

CASE = (0.1, 10.0, 1.0, 0.1, 0.99, 0.99, 10.0, 3, 40)


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def launch(world, n_total, fault=None):
    import _multirank_worker as w
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=w.run, args=(r, world, port, CASE, 7, n_total, fault, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = {}
    for _ in range(world):
        rank, status, payload = q.get(timeout=240)
        out[rank] = (status, payload)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    return out


def test_shard_ranges_partition_exactly():
    for n in (0, 1, 7, 1000, 12345):
        for world in (1, 2, 3, 8):
            parts = [shard.shard_range(r, world, n, first=100) for r in range(world)]
            assert sum(c for _, c in parts) == n
            assert parts[0][0] == 100
            for (f0, c0), (f1, _) in zip(parts, parts[1:]):
                assert f0 + c0 == f1


def test_two_ranks_merge_equals_one_run():
    n = 6000
    out = launch(2, n)
    case = oracle.Case(*CASE)
    ref = oracle.run(case, 7, 0, n)
    for rank in (0, 1):
        status, m = out[rank]
        assert status == "ok"
        for k, rk in (("nR", "nR"), ("nT", "nT"), ("nA", "nA"), ("n_coll", "n_coll"),
                      ("n_interface", "n_int"), ("n_events", "n_events"), ("n_histories", "n_histories")):
            assert m[k] == ref[rk]
        assert m["max_events"] == ref["max_events"]
        assert m["sum_t"] == pytest.approx(ref["sum_t"], rel=1e-12)
        np.testing.assert_allclose(m["flux_total"], ref["flux"].sum(0), rtol=1e-12)
        res = oracle.finalize(ref, case)
        assert m["R"] == pytest.approx(res["R"], rel=1e-15)
        assert m["total_flux"] == pytest.approx(res["total_flux"], rel=1e-12)


def test_lost_shard_is_detected():
    out = launch(2, 4000, fault=("drop", 1))
    assert all(status == "coverage" for status, _ in out.values())


def test_repeated_shard_is_detected():
    """Rank 1 walks rank 0's ids instead of its own: the merged history count is right
    (2 x 2000), but ids [0, 2000) were walked twice and [2000, 4000) never."""
    out = launch(2, 4000, fault=("repeat", 1))
    assert all(status == "coverage" for status, _ in out.values())
    assert all("more than once" in payload for _, payload in out.values())


def test_check_cover_on_the_host():
    shard.check_cover([(0, 10), (10, 5), (15, 0)], (0, 15))
    shard.check_cover([(100, 3), (103, 7)], (100, 10))
    for ranges, exp in (([(0, 10), (5, 10)], (0, 15)),   # overlap
                        ([(0, 10), (11, 4)], (0, 15)),   # gap
                        ([(0, 10), (10, 10)], (0, 15)),  # beyond the end
                        ([(1, 14)], (0, 15)),            # missing start
                        ([(0, 10), (0, 10)], (0, 20))):  # the same range twice, right total
        with pytest.raises(shard.CoverageError):
            shard.check_cover(ranges, exp)


def test_host_finalize_matches_oracle_finalize():
    """cls_finalize_raw (library, host) against the oracle's own normalisation."""
    import _multirank_worker as w
    case = oracle.Case(*CASE)
    raw_o = oracle.run(case, 3, 0, 20_000)
    raw = w.oracle_raw(case, 3, 0, 20_000)
    lib = _native.finalize_raw(raw, case.L)
    ref = oracle.finalize(raw_o, case)
    for k in ("R", "T", "A", "sigma_R", "sigma_T", "sigma_A", "total_flux", "sigma_total_flux"):
        assert lib[k] == pytest.approx(ref[k], rel=1e-12), k
    np.testing.assert_allclose(lib["flux"], ref["flux"], rtol=1e-12)
    np.testing.assert_allclose(lib["flux_sigma"], ref["flux_sigma"], rtol=1e-9)
