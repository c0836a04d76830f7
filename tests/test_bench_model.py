"""The benchmark's algorithmic work model against the oracle.

The roofline counts Algorithm A's own work from each run's counters; its draw
accounting (the source's draws, two per event, one per collision, one or two
per scatter) must equal the draws the oracle's walk actually takes, which each
history's trace reports as its final draw index."""
import os
import sys

import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


@pytest.mark.parametrize("params", [
    (0.5, 5.0, 2.0, 0.5, 0.5, 0.9, 10.0, 1, 100),        # rod
    (0.1, 10.0, 1.0, 0.1, 0.99, 0.99, 10.0, 3, 200),     # box
    (1.0, 3.0, 0.5, 0.7, 0.8, 0.6, 4.0, 11, 40),         # slab
    (1.0, 3.0, 0.5, 0.7, 0.8, 0.6, 4.0, 2, 40),          # extruded
    (1.0, 3.0, 0.5, 0.7, 0.8, 0.6, 4.0, 13, 40),         # x-projected box
])
def test_model_draws_equal_the_oracle_walks_draws(params):
    case = oracle.Case(*params[:7], int(params[7]), int(params[8]))
    n = 400
    raw = oracle.run(case, 3, 0, n)
    draws = 0
    for h in range(n):
        rows, _ = oracle.trace(case, 3, h)
        draws += int(rows[-1, 1])
    t = {"n_histories": raw["n_histories"], "n_events": raw["n_events"], "n_coll": raw["n_coll"], "nA": raw["nA"]}
    assert bench.model_draws(int(params[7]), t) == draws


def test_algorithmic_ops_grow_with_the_work():
    t = {"n_histories": 1000, "n_events": 47000, "n_coll": 15000, "nA": 160, "total_flux": 15.9}
    ops = bench.algorithmic_ops((0.1, 10.0, 1.0, 0.1, 0.99, 0.99, 10.0, 3, 200), t)
    per_event = ops / t["n_events"]
    # about 3.1 draws per event at 42 operations each, plus the flight's own ~40
    assert 150 < per_event < 200
    more_bins = bench.algorithmic_ops((0.1, 10.0, 1.0, 0.1, 0.99, 0.99, 10.0, 3, 2000), t)
    assert more_bins > ops


def test_count_z_is_the_pooled_z_for_large_counts_and_sane_for_few():
    """The bench compares two runs' R, T, A counts by the exact conditional test: for
    large counts it equals the combined-variance z with the pooled proportion (Eq.
    combined_var); for a rare outcome with a handful of counts, or none, in one run it
    stays a fair z (35 counts in 2e9 histories against none in 1e8 is not significant)."""
    import math
    for ka, na, kb, nb in ((72000, 100000, 71500, 100000), (1440000000, 2000000000, 72030000, 100000000),
                           (30, 100000, 52, 100000)):
        p = (ka + kb) / (na + nb)
        pooled = (ka / na - kb / nb) / math.sqrt(p * (1 - p) * (1 / na + 1 / nb))
        assert abs(bench.count_z(ka, na, kb, nb) - pooled) < 0.05 * max(1.0, abs(pooled))
    assert abs(bench.count_z(35, 2_000_000_000, 0, 100_000_000)) < 1.5
    assert bench.count_z(0, 100, 0, 100) is None and bench.count_z(100, 100, 50, 50) is None
    assert bench.count_z(0, 1000, 40, 1000) < -5
