"""FP64 parity at the benchmark workloads' full sizes, against the oracle on the
host cores: integer counts bit-exact, every flux bin within 1e-12 relative.

* the 3D box of side 10, all 1e8 histories, in the benchmark's launch shape;
* the 256-case sweep in its autotuned batched launch, every case on its first
  1e5 history ids;
* the diffusive box (L = 100, c = 0.999, 500 bins) on both schedules.
"""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1708_00765_gb300 as cls  # noqa: E402
from paper_1708_00765_gb300 import workloads  # noqa: E402

RTOL = 1e-12
BATCH_RTOL = 1e-10
COUNT_KEYS = ("nR", "nT", "nA", "n_coll", "n_int", "n_refl", "n_events", "max_events", "n_capped")
GPU_KEYS = {"n_int": "n_interface", "n_refl": "n_reflect"}


def ocase(p):
    return oracle.Case(*p[:7], int(p[7]), int(p[8]))


def assert_parity(raw_g, raw_o):
    for k in COUNT_KEYS:
        assert raw_g[GPU_KEYS.get(k, k)] == raw_o[k], k
    for k in ("sum_t", "sum_t2"):
        assert raw_g[k] == pytest.approx(raw_o[k], rel=RTOL), k
    fo = raw_o["flux"]
    fg = raw_g["flux"][: fo.shape[0]]
    scale = max(np.abs(fo).max(), 1e-300)
    np.testing.assert_allclose(fg.sum(0), fo.sum(0), rtol=RTOL, atol=1e-15 * scale)
    np.testing.assert_allclose(fg, fo, rtol=BATCH_RTOL, atol=1e-15 * scale)


def test_box_all_1e8_histories_match_the_oracle():
    """The benchmark's box workload, whole: 1e8 histories in one launch of the default
    launch shape against the oracle's 1e8 histories, split over the host cores."""
    p = workloads.BOX_L10
    n = workloads.BOX_L10_HISTORIES
    prob = cls.Problem(p)
    prob.run(n, 1)
    raw_g = prob.raw_tallies()
    prob.close()
    raw_o = oracle.run_parallel(ocase(p), 1, 0, n)
    assert raw_o["n_histories"] == n
    assert_parity(raw_g, raw_o)


def test_sweep_every_case_in_the_autotuned_batch_launch():
    """The 256-case sweep in FP64, in the launch the autotuner picks for it (as the
    benchmark does), every case's first 1e5 ids against the oracle."""
    cases = workloads.batch_sweep(256, seed=7, nbins=100)
    n = 100_000
    prob = cls.Problem(cases, batch=True)
    prob.autotune(max(4096, min(n // 16, 262_144)), seed=3)
    prob.run(n, 2)
    raws_g = [prob.raw_tallies(k) for k in range(len(cases))]
    prob.close()
    raws_o = oracle.run_many([ocase(c) for c in cases], 2, 0, n)
    for k, (g, o) in enumerate(zip(raws_g, raws_o)):
        try:
            assert_parity(g, o)
        except AssertionError as e:
            raise AssertionError(f"case {k}: {e}") from None


@pytest.mark.parametrize("schedule", ["history", "event"])
def test_diffusive_box_both_schedules(schedule):
    """L = 100, c = 0.999, 500 bins (histories of ~150 events, tails to 1e4): 1e6
    histories in FP64 on each schedule against the oracle."""
    p = workloads.BOX_DIFFUSIVE
    n = 1_000_000
    prob = cls.Problem(p)
    prob.set_option("schedule", schedule)
    prob.run(n, 5)
    raw_g = prob.raw_tallies()
    prob.close()
    raw_o = oracle.run_parallel(ocase(p), 5, 0, n)
    assert_parity(raw_g, raw_o)
