"""cls_run_noalloc: the tracker for callers that cannot allocate device memory.

Such callers (a plugin inside another framework's memory budget, a process
that reserved all device memory up front) hand the library device buffers they
already own; the library keeps its own scratch in a static device array.  The
test owns the output buffers (allocating them here is the caller's business,
not the library's) and checks that two calls in a row give the same tallies as
the allocating entry point, cls_run, over the same history ranges: integer
counts bit-exact, track-length sums within 1e-12 relative.

This file is named so that pytest collects it last.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import oracle  # noqa: E402
import paper_1708_00765_gb300 as cls  # noqa: E402
from paper_1708_00765_gb300 import _native, workloads  # noqa: E402

RTOL = 1e-12
# order of the u64 counters in d_counters (include/cls.h)
COUNTERS = ("nR", "nT", "nA", "n_coll", "n_interface", "n_reflect", "n_events", "n_capped", "max_events")


def test_noalloc_two_calls_match_cls_run():
    cases = np.array([workloads.BOX_L10, workloads.ROD_L10, workloads.suite_case("2c", nbins=37)])
    nbatch, nbs = 16, 200
    nc = cases.shape[0]
    flux = torch.zeros((nc, nbatch, nbs), dtype=torch.float64, device="cuda")
    stats = torch.zeros((nc, 4), dtype=torch.float64, device="cuda")
    counters = torch.zeros((nc, 9), dtype=torch.int64, device="cuda")
    stream = torch.cuda.current_stream()
    ranges = [(0, 20_000), (20_000, 7_001)]
    for i, (first, n) in enumerate(ranges):
        rc = _native.run_noalloc(cases, first, n, 5, nbatch, nbs, flux.data_ptr(), stats.data_ptr(),
                                 counters.data_ptr(), stream)
        assert rc == _native.CLS_OK, cls.strerror(rc)
        torch.cuda.synchronize()
        f = flux.cpu().numpy()
        st = stats.cpu().numpy()
        ct = counters.cpu().numpy().view(np.uint64)
        # the allocating path over the same history ranges: a batch handle's case k
        # draws with Philox counter word 3 = k, like case k of the no-alloc call
        ref = cls.Problem(cases, batch=True)
        ref.set_option("nbatch", nbatch)
        for _, n0 in ranges[: i + 1]:
            ref.run(n0, 5)
        for k in range(nc):
            raw = ref.raw_tallies(k)
            for j, key in enumerate(COUNTERS):
                assert int(ct[k, j]) == raw[key], (i, k, key)
            for j, key in enumerate(("sum_t", "sum_t2")):
                assert st[k, j] == pytest.approx(raw[key], rel=RTOL)
            nb = int(cases[k, 8])
            np.testing.assert_allclose(f[k, :, :nb], raw["flux"], rtol=RTOL, atol=1e-15 * raw["flux"].max())
        ref.close()
    # and against the oracle itself: the counts of every case over both ranges
    for k in range(nc):
        c = oracle.Case(*cases[k][:7], int(cases[k][7]), int(cases[k][8]))
        parts = [oracle.run(c, 5, first, n, case_id=k) for first, n in ranges]
        for j, key in enumerate(("nR", "nT", "nA", "n_coll", "n_int", "n_refl", "n_events", "n_capped")):
            assert int(ct[k, j]) == sum(p[key] for p in parts), (k, key)
        assert int(ct[k, 8]) == max(p["max_events"] for p in parts)
        assert st[k, 0] == pytest.approx(sum(p["sum_t"] for p in parts), rel=RTOL)


def test_noalloc_rejects_too_many_cases():
    cases = np.array([workloads.ROD_L10] * (_native.CLS_NOALLOC_MAX_CASES + 1))
    buf = torch.zeros(16, dtype=torch.float64, device="cuda")
    rc = _native.run_noalloc(cases, 0, 100, 1, 4, 100, buf.data_ptr(), buf.data_ptr(), buf.data_ptr())
    assert rc == _native.CLS_E_INVAL


def test_noalloc_rejects_a_stride_beyond_its_maximum():
    cases = np.array([workloads.ROD_L10])
    buf = torch.zeros(16, dtype=torch.float64, device="cuda")
    for nbs in (99, _native.CLS_NOALLOC_MAX_STRIDE + 1):  # below the case's 100 bins; above the maximum
        rc = _native.run_noalloc(cases, 0, 100, 1, 4, nbs, buf.data_ptr(), buf.data_ptr(), buf.data_ptr())
        assert rc == _native.CLS_E_INVAL
