"""Pins for the standard errors: the oracle's `finalize` and the library's host
normaliser (cls_finalize_raw) against the spread of independent runs.

The paper quotes every CLS result with a standard error and compares two
results in units of their combined error (Sec. 5, Eq. combined_var), but it
never says how a CLS error is computed.  The reading taken here: R, T and A are
per-history Bernoulli means, sigma^2 = p(1 - p)/(N - 1); <phi> is the mean
per-history track length, sigma^2 from its per-history squares; phi_k takes
the batch-means error B/(B - 1) sum_b (n_b/N)^2 (X_b - X)^2.  Each of these is
unbiased for the variance of its estimate, which fixes it independently of the
formula: over K runs on independent seeds, the sample variance of an estimate
must match the mean of the variances the runs report.  With K = 256 the ratio
of the two has a standard deviation near sqrt(2/255) = 0.089, so a sigma scaled
by sqrt(2) either way (ratio 2 or 1/2) is more than five standard deviations
out; the planted-mistake test below checks that the bounds catch it.
"""
import math

import numpy as np
import pytest

import oracle

K = 256                 # independent runs (seeds)
NBATCH = 16             # statistics batches per run, each of 1024 histories
N = NBATCH * 1024       # histories per run

CASES = {
    "rod": oracle.Case(0.5, 5.0, 2.0, 0.5, 0.5, 0.9, 10.0, 1, 100),
    "box": oracle.Case(1.0, 2.0, 0.3, 0.7, 0.5, 0.8, 2.0, 3, 20),
}
# one bin over the whole box: the bin's batch-means error and <phi>'s
# per-history error are two estimates of the same standard error
ONE_BIN = oracle.Case(1.0, 2.0, 0.3, 0.7, 0.5, 0.8, 2.0, 3, 1)

_cache = {}


def runs(case):
    if case not in _cache:
        _cache[case] = oracle.run_seeds(case, range(1000, 1000 + K), 0, N, nbatch=NBATCH)
    return _cache[case]


def variance_ratio(values, sigmas):
    """(sample variance of the K estimates) / (mean reported variance), and the
    standard deviation of that ratio under the hypothesis that the reported
    variances are right (chi-square with K - 1 degrees of freedom, widened by
    the estimates' excess kurtosis)."""
    v = np.asarray(values, dtype=np.float64)
    s2 = np.asarray(sigmas, dtype=np.float64) ** 2
    ratio = v.var(ddof=1) / s2.mean()
    d = v - v.mean()
    kurt = (d ** 4).mean() / max((d ** 2).mean() ** 2, 1e-300)
    sd = math.sqrt(2.0 / (len(v) - 1) + max(kurt - 3.0, 0.0) / len(v))
    return ratio, sd


def check_spread(results, nbins, kmax=4.5):
    """Every scalar's ratio within kmax of 1 (and within [0.7, 1.4]); every bin's
    within kmax of its own spread; the bins' mean ratio within [0.8, 1.25]."""
    bad = []
    for key in ("R", "T", "A", "total_flux"):
        vals = [r[key] for r in results]
        sig = [r["sigma_" + key] for r in results]
        ratio, sd = variance_ratio(vals, sig)
        if not (abs(ratio - 1) < kmax * sd and 0.7 < ratio < 1.4):
            bad.append((key, ratio, sd))
    rs = []
    for k in range(nbins):
        ratio, sd = variance_ratio([r["flux"][k] for r in results], [r["flux_sigma"][k] for r in results])
        rs.append(ratio)
        if not abs(ratio - 1) < max(kmax * sd, 0.3):
            bad.append((f"bin {k}", ratio, sd))
    if not 0.8 < float(np.mean(rs)) < 1.25:
        bad.append(("bins' mean", float(np.mean(rs)), None))
    return bad


def finalize_all(case, raws, scale=1.0):
    out = []
    for raw in raws:
        res = dict(oracle.finalize(raw, case))
        for key in ("sigma_R", "sigma_T", "sigma_A", "sigma_total_flux"):
            res[key] = res[key] * scale
        res["flux_sigma"] = res["flux_sigma"] * scale
        out.append(res)
    return out


@pytest.mark.parametrize("name", sorted(CASES))
def test_oracle_sigmas_match_the_spread_of_independent_runs(name):
    case = CASES[name]
    results = finalize_all(case, runs(case))
    assert check_spread(results, case.nbins) == []


@pytest.mark.parametrize("scale", [math.sqrt(2.0), 1.0 / math.sqrt(2.0)])
@pytest.mark.parametrize("name", sorted(CASES))
def test_a_sigma_off_by_sqrt2_fails_the_spread_check(name, scale):
    """A planted mistake in the oracle's normalisation (every sigma scaled by
    sqrt(2) or 1/sqrt(2)) is caught for every observable."""
    case = CASES[name]
    bad = check_spread(finalize_all(case, runs(case), scale=scale), case.nbins)
    flagged = {b[0] for b in bad}
    assert {"R", "A", "total_flux", "bins' mean"} <= flagged
    assert case.nbins - sum(1 for f in flagged if f.startswith("bin ")) <= case.nbins // 10


def test_library_finalizer_matches_the_spread_of_independent_runs():
    """cls_finalize_raw (the library's host normaliser, no GPU needed) on the same
    raw tallies: its errors pass the same spread check."""
    import _multirank_worker as w
    from paper_1708_00765_gb300 import _native
    case = CASES["box"]
    results = []
    for raw in runs(case):
        results.append(_native.finalize_raw(w.oracle_raw_from(raw, N), case.L))
    assert check_spread(results, case.nbins) == []


def test_batch_means_and_per_history_errors_of_the_total_flux_agree():
    """With one bin, phi_0 L = <phi>: the bin's batch-means error (16 batches) and
    <phi>'s per-history error estimate the same quantity.  Averaged over K runs
    their squares agree within 6% (the batch-means variance has 15 degrees of
    freedom per run: relative spread 0.37 per run, 0.023 over 256 runs)."""
    raws = runs(ONE_BIN)
    res = finalize_all(ONE_BIN, raws)
    bm = np.array([r["flux_sigma"][0] * ONE_BIN.L for r in res])
    ph = np.array([r["sigma_total_flux"] for r in res])
    np.testing.assert_allclose([r["flux"][0] * ONE_BIN.L for r in res], [r["total_flux"] for r in res], rtol=1e-12)
    ratio = float((bm ** 2).mean() / (ph ** 2).mean())
    assert abs(ratio - 1.0) < 0.06, ratio
    # and both against the spread of the runs
    ratio, sd = variance_ratio([r["total_flux"] for r in res], bm)
    assert abs(ratio - 1) < 4.5 * sd
