"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

FP64 mode: integer counts bit-exact, flux bins and track sums within 1e-12
relative (summation order only), traces event by event.  FP32 mode: within
4 combined standard errors of the oracle (paper Eq. combined_var), plus the
fraction of identical outcomes.
"""
import math

import numpy as np
import pytest

import oracle
from oracle import lp_ado

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


def ocase(p, source=0):
    return oracle.Case(*p[:7], int(p[7]), int(p[8]), source=source)


def gpu_raw(params, n, seed, first_runs=None, **opts):
    prob = cls.Problem(params)
    for k, v in opts.items():
        prob.set_option(k, v)
    for m in (first_runs or [n]):
        prob.run(m, seed)
    raw = prob.raw_tallies()
    tal = prob.tallies()
    prob.close()
    return raw, tal


def assert_parity(raw_g, raw_o, flux_o=None):
    for k in COUNT_KEYS:
        assert raw_g[GPU_KEYS.get(k, k)] == raw_o[k], k
    for k in ("sum_t", "sum_t2"):
        assert raw_g[k] == pytest.approx(raw_o[k], rel=RTOL), k
    for m in range(2):
        assert raw_g["track"][m] == pytest.approx(raw_o["track"][m], rel=RTOL, abs=1e-300)
    fo = raw_o["flux"] if flux_o is None else flux_o
    fg = raw_g["flux"][: fo.shape[0]]
    scale = max(np.abs(fo).max(), 1e-300)
    # flux per bin (summed over the statistics batches): 1e-12 relative
    np.testing.assert_allclose(fg.sum(0), fo.sum(0), rtol=RTOL, atol=1e-15 * scale)
    # the per-batch partial sums only feed standard errors; a flight that straddles
    # a bin edge at grazing incidence splits its length with a 1/|wx| sensitivity to
    # rounding of its start, so these are held to 1e-10
    np.testing.assert_allclose(fg, fo, rtol=BATCH_RTOL, atol=1e-15 * scale)


# ------------------------------------------------------------------ RNG

def test_philox_matches_curand_and_oracle():
    rng = np.random.default_rng(1)
    inp = rng.integers(0, 2**32, size=(1 << 20, 6), dtype=np.uint64).astype(np.uint32)
    inp[0] = 0
    inp[1] = 0xFFFFFFFF
    ours, theirs = cls.debug_philox(inp)
    assert np.array_equal(ours, theirs)
    for i in list(range(8)) + [12345, 999_999]:
        assert tuple(int(v) for v in ours[i]) == oracle.philox4x32_10(inp[i, :4], inp[i, 4:])


def test_uniform_mapping_matches_oracle():
    rng = np.random.default_rng(2)
    h = rng.integers(0, 2**40, size=4096, dtype=np.uint64)
    j = rng.integers(0, 2**31, size=4096, dtype=np.uint64)
    for seed, cid in ((1, 0), (2**45 + 7, 255)):
        u64, u32 = cls.debug_uniform(seed, cid, h, j)
        ref = np.array([oracle.uniform(seed, cid, int(a), int(b)) for a, b in zip(h, j)])
        assert np.array_equal(u64, ref)
        # FP32 draws are the same draw truncated to 24 bits
        assert np.array_equal(u32.astype(np.float64), np.floor(ref * 2**24) / 2**24)


def test_device_log_sincos_reciprocal_accuracy():
    """The FP64 walk's ln(1 - u) is within one ulp and its sin/cos(2 pi u)
    within 2^-52 of extended-precision references; u and mu = 2u - 1 are
    exact and 1/mu within one ulp; over random draws and the edges of the
    table ranges (u = 0, u < 2^-9, u near 1/2 and 1)."""
    rng = np.random.default_rng(11)
    edge = [0, 1, 2, 3, 2**44 - 1, 2**44, 2**44 + 1, 2**45 - 1, 2**45, 2**52 - 1, 2**52, 2**52 + 1,
            2**53 - 2, 2**53 - 1, 3 * 2**51, 2**51, 2**50]
    k = np.concatenate([np.array(edge, dtype=np.uint64),
                        rng.integers(0, 2**53, size=200_000, dtype=np.uint64),
                        (rng.integers(0, 2**53, size=50_000, dtype=np.uint64)
                         >> rng.integers(0, 53, size=50_000).astype(np.uint64))])
    out = cls.debug_math(k)
    ld = np.longdouble
    n = ld(2) ** 53

    def ulps(got, ref):
        return np.abs(got.astype(ld) - ref) / np.spacing(np.abs(ref.astype(np.float64))).astype(ld)

    ref_log = np.log((n - k.astype(ld)) / n)
    assert out["ln1m"][0] == 0.0 and float(ulps(out["ln1m"], ref_log)[1:].max()) <= 1.0
    two_pi = ld("6.283185307179586476925286766559005768394")
    ang = two_pi * (k.astype(ld) / n)
    assert float(np.max(np.abs(out["sin2pi"].astype(ld) - np.sin(ang)))) <= 2.0**-52
    assert float(np.max(np.abs(out["cos2pi"].astype(ld) - np.cos(ang)))) <= 2.0**-52
    u = k.astype(np.float64) * 2.0**-53  # exact: k < 2^53
    assert np.array_equal(out["u"], u)
    assert np.array_equal(out["mu"], 2.0 * u - 1.0)
    nz = out["mu"] != 0.0
    assert np.all(np.isinf(out["recip_mu"][~nz]))
    assert float(ulps(out["recip_mu"][nz], 1 / out["mu"][nz].astype(ld)).max()) <= 1.0


def _round_times_2_32(c):
    """round(c 2^32), ties to even, exactly, from the float32's significand and exponent."""
    bits = c.view(np.uint32).astype(np.int64)
    ex, fr = (bits >> 23) & 0xFF, bits & 0x7FFFFF
    m = np.where(ex > 0, fr | 0x800000, fr)             # c = m 2^(e - 23)
    sh = np.where(ex > 0, ex - 127, -126) - 23 + 32     # c 2^32 = m 2^sh
    out = np.zeros(c.size, dtype=np.uint64)
    up = sh >= 0
    out[up] = m[up].astype(np.uint64) << sh[up].astype(np.uint64)
    s = np.minimum(-sh[~up], 40)                        # m < 2^24: 2^40 rounds everything to 0
    q, r, half = m[~up] >> s, m[~up] & ((1 << s) - 1), 1 << (s - 1)
    out[~up] = (q + ((r > half) | ((r == half) & (q & 1 == 1)))).astype(np.uint64)
    return out


def test_fp32_fixed_point_conversion_rounds_exactly():
    """The FP32 walk adds track lengths to its tallies as round(c 2^32) with ties to
    even (exact integer sums): the device conversion against that value worked out
    from the float's bits, on ties, range ends and random floats across [0, 2^32)."""
    rng = np.random.default_rng(5)
    edge = np.array([0.0, 2.0**-33, 3 * 2.0**-33, 5 * 2.0**-33, 2.0**-32, 1.5 * 2.0**-32, 2.5 * 2.0**-32, 2.0**-40,
                     2.0**-126, 2.0**-8, 2.0**-8 + 2.0**-31, 0.5, 1.0, 1 - 2.0**-24, 1 + 2.0**-23, 2.0**23,
                     2.0**23 + 1, 2.0**24, 2.0**24 + 2, 2.0**31, 2.0**32 - 256, 12345.678], dtype=np.float32)
    scale = 2.0 ** rng.integers(-45, 32, 200_000).astype(np.float64)
    rnd = (rng.random(200_000) * scale).astype(np.float32)
    c = np.concatenate([edge, rnd, np.float32(2.0**-40) * np.arange(1, 2000, dtype=np.float32)])
    c = c[c < np.float32(2.0**32)]
    got = cls.debug_fixed32(c)
    ref = _round_times_2_32(c)
    bad = np.nonzero(got != ref)[0]
    assert bad.size == 0, [(float(c[i]), int(got[i]), int(ref[i])) for i in bad[:5]]
    assert got[0] == 0 and got[1] == 0 and got[2] == 2 and got[3] == 2 and got[5] == 2 and got[6] == 2
    with pytest.raises(cls.ClsError):
        cls.debug_fixed32(np.array([1.0, -1.0], dtype=np.float32))


# -------------------------------------------------------------- traces

@pytest.mark.parametrize("params", [workloads.ROD_L10, workloads.BOX_L10, workloads.suite_case("1c", nbins=10),
                                    workloads.suite_case("3c", d=11, nbins=10),
                                    workloads.suite_case("2c", d=2, nbins=10)])
def test_fp64_traces_replay_the_oracle(params):
    prob = cls.Problem(params)
    case = ocase(params)
    for h in list(range(48)) + [2**33 + 5, 10**8 - 1]:
        g = prob.trace(5, h)
        o, _ = oracle.trace(case, 5, h)
        assert g.shape == o.shape, h
        assert np.array_equal(g[:, [0, 1, 8]], o[:, [0, 1, 8]]), h  # events, draw indices, materials
        np.testing.assert_allclose(g[:, 2:8], o[:, 2:8], rtol=1e-11, atol=1e-12)
        np.testing.assert_allclose(g[:, 9], o[:, 9], rtol=1e-11, atol=1e-12)
    prob.close()


# ------------------------------------------------------- tallies parity

@pytest.mark.parametrize("chunk,block", [(256, 256), (32, 64), (1024, 128)])
def test_rod_config_full_parity(chunk, block):
    """The rod workload at its full size (1e5 histories): counts bit-exact, flux 1e-12."""
    p = workloads.ROD_L10
    raw_g, _ = gpu_raw(p, workloads.ROD_L10_HISTORIES, 1, chunk=chunk, block=block)
    raw_o = oracle.run_parallel(ocase(p), 1, 0, workloads.ROD_L10_HISTORIES)
    assert_parity(raw_g, raw_o)


@pytest.mark.parametrize("n", [1, 31, 1000, 20_037])
def test_box_parity_ragged(n):
    p = workloads.BOX_L10
    raw_g, _ = gpu_raw(p, n, 3)
    raw_o = oracle.run(ocase(p), 3, 0, n)
    assert_parity(raw_g, raw_o)


@pytest.mark.parametrize("params", [
    workloads.suite_case("1c", d=11, nbins=64),          # the paper's slab
    workloads.suite_case("2a", d=2, nbins=40),           # the paper's extruded 2D box
    workloads.BOX_L10_X,                                  # the box's x-marginal walk
    (0.7, 3.0, 0.4, 2.0, 0.8, 0.3, 3.0, 11, 13),         # slab, odd bin count
    (0.0, 2.0, 0.3, 0.7, 0.5, 0.5, 2.0, 3, 1),          # Sigma_0 = 0, one bin
    (1.0, 1.0, 1e-3, 2e-3, 1.0, 0.0, 1.0, 1, 4096),     # c = 1 / 0, maximum bins, tiny chords
    (3.0, 0.5, 50.0, 80.0, 0.0, 0.0, 0.01, 3, 7),      # pure absorbers, thin box, huge chords
    workloads.suite_case("3a", nbins=33),
])
def test_edge_cases_parity(params):
    raw_g, _ = gpu_raw(params, 5000, 11)
    raw_o = oracle.run(ocase(params), 11, 0, 5000)
    assert_parity(raw_g, raw_o)


def test_event_cap_parity():
    p = workloads.BOX_L10
    raw_g, tal = gpu_raw(p, 3000, 4, max_events=5)
    raw_o = oracle.run(ocase(p), 4, 0, 3000, max_events=5)
    assert raw_o["n_capped"] > 0
    assert tal["event_limit"]
    assert_parity(raw_g, raw_o)


def test_checkpoint_resume_equals_one_run():
    """run(a) + run(b) continues the history numbering: equal to the oracle over [0, a+b)."""
    p = workloads.ROD_L10
    raw_g, _ = gpu_raw(p, None, 7, first_runs=[30_000, 20_000])
    a = oracle.run(ocase(p), 7, 0, 30_000)
    b = oracle.run(ocase(p), 7, 30_000, 20_000)
    for k in COUNT_KEYS:
        ref = max(a[k], b[k]) if k == "max_events" else a[k] + b[k]
        assert raw_g[GPU_KEYS.get(k, k)] == ref
    assert raw_g["sum_t"] == pytest.approx(a["sum_t"] + b["sum_t"], rel=RTOL)
    np.testing.assert_allclose(raw_g["flux"][:a["flux"].shape[0]], a["flux"] + b["flux"], rtol=RTOL,
                               atol=1e-15 * a["flux"].max())


def test_box_full_size_sampled_range_and_properties():
    """The 1e8-history box workload in the benchmark's launch configuration: a sampled
    history range near the end of the id space matches the oracle exactly, and the full
    run satisfies the exact invariants and the LP expectation (paper Tables 3-5 pin the
    LP solver)."""
    p = workloads.BOX_L10
    n = workloads.BOX_L10_HISTORIES
    # sampled range at the top of the id space, same kernel and launch shape
    raw_o = oracle.run(ocase(p), 1, n - 10_000, 10_000)
    prob = cls.Problem(p)
    prob.run(n - 10_000, 1)
    head = prob.raw_tallies()
    prob.run(10_000, 1)
    full = prob.raw_tallies()
    tal = prob.tallies()
    prob.close()
    for k in ("nR", "nT", "nA", "n_coll", "n_events"):
        gk = GPU_KEYS.get(k, k)
        assert full[gk] - head[gk] == raw_o[k], k
    tail_flux = full["flux"] - head["flux"]
    np.testing.assert_allclose(tail_flux.sum(0), raw_o["flux"].sum(0), rtol=1e-6, atol=1e-9)
    # exact invariants of the whole run
    assert full["nR"] + full["nT"] + full["nA"] + full["n_capped"] == n
    assert full["n_events"] == full["n_coll"] + full["n_interface"] + full["n_reflect"] + full["nR"] + full["nT"]
    assert full["flux"].sum() == pytest.approx(full["sum_t"], rel=1e-9)
    lp = lp_ado.solve(p[0:2], p[2:4], p[4:6], p[6], "box3d", nbins=int(p[8]), n_half=48)
    for key in ("R", "T", "A"):
        assert abs(tal[key] - lp[key]) < 4 * tal["sigma_" + key]
    assert abs(tal["total_flux"] - lp["total_flux"]) < 4 * tal["sigma_total_flux"]
    z = (tal["flux"] - lp["flux"]) / tal["flux_sigma"]
    assert np.max(np.abs(z)) < 5 and np.mean(z * z) < 3.0


# ----------------------------------------------------------------- FP32

@pytest.mark.parametrize("params,kind", [(workloads.ROD_L10, "rod"), (workloads.BOX_L10, "box3d")])
def test_fp32_statistically_equal(params, kind):
    """FP32 tracking with FP64 tallies: within 4 combined sigma of the FP64 oracle on an
    independent seed, and most outcomes identical to FP64 on the same seed."""
    n = 200_000
    _, t32 = gpu_raw(params, n, 21, precision="fp32")
    raw_o = oracle.run_parallel(ocase(params), 22, 0, n)
    res_o = oracle.finalize(raw_o, ocase(params))
    for key in ("R", "T", "A"):
        comb = math.hypot(t32["sigma_" + key], res_o["sigma_" + key])
        if comb > 0:
            assert abs(t32[key] - res_o[key]) < 4 * comb, key
    comb = math.hypot(t32["sigma_total_flux"], res_o["sigma_total_flux"])
    assert abs(t32["total_flux"] - res_o["total_flux"]) < 4 * comb
    lp = lp_ado.solve(params[0:2], params[2:4], params[4:6], params[6], kind, nbins=int(params[8]))
    z = (t32["flux"] - lp["flux"]) / t32["flux_sigma"]
    assert np.max(np.abs(z)) < 5 and np.mean(z * z) < 3.0
    # identical outcomes between FP32 and FP64 on the same seed
    p32 = cls.Problem(params)
    p32.set_option("precision", "fp32")
    p64 = cls.Problem(params)
    same = 0
    for h in range(200):
        a = p32.trace(21, h)
        b = p64.trace(21, h)
        same += int(a[-1, 0]) == int(b[-1, 0])
    assert same >= 199  # measured: about one history in 10^6 ends differently


def _host_bins_of_fp32_flights(rows, L, nbins, source_x=0.0):
    """Score the flights of one FP32 trace on the host in FP64, by the rules of the
    track-length estimator (paper Sec. 2; the flight's x-extent clipped to [0, L]
    over |omega_x|, a flight inside one bin scores its length, omega_x = 0 scores
    in the bin of its start).  Row i holds the position and direction after event
    i, so flight i starts at row i - 1 (the source for i = 0) and moves along the
    direction of row i - 1; the first flight's omega_x is its x-extent over its
    length.  Returns (bins, per-material track)."""
    f32 = np.float32
    dx, inv_dx, Lf = f32(L / nbins), f32(nbins / L), f32(L)
    bins = np.zeros(nbins)
    track = [0.0, 0.0]
    x0 = f32(source_x)
    for i in range(rows.shape[0]):
        ev, l, x1, m_after = int(rows[i, 0]), float(rows[i, 9]), f32(rows[i, 2]), int(rows[i, 8])
        if ev == 6:
            break
        m = 1 - m_after if ev == 5 else m_after
        track[m] += l
        wx = float(rows[i - 1, 5]) if i > 0 else ((float(x1) - float(x0)) / l if l > 0 else 0.0)
        if l > 0:
            # bin coordinates in float, as the walk computes them: the bin a flight
            # end falls in is a decision, taken in the walk's precision
            lo, hi = max(min(x0, x1), f32(0)), min(max(x0, x1), Lf)
            if wx == 0.0:
                bins[min(int(f32(lo * inv_dx)), nbins - 1)] += l
            else:
                ulo, uhi = f32(lo * inv_dx), f32(hi * inv_dx)
                k0, k1 = min(int(ulo), nbins - 1), min(int(uhi), nbins - 1)
                if k0 == k1:
                    bins[k0] += l
                else:
                    c = float(dx) / abs(wx)
                    bins[k0] += (1.0 - float(f32(ulo - f32(k0)))) * c
                    bins[k1] += float(f32(uhi - f32(k1))) * c
                    bins[k0 + 1:k1] += c
        x0 = x1
    return bins, track


@pytest.mark.parametrize("params", [workloads.BOX_L10, workloads.ROD_L10, workloads.suite_case("2c", d=11, nbins=50),
                                    (1.0, 10.0, 0.5, 0.2, 0.99, 0.99, 10.0, 3, 500),
                                    # thin rod and box: most flights run from x = 0 to x = L, over whole end bins
                                    # (the short-history instance, whose deposits skip zero and end entries)
                                    (0.5, 5.0, 2.0, 0.5, 0.5, 0.9, 0.1, 1, 20),
                                    (0.5, 5.0, 2.0, 0.5, 0.5, 0.9, 0.1, 3, 20)])
def test_fp32_tallies_are_an_fp64_sum_of_the_fp32_flights(params):
    """FP32 tracking keeps its tallies in FP64 and exact fixed point: each history's
    flights are summed in float along the walk and widened once, every bin deposit
    is added exactly (32 fraction bits) and flushed into FP64.  Replayed from the FP32
    traces of the same histories -- the flights exactly as the walk made them, summed
    and binned on the host in FP64 -- the run's total track, its square sum and
    per-material tracks agree within 1e-6 relative (far below 0.01 standard
    errors), and every flux bin within 1e-4 of its FP64 binning (the walk's
    approximate reciprocal of omega_x against the host's division; a deposit that
    landed in the wrong bin, or a fixed-point entry lost, would be off by O(1))."""
    n = 3000
    prob = cls.Problem(params)
    prob.set_option("precision", "fp32")
    prob.run(n, 7)
    raw = prob.raw_tallies()
    tal = prob.tallies()
    L, nb = float(params[6]), int(params[8])
    t = np.zeros(n)
    bins = np.zeros(nb)
    track = np.zeros(2)
    for h in range(n):
        rows = prob.trace(7, h, cap=50_000)
        assert rows.shape[0] < 50_000
        t[h] = math.fsum(rows[:, 9])
        b, tr = _host_bins_of_fp32_flights(rows, L, nb)
        bins += b
        track += tr
    prob.close()
    sigma_sum = n * tal["sigma_total_flux"]
    assert abs(raw["sum_t"] - t.sum()) <= 1e-6 * t.sum()
    assert abs(raw["sum_t"] - t.sum()) <= 0.01 * sigma_sum
    assert raw["sum_t2"] == pytest.approx(float((t * t).sum()), rel=2e-6)
    np.testing.assert_allclose(raw["track"], track, rtol=1e-6)
    np.testing.assert_allclose(raw["flux"].sum(0), bins, rtol=1e-4, atol=1e-6 * bins.max())


@pytest.mark.parametrize("params", [workloads.ROD_L10, workloads.BOX_L10, workloads.suite_case("2c", d=11, nbins=50)])
@pytest.mark.parametrize("schedule", ["history", "event"])
def test_fp32_mode_runs_the_fp32_walk(params, schedule):
    """The same histories walked in FP32 and in FP64: outcomes all but identical, but the
    track sums differ at the float rounding level -- they would be bit-equal if the
    FP32 handle ran the FP64 kernels (the two precisions' launchers once collided at
    link time)."""
    raw32, _ = gpu_raw(params, 20_000, 3, precision="fp32", schedule=schedule)
    raw64, _ = gpu_raw(params, 20_000, 3, schedule=schedule)
    assert abs(raw32["nR"] - raw64["nR"]) <= 3
    rel = abs(raw32["sum_t"] - raw64["sum_t"]) / raw64["sum_t"]
    assert 1e-12 < rel < 1e-4


@pytest.mark.parametrize("schedule", ["history", "event"])
@pytest.mark.parametrize("nbins", [7, 200, 2000])
def test_fp32_flux_bins_add_up_to_the_track(schedule, nbins):
    """FP32 tallies: the bins -- the exact prefix sums of the fixed-point difference
    array -- add up to the histories' total track length, also on meshes whose tally
    regions need more than 48 KB of shared memory per block."""
    params = (1.0, 10.0, 0.5, 0.2, 0.99, 0.99, 10.0, 3, nbins)
    _, t = gpu_raw(params, 20_000, 5, precision="fp32", schedule=schedule)
    dx = params[6] / nbins
    assert t["flux"].sum() * dx == pytest.approx(t["total_flux"], rel=1e-5)
    assert t["nR"] + t["nT"] + t["nA"] == 20_000


# ---------------------------------------------------------------- batches

def test_batch_counts_exact_with_a_large_event_cap():
    """The short-history instance sums the histories' event counters over the warp in
    one 32-bit reduction while the event cap is below 2^27, and in 16-bit halves
    above it: with the cap at 2^28 the counts stay bit-exact against the oracle."""
    params = workloads.batch_sweep(12, seed=7, nbins=20)
    prob = cls.Problem(params, batch=True)
    prob.set_option("max_events", 1 << 28)
    prob.run(3000, 4)
    for k in range(params.shape[0]):
        raw_g = prob.raw_tallies(k)
        raw_o = oracle.run(ocase(params[k]), 4, 0, 3000, case_id=k, max_events=1 << 28)
        for key in COUNT_KEYS:
            assert raw_g[GPU_KEYS.get(key, key)] == raw_o[key], (k, key)
    prob.close()


@pytest.mark.parametrize("group_geometry", [1, 0])
def test_batch_cases_match_oracle_exactly(group_geometry):
    """Rods and boxes in one batch: one launch per geometry on parallel graph branches
    (the default), or one launch of the mixed-geometry walk."""
    params = workloads.batch_sweep(24, seed=7, nbins=20)
    prob = cls.Problem(params, batch=True)
    prob.set_option("group_geometry", group_geometry)
    prob.run(2000, 9)
    prob.run(1000, 9)  # graph replay with a new history range
    for k in range(params.shape[0]):
        raw_g = prob.raw_tallies(k)
        a = oracle.run(ocase(params[k]), 9, 0, 2000, case_id=k)
        b = oracle.run(ocase(params[k]), 9, 2000, 1000, case_id=k)
        for key in COUNT_KEYS:
            ref = max(a[key], b[key]) if key == "max_events" else a[key] + b[key]
            assert raw_g[GPU_KEYS.get(key, key)] == ref, (k, key)
        assert raw_g["sum_t"] == pytest.approx(a["sum_t"] + b["sum_t"], rel=RTOL)
    prob.close()


def _batch_exact(prob, params, seed, runs):
    """Every case's counts equal the oracle's over the given consecutive runs."""
    for k in range(params.shape[0]):
        raw_g = prob.raw_tallies(k)
        first = 0
        tot = {key: 0 for key in COUNT_KEYS}
        sum_t = 0.0
        for n in runs:
            o = oracle.run(ocase(params[k]), seed, first, n, case_id=k)
            for key in COUNT_KEYS:
                tot[key] = max(tot[key], o[key]) if key == "max_events" else tot[key] + o[key]
            sum_t += o["sum_t"]
            first += n
        for key in COUNT_KEYS:
            assert raw_g[GPU_KEYS.get(key, key)] == tot[key], (k, key)
        assert raw_g["sum_t"] == pytest.approx(sum_t, rel=RTOL)


def test_batch_with_mixed_case_schedules_matches_oracle_exactly():
    """Cases on the history and on the event schedule in one batch: two launches per
    replay of the captured graph, every case bit-exact against the oracle."""
    params = workloads.batch_sweep(12, seed=7, nbins=20)
    prob = cls.Problem(params, batch=True)
    prob.set_option("schedule", "history")
    for k in range(0, 12, 2):
        prob.set_case_schedule(k, "event")
    assert [prob.case_schedule(k) for k in range(12)] == [cls.CLS_SCHED_EVENT, cls.CLS_SCHED_HISTORY] * 6
    prob.run(2000, 9)
    prob.run(1000, 9)  # graph replay with a new history range
    _batch_exact(prob, params, 9, [2000, 1000])
    prob.close()


def test_batch_with_every_case_on_the_other_schedule():
    params = workloads.batch_sweep(6, seed=7, nbins=20)
    prob = cls.Problem(params, batch=True)
    prob.set_option("schedule", "history")
    for k in range(6):
        prob.set_case_schedule(k, "event")
    prob.run(1500, 4)
    _batch_exact(prob, params, 4, [1500])
    with pytest.raises(cls.ClsError):
        prob.set_case_schedule(6, "event")
    prob.close()


def test_autotune_cases_with_the_handle_schedule_still_automatic():
    """With the handle's schedule still to be tuned, every case keeps its own choice;
    the first run then tunes the handle's launch shape, and results stay exact."""
    params = workloads.batch_sweep(6, seed=7, nbins=20)
    prob = cls.Problem(params, batch=True)
    prob.set_option("schedule", "auto")
    chosen = prob.autotune_cases(4096, seed=3)
    assert set(chosen) <= {cls.CLS_SCHED_HISTORY, cls.CLS_SCHED_EVENT}
    prob.run(1200, 8)
    assert [prob.case_schedule(k) for k in range(6)] == chosen
    _batch_exact(prob, params, 8, [1200])
    prob.close()


def test_autotune_cases_keeps_results_exact():
    params = workloads.batch_sweep(8, seed=7, nbins=20)
    prob = cls.Problem(params, batch=True)
    prob.set_option("schedule", "history")
    chosen = prob.autotune_cases(4096, seed=3)
    assert len(chosen) == 8 and set(chosen) <= {cls.CLS_SCHED_HISTORY, cls.CLS_SCHED_EVENT}
    prob.run(1500, 6)
    _batch_exact(prob, params, 6, [1500])
    prob.close()


def test_fp32_batch_within_combined_sigma_of_oracle_per_case():
    """FP32-tracking batch, case by case, against the FP64 oracle on an independent seed
    and a history-id subset: R, T, A and <phi> within 4.5 combined standard errors
    (about 100 z-scores), their rms below 1.5."""
    params = workloads.batch_sweep(32, seed=7, nbins=20)
    prob = cls.Problem(params, batch=True)
    prob.set_option("precision", "fp32")
    prob.run(200_000, 31)
    t32 = [prob.tallies(k) for k in range(params.shape[0])]
    prob.close()
    cases = [ocase(p) for p in params]
    raws = oracle.run_many(cases, 32, 0, 20_000)
    zs = []
    for k, (c, raw) in enumerate(zip(cases, raws)):
        ref = oracle.finalize(raw, c)
        for key, skey in (("R", "sigma_R"), ("T", "sigma_T"), ("A", "sigma_A"), ("total_flux", "sigma_total_flux")):
            comb = math.hypot(t32[k][skey], ref[skey])
            if comb > 0:
                zs.append((t32[k][key] - ref[key]) / comb)
            else:
                assert t32[k][key] == ref[key], (k, key)
    zs = np.array(zs)
    assert len(zs) > 80
    assert np.max(np.abs(zs)) < 4.5
    assert np.sqrt(np.mean(zs * zs)) < 1.5


# ------------------------------------------------------- event schedule

@pytest.mark.parametrize("params", [workloads.ROD_L10, workloads.BOX_L10])
@pytest.mark.parametrize("epp,bank,block", [(1, 0, 256), (4, 256, 64), (16, 1024, 128)])
def test_event_schedule_fp64_parity(params, epp, bank, block):
    """The event-based tracker walks the same histories draw for draw: counts bit-exact."""
    n = 20_011
    raw_g, _ = gpu_raw(params, n, 13, schedule="event", events_per_pass=epp, bank=bank, block=block)
    raw_o = oracle.run(ocase(params), 13, 0, n)
    assert_parity(raw_g, raw_o)


def test_event_schedule_batch_parity():
    params = workloads.batch_sweep(12, seed=7, nbins=16)
    prob = cls.Problem(params, batch=True)
    prob.set_option("schedule", "event")
    prob.set_option("bank", 512)
    prob.run(1500, 9)
    for k in range(params.shape[0]):
        raw_g = prob.raw_tallies(k)
        raw_o = oracle.run(ocase(params[k]), 9, 0, 1500, case_id=k)
        assert_parity(raw_g, raw_o)
    prob.close()


def test_event_schedule_fp32_statistics():
    params = workloads.BOX_L10
    n = 200_000
    _, t_ev = gpu_raw(params, n, 31, precision="fp32", schedule="event")
    lp = lp_ado.solve(params[0:2], params[2:4], params[4:6], params[6], "box3d", nbins=int(params[8]))
    for key in ("R", "T", "A"):
        assert abs(t_ev[key] - lp[key]) < 4 * t_ev["sigma_" + key]
    z = (t_ev["flux"] - lp["flux"]) / t_ev["flux_sigma"]
    assert np.max(np.abs(z)) < 5 and np.mean(z * z) < 3.0


# ------------------------------------------------------------- autotuner

def test_autotune_keeps_results_exact():
    p = workloads.ROD_L10
    prob = cls.Problem(p)
    choice = prob.autotune(20_000, seed=3)
    assert choice["schedule"] in (cls.CLS_SCHED_HISTORY, cls.CLS_SCHED_EVENT)
    assert choice["block"] in (64, 128, 256)
    prob.run(30_000, 4)
    raw_g = prob.raw_tallies()
    prob.close()
    assert_parity(raw_g, oracle.run(ocase(p), 4, 0, 30_000))


def test_auto_schedule_tunes_on_first_run():
    p = workloads.BOX_L10
    prob = cls.Problem(p)
    prob.set_option("schedule", "auto")
    prob.run(20_000, 5)
    assert prob.get_option("schedule") in (cls.CLS_SCHED_HISTORY, cls.CLS_SCHED_EVENT)
    raw_g = prob.raw_tallies()
    prob.close()
    assert_parity(raw_g, oracle.run(ocase(p), 5, 0, 20_000))


TUNE_SCRIPT = """
import sys
sys.path.insert(0, {root!r})
import paper_1708_00765_gb300 as cls
p = cls.Problem([0.5, 5.0, 2.0, 0.5, 0.5, 0.9, 10.0, 1, 100])
print(p.autotune({pilot}, seed=1))
"""


def test_autotune_file_cache(tmp_path):
    """The autotuner's file cache: a second process finds the first one's result for a
    pilot of the same power of two (8192, then 12000), and a pilot of another size
    (65536) is tuned afresh under its own key."""
    import os
    import subprocess
    import sys
    cache = tmp_path / "tune.txt"
    env = dict(os.environ, CLS_AUTOTUNE_CACHE=str(cache))
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

    def tune(pilot):
        out = subprocess.run([sys.executable, "-c", TUNE_SCRIPT.format(root=root, pilot=pilot)], env=env,
                             capture_output=True, text=True, timeout=300)
        assert out.returncode == 0, out.stderr
        return cache.read_text().splitlines()

    assert len(tune(8192)) == 1
    lines = tune(12000)
    assert len(lines) == 1  # the second process found the first one's result
    key, sched, block, chunk, epp, gg = lines[0].split()
    assert "-s13-" in key and int(sched) in (1, 2) and int(block) in (64, 128, 256)
    lines = tune(65536)
    assert len(lines) == 2 and "-s16-" in lines[1].split()[0]


# ------------------------------------------------ the paper's printed values

def _paper_rows(d=3):
    import json
    import os
    from fractions import Fraction
    with open(os.path.join(os.path.dirname(__file__), "golden", "paper_cls_suite1.json")) as f:
        g = json.load(f)
    out = []
    for r in g["rows"]:
        if r["d"] != d:
            continue
        m = g["materials"]
        sig = [float(Fraction(v)) for v in m[r["case"][0]]["sigma"]]
        lam = [float(Fraction(v)) for v in m[r["case"][0]]["lambda"]]
        c = [float(v) for v in m[r["case"][1]]["c"]]
        out.append((r, (sig[0], sig[1], lam[0], lam[1], c[0], c[1], 10.0, {1: 11, 2: 2, 3: 3}[d], 100)))
    return out


@pytest.mark.parametrize("row,params", _paper_rows(3) + _paper_rows(1) + _paper_rows(2),
                         ids=lambda v: f"{v['case']}-d{v['d']}" if isinstance(v, dict) else "")
def test_fp64_reproduces_paper_tables(row, params):
    """Tables 3-5, d = 3 (box), d = 2 (extruded) and d = 1 (slab): the paper's Tripoli-4 CLS results
    (1e9 histories) against 1e8 FP64 GPU histories, within 4 combined standard
    errors (Eq. combined_var)."""
    prob = cls.Problem(params)
    prob.run(100_000_000, 2017)
    t = prob.tallies()
    prob.close()
    for key, ours, sd in (("R", t["R"], t["sigma_R"]), ("T", t["T"], t["sigma_T"]),
                          ("phi", t["total_flux"], t["sigma_total_flux"])):
        val, psd = float(row[key][0]), float(row[key][1])
        unit = 10.0 ** -len(row[key][0].split(".")[1])
        assert abs(ours - val) <= 4 * math.sqrt(sd * sd + psd * psd + (0.5 * unit) ** 2), (row["case"], key, ours, val)



# ------------------------------------------------------ suite II source

VOLUME_CASES = [workloads.ROD_L10, workloads.BOX_L10, workloads.suite_case("2c", d=11, nbins=30),
                workloads.suite_case("1b", d=2, nbins=30)]


@pytest.mark.parametrize("params", VOLUME_CASES)
def test_volume_source_traces_and_parity(params):
    """Suite II (uniform isotropic volume source): traces equal the oracle's event by
    event, and whole runs are bit-exact in counts."""
    prob = cls.Problem(params)
    prob.set_option("source", "volume")
    case = ocase(params, source=1)
    for h in range(24):
        g = prob.trace(9, h)
        o, _ = oracle.trace(case, 9, h)
        assert g.shape == o.shape and np.array_equal(g[:, [0, 1, 8]], o[:, [0, 1, 8]]), h
        np.testing.assert_allclose(g[:, 2:8], o[:, 2:8], rtol=1e-11, atol=1e-12)
    prob.run(10_007, 9)
    raw_g = prob.raw_tallies()
    prob.close()
    assert_parity(raw_g, oracle.run(case, 9, 0, 10_007))


def test_source_option_only_before_the_first_run():
    prob = cls.Problem(workloads.ROD_L10)
    prob.run(100, 1)
    with pytest.raises(cls.ClsError) as e:
        prob.set_option("source", "volume")
    assert e.value.code == cls._native.CLS_E_STATE
    prob.close()


def _paper_rows2(d):
    import json
    import os
    from fractions import Fraction
    here = os.path.dirname(__file__)
    with open(os.path.join(here, "golden", "paper_cls_suite2.json")) as f:
        g = json.load(f)
    with open(os.path.join(here, "golden", "paper_cls_suite1.json")) as f:
        m = json.load(f)["materials"]
    out = []
    for r in g["rows"]:
        if r["d"] != d:
            continue
        sig = [float(Fraction(v)) for v in m[r["case"][0]]["sigma"]]
        lam = [float(Fraction(v)) for v in m[r["case"][0]]["lambda"]]
        c = [float(v) for v in m[r["case"][1]]["c"]]
        out.append((r, (sig[0], sig[1], lam[0], lam[1], c[0], c[1], 10.0, {1: 11, 2: 2, 3: 3}[d], 100)))
    return out


@pytest.mark.parametrize("row,params", _paper_rows2(3) + _paper_rows2(1) + _paper_rows2(2),
                         ids=lambda v: f"{v['case']}-d{v['d']}" if isinstance(v, dict) else "")
def test_fp64_reproduces_paper_suite2_tables(row, params):
    """Tables 6-8 (suite II), d = 3, 2 and 1: leakage L = (T + R)/2 and <phi> from 1e8
    FP64 GPU histories against the paper's 1e9-history CLS values, 4 combined sigma."""
    prob = cls.Problem(params)
    prob.set_option("source", "volume")
    prob.run(100_000_000, 2018)
    t = prob.tallies()
    prob.close()
    N = t["n_histories"]
    pl = (t["nR"] + t["nT"]) / N
    lk, sd_lk = pl / 2, math.sqrt(pl * (1 - pl) / (N - 1)) / 2
    for key, ours, sd in (("L", lk, sd_lk), ("phi", t["total_flux"], t["sigma_total_flux"])):
        val, psd = float(row[key][0]), float(row[key][1])
        unit = 10.0 ** -len(row[key][0].split(".")[1])
        assert abs(ours - val) <= 4 * math.sqrt(sd * sd + psd * psd + (0.5 * unit) ** 2), (row["case"], key, ours, val)



def test_projected_box_matches_the_box_in_law():
    """Geometry 13 (the box walked in omega_x alone) against the canonical box on the
    GPU, 2e7 histories each on independent seeds: every observable within 4 combined
    standard errors, every flux bin within 5."""
    _, tb = gpu_raw(workloads.BOX_L10, 20_000_000, 41)
    _, tx = gpu_raw(workloads.BOX_L10_X, 20_000_000, 42)
    for key in ("R", "T", "A", "total_flux"):
        sk = "sigma_" + key
        assert abs(tb[key] - tx[key]) < 4 * math.hypot(tb[sk], tx[sk]), key
    z = (tb["flux"] - tx["flux"]) / np.hypot(tb["flux_sigma"], tx["flux_sigma"])
    assert np.max(np.abs(z)) < 5 and np.mean(z * z) < 3.0
    assert tx["n_reflect"] == 0 and tb["n_reflect"] > 0


@pytest.mark.parametrize("schedule", ["history", "event"])
@pytest.mark.parametrize("precision", ["fp64"])
def test_region_eviction_keeps_parity(schedule, precision):
    """1024 statistics batches and 32-history chunks: nearly every claim brings a new
    (case, batch) key, so warps keep evicting regions that still serve long histories,
    which then score into global memory.  Counts stay bit-exact and every batch's flux
    matches the oracle's."""
    p = workloads.BOX_L10
    n = 40_000
    raw_g, _ = gpu_raw(p, n, 23, schedule=schedule, precision=precision, nbatch=1024, chunk=32)
    raw_o = oracle.run(ocase(p), 23, 0, n, nbatch=1024)
    assert_parity(raw_g, raw_o)
