"""Plain FP64 CPU oracle for Chord Length Sampling (CLS) random walks.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  It shares no code with the CUDA library in
``paper_1708_00765_gb300``; the product path never falls back to it.

Contents
--------
* ``cls_oracle.c`` -- the Monte Carlo oracle: CLS Algorithm A (paper Sec. 4),
  3D source / scattering (Sec. 4.3), box boundary conditions (Sec. 2), the
  track-length flux estimator and R/T counts (Sec. 2, 3.3), driven by an
  independent Philox4x32-10 (Salmon et al., SC'11).
* ``lp_ado.py`` -- a deterministic solution of the Levermore-Pomraning
  equations (paper Eqs. ``boltzmann_ave`` + ``closure_lp_boltzmann``), which
  CLS solves in expectation; used to pin the Monte Carlo oracle.
* this module -- ctypes binding, a process-parallel driver and the
  normalisation of raw tallies into R, T, A, <phi>, phi(x) with standard errors
  (the per-batch statistics reading of sigma_CLS, paper Sec. 5).
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from dataclasses import dataclass, astuple

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "libcls_oracle.so")

DEFAULT_MAX_EVENTS = 100_000_000
DEFAULT_NBATCH = 64
BATCH_QUANTUM = 1024

EVENT_NAMES = {0: "leak_x0", 1: "leak_xL", 2: "reflect", 3: "scatter", 4: "absorb",
               5: "interface", 6: "capped"}


@dataclass(frozen=True)
class Case:
    """Parameters of one CLS problem (paper Tabs. 1-2 notation)."""
    sigma0: float
    sigma1: float
    lambda0: float
    lambda1: float
    c0: float
    c1: float
    L: float
    d: int          # 1 = rod (directions +-1), 2 = extruded 2D, 3 = box with reflective lateral faces, 11 = slab
    nbins: int
    source: int = 0  # 0 = incident flux on x = 0 (suite I), 1 = uniform isotropic volume source (suite II)

    @property
    def p0(self) -> float:
        """Volume fraction of material 0, p_0 = Lambda_0 / (Lambda_0 + Lambda_1) (paper Sec. 2)."""
        return self.lambda0 / (self.lambda0 + self.lambda1)


class _OrcCase(ctypes.Structure):
    _fields_ = [("sigma", ctypes.c_double * 2), ("lambda_", ctypes.c_double * 2),
                ("c", ctypes.c_double * 2), ("L", ctypes.c_double),
                ("d", ctypes.c_int32), ("nbins", ctypes.c_int32), ("source", ctypes.c_int32),
                ("pad", ctypes.c_int32)]


class _OrcCounts(ctypes.Structure):
    _fields_ = [(n, ctypes.c_uint64) for n in
                ("n_histories", "nR", "nT", "nA", "n_coll", "n_int", "n_refl", "n_events",
                 "max_events", "n_capped")] + [
        ("sum_t", ctypes.c_double), ("sum_t2", ctypes.c_double), ("track", ctypes.c_double * 2)]


COUNT_KEYS = ("n_histories", "nR", "nT", "nA", "n_coll", "n_int", "n_refl", "n_events",
              "max_events", "n_capped")


def build(force: bool = False) -> str:
    """Compile cls_oracle.c with plain gcc, FMA contraction off."""
    src = os.path.join(_HERE, "cls_oracle.c")
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= os.path.getmtime(src):
        return _SO
    os.makedirs(_BUILD, exist_ok=True)
    tmp = _SO + f".{os.getpid()}.tmp"
    subprocess.check_call(["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fno-fast-math",
                           "-fPIC", "-shared", "-o", tmp, src, "-lm"])
    os.replace(tmp, _SO)
    return _SO


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_SO)
        L.orc_philox4x32_10.argtypes = [ctypes.POINTER(ctypes.c_uint32)] * 3
        L.orc_philox4x32_10.restype = None
        L.orc_uniform.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_uint64]
        L.orc_uniform.restype = ctypes.c_double
        L.orc_run.argtypes = [ctypes.POINTER(_OrcCase), ctypes.c_uint32, ctypes.c_uint64,
                              ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64,
                              ctypes.c_uint32, ctypes.POINTER(_OrcCounts),
                              ctypes.POINTER(ctypes.c_double)]
        L.orc_run.restype = ctypes.c_int
        L.orc_trace.argtypes = [ctypes.POINTER(_OrcCase), ctypes.c_uint32, ctypes.c_uint64,
                                ctypes.c_uint64, ctypes.c_uint64, ctypes.POINTER(ctypes.c_double),
                                ctypes.c_int, ctypes.POINTER(_OrcCounts)]
        L.orc_trace.restype = ctypes.c_int
        L.orc_outcomes.argtypes = [ctypes.POINTER(_OrcCase), ctypes.c_uint32, ctypes.c_uint64,
                                   ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64,
                                   ctypes.POINTER(ctypes.c_uint8)]
        L.orc_outcomes.restype = ctypes.c_int
        _lib = L
    return _lib


def _ocase(case: Case) -> _OrcCase:
    oc = _OrcCase()
    oc.sigma[0], oc.sigma[1] = case.sigma0, case.sigma1
    oc.lambda_[0], oc.lambda_[1] = case.lambda0, case.lambda1
    oc.c[0], oc.c[1] = case.c0, case.c1
    oc.L, oc.d, oc.nbins, oc.source = case.L, int(case.d), int(case.nbins), int(case.source)
    return oc


def philox4x32_10(ctr, key):
    """Raw Philox4x32-10 block (4 x u32) for counter ctr (4 words) and key (2 words)."""
    c = (ctypes.c_uint32 * 4)(*[int(v) & 0xFFFFFFFF for v in ctr])
    k = (ctypes.c_uint32 * 2)(*[int(v) & 0xFFFFFFFF for v in key])
    o = (ctypes.c_uint32 * 4)()
    lib().orc_philox4x32_10(c, k, o)
    return tuple(int(v) for v in o)


def uniform(seed: int, case_id: int, h: int, j: int) -> float:
    """Draw j of history h (53-bit uniform in [0,1))."""
    return lib().orc_uniform(seed, case_id, h, j)


def batch_len(n: int, nbatch: int = DEFAULT_NBATCH) -> int:
    """Histories per statistics batch: 1024 * ceil(n / (1024 * nbatch))."""
    q = BATCH_QUANTUM * nbatch
    return BATCH_QUANTUM * max(1, -(-n // q))


def run(case: Case, seed: int, first: int, n: int, *, case_id: int = 0,
        max_events: int = DEFAULT_MAX_EVENTS, nbatch: int = DEFAULT_NBATCH) -> dict:
    """Run histories [first, first+n) and return raw tallies (counts, sums, flux[nbatch][nbins])."""
    oc = _ocase(case)
    cnt = _OrcCounts()
    bl = batch_len(n, nbatch)
    flux = np.zeros((nbatch, case.nbins), dtype=np.float64)
    rc = lib().orc_run(ctypes.byref(oc), case_id, seed, first, n, max_events, bl, nbatch,
                       ctypes.byref(cnt), flux.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    if rc != 0:
        raise ValueError("oracle rejected the case or arguments")
    out = {k: int(getattr(cnt, k)) for k in COUNT_KEYS}
    out.update(sum_t=cnt.sum_t, sum_t2=cnt.sum_t2, track=(cnt.track[0], cnt.track[1]),
               flux=flux, batch_len=bl, nbatch=nbatch, first=first, seed=seed)
    return out


def _run_piece(args):
    case_t, seed, first, n, case_id, max_events, bl, nbatch = args
    case = Case(*case_t)
    oc = _ocase(case)
    cnt = _OrcCounts()
    flux = np.zeros((nbatch, case.nbins), dtype=np.float64)
    rc = lib().orc_run(ctypes.byref(oc), case_id, seed, first, n, max_events, bl, nbatch,
                       ctypes.byref(cnt), flux.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    if rc != 0:
        raise ValueError("oracle rejected the case or arguments")
    return ({k: int(getattr(cnt, k)) for k in COUNT_KEYS}, cnt.sum_t, cnt.sum_t2,
            (cnt.track[0], cnt.track[1]), flux)


def run_parallel(case: Case, seed: int, first: int, n: int, *, workers: int | None = None,
                 case_id: int = 0, max_events: int = DEFAULT_MAX_EVENTS,
                 nbatch: int = DEFAULT_NBATCH) -> dict:
    """Same tallies as run(), computed by a spawn-started process pool over batch-aligned
    history ranges.  Counts are identical to run(); sums differ by summation order only."""
    import multiprocessing as mp
    workers = workers or os.cpu_count() or 1
    bl = batch_len(n, nbatch)
    nb_used = -(-n // bl)
    pieces = []
    per = max(1, -(-nb_used // workers))
    for b0 in range(0, nb_used, per):
        b1 = min(nb_used, b0 + per)
        lo, hi = b0 * bl, min(n, b1 * bl)
        pieces.append((b0, lo, hi))
    build()
    # pieces start on batch boundaries, so a piece's local batch k is global batch b0 + k
    args = [(astuple(case), seed, first + lo, hi - lo, case_id, max_events, bl,
             max(1, -(-(hi - lo) // bl))) for (b0, lo, hi) in pieces]
    ctx = mp.get_context("spawn")
    if len(args) == 1:
        results = [_run_piece(args[0])]
    else:
        with ctx.Pool(min(workers, len(args))) as pool:
            results = pool.map(_run_piece, args)
    out = {k: 0 for k in COUNT_KEYS}
    flux = np.zeros((nbatch, case.nbins))
    sum_t = sum_t2 = 0.0
    track = [0.0, 0.0]
    for (b0, lo, hi), (cnt, st, st2, tr, fl) in zip(pieces, results):
        for k in COUNT_KEYS:
            out[k] = max(out[k], cnt[k]) if k == "max_events" else out[k] + cnt[k]
        sum_t += st
        sum_t2 += st2
        track[0] += tr[0]
        track[1] += tr[1]
        flux[b0:b0 + fl.shape[0]] += fl
    out.update(sum_t=sum_t, sum_t2=sum_t2, track=tuple(track), flux=flux, batch_len=bl,
               nbatch=nbatch, first=first, seed=seed, workers=len(args))
    return out


def outcomes(case: Case, seed: int, first: int, n: int, *, case_id: int = 0,
             max_events: int = DEFAULT_MAX_EVENTS) -> np.ndarray:
    """Outcome of each history of [first, first+n): uint8 array, 0 reflected, 1 transmitted,
    2 absorbed, 3 event cap (paper Sec. 2 observables R, T, A)."""
    oc = _ocase(case)
    codes = np.zeros(n, dtype=np.uint8)
    rc = lib().orc_outcomes(ctypes.byref(oc), case_id, seed, first, n, max_events,
                            codes.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)))
    if rc != 0:
        raise ValueError("oracle rejected the case or arguments")
    return codes


def _run_case(args):
    case_t, seed, first, n, case_id = args
    return run(Case(*case_t), seed, first, n, case_id=case_id)


def run_many(cases, seed: int, first: int, n: int, *, case_ids=None, workers: int | None = None) -> list:
    """run() of several cases (case k with Philox counter word case_ids[k], default k),
    one task per case over a spawn-started process pool; a list of raw tallies."""
    import multiprocessing as mp
    case_ids = list(range(len(cases))) if case_ids is None else list(case_ids)
    build()
    args = [(astuple(c), seed, first, n, k) for c, k in zip(cases, case_ids)]
    workers = min(workers or os.cpu_count() or 1, len(args))
    if workers <= 1:
        return [_run_case(a) for a in args]
    with mp.get_context("spawn").Pool(workers) as pool:
        return pool.map(_run_case, args)


def _run_seed(args):
    case_t, seed, first, n, nbatch = args
    return run(Case(*case_t), seed, first, n, nbatch=nbatch)


def run_seeds(case: Case, seeds, first: int, n: int, *, nbatch: int = DEFAULT_NBATCH,
              workers: int | None = None) -> list:
    """run() of one case under several seeds (independent samples of the same
    histories' law), one task per seed over a spawn-started process pool."""
    import multiprocessing as mp
    build()
    args = [(astuple(case), int(s), first, n, nbatch) for s in seeds]
    workers = min(workers or os.cpu_count() or 1, len(args))
    if workers <= 1:
        return [_run_seed(a) for a in args]
    with mp.get_context("spawn").Pool(workers) as pool:
        return pool.map(_run_seed, args, chunksize=max(1, len(args) // (4 * workers)))


def trace(case: Case, seed: int, h: int, *, case_id: int = 0, max_events: int = DEFAULT_MAX_EVENTS,
          cap: int = 100_000):
    """Event-by-event trace of one history: array of rows
    (event, draw index after event, x, y, z, wx, wy, wz, material, flight length)."""
    oc = _ocase(case)
    cnt = _OrcCounts()
    rows = np.zeros((cap, 10), dtype=np.float64)
    nr = lib().orc_trace(ctypes.byref(oc), case_id, seed, h, max_events,
                         rows.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), cap, ctypes.byref(cnt))
    if nr < 0:
        raise ValueError("oracle rejected the case or arguments")
    out = {k: int(getattr(cnt, k)) for k in COUNT_KEYS}
    out.update(sum_t=cnt.sum_t, track=(cnt.track[0], cnt.track[1]))
    return rows[:nr].copy(), out


def finalize(raw: dict, case: Case) -> dict:
    """Normalise raw tallies per source particle (paper Sec. 2 observables).

    R, T, A are per-history Bernoulli means with standard error sqrt(p(1-p)/(N-1));
    <phi> is the mean total track length with its per-history standard error;
    phi_k = (track length in bin k) / (N dx) with a standard error from the
    batch means, sigma^2 = B/(B-1) sum_b (n_b/N)^2 (X_b - X)^2.
    """
    N = raw["n_histories"]
    dx = case.L / case.nbins
    res = {}
    for key, cnt in (("R", raw["nR"]), ("T", raw["nT"]), ("A", raw["nA"])):
        p = cnt / N
        res[key] = p
        res["sigma_" + key] = math.sqrt(p * (1 - p) / (N - 1)) if N > 1 else float("nan")
    mean_t = raw["sum_t"] / N
    res["total_flux"] = mean_t
    var_t = max(raw["sum_t2"] / N - mean_t * mean_t, 0.0)
    res["sigma_total_flux"] = math.sqrt(var_t / (N - 1)) if N > 1 else float("nan")
    flux = raw["flux"]
    bl = raw["batch_len"]
    nb_used = -(-N // bl)
    sizes = np.array([min(bl, N - b * bl) for b in range(nb_used)], dtype=np.float64)
    tot = flux[:nb_used].sum(axis=0)
    phi = tot / (N * dx)
    res["flux"] = phi
    if nb_used > 1:
        xb = flux[:nb_used] / (sizes[:, None] * dx)
        var = nb_used / (nb_used - 1) * (((sizes / N)[:, None] ** 2) * (xb - phi[None, :]) ** 2).sum(axis=0)
        res["flux_sigma"] = np.sqrt(var)
    else:
        res["flux_sigma"] = np.full(case.nbins, np.nan)
    res["track"] = (raw["track"][0] / N, raw["track"][1] / N)
    res["Lk"] = 0.5 * (res["R"] + res["T"])  # suite II leakage (paper Sec. 2)
    res["sigma_Lk"] = math.sqrt((raw["nR"] + raw["nT"]) / N * (1 - (raw["nR"] + raw["nT"]) / N) / (N - 1)) / 2 \
        if N > 1 else float("nan")
    for k in ("n_coll", "n_int", "n_refl", "n_events", "n_capped"):
        res[k] = raw[k]
    res["n_histories"] = N
    return res
