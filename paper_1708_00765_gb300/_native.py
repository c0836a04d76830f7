"""ctypes binding of libcls.so (include/cls.h): argument marshalling only.

Every step of the walk runs in the library's CUDA kernels.  If the library
has not been built this module raises; there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

CLS_OK = 0
CLS_E_INVAL = -1
CLS_E_NOMEM = -2
CLS_E_CUDA = -3
CLS_E_EVENT_LIMIT = -4
CLS_E_STATE = -5
CLS_E_NODEVICE = -6

CLS_OPT_PRECISION = 1
CLS_OPT_SCHEDULE = 2
CLS_OPT_BLOCK = 3
CLS_OPT_CHUNK = 4
CLS_OPT_NBATCH = 5
CLS_OPT_MAX_EVENTS = 6
CLS_OPT_BLOCKS_PER_SM = 7
CLS_OPT_BANK = 8
CLS_OPT_EVENTS_PER_PASS = 9
CLS_OPT_FIRST_HISTORY = 10
CLS_OPT_SOURCE = 11
CLS_OPT_GROUP_GEOMETRY = 12
CLS_SOURCE_INCIDENT = 0
CLS_SOURCE_VOLUME = 1

CLS_PREC_FP64 = 0
CLS_PREC_FP32 = 1
CLS_SCHED_AUTO = 0
CLS_SCHED_HISTORY = 1
CLS_SCHED_EVENT = 2

# every symbol include/cls.h declares
EXPORTED = ("cls_create", "cls_set_option", "cls_get_option", "cls_run", "cls_tallies", "cls_raw_tallies",
            "cls_reset", "cls_destroy", "cls_strerror", "cls_trace", "cls_batch_create", "cls_batch_run",
            "cls_batch_tallies", "cls_num_cases", "cls_debug_philox", "cls_debug_uniform", "cls_debug_math",
            "cls_debug_fixed32", "cls_run_noalloc", "cls_autotune", "cls_finalize_raw",
            "cls_record_outcomes", "cls_batch_set_case_schedule", "cls_batch_get_case_schedule",
            "cls_autotune_cases", "cls_workspace_bytes", "cls_bind_workspace")

CLS_NOALLOC_MAX_CASES = 64
CLS_NOALLOC_MAX_STRIDE = 4096
CLS_OUTCOME_REFLECTED = 0
CLS_OUTCOME_TRANSMITTED = 1
CLS_OUTCOME_ABSORBED = 2
CLS_OUTCOME_CAPPED = 3


class ClsError(RuntimeError):
    def __init__(self, code: int, what: str):
        self.code = code
        super().__init__(f"{what}: {strerror(code)} ({code})")


class cls_tallies_t(ctypes.Structure):
    _fields_ = [(n, ctypes.c_uint64) for n in
                ("n_histories", "nR", "nT", "nA", "n_coll", "n_interface", "n_reflect", "n_events",
                 "max_events", "n_capped")] + [
        (n, ctypes.c_double) for n in ("R", "T", "A", "total_flux", "sigma_R", "sigma_T", "sigma_A",
                                       "sigma_total_flux", "track0", "track1")] + [
        ("flux", ctypes.POINTER(ctypes.c_double)), ("flux_sigma", ctypes.POINTER(ctypes.c_double)),
        ("seconds", ctypes.c_double)]


class cls_raw_t(ctypes.Structure):
    _fields_ = [(n, ctypes.c_uint64) for n in
                ("n_histories", "nR", "nT", "nA", "n_coll", "n_interface", "n_reflect", "n_events",
                 "max_events", "n_capped")] + [
        ("sum_t", ctypes.c_double), ("sum_t2", ctypes.c_double), ("track", ctypes.c_double * 2),
        ("nbins", ctypes.c_int32), ("nbatch", ctypes.c_int32)]


_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = False) -> ctypes.CDLL:
    """Load libcls.so (building it first only if asked)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_build.LIB):
        if not build_if_missing:
            raise RuntimeError(f"libcls.so is not built ({_build.LIB}); run paper_1708_00765_gb300.build.build()")
        _build.build()
    L = ctypes.CDLL(_build.LIB)
    H = ctypes.c_void_p
    P = ctypes.POINTER
    d, i, u64, u32 = ctypes.c_double, ctypes.c_int, ctypes.c_uint64, ctypes.c_uint32
    sig = {
        "cls_create": ([d, d, d, d, d, d, d, i, i, P(H)], i),
        "cls_set_option": ([H, i, ctypes.c_int64], i),
        "cls_get_option": ([H, i, P(ctypes.c_int64)], i),
        "cls_run": ([H, u64, u64, H], i),
        "cls_tallies": ([H, P(cls_tallies_t)], i),
        "cls_raw_tallies": ([H, i, P(cls_raw_t), P(d), P(u64)], i),
        "cls_reset": ([H], i),
        "cls_destroy": ([H], None),
        "cls_strerror": ([i], ctypes.c_char_p),
        "cls_trace": ([H, i, u64, u64, P(d), i, P(i)], i),
        "cls_batch_create": ([P(d), i, P(H)], i),
        "cls_batch_run": ([H, u64, u64, H], i),
        "cls_batch_tallies": ([H, i, P(cls_tallies_t)], i),
        "cls_num_cases": ([H], i),
        "cls_debug_philox": ([P(u32), i, P(u32), P(u32)], i),
        "cls_debug_uniform": ([u64, u32, P(u64), P(u64), i, P(d), P(ctypes.c_float)], i),
        "cls_debug_math": ([P(u64), i, P(d), P(d), P(d), P(d), P(d), P(d)], i),
        "cls_debug_fixed32": ([P(ctypes.c_float), i, P(u64)], i),
        "cls_run_noalloc": ([P(d), i, u64, u64, u64, i, i, H, H, H, H], i),
        "cls_autotune": ([H, u64, u64, H], i),
        "cls_finalize_raw": ([P(cls_raw_t), P(d), P(u64), d, P(cls_tallies_t)], i),
        "cls_record_outcomes": ([H, H, u64], i),
        "cls_batch_set_case_schedule": ([H, i, i], i),
        "cls_batch_get_case_schedule": ([H, i, P(i)], i),
        "cls_autotune_cases": ([H, u64, u64, H], i),
        "cls_workspace_bytes": ([H, P(ctypes.c_size_t)], i),
        "cls_bind_workspace": ([H, H, ctypes.c_size_t], i),
    }
    for name, (args, res) in sig.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = res
    _lib = L
    return L


def strerror(code: int) -> str:
    return load().cls_strerror(code).decode()


def _check(code: int, what: str, ok=(CLS_OK,)) -> int:
    if code not in ok:
        raise ClsError(code, what)
    return code


def _ptr(a, ctype=ctypes.c_double):
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def _stream_handle(stream) -> int | None:
    """Accept None (default stream), an int handle, or a torch.cuda.Stream."""
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)


OPTIONS = {"precision": CLS_OPT_PRECISION, "schedule": CLS_OPT_SCHEDULE, "block": CLS_OPT_BLOCK,
           "chunk": CLS_OPT_CHUNK, "nbatch": CLS_OPT_NBATCH, "max_events": CLS_OPT_MAX_EVENTS,
           "blocks_per_sm": CLS_OPT_BLOCKS_PER_SM, "bank": CLS_OPT_BANK,
           "events_per_pass": CLS_OPT_EVENTS_PER_PASS, "first_history": CLS_OPT_FIRST_HISTORY, "source": CLS_OPT_SOURCE,
           "group_geometry": CLS_OPT_GROUP_GEOMETRY}
VALUES = {"fp64": CLS_PREC_FP64, "fp32": CLS_PREC_FP32, "history": CLS_SCHED_HISTORY, "event": CLS_SCHED_EVENT,
          "auto": CLS_SCHED_AUTO, "incident": CLS_SOURCE_INCIDENT, "volume": CLS_SOURCE_VOLUME}


class Problem:
    """One handle of libcls: a single case (cls_create) or a batch (cls_batch_create)."""

    def __init__(self, params, batch: bool = False):
        L = load()
        self._h = ctypes.c_void_p()
        params = np.ascontiguousarray(np.atleast_2d(np.asarray(params, dtype=np.float64)))
        if params.shape[1] != 9:
            raise ValueError("each case is (sigma0, sigma1, lambda0, lambda1, c0, c1, L, d, nbins)")
        self.params = params
        if batch:
            _check(L.cls_batch_create(_ptr(params), params.shape[0], ctypes.byref(self._h)), "cls_batch_create")
        else:
            if params.shape[0] != 1:
                raise ValueError("cls_create takes one case")
            p = params[0]
            _check(L.cls_create(*[float(v) for v in p[:7]], int(p[7]), int(p[8]), ctypes.byref(self._h)),
                   "cls_create")
        self.batch = batch
        self.nbins = [int(v) for v in params[:, 8]]

    # -- lifetime
    def close(self):
        if self._h:
            load().cls_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- options
    def set_option(self, key, value):
        k = OPTIONS[key] if isinstance(key, str) else key
        v = VALUES.get(value, value) if isinstance(value, str) else value
        _check(load().cls_set_option(self._h, k, int(v)), f"cls_set_option({key})")

    def get_option(self, key) -> int:
        k = OPTIONS[key] if isinstance(key, str) else key
        out = ctypes.c_int64()
        _check(load().cls_get_option(self._h, k, ctypes.byref(out)), f"cls_get_option({key})")
        return out.value

    # -- runs
    def run(self, n: int, seed: int, stream=None):
        fn = load().cls_batch_run if self.batch else load().cls_run
        _check(fn(self._h, n, seed, _stream_handle(stream)), "cls_batch_run" if self.batch else "cls_run")

    def reset(self):
        _check(load().cls_reset(self._h), "cls_reset")

    def record_outcomes(self, d_codes: int, capacity: int):
        """cls_record_outcomes: later runs write each history's CLS_OUTCOME_* code into the
        device buffer at address d_codes (capacity bytes; 0 stops recording)."""
        _check(load().cls_record_outcomes(self._h, d_codes or None, capacity if d_codes else 0),
               "cls_record_outcomes")

    def autotune(self, n_pilot: int, seed: int = 1, stream=None) -> dict:
        """cls_autotune: returns the chosen schedule and launch shape."""
        _check(load().cls_autotune(self._h, n_pilot, seed, _stream_handle(stream)), "cls_autotune")
        return {k: self.get_option(k) for k in ("schedule", "block", "chunk", "events_per_pass", "group_geometry")}

    def set_case_schedule(self, case: int, schedule):
        """cls_batch_set_case_schedule: "history", "event" or "auto" (follow the handle's)."""
        v = VALUES.get(schedule, schedule) if isinstance(schedule, str) else schedule
        _check(load().cls_batch_set_case_schedule(self._h, case, int(v)), "cls_batch_set_case_schedule")

    def case_schedule(self, case: int) -> int:
        out = ctypes.c_int()
        _check(load().cls_batch_get_case_schedule(self._h, case, ctypes.byref(out)), "cls_batch_get_case_schedule")
        return out.value

    def autotune_cases(self, n_pilot: int, seed: int = 1, stream=None) -> list:
        """cls_autotune_cases: returns every case's chosen schedule (CLS_SCHED_*)."""
        _check(load().cls_autotune_cases(self._h, n_pilot, seed, _stream_handle(stream)), "cls_autotune_cases")
        return [self.case_schedule(k) for k in range(self.params.shape[0])]

    def workspace_bytes(self) -> int:
        """cls_workspace_bytes: device bytes the handle needs for its current options."""
        out = ctypes.c_size_t()
        _check(load().cls_workspace_bytes(self._h, ctypes.byref(out)), "cls_workspace_bytes")
        return out.value

    def bind_workspace(self, d_ptr: int, nbytes: int):
        """cls_bind_workspace: hold the handle's device buffers in caller-owned device
        memory at address d_ptr (e.g. a torch tensor's data_ptr()); 0 unbinds."""
        _check(load().cls_bind_workspace(self._h, d_ptr or None, nbytes if d_ptr else 0), "cls_bind_workspace")

    def tallies(self, case: int = 0) -> dict:
        nb = self.nbins[case]
        flux = np.zeros(nb)
        fsig = np.zeros(nb)
        t = cls_tallies_t()
        t.flux = _ptr(flux)
        t.flux_sigma = _ptr(fsig)
        if self.batch:
            rc = load().cls_batch_tallies(self._h, case, ctypes.byref(t))
        else:
            rc = load().cls_tallies(self._h, ctypes.byref(t))
        _check(rc, "cls_tallies", ok=(CLS_OK, CLS_E_EVENT_LIMIT))
        out = {n: getattr(t, n) for n, _ in cls_tallies_t._fields_ if n not in ("flux", "flux_sigma")}
        out["flux"] = flux
        out["flux_sigma"] = fsig
        out["event_limit"] = rc == CLS_E_EVENT_LIMIT
        return out

    def raw_tallies(self, case: int = 0) -> dict:
        r = cls_raw_t()
        nbatch = self.get_option("nbatch")
        nb = self.nbins[case]
        fl = np.zeros((nbatch, nb))
        bh = np.zeros(nbatch, dtype=np.uint64)
        _check(load().cls_raw_tallies(self._h, case, ctypes.byref(r), _ptr(fl), _ptr(bh, ctypes.c_uint64)),
               "cls_raw_tallies")
        out = {n: getattr(r, n) for n, _ in cls_raw_t._fields_ if n != "track"}
        out["track"] = (r.track[0], r.track[1])
        out["flux"] = fl
        out["batch_histories"] = bh
        return out

    def trace(self, seed: int, history: int, case: int = 0, cap: int = 100_000):
        rows = np.zeros((cap, 10))
        n = ctypes.c_int()
        _check(load().cls_trace(self._h, case, seed, history, _ptr(rows), cap, ctypes.byref(n)), "cls_trace")
        return rows[:min(n.value, cap)].copy()


def debug_philox(inp: np.ndarray):
    inp = np.ascontiguousarray(inp, dtype=np.uint32).reshape(-1, 6)
    n = inp.shape[0]
    ours = np.zeros((n, 4), dtype=np.uint32)
    theirs = np.zeros((n, 4), dtype=np.uint32)
    _check(load().cls_debug_philox(_ptr(inp, ctypes.c_uint32), n, _ptr(ours, ctypes.c_uint32),
                                   _ptr(theirs, ctypes.c_uint32)), "cls_debug_philox")
    return ours, theirs


def debug_uniform(seed: int, case_id: int, h, j):
    h = np.ascontiguousarray(h, dtype=np.uint64)
    j = np.ascontiguousarray(j, dtype=np.uint64)
    n = h.size
    o64 = np.zeros(n)
    o32 = np.zeros(n, dtype=np.float32)
    _check(load().cls_debug_uniform(seed, case_id, _ptr(h, ctypes.c_uint64), _ptr(j, ctypes.c_uint64), n,
                                    _ptr(o64), _ptr(o32, ctypes.c_float)), "cls_debug_uniform")
    return o64, o32


def debug_math(k):
    """cls_debug_math: the FP64 walk's ln(1 - u), sin(2 pi u), cos(2 pi u), u, mu = 2u - 1
    and 1/mu for u = k 2^-53, as a dict of arrays."""
    k = np.ascontiguousarray(k, dtype=np.uint64)
    n = k.size
    out = {name: np.zeros(n) for name in ("ln1m", "sin2pi", "cos2pi", "u", "mu", "recip_mu")}
    _check(load().cls_debug_math(_ptr(k, ctypes.c_uint64), n, *(_ptr(out[name]) for name in out)), "cls_debug_math")
    return out


def debug_fixed32(c):
    """cls_debug_fixed32: the FP32 walk's conversion round(c 2^32) of floats c in [0, 2^32)."""
    c = np.ascontiguousarray(c, dtype=np.float32)
    out = np.zeros(c.size, dtype=np.uint64)
    _check(load().cls_debug_fixed32(_ptr(c, ctypes.c_float), c.size, _ptr(out, ctypes.c_uint64)),
           "cls_debug_fixed32")
    return out


def run_noalloc(params, first: int, n: int, seed: int, nbatch: int, nbins_stride: int, d_flux: int, d_stats: int,
                d_counters: int, stream=None) -> int:
    """cls_run_noalloc: tallies are added into caller-owned device buffers given as
    raw device addresses; returns the library's status code."""
    params = np.ascontiguousarray(np.atleast_2d(np.asarray(params, dtype=np.float64)))
    return load().cls_run_noalloc(_ptr(params), params.shape[0], first, n, seed, nbatch, nbins_stride, d_flux,
                                  d_stats, d_counters, _stream_handle(stream))


RAW_COUNT_KEYS = ("n_histories", "nR", "nT", "nA", "n_coll", "n_interface", "n_reflect", "n_events", "max_events",
                  "n_capped")


def finalize_raw(raw: dict, L: float) -> dict:
    """cls_finalize_raw: normalise (possibly merged) raw tallies on the host."""
    r = cls_raw_t()
    for k in RAW_COUNT_KEYS:
        setattr(r, k, int(raw[k]))
    r.sum_t, r.sum_t2 = float(raw["sum_t"]), float(raw["sum_t2"])
    r.track[0], r.track[1] = float(raw["track"][0]), float(raw["track"][1])
    flux = np.ascontiguousarray(raw["flux"], dtype=np.float64)
    r.nbatch, r.nbins = flux.shape
    bh = np.ascontiguousarray(raw["batch_histories"], dtype=np.uint64)
    out_flux = np.zeros(r.nbins)
    out_sig = np.zeros(r.nbins)
    t = cls_tallies_t()
    t.flux = _ptr(out_flux)
    t.flux_sigma = _ptr(out_sig)
    rc = load().cls_finalize_raw(ctypes.byref(r), _ptr(flux), _ptr(bh, ctypes.c_uint64), float(L), ctypes.byref(t))
    _check(rc, "cls_finalize_raw", ok=(CLS_OK, CLS_E_EVENT_LIMIT))
    out = {n: getattr(t, n) for n, _ in cls_tallies_t._fields_ if n not in ("flux", "flux_sigma")}
    out["flux"] = out_flux
    out["flux_sigma"] = out_sig
    return out
