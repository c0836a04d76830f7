"""GB300-native Chord Length Sampling (CLS) random walks.

The walks run in hand-written sm_103a CUDA kernels inside ``libcls.so``
(C ABI in ``include/cls.h``); this package is its thin ctypes binding plus the
build step.  There is no CPU fallback: loading fails loudly if the library
has not been built.
"""
from . import build
from ._native import (CLS_E_EVENT_LIMIT, CLS_E_INVAL, CLS_E_STATE, CLS_OK, CLS_OUTCOME_ABSORBED, CLS_OUTCOME_CAPPED,
                      CLS_OUTCOME_REFLECTED, CLS_OUTCOME_TRANSMITTED, CLS_PREC_FP32, CLS_PREC_FP64, CLS_SCHED_EVENT,
                      CLS_SCHED_HISTORY, EXPORTED, ClsError, Problem, debug_fixed32, debug_math, debug_philox,
                      debug_uniform, load, strerror)

__all__ = ["build", "load", "Problem", "ClsError", "strerror", "debug_philox", "debug_uniform", "debug_math",
           "debug_fixed32", "EXPORTED",
           "CLS_OK", "CLS_E_EVENT_LIMIT", "CLS_E_INVAL", "CLS_E_STATE", "CLS_PREC_FP32", "CLS_PREC_FP64",
           "CLS_SCHED_EVENT", "CLS_SCHED_HISTORY", "CLS_OUTCOME_REFLECTED", "CLS_OUTCOME_TRANSMITTED",
           "CLS_OUTCOME_ABSORBED", "CLS_OUTCOME_CAPPED"]
