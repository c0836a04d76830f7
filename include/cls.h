/*
 * cls.h -- C ABI of the GB300 Chord Length Sampling (CLS) library (libcls.so).
 *
 * The library runs CLS "Algorithm A" random walks (paper Sec. 4) for
 * single-speed transport with isotropic scattering through a binary Markov
 * mixture.  Geometries (the `d` argument):
 *   CLS_GEOM_ROD  (1)  rod of length L, directions +-1;
 *   CLS_GEOM_EXTRUDED (2) the paper's 2D extruded box (Sec. 4.2): x faces leak,
 *                      y faces reflect, invariant along z; the interface
 *                      distance is the in-plane chord along the flight,
 *                      Lambda/sqrt(1 - mu_z^2);
 *   CLS_GEOM_BOX  (3)  3D box of side L (paper Sec. 4.3) with leakage on the
 *                      faces normal to x and specular reflection on the four
 *                      lateral faces (paper Sec. 2);
 *   CLS_GEOM_SLAB (11) the paper's d = 1 slab (Sec. 4.1): continuous direction
 *                      cosine mu, interface distance projected on x
 *                      (Lambda/|mu|), leakage on both faces;
 *   CLS_GEOM_BOX_X (13) the box's x-marginal: since specular lateral faces keep
 *                      omega_x, the box's tallies have the law of a walk in
 *                      mu = omega_x alone (scatter mu = 2 xi - 1, chords along
 *                      the flight, no lateral events).  Same law as
 *                      CLS_GEOM_BOX, fewer draws, not draw-for-draw equal.
 * Sources (CLS_OPT_SOURCE): the isotropic incident flux on x = 0 of benchmark
 * suite I (cosine law mu = sqrt(xi), paper Sec. 4.1 / 4.3, the default), or
 * the uniform isotropic volume source of suite II.  Estimators: reflection R = J(x=0),
 * transmission T = J(x=L), absorption A, and the track-length scalar flux
 * phi(x) integrated over y and z on a uniform x mesh (paper Sec. 2).
 *
 * Everything runs on one CUDA device in hand-written kernels; there is no CPU
 * fallback.  Pointers are plain host pointers unless stated; streams are
 * cudaStream_t passed as void* (NULL = the legacy default stream).
 *
 * Error handling: every int-returning call returns CLS_OK (0) or a negative
 * CLS_E_* code; cls_strerror() names it.  A call that fails leaves the handle
 * usable unless it returned CLS_E_CUDA, after which the CUDA context may be
 * unusable (sticky device error).  Nothing is ever printed.
 *
 * Thread safety: a handle may be used by one host thread at a time.
 */
#ifndef CLS_H
#define CLS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------- geometries */
#define CLS_GEOM_ROD 1
#define CLS_GEOM_EXTRUDED 2
#define CLS_GEOM_BOX 3
#define CLS_GEOM_SLAB 11
#define CLS_GEOM_BOX_X 13

/* ------------------------------------------------------------ error codes */
#define CLS_OK 0
#define CLS_E_INVAL (-1)       /* invalid argument or parameter out of range          */
#define CLS_E_NOMEM (-2)       /* host or device allocation failed                    */
#define CLS_E_CUDA (-3)        /* a CUDA runtime call or kernel launch failed         */
#define CLS_E_EVENT_LIMIT (-4) /* some history hit the per-history event cap;        */
                               /* tallies are still filled (capped histories count    */
                               /* in n_capped and in no outcome)                      */
#define CLS_E_STATE (-5)       /* call not valid in the handle's state                */
#define CLS_E_NODEVICE (-6)    /* no CUDA device: the library never runs on the CPU   */

/* ---------------------------------------------------------------- options */
#define CLS_OPT_PRECISION 1     /* CLS_PREC_FP64 (default) or CLS_PREC_FP32                 */
#define CLS_OPT_SCHEDULE 2      /* CLS_SCHED_HISTORY (default), CLS_SCHED_EVENT, CLS_SCHED_AUTO */
#define CLS_OPT_BLOCK 3         /* threads per block, multiple of 32 in [32, 256]; the FP64
                                   history tracker uses at most 128, the FP32 history tracker
                                   for the 3D box at most 224 (their launch bounds)          */
#define CLS_OPT_CHUNK 4         /* histories a warp claims at once: 32, 64, ..., 1024       */
#define CLS_OPT_NBATCH 5        /* statistics batches per run, 2..1024 (default 64)         */
#define CLS_OPT_MAX_EVENTS 6    /* per-history event cap, 1..2^28 (default 1e8)             */
#define CLS_OPT_BLOCKS_PER_SM 7 /* persistent grid = SMs x this; 0 = occupancy maximum     */
#define CLS_OPT_BANK 8          /* event schedule: bank particles per warp, 0..4096, rounded  */
                                /* up to a multiple of 32 (0 = 128)                         */
#define CLS_OPT_EVENTS_PER_PASS 9 /* event schedule: events per particle per pass (1..64)  */
#define CLS_OPT_FIRST_HISTORY 10  /* set the next history id of every case (0..2^62); lets   */
                                  /* processes walk disjoint history ranges of one seed     */
#define CLS_OPT_SOURCE 11         /* CLS_SOURCE_INCIDENT (default) or CLS_SOURCE_VOLUME, for */
                                  /* every case; only before the first run (CLS_E_STATE)    */
#define CLS_OPT_GROUP_GEOMETRY 12 /* 1 (default): a batch whose cases have several geometries */
                                  /* runs one persistent launch per geometry, each compiled   */
                                  /* for its geometry, as parallel branches of its CUDA graph; */
                                  /* 0: one launch of the mixed-geometry walk                 */

#define CLS_SOURCE_INCIDENT 0 /* suite I: isotropic incident flux on x = 0, cosine law (Sec. 4.1/4.3) */
#define CLS_SOURCE_VOLUME 1   /* suite II: one particle, uniform in the volume, isotropic (Sec. 2,    */
                              /* 4.1, 4.3); the paper's leakage is L = (R + T) / 2                      */

#define CLS_PREC_FP64 0 /* all arithmetic in FP64 (draw-for-draw equal to the FP64 oracle) */
#define CLS_PREC_FP32 1 /* position / direction / distance in FP32, tallies in FP64          */

#define CLS_SCHED_AUTO 0    /* cls_autotune picks the schedule and launch shape at the first run */
#define CLS_SCHED_HISTORY 1 /* persistent history-based tracker, state in registers          */
#define CLS_SCHED_EVENT 2   /* event-based tracker over a structure-of-arrays particle bank   */

/* --------------------------------------------------------------- results */
typedef struct cls_handle cls_handle; /* opaque, owned by the library */

/* Normalised results of one case, filled by cls_tallies / cls_batch_tallies.
 * All per-source-particle (unit incident current).  Caller-owned. */
typedef struct {
    uint64_t n_histories; /* histories accumulated since create / reset            */
    uint64_t nR, nT, nA;  /* reflected, transmitted, absorbed histories            */
    uint64_t n_coll;      /* collisions                                            */
    uint64_t n_interface; /* material-interface crossings                          */
    uint64_t n_reflect;   /* specular reflections on lateral faces (box only)      */
    uint64_t n_events;    /* all events (flights)                                  */
    uint64_t max_events;  /* longest history, in events                            */
    uint64_t n_capped;    /* histories stopped by the event cap                    */
    double R, T, A;       /* nR/N, nT/N, nA/N                                       */
    double total_flux;    /* <phi> = int phi(x) dx = mean track length per history  */
    double sigma_R, sigma_T, sigma_A; /* standard errors (Bernoulli, per history)   */
    double sigma_total_flux;          /* standard error from per-history squares    */
    double track0, track1; /* mean track length in material 0 / 1                   */
    double *flux;       /* caller array [nbins] or NULL: phi_k = track in bin / (N dx) */
    double *flux_sigma; /* caller array [nbins] or NULL: standard error of the batch means */
    double seconds;     /* device time of all runs since create / reset (CUDA events) */
} cls_tallies_t;

/* Raw (un-normalised) accumulators of one case, for merging runs made on
 * several devices or processes: sums add, max_events takes the maximum. */
typedef struct {
    uint64_t n_histories, nR, nT, nA, n_coll, n_interface, n_reflect, n_events, max_events, n_capped;
    double sum_t;    /* sum over histories of the total track length */
    double sum_t2;   /* sum over histories of its square             */
    double track[2]; /* track length summed per material             */
    int32_t nbins, nbatch;
} cls_raw_t;

/* ------------------------------------------------------------ single case */

/* Create a handle for one CLS problem (paper Sec. 2, Tables 1-2 notation):
 *   sigma0, sigma1   total cross sections Sigma_i >= 0, finite
 *   lambda0, lambda1 mean chord lengths Lambda_i > 0, finite; material i is
 *                    picked at the source with p_i = Lambda_i / (Lambda_0 + Lambda_1)
 *   c0, c1           scattering probabilities c_i = Sigma_s,i / Sigma_i in [0, 1]
 *   L                rod length / box side, > 0
 *   d                CLS_GEOM_ROD, CLS_GEOM_EXTRUDED, CLS_GEOM_BOX, CLS_GEOM_SLAB or
 *                    CLS_GEOM_BOX_X
 *   nbins            uniform flux bins along x, 1..4096
 * Selects the current CUDA device, allocates the device tallies (library-
 * owned, freed by cls_destroy; see cls_bind_workspace for caller-owned
 * memory) and zeroes them.
 * Errors: CLS_E_INVAL, CLS_E_NOMEM, CLS_E_NODEVICE, CLS_E_CUDA. */
int cls_create(double sigma0, double sigma1, double lambda0, double lambda1, double c0, double c1,
               double L, int d, int nbins, cls_handle **out);

/* Set a CLS_OPT_* option (values above).  Takes effect at the next run.
 * Errors: CLS_E_INVAL (unknown key or value out of range). */
int cls_set_option(cls_handle *h, int key, int64_t value);

/* Read back a CLS_OPT_* option (after automatic choices have been made, the
 * value used by the last run).  Errors: CLS_E_INVAL. */
int cls_get_option(const cls_handle *h, int key, int64_t *value);

/* Walk histories [next, next + n_histories) of CLS Algorithm A (paper Sec. 4:
 * source, then per event the collision and interface distances drawn afresh,
 * the boundary distance, and the smallest of the three deciding between
 * leakage or reflection, scattering or absorption, and a material switch) on
 * `stream`, and add their track-length and current estimators (paper Sec. 2)
 * to the tallies; next starts at 0 and advances by n_histories, so a sequence
 * of runs equals one long run (checkpoint / resume).  History h draws its random
 * numbers from Philox4x32-10 with key `seed` and counter (j/2, h, case), so a
 * run is fully determined by (seed, first history, n).  Asynchronous; the
 * caller must keep the handle alive until the stream has finished.
 * Errors: CLS_E_INVAL (n == 0), CLS_E_CUDA. */
int cls_run(cls_handle *h, uint64_t n_histories, uint64_t seed, void *stream);

/* Synchronise with the last run's stream, copy the tallies to the host and
 * normalise them in FP64 into *out (out->flux / out->flux_sigma, if not NULL,
 * receive nbins values): the paper's observables (Sec. 2) R = J(x=0),
 * T = J(x=L), the total flux <phi> and the flux profile phi(x) per unit
 * incident current, with the standard errors the paper quotes but does not
 * define (Sec. 5): per-history Bernoulli errors for R, T, A, the per-history
 * error of <phi>, batch means for phi(x).  Errors: CLS_E_STATE (no history run yet),
 * CLS_E_CUDA, CLS_E_EVENT_LIMIT (out is filled; some histories were capped). */
int cls_tallies(cls_handle *h, cls_tallies_t *out);

/* Raw accumulators of case `case_idx` (0 for a single-case handle) and, if
 * flux_batches is not NULL, its raw track-length sums [nbatch][nbins]
 * (row-major, caller-owned) and, if batch_histories is not NULL, the number of
 * histories in each batch [nbatch].  Synchronises like cls_tallies.
 * Errors: CLS_E_INVAL, CLS_E_STATE, CLS_E_CUDA. */
int cls_raw_tallies(cls_handle *h, int case_idx, cls_raw_t *out, double *flux_batches,
                    uint64_t *batch_histories);

/* Normalise raw accumulators on the host, exactly as cls_tallies does: for
 * merging runs made on several devices or processes, sum their cls_raw_t
 * fields (max_events: maximum), their flux_batches and their batch_histories,
 * then call this.  flux_batches: [raw->nbatch][raw->nbins]; batch_histories:
 * [raw->nbatch]; L: the case's length.  Needs no GPU.
 * Errors: CLS_E_INVAL (no histories, bad sizes), CLS_E_EVENT_LIMIT (out is
 * filled; some histories were capped). */
int cls_finalize_raw(const cls_raw_t *raw, const double *flux_batches, const uint64_t *batch_histories, double L,
                     cls_tallies_t *out);

/* Zero the tallies and restart history numbering at 0 (synchronous). */
int cls_reset(cls_handle *h);

/* ------------------------------------------------ caller-owned device memory */
/* The paper has no counterpart: these let a caller that manages device memory
 * itself (a framework's caching allocator, e.g. a PyTorch tensor) hold the
 * handle's device buffers.
 *
 * cls_workspace_bytes: the bytes of device memory the handle needs for its
 * current cases and options -- flux tallies [cases][nbatch][nbins_stride]
 * doubles, statistics, counters, the case table, the work list, the work
 * counters and, when the handle's schedule (or a case's) is the event schedule
 * or still automatic, the event tracker's particle bank for the current launch
 * shape (for an automatic schedule, the larger of the autotuner's event
 * candidates).  Errors: CLS_E_INVAL, CLS_E_CUDA. */
int cls_workspace_bytes(cls_handle *h, size_t *bytes);

/* cls_bind_workspace: move every device buffer of the handle into the
 * caller's device memory d_workspace of `bytes` bytes (256-byte aligned, on
 * the handle's device, at least cls_workspace_bytes): the library frees its
 * own buffers, copies the case table into the workspace and zeroes the
 * tallies there (synchronous).  Bytes beyond the other buffers serve as the
 * event bank, so a larger workspace allows a larger bank.  The caller owns the
 * memory and must keep it allocated, and untouched, until the handle is
 * destroyed or unbound; later runs use it and allocate no device memory
 * (cls_trace and the autotuner's pilot handles still allocate their own).  An
 * option change whose buffers no longer fit fails with CLS_E_NOMEM (nbatch at
 * cls_set_option, a larger event bank at the next run); query again and bind
 * a larger workspace.  d_workspace = NULL returns the handle to library-owned
 * buffers.  Only before the first run or after cls_reset.
 * Errors: CLS_E_INVAL (misaligned, not device memory of the handle's device,
 * too small), CLS_E_STATE (the tallies hold results), CLS_E_NOMEM, CLS_E_CUDA. */
int cls_bind_workspace(cls_handle *h, void *d_workspace, size_t bytes);

/* Free all device and host resources of the handle (synchronises first). */
void cls_destroy(cls_handle *h);

/* Static string describing an error code. */
const char *cls_strerror(int code);

/* Trace history `history` of case `case_idx` event by event on the device in
 * the handle's precision: rows of 10 doubles (event, draw index after the
 * event, x, y, z, wx, wy, wz, material after the event, flight length) with
 * event codes 0 leak at x=0, 1 leak at x=L, 2 lateral reflection,
 * 3 scatter, 4 absorption, 5 interface crossing, 6 event cap.  Writes at most
 * `cap` rows to the caller array `rows` and the number of rows of the whole
 * history to *n_rows.  Synchronous; does not touch the tallies.
 * Errors: CLS_E_INVAL, CLS_E_CUDA. */
int cls_trace(cls_handle *h, int case_idx, uint64_t seed, uint64_t history, double *rows, int cap,
              int *n_rows);

/* Autotune the handle's launch: time pilot runs of n_pilot histories per case
 * (seed `seed`, history ids far above any a caller uses) for each candidate --
 * history schedule x block {64, 128, 256} x chunk {64, 256, 1024}, and event
 * schedule x block {128, 256} x events per pass {4, 16}, each with one launch
 * per geometry and with one mixed launch for a batch of several geometries
 * (CLS_OPT_GROUP_GEOMETRY) -- on a temporary twin
 * handle with the same cases and precision, so the handle's own tallies are
 * untouched, then set the fastest candidate's options on the handle.  Results
 * are cached by a signature of (precision, cases, floor(log2 n_pilot)) in
 * memory and, if the environment variable CLS_AUTOTUNE_CACHE names a file, in
 * that file: a shape tuned for small runs is not reused for large ones.  With
 * CLS_OPT_SCHEDULE = CLS_SCHED_AUTO the first run calls this itself with
 * n_pilot = n/16 clamped to [4096, 262144].  Synchronous on `stream`.
 * Errors: CLS_E_INVAL, CLS_E_NOMEM, CLS_E_CUDA. */
int cls_autotune(cls_handle *h, uint64_t n_pilot, uint64_t seed, void *stream);

/* --------------------------------------------------------------- batches */

/* Create a handle for `ncases` independent CLS problems run together in one
 * persistent launch.  params: ncases x 9 doubles, row-major
 * (sigma0, sigma1, lambda0, lambda1, c0, c1, L, d, nbins) with the meanings
 * and limits of cls_create; case k draws with Philox counter word 3 = k.
 * Errors: as cls_create; ncases in 1..65536. */
int cls_batch_create(const double *params, int ncases, cls_handle **out);

/* Run n_per_case histories of every case in one persistent launch per group of
 * cases (per geometry, CLS_OPT_GROUP_GEOMETRY, and per schedule,
 * cls_batch_set_case_schedule), each group's cases ordered by estimated cost
 * (largest first).  The launch sequence (counter reset, the groups' trackers
 * as parallel graph branches, nothing else) is captured once into a CUDA graph
 * and replayed on later calls with new history ranges.  Asynchronous on
 * `stream`.
 * Errors: CLS_E_INVAL, CLS_E_CUDA. */
int cls_batch_run(cls_handle *h, uint64_t n_per_case, uint64_t seed, void *stream);

/* Normalised results of case `case_idx`, as cls_tallies.
 * Errors: CLS_E_INVAL, CLS_E_STATE, CLS_E_CUDA, CLS_E_EVENT_LIMIT. */
int cls_batch_tallies(cls_handle *h, int case_idx, cls_tallies_t *out);

/* Number of cases of the handle (1 for cls_create handles). */
int cls_num_cases(const cls_handle *h);

/* Schedule of one case of a batch: CLS_SCHED_HISTORY, CLS_SCHED_EVENT, or
 * CLS_SCHED_AUTO (the default: the handle's CLS_OPT_SCHEDULE).  A batch whose
 * cases have different schedules runs one persistent launch per schedule (and
 * per geometry, CLS_OPT_GROUP_GEOMETRY) per cls_batch_run, each over its own
 * cases (largest estimated cost first) and all captured in the batch's CUDA
 * graph; the launch options (block, chunk, bank, events per pass) are the
 * handle's.  Results do not
 * depend on the schedule: both walk every history draw for draw.  Takes
 * effect at the next run.  Errors: CLS_E_INVAL. */
int cls_batch_set_case_schedule(cls_handle *h, int case_idx, int schedule);

/* The schedule case `case_idx` runs under at the next run (its own, else the
 * handle's; CLS_SCHED_AUTO while the handle's is still to be tuned).
 * Errors: CLS_E_INVAL. */
int cls_batch_get_case_schedule(const cls_handle *h, int case_idx, int *schedule);

/* Autotune the schedule of every case: each case alone, on a temporary
 * single-case twin with the handle's precision and launch options, runs
 * n_pilot histories (history ids far above any a caller uses, Philox key
 * `seed`) under the history and under the event schedule, timed with CUDA
 * events on `stream`; the faster is the case's choice.  A case's preference
 * alone need not carry over into the batch (a second launch adds its own
 * tail), so the choices are kept (cls_batch_set_case_schedule) only if a
 * pilot of the whole batch, n_pilot histories per case on a temporary twin,
 * runs faster with them than with every case on the handle's schedule;
 * otherwise every case follows the handle's schedule.  With the handle's
 * schedule still CLS_SCHED_AUTO the choices are kept untested.  The handle's
 * tallies are untouched.  Synchronous.
 * Errors: CLS_E_INVAL, CLS_E_NOMEM, CLS_E_CUDA. */
int cls_autotune_cases(cls_handle *h, uint64_t n_pilot, uint64_t seed, void *stream);

/* ------------------------------------------------------ per-history outcomes */

/* Outcome codes of cls_record_outcomes: how a history ended (paper Sec. 2:
 * leakage through x = 0 counts toward R, through x = L toward T; absorption
 * toward A; the event cap toward none of them). */
#define CLS_OUTCOME_REFLECTED 0
#define CLS_OUTCOME_TRANSMITTED 1
#define CLS_OUTCOME_ABSORBED 2
#define CLS_OUTCOME_CAPPED 3

/* Record every history's outcome, one byte per history, in the caller-owned
 * device buffer d_codes of `capacity` bytes: from the next cls_run or
 * cls_batch_run on, history h of case k writes
 * d_codes[k * n + (h - first)] = CLS_OUTCOME_*, where n is that run's
 * histories per case and first its first history id.  Each run overwrites the
 * codes of its own histories; the tallies are unaffected.  d_codes = NULL
 * stops recording.  The buffer must stay allocated while runs that record
 * into it are in flight.  A run then fails with CLS_E_INVAL when
 * ncases x n > capacity, and with CLS_E_STATE when the cases' next history
 * ids differ (CLS_OPT_FIRST_HISTORY sets them all alike).
 * Errors: CLS_E_INVAL (null handle, or capacity 0 with a buffer). */
int cls_record_outcomes(cls_handle *h, uint8_t *d_codes, uint64_t capacity);

/* ------------------------------------------------------------ diagnostics */

/* Evaluate this library's device Philox4x32-10 and, for comparison, CUDA's
 * curand_Philox4x32_10 on n counter/key sets.  in: n x 6 u32 (c0, c1, c2, c3,
 * k0, k1); ours, theirs: n x 4 u32 outputs.  Host arrays; synchronous.
 * Errors: CLS_E_INVAL, CLS_E_CUDA, CLS_E_NOMEM. */
int cls_debug_philox(const uint32_t *in, int n, uint32_t *ours, uint32_t *theirs);

/* Device uniforms: draw j of history h (case_id, seed) for n (h, j) pairs, in
 * FP64 (53 bits, out64) and FP32 (24 bits, out32); either may be NULL. */
int cls_debug_uniform(uint64_t seed, uint32_t case_id, const uint64_t *h, const uint64_t *j, int n,
                      double *out64, float *out32);

/* The FP64 walk's elementary functions of a draw: for u = k[i] 2^-53
 * (0 <= k[i] < 2^53), ln1m[i] = ln(1 - u) (the distances l_c = -ln(1-u)/Sigma
 * and l_i = -Lambda ln(1-u) of paper Sec. 4), sin2pi[i], cos2pi[i] = sin, cos
 * of 2 pi u (the azimuth of isotropic directions, paper Sec. 4.3), u[i] = u,
 * mu[i] = 2u - 1 (an isotropic direction cosine) and recip_mu[i] = 1/mu[i]
 * (the inverse direction cosines of the boundary distances).  Host arrays of
 * n entries; any output may be NULL; synchronous.
 * Errors: CLS_E_INVAL (k[i] >= 2^53, n < 1), CLS_E_CUDA, CLS_E_NOMEM. */
int cls_debug_math(const uint64_t *k, int n, double *ln1m, double *sin2pi, double *cos2pi, double *u, double *mu,
                   double *recip_mu);

/* The FP32 walk's fixed-point conversion: out[i] = round(c[i] 2^32), to the
 * nearest integer with ties to even, the form in which the FP32 walk adds its
 * flights' track lengths to the tallies (exact sums; paper Sec. 4's
 * track-length estimator).  c: n floats in [0, 2^32); out: n u64.  Host
 * arrays; synchronous.  Errors: CLS_E_INVAL (c[i] outside [0, 2^32) or NaN,
 * n < 1, NULL), CLS_E_CUDA, CLS_E_NOMEM. */
int cls_debug_fixed32(const float *c, int n, unsigned long long *out);

/* ------------------------------------------------- allocation-free run */

/* Largest number of cases one cls_run_noalloc call takes, and its largest
 * nbins_stride. */
#define CLS_NOALLOC_MAX_CASES 64
#define CLS_NOALLOC_MAX_STRIDE 4096

/* cls_run_noalloc -- run the FP64 history-based tracker without allocating
 * any device memory.  The paper has no counterpart: this exists for callers
 * that cannot call cudaMalloc (code living inside another framework's memory
 * budget, or a process that reserved all device memory up front), for whom
 * cls_create's allocations are not an option.
 *
 * Runs histories [first, first + n) of each of `ncases` cases
 * (1..CLS_NOALLOC_MAX_CASES; params: ncases x 9 doubles on the host, as in
 * cls_batch_create; case k draws with Philox counter word 3 = k) with key
 * `seed`, and ADDS the raw tallies into caller-owned device buffers, which the
 * caller zeroes before its first call:
 *   d_flux     [ncases][nbatch][nbins_stride] doubles: track length per
 *              statistics batch and bin (batch b holds histories
 *              first + b * L_b ..., L_b = 1024 * ceil(n / (1024 * nbatch)));
 *   d_stats    [ncases][4] doubles: sum of per-history track length, of its
 *              square, track length in material 0, in material 1;
 *   d_counters [ncases][9] u64: reflected, transmitted, absorbed, collisions,
 *              interface crossings, lateral reflections, events, capped
 *              histories (all added), longest history in events (maximum).
 * nbatch is 1..1024, nbins_stride is the largest nbins .. CLS_NOALLOC_MAX_STRIDE.
 * Results equal cls_run's for the same seed and history range (default
 * options; per-history event cap 1e8).  The call is asynchronous, so it cannot
 * report capped histories as CLS_E_EVENT_LIMIT: they show in d_counters[k][7].
 *
 * Scratch (case parameters, work list, work counter; about 16 KB) lives in a
 * static device array that every GPU loading the library holds until the
 * process exits.  The first call on each device looks up that array's device
 * address (with the device current) and keeps it for the life of the process;
 * make that first call before any stream capture, and do not call this entry
 * point again after cudaDeviceReset.  Each call hands its cases and work list
 * to a small set-up kernel as kernel arguments, which writes them into the
 * array ahead of the tracker on `stream`; nothing is read from host memory
 * after the call returns.  All calls share the array and each call rewrites
 * it, so calls that overlap on the GPU race and must be serialised by the
 * caller (one stream).  Asynchronous on `stream`.
 * Errors: CLS_E_INVAL (NULL buffer, ncases, n, nbatch or nbins_stride out of
 * range, invalid case), CLS_E_CUDA. */
int cls_run_noalloc(const double *params, int ncases, uint64_t first, uint64_t n, uint64_t seed, int nbatch,
                    int nbins_stride, double *d_flux, double *d_stats, unsigned long long *d_counters,
                    void *stream);

#ifdef __cplusplus
}
#endif

#endif /* CLS_H */
