// cls_host.cu -- host side of the C ABI declared in include/cls.h.
//
// Owns the device tallies, orders batched cases by estimated cost, builds the
// per-run work list, launches the trackers (directly for single cases,
// through a captured CUDA graph for batches) and normalises the tallies in
// FP64 (paper Sec. 2 observables; standard errors per Sec. 5 / Eq.
// combined_var usage: per-history for R, T, A and <phi>, batch means for phi(x)).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <map>
#include <mutex>
#include <string>
#include <cstdlib>
#include <cstring>
#include <new>
#include <numeric>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/cls.h"
#include "cls_case.h"
#include "cls_internal.h"

using namespace cls;

namespace {

constexpr int kBatchQuantum = 1024;   // statistics batches are multiples of this many histories
constexpr int kMaxCases = 65536;
constexpr uint32_t kMaxEventsLimit = 1u << 28;
constexpr size_t kMaxSmemPerBlock = 200 * 1024;  // opt-in dynamic shared memory per block

struct Options {
    int precision = CLS_PREC_FP64;
    int schedule = CLS_SCHED_HISTORY;
    int block = 256;
    int chunk = 256;
    int nbatch = 64;
    uint32_t max_events = 100000000u;
    int blocks_per_sm = 0;
    int bank = 0;
    int events_per_pass = 4;
    int group_geometry = 1;  // a batch of mixed geometries: one launch per geometry
};

// Launch groups of one run: (schedule, geometry) pairs, each its own
// persistent launch with its own chunk counter.
constexpr int kMaxGroups = 10;  // 2 schedules x 5 geometries

}  // namespace

struct cls_handle {
    int device = 0;
    int sm_count = 0;
    bool batch = false;
    std::vector<double> params;  // ncases x 9, as created
    int geom = 0;                // geometry shared by every case, 0 if mixed
    Options opt;
    int used_blocks_per_sm = 0;
    std::vector<CaseParams> cases;
    CaseParams *d_cases = nullptr;
    // tallies
    int nbatch = 0;        // allocated batches (fixed at the first run / reset)
    int nbins_stride = 0;
    int nbins_max = 0;
    double *d_flux = nullptr;
    double *d_stats = nullptr;
    unsigned long long *d_counters = nullptr;
    unsigned long long *d_chunk_counter = nullptr;
    // per-run work
    RunCase *h_runs = nullptr;  // pinned; the OutcomeRecord follows the cases' RunCases
    RunCase *d_runs = nullptr;
    uint8_t *outcome_codes = nullptr;  // caller's per-history outcome buffer (device), or null
    uint64_t outcome_cap = 0;
    // batches: per-case schedule (CLS_SCHED_AUTO: the handle's CLS_OPT_SCHEDULE).
    // Cases of different schedules run as two groups, one launch each, with
    // their own slices of the work list and their own chunk counters.
    std::vector<int> case_sched;
    cudaEvent_t runs_copied = nullptr;
    std::vector<int> order;  // case indices, largest estimated cost first
    std::vector<uint64_t> next_history;
    std::vector<std::vector<uint64_t>> batch_hist;  // [case][nbatch]
    std::vector<uint64_t> n_hist;
    // event-schedule bank
    void *d_bank = nullptr;
    size_t bank_bytes = 0;
    // caller-owned device workspace (cls_bind_workspace) holding every device
    // buffer above, or null: the library's own allocations
    unsigned char *ws = nullptr;
    size_t ws_bytes = 0;
    size_t ws_bank_off = 0;
    // timing / sync
    cudaStream_t last_stream = nullptr;
    bool ran = false;
    std::vector<cudaEvent_t> ev_pairs;  // start/stop per pending run
    double seconds = 0.0;
    // batch graph: group 0 is captured on capture_stream, group g > 0 on
    // aux_streams[g - 1], forked after the counter reset and joined at the end
    cudaStream_t capture_stream = nullptr;
    std::vector<cudaStream_t> aux_streams;
    std::vector<cudaEvent_t> join_events;  // [0]: the fork, [g]: group g's end
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t graph_exec = nullptr;
    std::vector<uint64_t> graph_total_chunks;
    int graph_key[10] = {0};
};

namespace {

int cuda_fail(cudaError_t e) { return e == cudaSuccess ? CLS_OK : CLS_E_CUDA; }

#define CLS_CUDA(call)                              \
    do {                                            \
        cudaError_t _e = (call);                    \
        if (_e != cudaSuccess) return CLS_E_CUDA;   \
    } while (0)

// The run's work list: one RunCase per case, then the OutcomeRecord.
size_t runs_bytes(size_t ncases) { return ncases * sizeof(RunCase) + sizeof(OutcomeRecord); }

OutcomeRecord *outcome_record(RunCase *runs, size_t ncases) {
    return reinterpret_cast<OutcomeRecord *>(reinterpret_cast<unsigned char *>(runs) + ncases * sizeof(RunCase));
}

void free_tallies(cls_handle *h) {
    if (!h->ws) {
        cudaFree(h->d_flux);
        cudaFree(h->d_stats);
        cudaFree(h->d_counters);
    }
    h->d_flux = nullptr;
    h->d_stats = nullptr;
    h->d_counters = nullptr;
}

// The library's own device buffers (none while a caller's workspace is bound).
void free_device(cls_handle *h) {
    free_tallies(h);
    if (!h->ws) {
        cudaFree(h->d_cases);
        cudaFree(h->d_runs);
        cudaFree(h->d_chunk_counter);
        cudaFree(h->d_bank);
    }
    h->d_cases = nullptr;
    h->d_runs = nullptr;
    h->d_chunk_counter = nullptr;
    h->d_bank = nullptr;
    h->bank_bytes = 0;
}

// Byte offsets of the device buffers in a caller's workspace, each 256-byte
// aligned: flux [cases][nbatch][nbins_stride] doubles, statistics, counters,
// the case table, the work list, the two work counters, then the event bank.
struct DevLayout {
    size_t flux, stats, counters, cases, runs, chunk, bank, total;
};

DevLayout dev_layout(const cls_handle *h, size_t bank) {
    auto up = [](size_t v) { return (v + 255) & ~(size_t)255; };
    const size_t nc = h->cases.size();
    DevLayout L;
    size_t o = 0;
    L.flux = o;
    o = up(o + nc * (size_t)h->nbatch * (size_t)h->nbins_stride * sizeof(double));
    L.stats = o;
    o = up(o + nc * S_NUM * sizeof(double));
    L.counters = o;
    o = up(o + nc * C_NUM * sizeof(unsigned long long));
    L.cases = o;
    o = up(o + nc * sizeof(CaseParams));
    L.runs = o;
    o = up(o + runs_bytes(nc));
    L.chunk = o;
    o = up(o + kMaxGroups * sizeof(unsigned long long));
    L.bank = o;
    L.total = up(o + bank);
    return L;
}

int alloc_tallies(cls_handle *h) {
    if (h->ws) return CLS_E_STATE;  // a bound workspace is re-carved, not reallocated
    const size_t nc = h->cases.size();
    const size_t nflux = nc * (size_t)h->nbatch * (size_t)h->nbins_stride;
    if (cudaMalloc(&h->d_flux, nflux * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&h->d_stats, nc * S_NUM * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&h->d_counters, nc * C_NUM * sizeof(unsigned long long)) != cudaSuccess) {
        free_tallies(h);
        cudaGetLastError();
        return CLS_E_NOMEM;
    }
    return CLS_OK;
}

int zero_tallies(cls_handle *h) {
    const size_t nc = h->cases.size();
    CLS_CUDA(cudaMemset(h->d_flux, 0, nc * (size_t)h->nbatch * h->nbins_stride * sizeof(double)));
    CLS_CUDA(cudaMemset(h->d_stats, 0, nc * S_NUM * sizeof(double)));
    CLS_CUDA(cudaMemset(h->d_counters, 0, nc * C_NUM * sizeof(unsigned long long)));
    h->next_history.assign(nc, 0);
    h->n_hist.assign(nc, 0);
    h->batch_hist.assign(nc, std::vector<uint64_t>(h->nbatch, 0));
    for (cudaEvent_t e : h->ev_pairs) cudaEventDestroy(e);
    h->ev_pairs.clear();
    h->seconds = 0.0;
    h->ran = false;
    return CLS_OK;
}

void destroy_graph(cls_handle *h) {
    if (h->graph_exec) cudaGraphExecDestroy(h->graph_exec);
    if (h->graph) cudaGraphDestroy(h->graph);
    h->graph_exec = nullptr;
    h->graph = nullptr;
}

int create_common(const double *params, int ncases, bool batch, cls_handle **out) {
    if (!out || !params || ncases < 1 || ncases > kMaxCases) return CLS_E_INVAL;
    *out = nullptr;
    for (int k = 0; k < ncases; ++k) {
        int rc = validate_case(params + 9 * (size_t)k);
        if (rc) return rc;
    }
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
        cudaGetLastError();
        return CLS_E_NODEVICE;
    }
    cls_handle *h = new (std::nothrow) cls_handle();
    if (!h) return CLS_E_NOMEM;
    h->batch = batch;
    h->params.assign(params, params + 9 * (size_t)ncases);
    if (cudaGetDevice(&h->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&h->sm_count, cudaDevAttrMultiProcessorCount, h->device) != cudaSuccess) {
        delete h;
        return CLS_E_CUDA;
    }
    h->cases.reserve(ncases);
    for (int k = 0; k < ncases; ++k) {
        h->cases.push_back(make_case(params + 9 * (size_t)k, (uint32_t)k));
        h->nbins_max = std::max(h->nbins_max, h->cases.back().nbins);
    }
    h->nbins_stride = (h->nbins_max + 1) & ~1;
    h->geom = h->cases[0].d;
    for (const CaseParams &c : h->cases)
        if (c.d != h->geom) h->geom = 0;
    h->case_sched.assign(ncases, CLS_SCHED_AUTO);
    h->order.resize(ncases);
    std::iota(h->order.begin(), h->order.end(), 0);
    std::stable_sort(h->order.begin(), h->order.end(),
                     [&](int a, int b) { return h->cases[a].cost > h->cases[b].cost; });
    h->nbatch = h->opt.nbatch;
    int rc = CLS_OK;
    if (cudaMalloc(&h->d_cases, ncases * sizeof(CaseParams)) != cudaSuccess ||
        cudaMalloc(&h->d_runs, runs_bytes(ncases)) != cudaSuccess ||
        cudaMalloc(&h->d_chunk_counter, kMaxGroups * sizeof(unsigned long long)) != cudaSuccess ||
        cudaMallocHost(&h->h_runs, runs_bytes(ncases)) != cudaSuccess) {
        rc = CLS_E_NOMEM;
    }
    if (!rc) rc = alloc_tallies(h);
    if (!rc && cudaMemcpy(h->d_cases, h->cases.data(), ncases * sizeof(CaseParams), cudaMemcpyHostToDevice) != cudaSuccess)
        rc = CLS_E_CUDA;
    if (!rc && cudaEventCreateWithFlags(&h->runs_copied, cudaEventDisableTiming) != cudaSuccess) rc = CLS_E_CUDA;
    if (!rc) rc = zero_tallies(h);
    if (rc) {
        cudaGetLastError();
        cls_destroy(h);
        return rc;
    }
    *out = h;
    return CLS_OK;
}

uint64_t batch_len_for(uint64_t n, int nbatch) {
    const uint64_t q = (uint64_t)kBatchQuantum * (uint64_t)nbatch;
    return (uint64_t)kBatchQuantum * std::max<uint64_t>(1, (n + q - 1) / q);
}

int region_bytes_for(const cls_handle *h) {
    return region_bytes(h->opt.precision == CLS_PREC_FP32, h->nbins_stride);
}

// FP32 regions are flushed into the FP64 global tallies after this many
// histories, which keeps each bin's fixed-point sum far below its 2^31 range.
constexpr int kFp32FlushHistories = 1024;

// Schedule of case k: its own, or the handle's.
int case_schedule(const cls_handle *h, int k) {
    const int cs = h->case_sched.empty() ? CLS_SCHED_AUTO : h->case_sched[k];
    return cs != CLS_SCHED_AUTO ? cs : h->opt.schedule;
}

// The launch groups of a run: cases grouped by schedule and, when launches
// are split by geometry, by geometry (a batch of rods and boxes runs the rod
// walk and the box walk each compiled for its geometry); the handle's schedule
// first, then the group of largest estimated cost first.  gk[k]: case k's group.
struct Group {
    int sched, geom;
    double cost;   // summed estimated events per history of its cases
    int ncases;
};

// A launch whose cases average fewer estimated events per history than this
// runs the tracker's short-history instance (history-end counters summed over
// the warp, deposits that skip zero and past-the-mesh difference entries).
constexpr double kWarpCountCost = 32.0;

std::vector<Group> plan_groups(const cls_handle *h, std::vector<int> *gk) {
    std::vector<Group> groups;
    const int nc = (int)h->cases.size();
    std::vector<int> of(nc);
    for (int k = 0; k < nc; ++k) {
        const int sc = case_schedule(h, k);
        const int ge = h->opt.group_geometry ? h->cases[k].d : h->geom;
        int g = 0;
        while (g < (int)groups.size() && !(groups[g].sched == sc && groups[g].geom == ge)) ++g;
        if (g == (int)groups.size()) groups.push_back({sc, ge, 0.0, 0});
        groups[g].cost += h->cases[k].cost;
        groups[g].ncases += 1;
        of[k] = g;
    }
    std::vector<int> order(groups.size());
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
        const bool ha = groups[a].sched == h->opt.schedule, hb = groups[b].sched == h->opt.schedule;
        return ha != hb ? ha : groups[a].cost > groups[b].cost;
    });
    std::vector<int> rank(groups.size());
    std::vector<Group> sorted;
    for (size_t i = 0; i < order.size(); ++i) {
        rank[order[i]] = (int)i;
        sorted.push_back(groups[order[i]]);
    }
    if (gk) {
        gk->resize(nc);
        for (int k = 0; k < nc; ++k) (*gk)[k] = rank[of[k]];
    }
    return sorted;
}

// One run: a launch per group.  Group g's cases sit in the work list at
// runs[off .. off + nruns), largest estimated cost first, with chunk numbers
// from 0 and chunk counter g.
struct RunPlan {
    int ngroups = 0;
    int sched[kMaxGroups];
    int geom[kMaxGroups];
    LaunchArgs a[kMaxGroups];
};

// Fill the pinned work list for n histories per case and describe the launches.
int prepare_run(cls_handle *h, uint64_t n, uint64_t seed, RunPlan *plan) {
    // the previous run's copy of the pinned work list must have completed
    CLS_CUDA(cudaEventSynchronize(h->runs_copied));
    const int nc = (int)h->cases.size();
    std::vector<int> gk;
    const std::vector<Group> groups = plan_groups(h, &gk);
    if ((int)groups.size() > kMaxGroups) return CLS_E_INVAL;
    LaunchArgs a;
    std::memset(&a, 0, sizeof(a));
    a.cases = h->d_cases;
    a.chunk = (uint32_t)h->opt.chunk;
    a.t = Tallies{h->d_flux, h->d_stats, h->d_counters, h->nbatch, h->nbins_stride};
    a.seed = seed;
    a.rk = make_round_keys(seed);
    a.max_events = h->opt.max_events;
    a.region_bytes = region_bytes_for(h);
    a.flush_every = (h->opt.precision == CLS_PREC_FP32) ? kFp32FlushHistories : 0;
    // the record's binding is read from device memory at every launch (graph
    // replays see the current buffer); while nothing is recorded the kernels are
    // given no record at all and skip that read
    a.outcomes = h->outcome_codes ? outcome_record(h->d_runs, nc) : nullptr;
    int idx = 0;
    plan->ngroups = (int)groups.size();
    for (int g = 0; g < plan->ngroups; ++g) {
        const int off = idx;
        uint64_t chunks = 0;
        for (int i = 0; i < nc; ++i) {
            const int k = h->order[i];
            if (gk[k] != g) continue;
            RunCase &r = h->h_runs[idx++];
            r.first = h->next_history[k];
            r.n = n;
            r.batch_len = batch_len_for(n, h->nbatch);
            r.chunk_begin = chunks;
            r.case_index = k;
            r.pad = 0;
            chunks += (n + h->opt.chunk - 1) / h->opt.chunk;
        }
        LaunchArgs &ag = plan->a[g];
        ag = a;
        ag.runs = h->d_runs + off;
        ag.nruns = idx - off;
        ag.total_chunks = chunks;
        ag.chunk_counter = h->d_chunk_counter + g;
        ag.warp_counts = (groups[g].geom == 0 || groups[g].cost < kWarpCountCost * groups[g].ncases) ? 1 : 0;
        plan->sched[g] = groups[g].sched;
        plan->geom[g] = groups[g].geom;
    }
    OutcomeRecord *rec = outcome_record(h->h_runs, nc);
    *rec = OutcomeRecord{nullptr, 0, 0};
    if (h->outcome_codes) {
        // every case's row starts at the same history id and holds n codes
        for (int k = 1; k < nc; ++k)
            if (h->next_history[k] != h->next_history[0]) return CLS_E_STATE;
        if (n > h->outcome_cap / (uint64_t)nc) return CLS_E_INVAL;
        *rec = OutcomeRecord{h->outcome_codes, h->next_history[0], n};
    }
    return CLS_OK;
}

void account_run(cls_handle *h, uint64_t n) {
    const uint64_t bl = batch_len_for(n, h->nbatch);
    for (size_t k = 0; k < h->cases.size(); ++k) {
        for (uint64_t b = 0; b * bl < n; ++b) h->batch_hist[k][b] += std::min(bl, n - b * bl);
        h->next_history[k] += n;
        h->n_hist[k] += n;
    }
    h->ran = true;
}

// Launch shape of the tracker for the handle's options.
struct Shape {
    int grid, block;
    size_t smem;
    uint32_t bank_slots;  // event schedule: slots per block and buffer
    size_t bank_off;      // event schedule: this launch's slice of the bank
};

size_t shape_bank_bytes(const cls_handle *h, const Shape &sh) {
    return (size_t)sh.grid * (sh.block / 32) * 2 * sh.bank_slots * (size_t)event_bank_fields(h->opt.precision) * 16;
}

int tracker_shape(cls_handle *h, int region_bytes, int sched, int geom, Shape *out) {
    const bool event = sched == CLS_SCHED_EVENT;
    const bool fp64 = h->opt.precision == CLS_PREC_FP64;
    // each warp owns two tally regions; wide meshes get fewer warps per block
    const size_t per_warp = 2 * (size_t)region_bytes;
    const int fit_warps = (int)std::min<size_t>(kMaxSmemPerBlock / per_warp, 8);
    if (fit_warps < 1) return CLS_E_INVAL;
    // the history trackers' launch bounds
    const int cap_warps = event ? kEventBlockThreads / 32 : fp64 ? kHistoryBlockFp64 / 32 : history_threads_fp32(geom) / 32;
    const int block = 32 * std::min(std::min(h->opt.block / 32, fit_warps), cap_warps);
    const size_t smem = (size_t)(block / 32) * per_warp;
    int bps = h->opt.blocks_per_sm;
    if (bps <= 0) {
        const int g = geom;
        cudaError_t e = event ? (fp64 ? occupancy_event_fp64(block, smem, &bps, g) : occupancy_event_fp32(block, smem, &bps, g))
                              : (fp64 ? occupancy_history_fp64(block, smem, &bps, g)
                                      : occupancy_history_fp32(block, smem, &bps, g));
        if (e != cudaSuccess) return CLS_E_CUDA;
        if (bps < 1) return CLS_E_INVAL;  // the block does not fit on an SM
    }
    h->used_blocks_per_sm = bps;
    out->grid = h->sm_count * bps;
    out->block = block;
    out->smem = smem;
    out->bank_slots = event ? (uint32_t)(h->opt.bank > 0 ? ((h->opt.bank + 31) & ~31) : 128) : 0u;
    out->bank_off = 0;
    return CLS_OK;
}

// Shapes of a run's launches; the event launches take consecutive slices of
// one particle bank (grid warps x 2 buffers x slots x fields x 16 B each, all
// of a run's launches may run at once).  *bank: the bytes they need together.
int plan_shapes(cls_handle *h, const RunPlan &plan, Shape *sh, size_t *bank) {
    *bank = 0;
    for (int g = 0; g < plan.ngroups; ++g) {
        const int rc = tracker_shape(h, plan.a[g].region_bytes, plan.sched[g], plan.geom[g], &sh[g]);
        if (rc) return rc;
        if (plan.sched[g] == CLS_SCHED_EVENT) {
            sh[g].bank_off = *bank;
            *bank += (shape_bank_bytes(h, sh[g]) + 255) & ~(size_t)255;
        }
    }
    return CLS_OK;
}

// Make sure the particle bank holds `need` bytes.  Done before any graph capture.
int ensure_bank(cls_handle *h, size_t need) {
    if (need == 0) return CLS_OK;
    if (h->ws) {
        // the bank takes the bound workspace's bytes after its other buffers
        if (need > h->ws_bytes - h->ws_bank_off) return CLS_E_NOMEM;
        h->d_bank = h->ws + h->ws_bank_off;
        h->bank_bytes = h->ws_bytes - h->ws_bank_off;
        return CLS_OK;
    }
    if (need <= h->bank_bytes) return CLS_OK;
    CLS_CUDA(cudaDeviceSynchronize());
    cudaFree(h->d_bank);
    h->d_bank = nullptr;
    h->bank_bytes = 0;
    if (cudaMalloc(&h->d_bank, need) != cudaSuccess) {
        cudaGetLastError();
        return CLS_E_NOMEM;
    }
    h->bank_bytes = need;
    return CLS_OK;
}

// Bytes of event bank the handle's current options need: none unless the
// handle's schedule (or a case's) is the event schedule or still automatic
// (then the larger of the autotuner's event candidates, every group on the
// event schedule).
int bank_need(cls_handle *h, size_t *need) {
    *need = 0;
    bool event = h->opt.schedule == CLS_SCHED_EVENT || h->opt.schedule == CLS_SCHED_AUTO;
    for (size_t k = 0; k < h->cases.size(); ++k) event |= case_schedule(h, (int)k) == CLS_SCHED_EVENT;
    if (!event) return CLS_OK;
    const Options saved = h->opt;
    const int saved_bps = h->used_blocks_per_sm;
    int rc = CLS_OK;
    for (int block : {h->opt.block, 128, 256}) {
        if (block != saved.block && saved.schedule != CLS_SCHED_AUTO) continue;
        h->opt.block = block;
        if (saved.schedule == CLS_SCHED_AUTO) h->opt.schedule = CLS_SCHED_EVENT;
        RunPlan plan;
        const std::vector<Group> groups = plan_groups(h, nullptr);
        plan.ngroups = (int)groups.size();
        for (int g = 0; g < plan.ngroups; ++g) {
            plan.sched[g] = groups[g].sched;
            plan.geom[g] = groups[g].geom;
            plan.a[g].region_bytes = region_bytes_for(h);
        }
        Shape sh[kMaxGroups];
        size_t bank = 0;
        rc = plan_shapes(h, plan, sh, &bank);
        h->opt = saved;
        if (rc) break;
        *need = std::max(*need, bank);
    }
    h->opt = saved;
    h->used_blocks_per_sm = saved_bps;
    return rc;
}

// Point every device buffer into the bound workspace (layout dev_layout), copy
// the case table there and zero the tallies.  Synchronous.
int carve_workspace(cls_handle *h, size_t bank) {
    const DevLayout L = dev_layout(h, bank);
    if (L.total > h->ws_bytes) return CLS_E_NOMEM;
    h->d_flux = reinterpret_cast<double *>(h->ws + L.flux);
    h->d_stats = reinterpret_cast<double *>(h->ws + L.stats);
    h->d_counters = reinterpret_cast<unsigned long long *>(h->ws + L.counters);
    h->d_cases = reinterpret_cast<CaseParams *>(h->ws + L.cases);
    h->d_runs = reinterpret_cast<RunCase *>(h->ws + L.runs);
    h->d_chunk_counter = reinterpret_cast<unsigned long long *>(h->ws + L.chunk);
    h->ws_bank_off = L.bank;
    h->d_bank = nullptr;
    h->bank_bytes = 0;
    destroy_graph(h);  // the captured launches name the old buffers
    CLS_CUDA(cudaMemcpy(h->d_cases, h->cases.data(), h->cases.size() * sizeof(CaseParams), cudaMemcpyHostToDevice));
    return zero_tallies(h);
}

int launch_tracker(cls_handle *h, LaunchArgs a, int sched, int geom, const Shape &sh, cudaStream_t s) {
    cudaError_t e;
    const bool fp64 = h->opt.precision == CLS_PREC_FP64;
    if (sched == CLS_SCHED_EVENT) {
        a.bank = static_cast<unsigned char *>(h->d_bank) + sh.bank_off;
        a.bank_slots = sh.bank_slots;
        a.events_per_pass = (uint32_t)h->opt.events_per_pass;
        e = fp64 ? launch_event_fp64(a, sh.grid, sh.block, sh.smem, s, geom)
                 : launch_event_fp32(a, sh.grid, sh.block, sh.smem, s, geom);
    } else {
        e = fp64 ? launch_history_fp64(a, sh.grid, sh.block, sh.smem, s, geom)
                 : launch_history_fp32(a, sh.grid, sh.block, sh.smem, s, geom);
    }
    return cuda_fail(e);
}

int record_pair(cls_handle *h, cudaStream_t s, bool start) {
    if (start) {
        cudaEvent_t e0, e1;
        CLS_CUDA(cudaEventCreate(&e0));
        if (cudaEventCreate(&e1) != cudaSuccess) {
            cudaEventDestroy(e0);
            return CLS_E_CUDA;
        }
        h->ev_pairs.push_back(e0);
        h->ev_pairs.push_back(e1);
    }
    return cuda_fail(cudaEventRecord(h->ev_pairs[h->ev_pairs.size() - (start ? 2 : 1)], s));
}

int sync_and_time(cls_handle *h) {
    if (!h->ran) return CLS_E_STATE;
    CLS_CUDA(cudaSetDevice(h->device));
    CLS_CUDA(cudaStreamSynchronize(h->last_stream));
    for (size_t i = 0; i + 1 < h->ev_pairs.size(); i += 2) {
        float ms = 0.f;
        CLS_CUDA(cudaEventElapsedTime(&ms, h->ev_pairs[i], h->ev_pairs[i + 1]));
        h->seconds += ms * 1e-3;
        cudaEventDestroy(h->ev_pairs[i]);
        cudaEventDestroy(h->ev_pairs[i + 1]);
    }
    h->ev_pairs.clear();
    return CLS_OK;
}

int fetch_case(cls_handle *h, int k, std::vector<double> &flux, double stats[S_NUM], unsigned long long ct[C_NUM]) {
    const size_t nfl = (size_t)h->nbatch * h->nbins_stride;
    flux.resize(nfl);
    CLS_CUDA(cudaMemcpy(flux.data(), h->d_flux + (size_t)k * nfl, nfl * sizeof(double), cudaMemcpyDeviceToHost));
    CLS_CUDA(cudaMemcpy(stats, h->d_stats + (size_t)k * S_NUM, S_NUM * sizeof(double), cudaMemcpyDeviceToHost));
    CLS_CUDA(cudaMemcpy(ct, h->d_counters + (size_t)k * C_NUM, C_NUM * sizeof(unsigned long long),
                        cudaMemcpyDeviceToHost));
    return CLS_OK;
}

// FP64 normalisation of raw accumulators (paper Sec. 2 observables):
// R, T, A per-history Bernoulli means with sqrt(p(1-p)/(N-1)); <phi> the mean
// track length with its per-history standard error; phi_k = sum_b flux[b][k] /
// (N dx) with the batch-means error B/(B-1) sum_b (n_b/N)^2 (X_b - X)^2.
int finalize_raw(const cls_raw_t &raw, const double *flux, int flux_stride, const uint64_t *bh, double L,
                 cls_tallies_t *out) {
    const double N = (double)raw.n_histories;
    if (!(N > 0) || raw.nbins < 1 || raw.nbatch < 1 || !(L > 0)) return CLS_E_INVAL;
    out->n_histories = raw.n_histories;
    out->nR = raw.nR;
    out->nT = raw.nT;
    out->nA = raw.nA;
    out->n_coll = raw.n_coll;
    out->n_interface = raw.n_interface;
    out->n_reflect = raw.n_reflect;
    out->n_events = raw.n_events;
    out->max_events = raw.max_events;
    out->n_capped = raw.n_capped;
    auto bern = [&](uint64_t c, double *p, double *sd) {
        *p = (double)c / N;
        *sd = N > 1 ? std::sqrt(*p * (1.0 - *p) / (N - 1.0)) : NAN;
    };
    bern(raw.nR, &out->R, &out->sigma_R);
    bern(raw.nT, &out->T, &out->sigma_T);
    bern(raw.nA, &out->A, &out->sigma_A);
    const double mean = raw.sum_t / N;
    out->total_flux = mean;
    const double var = std::max(raw.sum_t2 / N - mean * mean, 0.0);
    out->sigma_total_flux = N > 1 ? std::sqrt(var / (N - 1.0)) : NAN;
    out->track0 = raw.track[0] / N;
    out->track1 = raw.track[1] / N;
    const int nb = raw.nbins;
    const double dx = L / nb;
    int B = 0;
    for (int b = 0; b < raw.nbatch; ++b) B += bh[b] > 0;
    for (int j = 0; j < nb; ++j) {
        double tot = 0.0;
        for (int b = 0; b < raw.nbatch; ++b) tot += flux[(size_t)b * flux_stride + j];
        const double phi = tot / (N * dx);
        if (out->flux) out->flux[j] = phi;
        if (out->flux_sigma) {
            if (B < 2) {
                out->flux_sigma[j] = NAN;
                continue;
            }
            double acc = 0.0;
            for (int b = 0; b < raw.nbatch; ++b) {
                if (!bh[b]) continue;
                const double nbh = (double)bh[b];
                const double xb = flux[(size_t)b * flux_stride + j] / (nbh * dx);
                const double wgt = nbh / N;
                acc += wgt * wgt * (xb - phi) * (xb - phi);
            }
            out->flux_sigma[j] = std::sqrt(acc * B / (B - 1.0));
        }
    }
    return raw.n_capped ? CLS_E_EVENT_LIMIT : CLS_OK;
}

void raw_of(const cls_handle *h, int k, const double st[S_NUM], const unsigned long long ct[C_NUM], cls_raw_t *out) {
    out->n_histories = h->n_hist[k];
    out->nR = ct[C_R];
    out->nT = ct[C_T];
    out->nA = ct[C_A];
    out->n_coll = ct[C_COLL];
    out->n_interface = ct[C_INT];
    out->n_reflect = ct[C_REFL];
    out->n_events = ct[C_EVENTS];
    out->max_events = ct[C_MAXEV];
    out->n_capped = ct[C_CAPPED];
    out->sum_t = st[S_T];
    out->sum_t2 = st[S_T2];
    out->track[0] = st[S_TRACK0];
    out->track[1] = st[S_TRACK1];
    out->nbins = h->cases[k].nbins;
    out->nbatch = h->nbatch;
}

int tallies_of(cls_handle *h, int k, cls_tallies_t *out) {
    if (!h || !out || k < 0 || k >= (int)h->cases.size()) return CLS_E_INVAL;
    int rc = sync_and_time(h);
    if (rc) return rc;
    std::vector<double> flux;
    double st[S_NUM];
    unsigned long long ct[C_NUM];
    rc = fetch_case(h, k, flux, st, ct);
    if (rc) return rc;
    cls_raw_t raw;
    raw_of(h, k, st, ct, &raw);
    rc = finalize_raw(raw, flux.data(), h->nbins_stride, h->batch_hist[k].data(), h->cases[k].L, out);
    out->seconds = h->seconds;
    return rc;
}

// ------------------------------------------------------------- autotuner
struct Tuned {
    int schedule, block, chunk, events_per_pass, group_geometry;
};

std::mutex g_tune_mutex;
std::map<std::string, Tuned> g_tune_cache;
bool g_tune_file_read = false;

// FNV-1a over (precision, case parameters), and the pilot size's power of
// two: identifies a tuning problem.  The best shape depends on the run's size
// (small chunks balance a short run, large ones amortise chunk claims in a long
// one), so a shape tuned on a small pilot is not reused for a large one.
std::string tune_signature(const cls_handle *h, uint64_t n_pilot) {
    unsigned long long x = 1469598103934665603ull;
    auto mix = [&](const void *p, size_t n) {
        const unsigned char *c = static_cast<const unsigned char *>(p);
        for (size_t i = 0; i < n; ++i) {
            x ^= c[i];
            x *= 1099511628211ull;
        }
    };
    mix(&h->opt.precision, sizeof(int));
    mix(h->params.data(), h->params.size() * sizeof(double));
    int size_bits = 0;
    while ((n_pilot >> size_bits) > 1) ++size_bits;
    char buf[80];
    std::snprintf(buf, sizeof(buf), "p%d-n%zu-s%d-%016llx", h->opt.precision, h->params.size() / 9, size_bits, x);
    return buf;
}

void tune_file_load() {
    if (g_tune_file_read) return;
    g_tune_file_read = true;
    const char *path = std::getenv("CLS_AUTOTUNE_CACHE");
    if (!path) return;
    FILE *f = std::fopen(path, "r");
    if (!f) return;
    char key[128];
    Tuned t;
    while (std::fscanf(f, "%127s %d %d %d %d %d", key, &t.schedule, &t.block, &t.chunk, &t.events_per_pass,
                       &t.group_geometry) == 6)
        g_tune_cache[key] = t;
    std::fclose(f);
}

void tune_file_append(const std::string &key, const Tuned &t) {
    const char *path = std::getenv("CLS_AUTOTUNE_CACHE");
    if (!path) return;
    FILE *f = std::fopen(path, "a");
    if (!f) return;
    std::fprintf(f, "%s %d %d %d %d %d\n", key.c_str(), t.schedule, t.block, t.chunk, t.events_per_pass,
                 t.group_geometry);
    std::fclose(f);
}

void apply_tuned(cls_handle *h, const Tuned &t) {
    h->opt.schedule = t.schedule;
    h->opt.block = t.block;
    h->opt.chunk = t.chunk;
    h->opt.events_per_pass = t.events_per_pass;
    h->opt.group_geometry = t.group_geometry;
    destroy_graph(h);
}

}  // namespace

extern "C" {

int cls_autotune(cls_handle *h, uint64_t n_pilot, uint64_t seed, void *stream) {
    if (!h || n_pilot == 0 || n_pilot > (1ull << 32)) return CLS_E_INVAL;
    CLS_CUDA(cudaSetDevice(h->device));
    const std::string key = tune_signature(h, n_pilot);
    {
        std::lock_guard<std::mutex> lock(g_tune_mutex);
        tune_file_load();
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) {
            apply_tuned(h, it->second);
            return CLS_OK;
        }
    }
    const int ncases = (int)h->cases.size();
    cls_handle *t = nullptr;
    int rc = create_common(h->params.data(), ncases, h->batch, &t);
    if (rc) return rc;
    t->opt = h->opt;
    std::vector<Tuned> cand;
    // a batch of several geometries also tries one launch per geometry against one mixed launch
    std::vector<int> groupings = {h->opt.group_geometry};
    if (h->geom == 0) groupings = {1, 0};
    for (int gg : groupings) {
        for (int b : {64, 128, 256})
            for (int c : {64, 256, 1024}) cand.push_back({CLS_SCHED_HISTORY, b, c, h->opt.events_per_pass, gg});
        for (int b : {128, 256})
            for (int e : {4, 16}) cand.push_back({CLS_SCHED_EVENT, b, h->opt.chunk, e, gg});
    }
    cudaStream_t s = (cudaStream_t)stream;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        cls_destroy(t);
        return CLS_E_CUDA;
    }
    float best_ms = 0.f;
    Tuned best = cand[0];
    bool have = false;
    const uint64_t base = 1ull << 61;  // pilot history ids, far from a caller's
    for (size_t i = 0; i < cand.size() && !rc; ++i) {
        apply_tuned(t, cand[i]);
        t->opt.max_events = h->opt.max_events;
        // warm-up (module load, bank allocation, graph capture), then one timed run
        for (int rep = 0; rep < 2 && !rc; ++rep) {
            for (auto &nh : t->next_history) nh = base + (uint64_t)(2 * i + rep) * n_pilot;
            if (rep == 1 && cudaEventRecord(e0, s) != cudaSuccess) rc = CLS_E_CUDA;
            if (!rc) rc = t->batch ? cls_batch_run(t, rep ? n_pilot : std::max<uint64_t>(n_pilot / 4, 1), seed, stream)
                                   : cls_run(t, rep ? n_pilot : std::max<uint64_t>(n_pilot / 4, 1), seed, stream);
            if (!rc && rep == 1 && cudaEventRecord(e1, s) != cudaSuccess) rc = CLS_E_CUDA;
        }
        if (rc) {
            // a candidate that does not fit (e.g. shared memory) is skipped
            if (rc == CLS_E_INVAL || rc == CLS_E_NOMEM) rc = CLS_OK;
            continue;
        }
        float ms = 0.f;
        if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
            rc = CLS_E_CUDA;
            break;
        }
        if (!have || ms < best_ms) {
            best_ms = ms;
            best = cand[i];
            have = true;
        }
        zero_tallies(t);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cls_destroy(t);
    if (rc) return rc;
    if (!have) return CLS_E_INVAL;
    apply_tuned(h, best);
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    g_tune_cache[key] = best;
    tune_file_append(key, best);
    return CLS_OK;
}


int cls_create(double sigma0, double sigma1, double lambda0, double lambda1, double c0, double c1, double L,
               int d, int nbins, cls_handle **out) {
    const double p[9] = {sigma0, sigma1, lambda0, lambda1, c0, c1, L, (double)d, (double)nbins};
    return create_common(p, 1, false, out);
}

int cls_batch_create(const double *params, int ncases, cls_handle **out) {
    return create_common(params, ncases, true, out);
}

int cls_num_cases(const cls_handle *h) { return h ? (int)h->cases.size() : 0; }

int cls_set_option(cls_handle *h, int key, int64_t v) {
    if (!h) return CLS_E_INVAL;
    Options &o = h->opt;
    switch (key) {
    case CLS_OPT_PRECISION:
        if (v != CLS_PREC_FP64 && v != CLS_PREC_FP32) return CLS_E_INVAL;
        o.precision = (int)v;
        break;
    case CLS_OPT_SCHEDULE:
        if (v != CLS_SCHED_HISTORY && v != CLS_SCHED_EVENT && v != CLS_SCHED_AUTO) return CLS_E_INVAL;
        o.schedule = (int)v;
        break;
    case CLS_OPT_BLOCK:
        if (v < 32 || v > 256 || v % 32) return CLS_E_INVAL;
        o.block = (int)v;
        break;
    case CLS_OPT_CHUNK:
        if (v < 32 || v > kBatchQuantum || (v & (v - 1))) return CLS_E_INVAL;
        o.chunk = (int)v;
        break;
    case CLS_OPT_NBATCH:
        if (v < 2 || v > 1024) return CLS_E_INVAL;
        if (v != h->nbatch) {
            // changes the tally layout: only allowed before the first run
            if (h->ran) return CLS_E_STATE;
            CLS_CUDA(cudaSetDevice(h->device));
            if (h->ws) {
                // re-carve the bound workspace, if the new layout fits it
                const int old = h->nbatch;
                size_t bank = 0;
                h->nbatch = (int)v;
                int rc = bank_need(h, &bank);
                if (!rc && dev_layout(h, bank).total > h->ws_bytes) rc = CLS_E_NOMEM;
                if (rc) {
                    h->nbatch = old;
                    return rc;
                }
                o.nbatch = (int)v;
                rc = carve_workspace(h, bank);
                if (rc) return rc;
            } else {
                free_tallies(h);
                h->nbatch = (int)v;
                o.nbatch = (int)v;
                int rc = alloc_tallies(h);
                if (rc) return rc;
                rc = zero_tallies(h);
                if (rc) return rc;
            }
        }
        break;
    case CLS_OPT_MAX_EVENTS:
        if (v < 1 || v > (int64_t)kMaxEventsLimit) return CLS_E_INVAL;
        o.max_events = (uint32_t)v;
        break;
    case CLS_OPT_BLOCKS_PER_SM:
        if (v < 0 || v > 32) return CLS_E_INVAL;
        o.blocks_per_sm = (int)v;
        break;
    case CLS_OPT_BANK:
        if (v < 0 || v > 4096) return CLS_E_INVAL;
        o.bank = (int)v;
        break;
    case CLS_OPT_EVENTS_PER_PASS:
        if (v < 1 || v > 64) return CLS_E_INVAL;
        o.events_per_pass = (int)v;
        break;
    case CLS_OPT_SOURCE:
        if (v != CLS_SOURCE_INCIDENT && v != CLS_SOURCE_VOLUME) return CLS_E_INVAL;
        if (h->ran) return CLS_E_STATE;
        for (auto &c : h->cases) c.source = (int32_t)v;
        CLS_CUDA(cudaSetDevice(h->device));
        CLS_CUDA(cudaMemcpy(h->d_cases, h->cases.data(), h->cases.size() * sizeof(CaseParams), cudaMemcpyHostToDevice));
        break;
    case CLS_OPT_GROUP_GEOMETRY:
        if (v != 0 && v != 1) return CLS_E_INVAL;
        o.group_geometry = (int)v;
        break;
    case CLS_OPT_FIRST_HISTORY:
        if (v < 0 || v > ((int64_t)1 << 62)) return CLS_E_INVAL;
        for (auto &nh : h->next_history) nh = (uint64_t)v;
        return CLS_OK;
    default:
        return CLS_E_INVAL;
    }
    destroy_graph(h);
    return CLS_OK;
}

int cls_get_option(const cls_handle *h, int key, int64_t *v) {
    if (!h || !v) return CLS_E_INVAL;
    const Options &o = h->opt;
    switch (key) {
    case CLS_OPT_PRECISION: *v = o.precision; break;
    case CLS_OPT_SCHEDULE: *v = o.schedule; break;
    case CLS_OPT_BLOCK: *v = o.block; break;
    case CLS_OPT_CHUNK: *v = o.chunk; break;
    case CLS_OPT_NBATCH: *v = h->nbatch; break;
    case CLS_OPT_MAX_EVENTS: *v = o.max_events; break;
    case CLS_OPT_BLOCKS_PER_SM: *v = o.blocks_per_sm ? o.blocks_per_sm : h->used_blocks_per_sm; break;
    case CLS_OPT_BANK: *v = o.bank; break;
    case CLS_OPT_EVENTS_PER_PASS: *v = o.events_per_pass; break;
    case CLS_OPT_FIRST_HISTORY: *v = h->next_history.empty() ? 0 : (int64_t)h->next_history[0]; break;
    case CLS_OPT_SOURCE: *v = h->cases.empty() ? 0 : h->cases[0].source; break;
    case CLS_OPT_GROUP_GEOMETRY: *v = o.group_geometry; break;
    default: return CLS_E_INVAL;
    }
    return CLS_OK;
}

int cls_run(cls_handle *h, uint64_t n, uint64_t seed, void *stream) {
    if (!h || n == 0 || n > (1ull << 62)) return CLS_E_INVAL;
    CLS_CUDA(cudaSetDevice(h->device));
    if (h->opt.schedule == CLS_SCHED_AUTO) {
        int arc = cls_autotune(h, std::min<uint64_t>(std::max<uint64_t>(n / 16, 4096), 262144), seed ^ 0x5bd1e995ull,
                               stream);
        if (arc) return arc;
    }
    cudaStream_t s = (cudaStream_t)stream;
    RunPlan plan;
    int rc = prepare_run(h, n, seed, &plan);
    if (rc) return rc;
    Shape sh[kMaxGroups];
    size_t bank = 0;
    rc = plan_shapes(h, plan, sh, &bank);
    if (!rc) rc = ensure_bank(h, bank);
    if (rc) return rc;
    rc = record_pair(h, s, true);
    if (rc) return rc;
    CLS_CUDA(cudaMemcpyAsync(h->d_runs, h->h_runs, runs_bytes(h->cases.size()), cudaMemcpyHostToDevice, s));
    CLS_CUDA(cudaEventRecord(h->runs_copied, s));
    CLS_CUDA(cudaMemsetAsync(h->d_chunk_counter, 0, kMaxGroups * sizeof(unsigned long long), s));
    for (int g = 0; g < plan.ngroups && !rc; ++g) rc = launch_tracker(h, plan.a[g], plan.sched[g], plan.geom[g], sh[g], s);
    if (rc) return rc;
    rc = record_pair(h, s, false);
    if (rc) return rc;
    h->last_stream = s;
    account_run(h, n);
    return CLS_OK;
}

int cls_batch_run(cls_handle *h, uint64_t n, uint64_t seed, void *stream) {
    if (!h || n == 0 || n > (1ull << 62)) return CLS_E_INVAL;
    CLS_CUDA(cudaSetDevice(h->device));
    if (h->opt.schedule == CLS_SCHED_AUTO) {
        int arc = cls_autotune(h, std::min<uint64_t>(std::max<uint64_t>(n / 16, 4096), 262144), seed ^ 0x5bd1e995ull,
                               stream);
        if (arc) return arc;
    }
    cudaStream_t s = (cudaStream_t)stream;
    RunPlan plan;
    int rc = prepare_run(h, n, seed, &plan);
    if (rc) return rc;
    // capture {counter reset, one tracker per launch group} once per (launch
    // shape, seed, grouping); later calls only refresh the work list (history
    // ranges) before replaying the graph.  The groups' launches are parallel
    // branches of the graph: the second starts its blocks as the first one's
    // drain, so their tails overlap.
    const int key[10] = {h->opt.precision, h->opt.schedule, h->opt.block, h->opt.chunk, (int)h->opt.max_events,
                         h->opt.blocks_per_sm, (int)(seed & 0x7fffffff), (int)(seed >> 31), h->opt.group_geometry,
                         h->outcome_codes != nullptr};
    std::vector<uint64_t> tc(plan.ngroups);
    for (int g = 0; g < plan.ngroups; ++g) tc[g] = plan.a[g].total_chunks;
    if (h->graph_exec && (tc != h->graph_total_chunks || std::memcmp(key, h->graph_key, sizeof(key))))
        destroy_graph(h);
    if (!h->graph_exec) {
        Shape sh[kMaxGroups];
        size_t bank = 0;
        rc = plan_shapes(h, plan, sh, &bank);
        if (!rc) rc = ensure_bank(h, bank);
        if (rc) return rc;
        if (!h->capture_stream) CLS_CUDA(cudaStreamCreateWithFlags(&h->capture_stream, cudaStreamNonBlocking));
        while ((int)h->aux_streams.size() < plan.ngroups - 1) {
            cudaStream_t a = nullptr;
            CLS_CUDA(cudaStreamCreateWithFlags(&a, cudaStreamNonBlocking));
            h->aux_streams.push_back(a);
        }
        while ((int)h->join_events.size() < plan.ngroups) {
            cudaEvent_t e = nullptr;
            CLS_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
            h->join_events.push_back(e);
        }
        CLS_CUDA(cudaStreamBeginCapture(h->capture_stream, cudaStreamCaptureModeThreadLocal));
        cudaError_t e = cudaMemsetAsync(h->d_chunk_counter, 0, kMaxGroups * sizeof(unsigned long long), h->capture_stream);
        if (e == cudaSuccess && plan.ngroups > 1) e = cudaEventRecord(h->join_events[0], h->capture_stream);
        int lrc = (e == cudaSuccess) ? CLS_OK : CLS_E_CUDA;
        for (int g = 0; g < plan.ngroups && !lrc; ++g) {
            cudaStream_t gs = g == 0 ? h->capture_stream : h->aux_streams[g - 1];
            if (g > 0 && cudaStreamWaitEvent(gs, h->join_events[0], 0) != cudaSuccess) lrc = CLS_E_CUDA;
            if (!lrc) lrc = launch_tracker(h, plan.a[g], plan.sched[g], plan.geom[g], sh[g], gs);
            if (!lrc && g > 0 && (cudaEventRecord(h->join_events[g], gs) != cudaSuccess ||
                                  cudaStreamWaitEvent(h->capture_stream, h->join_events[g], 0) != cudaSuccess))
                lrc = CLS_E_CUDA;
        }
        cudaGraph_t g = nullptr;
        cudaError_t e2 = cudaStreamEndCapture(h->capture_stream, &g);
        if (lrc || e2 != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            cudaGetLastError();
            return lrc ? lrc : CLS_E_CUDA;
        }
        h->graph = g;
        if (cudaGraphInstantiate(&h->graph_exec, g, 0) != cudaSuccess) {
            destroy_graph(h);
            return CLS_E_CUDA;
        }
        h->graph_total_chunks = tc;
        std::memcpy(h->graph_key, key, sizeof(key));
    }
    rc = record_pair(h, s, true);
    if (rc) return rc;
    CLS_CUDA(cudaMemcpyAsync(h->d_runs, h->h_runs, runs_bytes(h->cases.size()), cudaMemcpyHostToDevice, s));
    CLS_CUDA(cudaEventRecord(h->runs_copied, s));
    CLS_CUDA(cudaGraphLaunch(h->graph_exec, s));
    rc = record_pair(h, s, false);
    if (rc) return rc;
    h->last_stream = s;
    account_run(h, n);
    return CLS_OK;
}

int cls_batch_set_case_schedule(cls_handle *h, int case_idx, int schedule) {
    if (!h || case_idx < 0 || case_idx >= (int)h->cases.size()) return CLS_E_INVAL;
    if (schedule != CLS_SCHED_AUTO && schedule != CLS_SCHED_HISTORY && schedule != CLS_SCHED_EVENT) return CLS_E_INVAL;
    if (h->case_sched[case_idx] != schedule) {
        h->case_sched[case_idx] = schedule;
        destroy_graph(h);  // the grouping of the captured launches changes
    }
    return CLS_OK;
}

int cls_batch_get_case_schedule(const cls_handle *h, int case_idx, int *schedule) {
    if (!h || !schedule || case_idx < 0 || case_idx >= (int)h->cases.size()) return CLS_E_INVAL;
    *schedule = case_schedule(h, case_idx);
    return CLS_OK;
}

int cls_autotune_cases(cls_handle *h, uint64_t n_pilot, uint64_t seed, void *stream) {
    if (!h || n_pilot == 0 || n_pilot > (1ull << 32)) return CLS_E_INVAL;
    CLS_CUDA(cudaSetDevice(h->device));
    cudaStream_t s = (cudaStream_t)stream;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        return CLS_E_CUDA;
    }
    const uint64_t base = 1ull << 61;  // pilot history ids, far from a caller's
    const int nc = (int)h->cases.size();
    std::vector<int> chosen(nc, CLS_SCHED_AUTO);
    int rc = CLS_OK;
    for (int k = 0; k < nc && !rc; ++k) {
        cls_handle *t = nullptr;
        rc = create_common(h->params.data() + 9 * (size_t)k, 1, false, &t);
        if (rc) break;
        t->opt = h->opt;
        t->cases[0].case_id = h->cases[k].case_id;  // the case's own random numbers
        rc = cudaMemcpy(t->d_cases, t->cases.data(), sizeof(CaseParams), cudaMemcpyHostToDevice) == cudaSuccess
                 ? CLS_OK : CLS_E_CUDA;
        float ms[2] = {0.f, 0.f};
        const int scheds[2] = {CLS_SCHED_HISTORY, CLS_SCHED_EVENT};
        for (int i = 0; i < 2 && !rc; ++i) {
            t->opt.schedule = scheds[i];
            for (int rep = 0; rep < 2 && !rc; ++rep) {
                t->next_history[0] = base + (uint64_t)(2 * i + rep) * n_pilot;
                if (rep == 1 && cudaEventRecord(e0, s) != cudaSuccess) rc = CLS_E_CUDA;
                if (!rc) rc = cls_run(t, rep ? n_pilot : std::max<uint64_t>(n_pilot / 4, 1), seed, stream);
                if (!rc && rep == 1 && cudaEventRecord(e1, s) != cudaSuccess) rc = CLS_E_CUDA;
            }
            if (!rc && (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms[i], e0, e1) != cudaSuccess))
                rc = CLS_E_CUDA;
        }
        cls_destroy(t);
        if (!rc) chosen[k] = ms[1] < ms[0] ? CLS_SCHED_EVENT : CLS_SCHED_HISTORY;
    }
    // a case's preference alone need not carry over into the batch, where a
    // second launch adds its own tail: keep the per-case grouping only if a
    // pilot of the whole batch runs faster with it than with every case on
    // the handle's schedule
    bool mixed = false;
    for (int k = 0; k < nc; ++k) mixed |= chosen[k] != h->opt.schedule;
    float batch_ms[2] = {0.f, 0.f};
    if (!rc && mixed && h->opt.schedule != CLS_SCHED_AUTO) {
        cls_handle *t = nullptr;
        rc = create_common(h->params.data(), nc, true, &t);
        if (!rc) {
            t->opt = h->opt;
            for (int i = 0; i < 2 && !rc; ++i) {
                for (int k = 0; k < nc; ++k) t->case_sched[k] = i ? chosen[k] : CLS_SCHED_AUTO;
                destroy_graph(t);
                for (int rep = 0; rep < 2 && !rc; ++rep) {
                    for (auto &nh : t->next_history) nh = base + (uint64_t)(8 + 2 * i + rep) * n_pilot;
                    if (rep == 1 && cudaEventRecord(e0, s) != cudaSuccess) rc = CLS_E_CUDA;
                    if (!rc) rc = cls_batch_run(t, rep ? n_pilot : std::max<uint64_t>(n_pilot / 4, 1), seed, stream);
                    if (!rc && rep == 1 && cudaEventRecord(e1, s) != cudaSuccess) rc = CLS_E_CUDA;
                }
                if (!rc && (cudaEventSynchronize(e1) != cudaSuccess ||
                            cudaEventElapsedTime(&batch_ms[i], e0, e1) != cudaSuccess))
                    rc = CLS_E_CUDA;
            }
            cls_destroy(t);
        }
        if (!rc && !(batch_ms[1] < batch_ms[0])) mixed = false;
    }
    for (int k = 0; k < nc && !rc; ++k) rc = cls_batch_set_case_schedule(h, k, mixed ? chosen[k] : CLS_SCHED_AUTO);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return rc;
}

int cls_record_outcomes(cls_handle *h, uint8_t *d_codes, uint64_t capacity) {
    if (!h || (d_codes && capacity == 0)) return CLS_E_INVAL;
    // switching recording on or off changes the launches' arguments: recapture
    if ((d_codes != nullptr) != (h->outcome_codes != nullptr)) destroy_graph(h);
    h->outcome_codes = d_codes;
    h->outcome_cap = d_codes ? capacity : 0;
    return CLS_OK;
}

int cls_tallies(cls_handle *h, cls_tallies_t *out) { return tallies_of(h, 0, out); }

int cls_batch_tallies(cls_handle *h, int case_idx, cls_tallies_t *out) { return tallies_of(h, case_idx, out); }

int cls_raw_tallies(cls_handle *h, int k, cls_raw_t *out, double *flux_batches, uint64_t *batch_histories) {
    if (!h || !out || k < 0 || k >= (int)h->cases.size()) return CLS_E_INVAL;
    int rc = sync_and_time(h);
    if (rc) return rc;
    std::vector<double> flux;
    double st[S_NUM];
    unsigned long long ct[C_NUM];
    rc = fetch_case(h, k, flux, st, ct);
    if (rc) return rc;
    raw_of(h, k, st, ct, out);
    if (flux_batches)
        for (int b = 0; b < h->nbatch; ++b)
            std::memcpy(flux_batches + (size_t)b * out->nbins, flux.data() + (size_t)b * h->nbins_stride,
                        out->nbins * sizeof(double));
    if (batch_histories)
        for (int b = 0; b < h->nbatch; ++b) batch_histories[b] = h->batch_hist[k][b];
    return CLS_OK;
}

int cls_finalize_raw(const cls_raw_t *raw, const double *flux_batches, const uint64_t *batch_histories, double L,
                     cls_tallies_t *out) {
    if (!raw || !flux_batches || !batch_histories || !out) return CLS_E_INVAL;
    const int rc = finalize_raw(*raw, flux_batches, raw->nbins, batch_histories, L, out);
    out->seconds = 0.0;
    return rc;
}

int cls_reset(cls_handle *h) {
    if (!h) return CLS_E_INVAL;
    CLS_CUDA(cudaSetDevice(h->device));
    if (h->last_stream || h->ran) CLS_CUDA(cudaDeviceSynchronize());
    return zero_tallies(h);
}

void cls_destroy(cls_handle *h) {
    if (!h) return;
    cudaSetDevice(h->device);
    cudaDeviceSynchronize();
    destroy_graph(h);
    if (h->capture_stream) cudaStreamDestroy(h->capture_stream);
    for (cudaStream_t a : h->aux_streams) cudaStreamDestroy(a);
    for (cudaEvent_t e : h->join_events) cudaEventDestroy(e);
    for (cudaEvent_t e : h->ev_pairs) cudaEventDestroy(e);
    if (h->runs_copied) cudaEventDestroy(h->runs_copied);
    free_device(h);
    if (h->h_runs) cudaFreeHost(h->h_runs);
    cudaGetLastError();
    delete h;
}

int cls_workspace_bytes(cls_handle *h, size_t *bytes) {
    if (!h || !bytes) return CLS_E_INVAL;
    CLS_CUDA(cudaSetDevice(h->device));
    size_t bank = 0;
    const int rc = bank_need(h, &bank);
    if (rc) return rc;
    *bytes = dev_layout(h, bank).total;
    return CLS_OK;
}

int cls_bind_workspace(cls_handle *h, void *d_workspace, size_t bytes) {
    if (!h) return CLS_E_INVAL;
    if (h->ran) return CLS_E_STATE;  // the tallies hold results: cls_reset first
    CLS_CUDA(cudaSetDevice(h->device));
    if (!d_workspace) {
        if (!h->ws) return CLS_OK;
        // back to the library's own buffers
        CLS_CUDA(cudaDeviceSynchronize());
        free_device(h);
        h->ws = nullptr;
        h->ws_bytes = h->ws_bank_off = 0;
        destroy_graph(h);
        int rc = CLS_OK;
        if (cudaMalloc(&h->d_cases, h->cases.size() * sizeof(CaseParams)) != cudaSuccess ||
            cudaMalloc(&h->d_runs, runs_bytes(h->cases.size())) != cudaSuccess ||
            cudaMalloc(&h->d_chunk_counter, kMaxGroups * sizeof(unsigned long long)) != cudaSuccess) {
            cudaGetLastError();
            rc = CLS_E_NOMEM;
        }
        if (!rc) rc = alloc_tallies(h);
        if (!rc && cudaMemcpy(h->d_cases, h->cases.data(), h->cases.size() * sizeof(CaseParams),
                              cudaMemcpyHostToDevice) != cudaSuccess)
            rc = CLS_E_CUDA;
        if (!rc) rc = zero_tallies(h);
        return rc;
    }
    if (reinterpret_cast<uintptr_t>(d_workspace) & 255u) return CLS_E_INVAL;
    cudaPointerAttributes attr;
    if (cudaPointerGetAttributes(&attr, d_workspace) != cudaSuccess) {
        cudaGetLastError();
        return CLS_E_INVAL;
    }
    if (attr.type != cudaMemoryTypeDevice || attr.device != h->device) return CLS_E_INVAL;
    size_t bank = 0;
    int rc = bank_need(h, &bank);
    if (rc) return rc;
    if (bytes < dev_layout(h, bank).total) return CLS_E_INVAL;
    CLS_CUDA(cudaDeviceSynchronize());  // no launch of this handle still uses the old buffers
    free_device(h);
    h->ws = static_cast<unsigned char *>(d_workspace);
    h->ws_bytes = bytes;
    return carve_workspace(h, bank);
}

const char *cls_strerror(int code) {
    switch (code) {
    case CLS_OK: return "success";
    case CLS_E_INVAL: return "invalid argument";
    case CLS_E_NOMEM: return "out of memory";
    case CLS_E_CUDA: return "CUDA error";
    case CLS_E_EVENT_LIMIT: return "a history reached the event cap";
    case CLS_E_STATE: return "call not valid in this state";
    case CLS_E_NODEVICE: return "no CUDA device";
    default: return "unknown error";
    }
}

int cls_trace(cls_handle *h, int k, uint64_t seed, uint64_t history, double *rows, int cap, int *n_rows) {
    if (!h || !rows || cap < 1 || !n_rows || k < 0 || k >= (int)h->cases.size()) return CLS_E_INVAL;
    CLS_CUDA(cudaSetDevice(h->device));
    double *d_rows = nullptr;
    int *d_n = nullptr;
    if (cudaMalloc(&d_rows, (size_t)cap * 10 * sizeof(double)) != cudaSuccess) return CLS_E_NOMEM;
    if (cudaMalloc(&d_n, sizeof(int)) != cudaSuccess) {
        cudaFree(d_rows);
        return CLS_E_NOMEM;
    }
    TraceArgs ta{h->d_cases, k, seed, history, h->opt.max_events, d_rows, cap, d_n};
    cudaError_t e = (h->opt.precision == CLS_PREC_FP64) ? launch_trace_fp64(ta, 0) : launch_trace_fp32(ta, 0);
    int n = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&n, d_n, sizeof(int), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess)
        e = cudaMemcpy(rows, d_rows, (size_t)std::min(n, cap) * 10 * sizeof(double), cudaMemcpyDeviceToHost);
    cudaFree(d_rows);
    cudaFree(d_n);
    if (e != cudaSuccess) return CLS_E_CUDA;
    *n_rows = n;
    return CLS_OK;
}

}  // extern "C"
