// cls_noalloc.cu -- cls_run_noalloc: the FP64 history-based tracker for callers
// that must not allocate device memory.
//
// Some callers cannot call cudaMalloc: code that runs inside another
// framework's memory budget (a plugin whose host owns every device byte
// through its own pool allocator), or a process that has reserved all device
// memory up front and forbids the library from growing it.  cls_create()
// allocates its tallies and work list, so it is not usable there.  This entry
// point instead keeps its scratch -- the case parameters, the per-case work
// list and the chunk counter the persistent kernel claims work from -- in a
// file-scope __device__ array of fixed size, and writes results into tally
// buffers the caller already owns.  It calls no cudaMalloc, cudaFree or other
// allocating routine.
//
// Every call shares the one scratch array, which keeps the last call's
// contents; each call rewrites the parameters and work list and clears the
// chunk counter before its kernel starts.  Calls whose work overlaps on the
// GPU (different streams, or another host thread) race on it.
#include <cstring>
#include <mutex>

#include "../../include/cls.h"
#include "cls_device.cuh"

namespace {

using namespace cls;

struct NoallocScratch {
    CaseParams cases[CLS_NOALLOC_MAX_CASES];
    RunCase runs[CLS_NOALLOC_MAX_CASES];
    unsigned long long chunk_counter;
};

// The static scratch: every device that loads the library holds one copy of
// it (about 12 KB) until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[sizeof(NoallocScratch)];

constexpr int kMaxDevices = 64;
NoallocScratch *g_scratch_ptr[kMaxDevices] = {nullptr};
int g_sm_count[kMaxDevices] = {0};
std::mutex g_setup_mutex;

// Device address of the scratch array for the current device.  In host code
// the array's name is only a host-side stand-in, so the address must come
// from cudaGetSymbolAddress, once per device, with that device current.
int scratch_for_current_device(NoallocScratch **out, int *sm_count) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return CLS_E_CUDA;
    if (dev < 0 || dev >= kMaxDevices) return CLS_E_INVAL;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess) return CLS_E_CUDA;
        int sms = 0;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return CLS_E_CUDA;
        if (cudaFuncSetAttribute(history_kernel<double, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 200 * 1024) != cudaSuccess)
            return CLS_E_CUDA;
        g_sm_count[dev] = sms;
        g_scratch_ptr[dev] = static_cast<NoallocScratch *>(p);
    }
    *out = g_scratch_ptr[dev];
    *sm_count = g_sm_count[dev];
    return CLS_OK;
}

bool valid_case(const double *p) {
    const double s0 = p[0], s1 = p[1], l0 = p[2], l1 = p[3], c0 = p[4], c1 = p[5], L = p[6], d = p[7], nb = p[8];
    auto fin = [](double v) { return v == v && v - v == 0.0; };
    return fin(s0) && s0 >= 0 && fin(s1) && s1 >= 0 && fin(l0) && l0 > 0 && fin(l1) && l1 > 0 && c0 >= 0 &&
           c0 <= 1 && c1 >= 0 && c1 <= 1 && fin(L) && L > 0 && (d == 1.0 || d == 2.0 || d == 3.0 || d == 11.0 || d == 13.0) && nb >= 1 && nb <= 4096 &&
           nb == (double)(int)nb;
}

}  // namespace

extern "C" int cls_run_noalloc(const double *params, int ncases, uint64_t first, uint64_t n, uint64_t seed,
                               int nbatch, int nbins_stride, double *d_flux, double *d_stats,
                               unsigned long long *d_counters, void *stream) {
    if (!params || !d_flux || !d_stats || !d_counters) return CLS_E_INVAL;
    if (ncases < 1 || ncases > CLS_NOALLOC_MAX_CASES) return CLS_E_INVAL;
    if (n == 0 || n > (1ull << 62) || first > (1ull << 62)) return CLS_E_INVAL;
    if (nbatch < 1 || nbatch > 1024) return CLS_E_INVAL;
    int nbins_max = 0;
    for (int k = 0; k < ncases; ++k) {
        if (!valid_case(params + 9 * (size_t)k)) return CLS_E_INVAL;
        nbins_max = nbins_max > (int)params[9 * k + 8] ? nbins_max : (int)params[9 * k + 8];
    }
    if (nbins_stride < nbins_max) return CLS_E_INVAL;

    NoallocScratch *scratch = nullptr;
    int sm_count = 0;
    int rc = scratch_for_current_device(&scratch, &sm_count);
    if (rc) return rc;

    // host image of the parameters and work list (stack memory: no allocation)
    NoallocScratch host;
    std::memset(&host, 0, sizeof(host));
    const uint64_t q = 1024ull * (uint64_t)nbatch;
    const uint64_t batch_len = 1024ull * ((n + q - 1) / q > 0 ? (n + q - 1) / q : 1);
    const int chunk = 256;
    uint64_t chunk_begin = 0;
    for (int k = 0; k < ncases; ++k) {
        const double *p = params + 9 * (size_t)k;
        CaseParams &c = host.cases[k];
        for (int i = 0; i < 2; ++i) {
            c.sigma[i] = p[i];
            c.inv_sigma[i] = p[i] > 0 ? 1.0 / p[i] : 0.0;
            c.lambda[i] = p[2 + i];
            c.c[i] = p[4 + i];
            c.sigma_f[i] = (float)p[i];
            c.inv_sigma_f[i] = p[i] > 0 ? (float)(1.0 / p[i]) : 0.0f;
            c.lambda_f[i] = (float)p[2 + i];
            c.c_f[i] = (float)p[4 + i];
        }
        c.L = p[6];
        c.d = (int32_t)p[7];
        c.nbins = (int32_t)p[8];
        c.p0 = c.lambda[0] / (c.lambda[0] + c.lambda[1]);
        c.dx = c.L / c.nbins;
        c.inv_dx = c.nbins / c.L;
        c.L_f = (float)c.L;
        c.p0_f = (float)c.p0;
        c.dx_f = (float)c.dx;
        c.inv_dx_f = (float)c.inv_dx;
        c.case_id = (uint32_t)k;
        for (int i = 0; i < 2; ++i) {
            c.thr_c53[i] = unit_threshold(c.c[i], 53);
            c.thr_c24[i] = (uint32_t)unit_threshold((double)c.c_f[i], 24);
        }
        c.thr_p053 = unit_threshold(c.p0, 53);
        c.thr_p024 = (uint32_t)unit_threshold((double)c.p0_f, 24);
        RunCase &r = host.runs[k];
        r.first = first;
        r.n = n;
        r.batch_len = batch_len;
        r.chunk_begin = chunk_begin;
        r.case_index = k;
        chunk_begin += (n + chunk - 1) / chunk;
    }

    cudaStream_t s = (cudaStream_t)stream;
    // pageable source: the copy is staged before cudaMemcpyAsync returns, so the
    // stack image may go out of scope afterwards
    if (cudaMemcpyAsync(scratch->cases, host.cases, ncases * sizeof(CaseParams), cudaMemcpyHostToDevice, s) !=
            cudaSuccess ||
        cudaMemcpyAsync(scratch->runs, host.runs, ncases * sizeof(RunCase), cudaMemcpyHostToDevice, s) !=
            cudaSuccess ||
        cudaMemsetAsync(&scratch->chunk_counter, 0, sizeof(unsigned long long), s) != cudaSuccess)
        return CLS_E_CUDA;

    LaunchArgs a;
    std::memset(&a, 0, sizeof(a));
    a.cases = scratch->cases;
    a.runs = scratch->runs;
    a.nruns = ncases;
    a.chunk = chunk;
    a.total_chunks = chunk_begin;
    a.chunk_counter = &scratch->chunk_counter;
    a.t = Tallies{d_flux, d_stats, d_counters, nbatch, nbins_stride};
    a.seed = seed;
    a.rk = make_round_keys(seed);
    a.max_events = 100000000u;
    a.region_bytes = region_bytes((int)sizeof(double), nbins_stride);
    a.dif = 0;
    a.flush_every = 0;

    const size_t per_warp = 2 * (size_t)a.region_bytes;
    int warps = (int)((200 * 1024) / per_warp);
    warps = warps > kHistoryBlockFp64 / 32 ? kHistoryBlockFp64 / 32 : warps;
    if (warps < 1) return CLS_E_INVAL;
    const int block = 32 * warps;
    const size_t smem = (size_t)warps * per_warp;
    int bps = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, history_kernel<double, 0>, block, smem) != cudaSuccess)
        return CLS_E_CUDA;
    if (bps < 1) return CLS_E_INVAL;
    history_kernel<double, 0><<<sm_count * bps, block, smem, s>>>(a);
    return cudaGetLastError() == cudaSuccess ? CLS_OK : CLS_E_CUDA;
}
