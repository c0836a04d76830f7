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
// chunk counter in a small set-up kernel before its tracker starts.  Calls
// whose work overlaps on the GPU (different streams, or another host thread)
// race on it.
#include <cstring>
#include <mutex>

#include "../../include/cls.h"
#include "cls_case.h"
#include "cls_device.cuh"

namespace {

using namespace cls;

struct NoallocScratch {
    CaseParams cases[CLS_NOALLOC_MAX_CASES];
    RunCase runs[CLS_NOALLOC_MAX_CASES];
    unsigned long long chunk_counter;
};

// The static scratch: every device that loads the library holds one copy of
// it (about 16 KB) until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[sizeof(NoallocScratch)];

// One call's case parameters and work list, handed to the set-up kernel by
// value: kernel arguments are copied when the launch is enqueued, so nothing
// is read from host memory after this call returns (a stream-ordered copy
// from a host buffer would have to keep that buffer alive until it runs).
struct NoallocImage {
    CaseParams cases[CLS_NOALLOC_MAX_CASES];
    RunCase runs[CLS_NOALLOC_MAX_CASES];
    int ncases;
};
static_assert(sizeof(NoallocImage) < 32000, "kernel arguments are limited to 32 KB");

// Writes the call's cases and work list into the scratch and clears the work
// counter; runs before the tracker on the same stream.
__global__ void noalloc_setup(NoallocScratch *scratch, const NoallocImage img) {
    for (int i = threadIdx.x; i < img.ncases; i += blockDim.x) {
        scratch->cases[i] = img.cases[i];
        scratch->runs[i] = img.runs[i];
    }
    if (threadIdx.x == 0) scratch->chunk_counter = 0ull;
}

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

}  // namespace

extern "C" int cls_run_noalloc(const double *params, int ncases, uint64_t first, uint64_t n, uint64_t seed,
                               int nbatch, int nbins_stride, double *d_flux, double *d_stats,
                               unsigned long long *d_counters, void *stream) {
    if (!params || !d_flux || !d_stats || !d_counters) return CLS_E_INVAL;
    if (ncases < 1 || ncases > CLS_NOALLOC_MAX_CASES) return CLS_E_INVAL;
    if (n == 0 || n > (1ull << 62) || first > (1ull << 62)) return CLS_E_INVAL;
    if (nbatch < 1 || nbatch > 1024) return CLS_E_INVAL;
    if (nbins_stride < 1 || nbins_stride > CLS_NOALLOC_MAX_STRIDE) return CLS_E_INVAL;
    for (int k = 0; k < ncases; ++k) {
        const double *p = params + 9 * (size_t)k;
        if (validate_case(p) != CLS_OK || p[8] > nbins_stride) return CLS_E_INVAL;
    }

    NoallocScratch *scratch = nullptr;
    int sm_count = 0;
    int rc = scratch_for_current_device(&scratch, &sm_count);
    if (rc) return rc;

    // this call's cases and work list (stack memory: no allocation), the same
    // case set-up as cls_batch_create: case k draws with Philox counter word 3 = k
    NoallocImage img;
    std::memset(&img, 0, sizeof(img));
    img.ncases = ncases;
    const uint64_t q = 1024ull * (uint64_t)nbatch;
    const uint64_t batch_len = 1024ull * ((n + q - 1) / q > 0 ? (n + q - 1) / q : 1);
    const int chunk = 256;
    uint64_t chunk_begin = 0;
    for (int k = 0; k < ncases; ++k) {
        img.cases[k] = make_case(params + 9 * (size_t)k, (uint32_t)k);
        RunCase &r = img.runs[k];
        r.first = first;
        r.n = n;
        r.batch_len = batch_len;
        r.chunk_begin = chunk_begin;
        r.case_index = k;
        chunk_begin += (n + chunk - 1) / chunk;
    }

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
    a.region_bytes = region_bytes(false, nbins_stride);
    a.flush_every = 0;
    a.warp_counts = 1;

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

    cudaStream_t s = (cudaStream_t)stream;
    noalloc_setup<<<1, 64, 0, s>>>(scratch, img);
    if (cudaGetLastError() != cudaSuccess) return CLS_E_CUDA;
    history_kernel<double, 0><<<sm_count * bps, block, smem, s>>>(a);
    return cudaGetLastError() == cudaSuccess ? CLS_OK : CLS_E_CUDA;
}
