// cls_internal.h -- structures shared by the host API and the kernels of libcls.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace cls {

// One CLS problem as the kernels read it (paper Sec. 2: Sigma_i, Lambda_i, c_i,
// p_i = Lambda_i / (Lambda_0 + Lambda_1); box side L; uniform x mesh).
struct CaseParams {
    double sigma[2];
    double inv_sigma[2];  // 1 / Sigma_i (0 when Sigma_i = 0, unused then)
    double lambda[2];
    double c[2];
    double L;
    double p0;      // Lambda_0 / (Lambda_0 + Lambda_1)
    double dx;      // L / nbins
    double inv_dx;  // nbins / L
    float sigma_f[2];
    float inv_sigma_f[2];  // 1 / Sigma_i (0 when Sigma_i = 0, unused then)
    float lambda_f[2];
    float c_f[2];
    float L_f, p0_f, dx_f, inv_dx_f;
    // integer thresholds: a draw u = k 2^-53 (FP64) or k 2^-24 (FP32) is below
    // c_i or p_0 exactly when k is below ceil(c_i 2^53) (resp. 2^24)
    unsigned long long thr_c53[2];
    unsigned long long thr_p053;
    uint32_t thr_c24[2];
    uint32_t thr_p024;
    int32_t d;      // 1 rod, 3 box
    int32_t nbins;
    uint32_t case_id;  // Philox counter word 3
    int32_t source;    // 0 incident flux on x = 0 (suite I), 1 uniform isotropic volume source (suite II)
    double cost;    // host estimate of events per history (ordering only)
};

// Per-run work of one case: histories [first, first + n), statistics batch
// length, and the case's first global chunk index.
struct RunCase {
    uint64_t first;
    uint64_t n;
    uint64_t batch_len;
    uint64_t chunk_begin;
    int32_t case_index;  // index into the CaseParams array / tally blocks
    int32_t pad;
};

// The caller's per-history outcome record (cls_record_outcomes), kept in
// device memory right after the run's RunCase array, so that a captured batch
// graph reads the current binding at every replay.  History h of case k
// writes codes[k * stride + (h - first)]: CLS_OUTCOME_* (0 reflected, 1
// transmitted, 2 absorbed, 3 capped).  codes == nullptr: nothing is recorded.
struct OutcomeRecord {
    uint8_t *codes;
    uint64_t first;   // first history id of the run (the same for every case)
    uint64_t stride;  // the run's histories per case
};

// Order of the counters and statistics in every tally block and smem region.
enum Counter { C_R = 0, C_T, C_A, C_COLL, C_INT, C_REFL, C_EVENTS, C_CAPPED, C_MAXEV, C_NUM };
enum Stat { S_T = 0, S_T2, S_TRACK0, S_TRACK1, S_NUM };

// Event codes of traces (shared with the public trace format).
enum Event { EV_LEAK_X0 = 0, EV_LEAK_XL = 1, EV_REFLECT = 2, EV_SCATTER = 3, EV_ABSORB = 4,
             EV_INTERFACE = 5, EV_CAPPED = 6 };

// Device tallies of all cases.  Case k owns
//   flux     + k * nbatch * nbins_stride   [nbatch][nbins_stride] doubles
//   stats    + k * S_NUM                   doubles
//   counters + k * C_NUM                   u64
struct Tallies {
    double *flux;
    double *stats;
    unsigned long long *counters;
    int nbatch;
    int nbins_stride;
};

// The ten round keys of Philox4x32-10 for one seed: (k0, k1) of round r are
// (seed_lo + r * 0x9E3779B9, seed_hi + r * 0xBB67AE85) mod 2^32.  Every thread
// of a launch shares them, so they travel in the kernel arguments (constant
// bank) instead of being recomputed in every Philox block.
struct RoundKeys {
    uint32_t k[20];
};

__host__ __device__ inline RoundKeys make_round_keys(uint64_t seed) {
    RoundKeys rk;
    uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
    for (int r = 0; r < 10; ++r) {
        rk.k[2 * r] = k0;
        rk.k[2 * r + 1] = k1;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return rk;
}

struct LaunchArgs {
    RoundKeys rk;  // from the seed
    const CaseParams *cases;
    const RunCase *runs;  // in chunk order (largest estimated cost first)
    int nruns;
    uint32_t chunk;       // histories per chunk (divides 1024)
    uint64_t total_chunks;
    unsigned long long *chunk_counter;  // zeroed before each launch
    Tallies t;
    uint64_t seed;
    uint32_t max_events;
    int region_bytes;     // bytes per warp tally region (see region_bytes())
    int flush_every;      // flush a region after this many histories were fed into it (0: never)
    int warp_counts;      // history tracker: its short-history instance (warp-summed counters, sparse deposits)
    const OutcomeRecord *outcomes;  // per-history outcome record, or nullptr (never recorded)
    // event schedule only
    void *bank;            // grid warps x 2 buffers x bank_slots particles (SoA)
    uint32_t bank_slots;   // particles per warp and buffer, a multiple of 32
    uint32_t events_per_pass;
};

// Trace kernel arguments (one history).
struct TraceArgs {
    const CaseParams *cases;
    int case_index;
    uint64_t seed;
    uint64_t history;
    uint32_t max_events;
    double *rows;  // cap x 10
    int cap;
    int *n_rows;
};

// A warp tally region: the bins, then S_NUM FP64 statistics and C_NUM u64
// counters, then each lane's own copy of the per-history statistics (S_NUM x
// 32 doubles, statistic-major), which a lane updates without atomics when its
// history ends and the flush sums over the warp; padded to 16 bytes.
//   FP64 walk: nbins_stride FP64 bins, each flight scored bin by bin.
//   FP32 walk: nbins_stride + 1 entries of a fixed-point difference array
//     (u64, 32 fraction bits): a flight adds its end-bin partials and its
//     interior-bin length with at most four integer atomics, and the flush
//     takes the exact prefix sum, so the FP32 walk's deposits are summed
//     without rounding (FP64 is used from the flush on).
__host__ __device__ inline int region_bins_bytes(bool fixed, int nbins_stride) {
    return 8 * (nbins_stride + (fixed ? 1 : 0));
}
__host__ __device__ inline int region_lane_stats_offset(bool fixed, int nbins_stride) {
    return region_bins_bytes(fixed, nbins_stride) + 8 * (S_NUM + C_NUM);
}
__host__ __device__ inline int region_bytes(bool fixed, int nbins_stride) {
    return (region_lane_stats_offset(fixed, nbins_stride) + 8 * 32 * S_NUM + 15) & ~15;
}

// Largest block of the event tracker (its launch bounds: 2 such blocks per SM).
constexpr int kEventBlockThreads = 256;

// Largest block of the FP64 history tracker (its launch bounds allow 5 such
// blocks per SM; the host caps the block option at this size for it).
constexpr int kHistoryBlockFp64 = 128;

// Threads per block the FP32 history tracker is built for (its launch bound,
// and the host's cap on CLS_OPT_BLOCK): 224 for the 3D box, whose 72
// registers then hold its state without spills (3.6% faster than 256 threads
// at 64 registers), else 256.
constexpr int history_threads_fp32(int geom) { return geom == 3 ? 224 : 256; }

// ceil(v 2^bits) for v in [0, 1], exact (scaling by a power of two is exact).
inline unsigned long long unit_threshold(double v, int bits) {
    const double scaled = v * (double)(1ull << bits);
    const double c = (scaled == (double)(unsigned long long)scaled) ? scaled : (double)(unsigned long long)scaled + 1.0;
    return (unsigned long long)c;
}

// Launchers, one set per precision translation unit.
// `geom`: the geometry code every case of the launch shares, or 0 (mixed)
cudaError_t launch_history_fp64(const LaunchArgs &a, int grid, int block, size_t smem, cudaStream_t s, int geom);
cudaError_t launch_history_fp32(const LaunchArgs &a, int grid, int block, size_t smem, cudaStream_t s, int geom);
cudaError_t launch_event_fp64(const LaunchArgs &a, int grid, int block, size_t smem, cudaStream_t s, int geom);
cudaError_t launch_event_fp32(const LaunchArgs &a, int grid, int block, size_t smem, cudaStream_t s, int geom);
cudaError_t launch_trace_fp64(const TraceArgs &a, cudaStream_t s);
cudaError_t launch_trace_fp32(const TraceArgs &a, cudaStream_t s);
cudaError_t occupancy_history_fp64(int block, size_t smem, int *blocks_per_sm, int geom);
cudaError_t occupancy_history_fp32(int block, size_t smem, int *blocks_per_sm, int geom);
cudaError_t occupancy_event_fp64(int block, size_t smem, int *blocks_per_sm, int geom);
cudaError_t occupancy_event_fp32(int block, size_t smem, int *blocks_per_sm, int geom);
int event_bank_fields(int precision); // 16-byte SoA fields per particle (0 = FP64)

}  // namespace cls
