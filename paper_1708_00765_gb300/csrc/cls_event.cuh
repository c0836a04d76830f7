// cls_event.cuh -- event-based CLS tracker over a structure-of-arrays particle bank.
//
// Each warp of the persistent grid owns a slice of a particle bank in global
// memory: `bank_slots` particles, held as structure-of-arrays of 16-byte
// vectors (one coalesced 128-bit load or store per field per particle) and
// double-buffered.  A pass of the warp:
//   1. refill: empty slots take new histories from the global work counter, 32
//      at a time, so sources are sampled by full warps;
//   2. flights: the live particles are loaded 32 at a time, advanced by up to
//      `events_per_pass` events of Algorithm A (same `step` as the history
//      tracker, warp-cooperative tallies), and the survivors are compacted into
//      the other buffer (ballot + prefix popcount), squeezing dead lanes out.
// No block-wide synchronisation: warps progress independently.  Tallies go to
// two warp-private regions keyed by (case, batch), as in the history tracker;
// per-region live counts tell when a region is free.  When a new key arrives
// and both regions are in use, a region with only a few particles left is
// flushed and given a new generation, after which those particles score into
// the FP64 global tallies; otherwise the warp keeps walking its bank and
// retries the chunk after the next pass.
#pragma once

#include "cls_device.cuh"

namespace cls {

// Bank fields (16 bytes each, SoA): FP32 uses 4, FP64 uses 8.
//   FP32: [0] (x, y, z, track0) [1] (wx, wy, wz, track1) [2] meta0 [3] meta1
//   FP64: [0] (x, y) [1] (z, track0) [2] (wx, wy) [3] (wz, track1) [4] (iwx, iwy)
//         [5] (iwz, -) [6] meta0 [7] meta1
//   meta0 = (h_lo, h_hi, j, c2); meta1 = (c3, m | region << 1 | generation << 3, events, run)
//   (region 0 or 1: a warp tally region of that generation; 2: global tallies)
template <typename P>
struct BankLayout;
template <>
struct BankLayout<float> {
    static constexpr int kFields = 4;
};
template <>
struct BankLayout<double> {
    static constexpr int kFields = 8;
};

template <typename P>
__device__ __forceinline__ void bank_store(unsigned char *buf, uint32_t S, uint32_t slot, const History<P> &s, int run,
                                           int reg);
template <typename P>
__device__ __forceinline__ void bank_load(const unsigned char *buf, uint32_t S, uint32_t slot, History<P> &s, int &run,
                                          int &reg);

template <>
__device__ __forceinline__ void bank_store<float>(unsigned char *buf, uint32_t S, uint32_t slot, const History<float> &s,
                                                  int run, int reg) {
    const size_t f = (size_t)S * 16;
    reinterpret_cast<float4 *>(buf)[slot] = make_float4(s.r[0], s.r[1], s.r[2], s.track0);
    reinterpret_cast<float4 *>(buf + f)[slot] = make_float4(s.w[0], s.w[1], s.w[2], s.track1);
    reinterpret_cast<uint4 *>(buf + 2 * f)[slot] = make_uint4(s.h_lo, s.h_hi, s.j, s.c2);
    reinterpret_cast<uint4 *>(buf + 3 * f)[slot] =
        make_uint4(s.c3, (uint32_t)s.m | ((uint32_t)reg << 1), s.events, (uint32_t)run);
}

template <>
__device__ __forceinline__ void bank_load<float>(const unsigned char *buf, uint32_t S, uint32_t slot, History<float> &s,
                                                 int &run, int &reg) {
    const size_t f = (size_t)S * 16;
    const float4 a = reinterpret_cast<const float4 *>(buf)[slot];
    const float4 b = reinterpret_cast<const float4 *>(buf + f)[slot];
    const uint4 c = reinterpret_cast<const uint4 *>(buf + 2 * f)[slot];
    const uint4 d = reinterpret_cast<const uint4 *>(buf + 3 * f)[slot];
    s.r[0] = a.x;
    s.r[1] = a.y;
    s.r[2] = a.z;
    s.track0 = a.w;
    set_direction<float>(s, b.x, b.y, b.z);
    s.track1 = b.w;
    s.h_lo = c.x;
    s.h_hi = c.y;
    s.j = c.z;
    s.c2 = c.w;
    s.c3 = d.x;
    s.m = (int)(d.y & 1u);
    reg = (int)(d.y >> 1);
    s.events = d.z;
    run = (int)d.w;
}

template <>
__device__ __forceinline__ void bank_store<double>(unsigned char *buf, uint32_t S, uint32_t slot,
                                                   const History<double> &s, int run, int reg) {
    const size_t f = (size_t)S * 16;
    reinterpret_cast<double2 *>(buf)[slot] = make_double2(s.r[0], s.r[1]);
    reinterpret_cast<double2 *>(buf + f)[slot] = make_double2(s.r[2], s.track0);
    reinterpret_cast<double2 *>(buf + 2 * f)[slot] = make_double2(s.w[0], s.w[1]);
    reinterpret_cast<double2 *>(buf + 3 * f)[slot] = make_double2(s.w[2], s.track1);
    reinterpret_cast<double2 *>(buf + 4 * f)[slot] = make_double2(s.iw[0], s.iw[1]);
    reinterpret_cast<double2 *>(buf + 5 * f)[slot] = make_double2(s.iw[2], 0.0);
    reinterpret_cast<uint4 *>(buf + 6 * f)[slot] = make_uint4(s.h_lo, s.h_hi, s.j, s.c2);
    reinterpret_cast<uint4 *>(buf + 7 * f)[slot] =
        make_uint4(s.c3, (uint32_t)s.m | ((uint32_t)reg << 1), s.events, (uint32_t)run);
}

template <>
__device__ __forceinline__ void bank_load<double>(const unsigned char *buf, uint32_t S, uint32_t slot,
                                                  History<double> &s, int &run, int &reg) {
    const size_t f = (size_t)S * 16;
    const double2 a = reinterpret_cast<const double2 *>(buf)[slot];
    const double2 b = reinterpret_cast<const double2 *>(buf + f)[slot];
    const double2 c = reinterpret_cast<const double2 *>(buf + 2 * f)[slot];
    const double2 d = reinterpret_cast<const double2 *>(buf + 3 * f)[slot];
    const double2 e = reinterpret_cast<const double2 *>(buf + 4 * f)[slot];
    const double2 g = reinterpret_cast<const double2 *>(buf + 5 * f)[slot];
    const uint4 m0 = reinterpret_cast<const uint4 *>(buf + 6 * f)[slot];
    const uint4 m1 = reinterpret_cast<const uint4 *>(buf + 7 * f)[slot];
    s.r[0] = a.x;
    s.r[1] = a.y;
    s.r[2] = b.x;
    s.track0 = b.y;
    s.w[0] = c.x;
    s.w[1] = c.y;
    s.w[2] = d.x;
    s.track1 = d.y;
    s.iw[0] = e.x;
    s.iw[1] = e.y;
    s.iw[2] = g.x;
    s.h_lo = m0.x;
    s.h_hi = m0.y;
    s.j = m0.z;
    s.c2 = m0.w;
    s.c3 = m1.x;
    s.m = (int)(m1.y & 1u);
    reg = (int)(m1.y >> 1);
    s.events = m1.z;
    run = (int)m1.w;
}


// Sum over the warp.
__device__ __forceinline__ unsigned long long warp_sum(unsigned long long v) {
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) v += __shfl_xor_sync(CLS_FULL_MASK, v, o);
    return v;
}

// History end in the event tracker: per-history FP64 statistics, outcome and
// event maximum (event and collision counts are added per pass).
template <typename P>
__device__ __forceinline__ void finish_event_history(unsigned char *region, int nbs, const History<P> &s, int outcome) {
    double *st = region_stats<P>(region, nbs);
    unsigned long long *ct = reinterpret_cast<unsigned long long *>(st + S_NUM);
    const double t0 = (double)s.track0;
    const double t1 = (double)s.track1;
    const double t = t0 + t1;
    atomicAdd(&st[S_T], t);
    atomicAdd(&st[S_T2], t * t);
    if (__double_as_longlong(t0) != 0) atomicAdd(&st[S_TRACK0], t0);
    if (__double_as_longlong(t1) != 0) atomicAdd(&st[S_TRACK1], t1);
    const int c = (outcome == EV_LEAK_X0) ? C_R : (outcome == EV_LEAK_XL) ? C_T : (outcome == EV_ABSORB) ? C_A : C_CAPPED;
    atomicAdd(&ct[c], 1ull);
    atomicMax(&ct[C_MAXEV], (unsigned long long)s.events);
}

// Launch bounds of the event tracker: blocks of up to kEventBlock = 256
// threads, 2 per SM (16 warps, up to 128 registers a thread).  Measured on the
// diffusive box (FP32, 2e7 histories): 5 blocks of 128 threads (20 warps, 96
// registers, about 100 bytes spilled) ran 15% slower, and 3 blocks of 256 at
// 80 registers (about 350 bytes spilled) 1.3x slower.
constexpr int kEventBlock = kEventBlockThreads;
constexpr int kEventMinBlocks = 2;

template <typename P, int G>
__global__ void __launch_bounds__(kEventBlock, kEventMinBlocks) event_kernel(const LaunchArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int rb = a.region_bytes;
    unsigned char *regions = smem + (size_t)warp * 2 * rb;
    for (int i = lane; i < 2 * rb / 8; i += 32) reinterpret_cast<unsigned long long *>(regions)[i] = 0ull;
    load_math_tables<P>(threadIdx.x, blockDim.x);
    if constexpr (sizeof(P) == 8) __syncthreads();
    __syncwarp();
    const uint32_t W = a.bank_slots;  // particles per warp and buffer (multiple of 32)
    const size_t buf_bytes = (size_t)W * 16 * BankLayout<P>::kFields;
    const size_t gwarp = (size_t)blockIdx.x * (blockDim.x >> 5) + warp;
    unsigned char *bank = reinterpret_cast<unsigned char *>(a.bank) + gwarp * 2 * buf_bytes;
    const RoundKeys &key = a.rk;
    const int nbs = a.t.nbins_stride;
    const unsigned lt_mask = (1u << lane) - 1u;

    // warp-uniform feeding state (as in the history tracker), live counts and
    // region generations: a banked particle names its region and that region's
    // generation; a region handed to a newer key gets a new generation, and
    // particles of an older one score into global memory
    int key_run[2] = {-1, -1};
    uint32_t key_batch[2] = {0, 0};
    int fed[2] = {0, 0};
    int live[2] = {0, 0};
    uint32_t gen[2] = {0, 0};
    uint64_t cursor = 0, end = 0;
    int feed_reg = 0, feed_run = 0;
    bool exhausted = false, have_pending = false;
    unsigned long long pending = 0;
    // a region still serving more particles than this is drained rather than evicted
    const int evict_max = (int)(W >> 4);
    uint32_t nlive = 0;
    int cur = 0;

    while (true) {
        unsigned char *buf = bank + cur * buf_bytes;
        unsigned char *nxt = bank + (cur ^ 1) * buf_bytes;
        // ------------------------------------------------------------ refill
        while (nlive < W && !exhausted) {
            if (cursor == end) {
                unsigned long long ch;
                if (have_pending) {
                    ch = pending;
                    have_pending = false;
                } else {
                    if (lane == 0) ch = atomicAdd(a.chunk_counter, 1ull);
                    ch = __shfl_sync(CLS_FULL_MASK, ch, 0);
                }
                if (ch >= a.total_chunks) {
                    exhausted = true;
                    break;
                }
                const int run = find_run(a, ch);
                const RunCase &rc = a.runs[run];
                const uint64_t local0 = (ch - rc.chunk_begin) * (uint64_t)a.chunk;
                const uint64_t cnt = min((uint64_t)a.chunk, rc.n - local0);
                const uint32_t batch = (uint32_t)(local0 / rc.batch_len);
                int r = -1;
                if (key_run[0] == run && key_batch[0] == batch) r = 0;
                else if (key_run[1] == run && key_batch[1] == batch) r = 1;
                if (r < 0) {
                    const int other = feed_reg ^ 1;
                    if (live[other] == 0) r = other;
                    else if (live[feed_reg] == 0) r = feed_reg;
                    else if (live[other] <= evict_max) r = other;  // a few stragglers: evict
                    if (r < 0) {  // both regions busy: keep walking the bank, retry next pass
                        pending = ch;
                        have_pending = true;
                        break;
                    }
                    if (key_run[r] >= 0) {
                        flush_region<P>(regions + r * rb, a, a.runs[key_run[r]].case_index, key_batch[r], lane);
                        gen[r] += 1;  // its banked particles now score into global memory
                        live[r] = 0;
                    }
                    key_run[r] = run;
                    key_batch[r] = batch;
                    fed[r] = 0;
                }
                feed_reg = r;
                feed_run = run;
                cursor = rc.first + local0;
                end = cursor + cnt;
            }
            const uint64_t avail = end - cursor;
            const uint32_t room = W - nlive;
            const uint32_t take = (uint32_t)min((uint64_t)min(room, 32u), avail);
            if ((uint32_t)lane < take) {
                const CaseParams &cp = a.cases[a.runs[feed_run].case_index];
                History<P> s;
                source<P, G>(s, cp, key, cursor + lane);
                bank_store<P>(buf, W, nlive + lane, s, feed_run, feed_reg | (int)(gen[feed_reg] << 2));
            }
            cursor += take;
            nlive += take;
            live[feed_reg] += (int)take;
            fed[feed_reg] += (int)take;
        }
        if (nlive == 0) break;
        __syncwarp();

        // ----------------------------------------------------------- flights
        // Once no history is left to start and the bank fits one row of lanes,
        // the warp walks its last particles to their ends in registers, as the
        // history tracker does, instead of storing and reloading them through the
        // bank every events_per_pass events: the longest histories of a launch
        // (10^4 events and more) would otherwise pay a bank round trip every few
        // events while the rest of the GPU idles.
        const bool tail = exhausted && nlive <= 32u;
        const uint32_t epp = tail ? 0xFFFFFFFFu : a.events_per_pass;
        // collisions, interface crossings, reflections, events of this pass, per region
        uint32_t c0 = 0, i0 = 0, f0 = 0, e0 = 0, c1 = 0, i1 = 0, f1 = 0, e1 = 0;
        uint32_t out = 0;
        for (uint32_t r0 = 0; r0 < nlive; r0 += 32) {
            const uint32_t slot = r0 + lane;
            History<P> s;
            Flight<P> f;
            int run = 0, packed = 0;
            bool alive = slot < nlive;
            if (alive) bank_load<P>(buf, W, slot, s, run, packed);
            const int ci = alive ? a.runs[run].case_index : 0;
            s.cid = a.cases[ci].case_id;  // Philox counter word 3 (not stored in the bank)
            // the particle's region, or 2 if that region has since changed key
            int reg = packed & 3;
            if (reg < 2 && (uint32_t)(packed >> 2) != gen[reg]) reg = 2;
            uint64_t goff = 0;
            if (alive && reg == 2) {
                const RunCase &rc = a.runs[run];
                const uint64_t h = ((uint64_t)s.h_hi << 32) | s.h_lo;
                const uint64_t batch = (h - rc.first) / rc.batch_len;
                goff = ((uint64_t)ci * (uint64_t)a.t.nbatch + batch) * (uint64_t)nbs;
            }
            const uint32_t ev0 = alive ? s.events : 0u;
            s.n_coll = s.n_int = s.n_refl = 0;
            bool died = false;
            for (uint32_t e = 0; e < epp; ++e) {
                if (!__any_sync(CLS_FULL_MASK, alive)) break;
                int o = -1;
                f.k0 = 0;
                f.k1 = -1;
                if (alive) o = step<P, false, G>(s, a.cases[ci], key, a.max_events, f, nullptr);
                warp_deposit<P>(regions, rb, nbs, reg, a.t.flux, goff, f, lane);
                if (o >= 0) {
                    record_outcome(a, ci, s.h_lo, s.h_hi, o);
                    if (reg < 2) finish_event_history<P>(regions + reg * rb, nbs, s, o);
                    else finish_history_global<P>(a, ci, s, o, false);
                    alive = false;
                    died = true;
                }
            }
            if (slot < nlive) {
                if (reg == 0) {
                    c0 += s.n_coll;
                    i0 += s.n_int;
                    f0 += s.n_refl;
                    e0 += s.events - ev0;
                } else if (reg == 1) {
                    c1 += s.n_coll;
                    i1 += s.n_int;
                    f1 += s.n_refl;
                    e1 += s.events - ev0;
                } else {
                    unsigned long long *gc = a.t.counters + (size_t)ci * C_NUM;
                    if (s.n_coll) atomicAdd(&gc[C_COLL], (unsigned long long)s.n_coll);
                    if (s.n_int) atomicAdd(&gc[C_INT], (unsigned long long)s.n_int);
                    if (s.n_refl) atomicAdd(&gc[C_REFL], (unsigned long long)s.n_refl);
                    atomicAdd(&gc[C_EVENTS], (unsigned long long)(s.events - ev0));
                }
            }
            live[0] -= __popc(__ballot_sync(CLS_FULL_MASK, died && reg == 0));
            live[1] -= __popc(__ballot_sync(CLS_FULL_MASK, died && reg == 1));
            const int store_tag = (reg < 2) ? (reg | (int)(gen[reg] << 2)) : 2;
            const unsigned b = __ballot_sync(CLS_FULL_MASK, alive);
            if (alive) bank_store<P>(nxt, W, out + __popc(b & lt_mask), s, run, store_tag);
            out += __popc(b);
        }
        // warp-aggregated event counters: one shared-memory atomic per counter
        for (int r = 0; r < 2; ++r) {
            unsigned long long *ct = reinterpret_cast<unsigned long long *>(region_stats<P>(regions + r * rb, nbs) + S_NUM);
            const unsigned long long v0 = warp_sum(r ? c1 : c0), v1 = warp_sum(r ? i1 : i0);
            const unsigned long long v2 = warp_sum(r ? f1 : f0), v3 = warp_sum(r ? e1 : e0);
            if (lane == 0) {
                if (v0) atomicAdd(&ct[C_COLL], v0);
                if (v1) atomicAdd(&ct[C_INT], v1);
                if (v2) atomicAdd(&ct[C_REFL], v2);
                if (v3) atomicAdd(&ct[C_EVENTS], v3);
            }
        }
        __syncwarp();
        nlive = out;
        cur ^= 1;
        // FP32 regions: bound the partial sums
        if (a.flush_every) {
            for (int r = 0; r < 2; ++r) {
                if (fed[r] >= a.flush_every && key_run[r] >= 0) {
                    flush_region<P>(regions + r * rb, a, a.runs[key_run[r]].case_index, key_batch[r], lane);
                    fed[r] = 0;
                }
            }
        }
    }
    __syncwarp();
    for (int r = 0; r < 2; ++r)
        if (key_run[r] >= 0) flush_region<P>(regions + r * rb, a, a.runs[key_run[r]].case_index, key_batch[r], lane);
}

template <typename P, int G>
cudaError_t launch_event_g(const LaunchArgs &a, int grid, int block, size_t smem, cudaStream_t st) {
    static std::atomic<unsigned long long> optin{0};
    const cudaError_t e = ensure_smem_optin(event_kernel<P, G>, optin);
    if (e != cudaSuccess) return e;
    event_kernel<P, G><<<grid, block, smem, st>>>(a);
    return cudaGetLastError();
}

template <typename P>
cudaError_t launch_event_impl(const LaunchArgs &a, int grid, int block, size_t smem, cudaStream_t st, int geom) {
    switch (geom) {
    case 1: return launch_event_g<P, 1>(a, grid, block, smem, st);
    case 2: return launch_event_g<P, 2>(a, grid, block, smem, st);
    case 3: return launch_event_g<P, 3>(a, grid, block, smem, st);
    case 11: return launch_event_g<P, 11>(a, grid, block, smem, st);
    case 13: return launch_event_g<P, 13>(a, grid, block, smem, st);
    default: return launch_event_g<P, 0>(a, grid, block, smem, st);
    }
}

template <typename P, int G>
cudaError_t occupancy_event_g(int block, size_t smem, int *blocks_per_sm) {
    return occupancy_with_smem(blocks_per_sm, event_kernel<P, G>, block, smem);
}

template <typename P>
cudaError_t occupancy_event_impl(int block, size_t smem, int *blocks_per_sm, int geom) {
    switch (geom) {
    case 1: return occupancy_event_g<P, 1>(block, smem, blocks_per_sm);
    case 2: return occupancy_event_g<P, 2>(block, smem, blocks_per_sm);
    case 3: return occupancy_event_g<P, 3>(block, smem, blocks_per_sm);
    case 11: return occupancy_event_g<P, 11>(block, smem, blocks_per_sm);
    case 13: return occupancy_event_g<P, 13>(block, smem, blocks_per_sm);
    default: return occupancy_event_g<P, 0>(block, smem, blocks_per_sm);
    }
}

}  // namespace cls
