// cls_event.cuh -- event-based CLS tracker over a structure-of-arrays particle bank.
//
// Each persistent block owns a slice of a particle bank in global memory, held
// as structure-of-arrays of 16-byte vectors (one coalesced 128-bit load or
// store per field per particle) and double-buffered.  A pass of the block:
//   1. refill: empty slots take new histories from the global work counter;
//      their sources are sampled by full warps;
//   2. flights: every live particle is loaded, advanced by up to
//      `events_per_pass` events of Algorithm A (same `step` as the history
//      tracker, warp-cooperative tallies), and the survivors are compacted into
//      the other buffer (warp ballot + block prefix sum), so dead lanes are
//      squeezed out before the next pass.
// Tallies go to two block-shared regions keyed by (case, batch); a region is
// flushed when it must change key (no live particle refers to it any more),
// periodically in FP32 mode, and when the block retires.
#pragma once

#include "cls_device.cuh"

namespace cls {

// Bank fields (16 bytes each, SoA): FP32 uses 4, FP64 uses 8.
//   FP32: [0] (x, y, z, track0) [1] (wx, wy, wz, track1) [2] meta0 [3] meta1
//   FP64: [0] (x, y) [1] (z, track0) [2] (wx, wy) [3] (wz, track1) [4] (iwx, iwy)
//         [5] (iwz, -) [6] meta0 [7] meta1
//   meta0 = (h_lo, h_hi, j, c2); meta1 = (c3, m | region << 1, events, run)
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
    reg = (int)((d.y >> 1) & 1u);
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
    reg = (int)((m1.y >> 1) & 1u);
    s.events = m1.z;
    run = (int)m1.w;
}

// Block-shared bookkeeping of the event tracker.
struct EventBlock {
    unsigned long long cursor, end, pending;
    int key_run[2];
    uint32_t key_batch[2];
    int live[2];  // live particles whose tallies go to region r
    int fed[2];   // histories fed into region r since its last flush
    int feed_reg, feed_run;
    int exhausted, have_pending;
    int nfill;    // slots filled in the current buffer
    // action broadcast by thread 0 during refill (for a flush: act_run is the
    // case index and act_first the batch of the region's old key)
    int act, act_reg, act_take, act_start, act_run;
    unsigned long long act_first;
    int warp_tot[32];
};

enum { ACT_DONE = 0, ACT_FILL = 1, ACT_FLUSH = 2 };

// Block-wide flush of a region into the global tallies of (case, batch).
template <typename P>
__device__ __forceinline__ void block_flush(unsigned char *region, const LaunchArgs &a, int case_index, uint32_t batch) {
    using B = typename Real<P>::Bin;
    const int nbs = a.t.nbins_stride;
    const int nb = a.cases[case_index].nbins;
    B *bins = reinterpret_cast<B *>(region);
    double *g = a.t.flux + ((size_t)case_index * a.t.nbatch + batch) * (size_t)nbs;
    for (int k = threadIdx.x; k < nb; k += blockDim.x) {
        const B v = bins[k];
        if (v != B(0)) {
            atomicAdd(&g[k], (double)v);
            bins[k] = B(0);
        }
    }
    double *st = region_stats<P>(region, nbs);
    const int t = threadIdx.x;
    if (t < S_NUM) {
        const double v = st[t];
        if (v != 0.0) {
            atomicAdd(&a.t.stats[(size_t)case_index * S_NUM + t], v);
            st[t] = 0.0;
        }
    } else if (t < S_NUM + C_NUM) {
        const int c = t - S_NUM;
        unsigned long long *ct = reinterpret_cast<unsigned long long *>(st + S_NUM);
        const unsigned long long v = ct[c];
        if (v != 0ull) {
            unsigned long long *gc = &a.t.counters[(size_t)case_index * C_NUM + c];
            if (c == C_MAXEV) atomicMax(gc, v);
            else atomicAdd(gc, v);
            ct[c] = 0ull;
        }
    }
}

// History end: per-history FP64 statistics, outcome and event maximum.
template <typename P>
__device__ __forceinline__ void finish_event_history(unsigned char *region, int nbs, const History<P> &s, int outcome) {
    double *st = region_stats<P>(region, nbs);
    unsigned long long *ct = reinterpret_cast<unsigned long long *>(st + S_NUM);
    const double t0 = (double)s.track0;
    const double t1 = (double)s.track1;
    const double t = t0 + t1;
    atomicAdd(&st[S_T], t);
    atomicAdd(&st[S_T2], t * t);
    if (t0 != 0.0) atomicAdd(&st[S_TRACK0], t0);
    if (t1 != 0.0) atomicAdd(&st[S_TRACK1], t1);
    const int c = (outcome == EV_LEAK_X0) ? C_R : (outcome == EV_LEAK_XL) ? C_T : (outcome == EV_ABSORB) ? C_A : C_CAPPED;
    atomicAdd(&ct[c], 1ull);
    atomicMax(&ct[C_MAXEV], (unsigned long long)s.events);
}

// Exclusive block prefix sum of a 0/1 flag (warp ballots, then warp totals).
__device__ __forceinline__ int block_flag_scan(bool flag, EventBlock *eb, int *total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const unsigned b = __ballot_sync(CLS_FULL_MASK, flag);
    const int in_warp = __popc(b & ((1u << lane) - 1u));
    if (lane == 0) eb->warp_tot[warp] = __popc(b);
    __syncthreads();
    int before = 0, tot = 0;
    for (int w = 0; w < nw; ++w) {
        const int v = eb->warp_tot[w];
        before += (w < warp) ? v : 0;
        tot += v;
    }
    *total = tot;
    return before + in_warp;
}

template <typename P, int G>
__global__ void __launch_bounds__(256) event_kernel(const LaunchArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int rb = a.region_bytes;
    unsigned char *regions = smem;
    EventBlock *eb = reinterpret_cast<EventBlock *>(smem + 2 * rb);
    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const uint32_t S = a.bank_slots;  // slots per block and buffer
    const size_t buf_bytes = (size_t)S * 16 * BankLayout<P>::kFields;
    unsigned char *bank = reinterpret_cast<unsigned char *>(a.bank) + (size_t)blockIdx.x * 2 * buf_bytes;
    const RoundKeys &key = a.rk;
    const int nbs = a.t.nbins_stride;

    for (int i = tid; i < 2 * rb / 8; i += blockDim.x) reinterpret_cast<unsigned long long *>(regions)[i] = 0ull;
    if (tid == 0) {
        eb->cursor = eb->end = 0;
        eb->key_run[0] = eb->key_run[1] = -1;
        eb->key_batch[0] = eb->key_batch[1] = 0;
        eb->live[0] = eb->live[1] = 0;
        eb->fed[0] = eb->fed[1] = 0;
        eb->feed_reg = 0;
        eb->feed_run = 0;
        eb->exhausted = 0;
        eb->have_pending = 0;
        eb->nfill = 0;
    }
    __syncthreads();

    int cur = 0;
    while (true) {
        unsigned char *buf = bank + cur * buf_bytes;
        unsigned char *nxt = bank + (cur ^ 1) * buf_bytes;
        // ---------------------------------------------------------- refill
        // Thread 0 picks one action per round; the whole block carries it out.
        while (true) {
            if (tid == 0) {
                int act = ACT_DONE;
                while (true) {
                    const int free_slots = (int)S - eb->nfill;
                    if (free_slots <= 0) break;
                    if (eb->cursor < eb->end) {
                        const unsigned long long avail = eb->end - eb->cursor;
                        const int take = (avail < (unsigned long long)free_slots) ? (int)avail : free_slots;
                        act = ACT_FILL;
                        eb->act_take = take;
                        eb->act_start = eb->nfill;
                        eb->act_first = eb->cursor;
                        eb->act_reg = eb->feed_reg;
                        eb->act_run = eb->feed_run;
                        eb->cursor += take;
                        eb->nfill += take;
                        eb->live[eb->feed_reg] += take;
                        eb->fed[eb->feed_reg] += take;
                        break;
                    }
                    if (eb->exhausted) break;
                    unsigned long long ch;
                    if (eb->have_pending) {
                        ch = eb->pending;
                        eb->have_pending = 0;
                    } else {
                        ch = atomicAdd(a.chunk_counter, 1ull);
                    }
                    if (ch >= a.total_chunks) {
                        eb->exhausted = 1;
                        break;
                    }
                    const int run = find_run(a, ch);
                    const RunCase &rc = a.runs[run];
                    const uint64_t local0 = (ch - rc.chunk_begin) * (uint64_t)a.chunk;
                    const uint64_t cnt = min((uint64_t)a.chunk, rc.n - local0);
                    const uint32_t batch = (uint32_t)(local0 / rc.batch_len);
                    int r = -1;
                    if (eb->key_run[0] == run && eb->key_batch[0] == batch) r = 0;
                    else if (eb->key_run[1] == run && eb->key_batch[1] == batch) r = 1;
                    if (r < 0) {
                        const int other = eb->feed_reg ^ 1;
                        int rr = -1;
                        if (eb->live[other] == 0) rr = other;
                        else if (eb->live[eb->feed_reg] == 0) rr = eb->feed_reg;
                        if (rr < 0) {  // both regions still referenced: drain first
                            eb->pending = ch;
                            eb->have_pending = 1;
                            break;
                        }
                        if (eb->key_run[rr] >= 0) {  // flush the old key, then retry this chunk
                            act = ACT_FLUSH;
                            eb->act_reg = rr;
                            eb->act_run = a.runs[eb->key_run[rr]].case_index;
                            eb->act_first = eb->key_batch[rr];
                            eb->key_run[rr] = -1;
                            eb->pending = ch;
                            eb->have_pending = 1;
                            break;
                        }
                        eb->key_run[rr] = run;
                        eb->key_batch[rr] = batch;
                        eb->fed[rr] = 0;
                        r = rr;
                    }
                    eb->feed_reg = r;
                    eb->feed_run = run;
                    eb->cursor = rc.first + local0;
                    eb->end = eb->cursor + cnt;
                }
                eb->act = act;
            }
            __syncthreads();
            const int act = eb->act;
            if (act == ACT_DONE) break;
            if (act == ACT_FLUSH) {
                block_flush<P>(regions + eb->act_reg * rb, a, eb->act_run, (uint32_t)eb->act_first);
            } else {
                const int take = eb->act_take, start = eb->act_start, reg = eb->act_reg, run = eb->act_run;
                const unsigned long long first = eb->act_first;
                const CaseParams &cp = a.cases[a.runs[run].case_index];
                for (int i = tid; i < take; i += blockDim.x) {
                    History<P> s;
                    source<P, G>(s, cp, key, first + (unsigned long long)i);
                    bank_store<P>(buf, S, (uint32_t)(start + i), s, run, reg);
                }
            }
            __syncthreads();
        }
        const int nlive = eb->nfill;
        if (nlive == 0) break;

        // --------------------------------------------------------- flights
        int out_base = 0;
        for (int r0 = 0; r0 < nlive; r0 += blockDim.x) {
            const int slot = r0 + tid;
            History<P> s;
            Flight<P> f;
            int run = 0, reg = 0;
            bool alive = slot < nlive;
            if (alive) bank_load<P>(buf, S, (uint32_t)slot, s, run, reg);
            const uint32_t ev0 = alive ? s.events : 0u;
            s.n_coll = s.n_int = s.n_refl = 0;
            const int ci = alive ? a.runs[run].case_index : 0;
            s.cid = a.cases[ci].case_id;  // Philox counter word 3 (not stored in the bank)
            for (uint32_t e = 0; e < a.events_per_pass; ++e) {
                if (!__any_sync(CLS_FULL_MASK, alive)) break;
                int out = -1;
                f.k0 = 0;
                f.k1 = -1;
                if (alive) out = step<P, false, G>(s, a.cases[ci], key, a.max_events, f, nullptr);
                warp_deposit<P>(regions, rb, reg, f, lane);
                if (out >= 0) {
                    finish_event_history<P>(regions + reg * rb, nbs, s, out);
                    atomicSub(&eb->live[reg], 1);
                    alive = false;
                }
            }
            if (slot < nlive) {
                double *st = region_stats<P>(regions + reg * rb, nbs);
                unsigned long long *ct = reinterpret_cast<unsigned long long *>(st + S_NUM);
                if (s.n_coll) atomicAdd(&ct[C_COLL], (unsigned long long)s.n_coll);
                if (s.n_int) atomicAdd(&ct[C_INT], (unsigned long long)s.n_int);
                if (s.n_refl) atomicAdd(&ct[C_REFL], (unsigned long long)s.n_refl);
                atomicAdd(&ct[C_EVENTS], (unsigned long long)(s.events - ev0));
            }
            int total = 0;
            const int idx = block_flag_scan(alive, eb, &total);
            if (alive) bank_store<P>(nxt, S, (uint32_t)(out_base + idx), s, run, reg);
            out_base += total;
            __syncthreads();
        }
        if (tid == 0) eb->nfill = out_base;
        cur ^= 1;
        // FP32 regions: bound the partial sums
        if (a.flush_every) {
            for (int r = 0; r < 2; ++r) {
                if (eb->fed[r] >= a.flush_every && eb->key_run[r] >= 0) {
                    block_flush<P>(regions + r * rb, a, a.runs[eb->key_run[r]].case_index, eb->key_batch[r]);
                    __syncthreads();
                    if (tid == 0) eb->fed[r] = 0;
                }
            }
        }
        __syncthreads();
    }
    for (int r = 0; r < 2; ++r)
        if (eb->key_run[r] >= 0) block_flush<P>(regions + r * rb, a, a.runs[eb->key_run[r]].case_index, eb->key_batch[r]);
}

template <typename P, int G>
cudaError_t launch_event_g(const LaunchArgs &a, int grid, int block, size_t smem, cudaStream_t st) {
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(event_kernel<P, G>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
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

template <typename P>
cudaError_t occupancy_event_impl(int block, size_t smem, int *blocks_per_sm, int geom) {
    switch (geom) {
    case 1: return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, event_kernel<P, 1>, block, smem);
    case 2: return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, event_kernel<P, 2>, block, smem);
    case 3: return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, event_kernel<P, 3>, block, smem);
    case 11: return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, event_kernel<P, 11>, block, smem);
    case 13: return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, event_kernel<P, 13>, block, smem);
    default: return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, event_kernel<P, 0>, block, smem);
    }
}

}  // namespace cls
