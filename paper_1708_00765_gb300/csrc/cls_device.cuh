// cls_device.cuh -- device side of the CLS random walk (paper Sec. 4, "Algorithm A").
//
// One history: sample the source (paper Sec. 4.3 for the box: y, z uniform on
// the x = 0 face, cosine-law direction; rod: x = 0 moving +x), sample the
// material label from p_0, then repeat: draw the collision distance
// l_c = -ln(1-u)/Sigma_m and the interface distance l_i = -Lambda_m ln(1-u),
// compute the boundary distance l_b, and take the smallest.  Boundary: leak
// through an x face (R or T) or reflect specularly on a lateral face.
// Collision: scatter isotropically with probability c_m, else absorb.
// Interface: switch the label.  Every flight is scored by the track-length
// estimator on the uniform x mesh.
//
// Ties: boundary wins over collision and interface, collision over interface;
// an x face wins over a lateral face; equal lateral distances reflect both.
// The collision draw is consumed even when Sigma_m = 0.
#pragma once

#include <atomic>
#include <type_traits>
#include <cstdint>
#include <cuda_runtime.h>

#include "cls_internal.h"
#include "cls_intmath.h"

namespace cls {

#define CLS_FULL_MASK 0xffffffffu

// Blocks per SM of a kernel at a given dynamic shared memory.  The opt-in for
// more than 48 KB is set first: without it the occupancy query reports zero
// blocks for such sizes.
template <typename K>
__host__ cudaError_t occupancy_with_smem(int *blocks_per_sm, K kernel, int block, size_t smem) {
    const cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, kernel, block, smem);
}

// The opt-in to 200 KB of dynamic shared memory, set once per device and
// kernel (`done` holds one bit per device index below 64, set after a
// successful call; two threads racing on it only repeat the call).
template <typename K>
__host__ cudaError_t ensure_smem_optin(K kernel, std::atomic<unsigned long long> &done) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const unsigned long long bit = (dev >= 0 && dev < 64) ? (1ull << dev) : 0ull;
    if (bit && (done.load(std::memory_order_acquire) & bit)) return cudaSuccess;
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    if (e == cudaSuccess && bit) done.fetch_or(bit, std::memory_order_release);
    return e;
}

// ------------------------------------------------- FP64 logarithm, sine/cosine
// The FP64 walk takes its logarithms and its sine/cosine pairs straight from
// the 53-bit integer k of a draw (u = k 2^-53), in integer arithmetic
// (cls_intmath.h), through tables that every FP64 kernel copies into shared
// memory when it starts (load_math_tables): the FP64 pipe, the walk's
// bottleneck, sees neither.
__shared__ uint16_t cls_logn_tab[CLS_LOG_TABLE_N];
__shared__ __align__(16) uint64_t cls_logt_tab[CLS_LOG_TABLE_N][2];
__shared__ __align__(16) int64_t cls_sincos_tab[CLS_SINCOS_TABLE_N][2];

template <typename P>
__device__ __forceinline__ void load_math_tables(int tid, int nthreads) {
    if constexpr (sizeof(P) == 8) {
        for (int i = tid; i < CLS_LOG_TABLE_N; i += nthreads) {
            cls_logn_tab[i] = cls_log_n_init[i];
            cls_logt_tab[i][0] = cls_log_t_init[i][0];
            cls_logt_tab[i][1] = cls_log_t_init[i][1];
        }
        for (int i = tid; i < CLS_SINCOS_TABLE_N; i += nthreads) {
            cls_sincos_tab[i][0] = cls_sincos_q62_init[i][0];
            cls_sincos_tab[i][1] = cls_sincos_q62_init[i][1];
        }
    }
}

// -ln(1 - u) for u = k 2^-53, from the shared-memory tables
__device__ __forceinline__ double exp_variate_shared(unsigned long long k) {
    return exp_variate(k, IntLogTables{cls_logn_tab, cls_logt_tab});
}

// (sin, cos) of 2 pi u for u = k 2^-53, from the shared-memory table
__device__ __forceinline__ void sincos_2pi_shared(unsigned long long k, double *sn, double *cs) {
    sincos_2pi_int(k, cls_sincos_tab, sn, cs);
}

// the integer E as a double, exactly (|E| < 2^51), by the 1.5 2^52 shift
__device__ __forceinline__ double small_int_to_double(long long e) {
    return __longlong_as_double(0x4338000000000000ll + e) - 0x1.8p52;
}

// ------------------------------------------------------------------ Philox
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of two
// 32x32->64 multiplies mixed with the other two words and the round key; the
// key advances by the Weyl increments between rounds.  The round keys come
// precomputed (RoundKeys, cls_internal.h): all threads of a launch share them.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, const RoundKeys &rk) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo0 = 0xD2511F53u * c.x;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z);
        const uint32_t lo1 = 0xCD9E8D57u * c.z;
        c = make_uint4(hi1 ^ c.y ^ rk.k[2 * r], lo1, hi0 ^ c.w ^ rk.k[2 * r + 1], lo0);
    }
    return c;
}

// ------------------------------------------------------- precision traits
template <typename P>
struct Real;

// FP64 walk: every quantity in double; shared-memory tally bins in double.
// Comparisons of distances (non-negative after clamping) and sign tests run on
// the IEEE bit patterns in the integer pipes, which order non-negative doubles
// like the numbers they encode; the FP64 pipe is left to the arithmetic.
template <>
struct Real<double> {
    static __device__ __forceinline__ unsigned long long k53(uint32_t hi, uint32_t lo) {
        return (((unsigned long long)hi << 32) | (unsigned long long)lo) >> 11;
    }
    // m 2^e, exactly, for |m| < 2^53: the bit pattern is assembled in the
    // integer pipes (leading-zero count, shift), keeping the conversion off
    // the FP64 pipe
    static __device__ __forceinline__ double scaled_int(long long m, int e) {
        const unsigned long long sgn = m < 0 ? (1ull << 63) : 0ull;
        const unsigned long long a = (unsigned long long)(m < 0 ? -m : m);
        const int p = 63 - __clzll((long long)(a | 1ull));  // leading bit
        const unsigned long long bits =
            sgn | ((unsigned long long)(p + e + 1023) << 52) | ((a << (52 - p)) & 0xFFFFFFFFFFFFFull);
        return a == 0ull ? 0.0 : __longlong_as_double((long long)bits);
    }
    // 53-bit uniform u = k 2^-53 in [0, 1) from the (hi, lo) output words
    static __device__ __forceinline__ double uniform(uint32_t hi, uint32_t lo) {
        return scaled_int((long long)k53(hi, lo), -53);
    }
    // 2u - 1 = (k - 2^52) 2^-52, exactly
    static __device__ __forceinline__ double two_u_minus_one(uint32_t hi, uint32_t lo) {
        return scaled_int((long long)k53(hi, lo) - (1ll << 52), -52);
    }
    // sqrt(u) = sqrt(2k 2^-54), in integer arithmetic
    static __device__ __forceinline__ double sqrt_uniform(uint32_t hi, uint32_t lo) {
        return sqrt_int(U128{k53(hi, lo) << 1, 0ull}, 54);
    }
    // A new direction's cosine mu and st = sqrt(1 - mu^2) from the draw u of mu:
    // cosine law mu = sqrt(u), st = sqrt(1 - u); isotropic mu = 2u - 1,
    // st = sqrt(4 u (1 - u)), with 1 - u and 4 u (1 - u) exact integers
    static __device__ __forceinline__ void direction_cosines(uint32_t hi, uint32_t lo, bool cosine, double *mu,
                                                             double *st) {
        const unsigned long long k = k53(hi, lo), n = (1ull << 53) - k;
        // sqrt(u) (the cosine law only: a lane starts the loop at t = 1
        // otherwise), then st, through one copy of sqrt_int
        const U128 x1 = cosine ? U128{n << 1, 0ull} : U128{(k * n) << 2, (umulhi64(k, n) << 2) | ((k * n) >> 62)};
        const int s1 = cosine ? 54 : 106;
        U128 x = cosine ? U128{k << 1, 0ull} : x1;
        int scale = s1;
        double r0 = 0.0, r1 = 0.0;
#pragma unroll 1
        for (int t = cosine ? 0 : 1; t < 2; ++t) {
            r0 = r1;
            r1 = sqrt_int(x, scale);
            x = x1;
            scale = s1;
        }
        *mu = cosine ? r0 : two_u_minus_one(hi, lo);
        *st = r1;
    }
    // 1 - u, exactly: (2^53 - k) 2^-53
    static __device__ __forceinline__ double one_minus(uint32_t hi, uint32_t lo) {
        return (double)((1ull << 53) - k53(hi, lo)) * 0x1p-53;
    }
    // u < v for the threshold ceil(v 2^53)
    static __device__ __forceinline__ bool below(uint32_t hi, uint32_t lo, unsigned long long thr53, uint32_t) {
        return k53(hi, lo) < thr53;
    }
    static __device__ __forceinline__ double inf() { return __longlong_as_double(0x7ff0000000000000ll); }
    static __device__ __forceinline__ bool pos(double w) { return __double_as_longlong(w) > 0; }
    static __device__ __forceinline__ bool neg(double w) {
        const long long b = __double_as_longlong(w);
        return b < 0 && (b << 1) != 0;
    }
    // negative values and -0 become +0
    static __device__ __forceinline__ double nonneg(double x) { return __double_as_longlong(x) < 0 ? 0.0 : x; }
    static __device__ __forceinline__ bool le(double a, double b) { return __double_as_longlong(a) <= __double_as_longlong(b); }
    static __device__ __forceinline__ bool lt(double a, double b) { return __double_as_longlong(a) < __double_as_longlong(b); }
    static __device__ __forceinline__ bool eq(double a, double b) { return __double_as_longlong(a) == __double_as_longlong(b); }
    static __device__ __forceinline__ double sigma(const CaseParams &c, int m) { return c.sigma[m]; }
    static __device__ __forceinline__ unsigned long long thr_c53(const CaseParams &c, int m) { return c.thr_c53[m]; }
    static __device__ __forceinline__ uint32_t thr_c24(const CaseParams &c, int m) { return c.thr_c24[m]; }
    static __device__ __forceinline__ double L(const CaseParams &c) { return c.L; }
    static __device__ __forceinline__ double dx(const CaseParams &c) { return c.dx; }
    static __device__ __forceinline__ double inv_dx(const CaseParams &c) { return c.inv_dx; }
    static __device__ __forceinline__ bool is_zero(double x) { return (__double_as_longlong(x) << 1) == 0; }
    // |x| and -x on the bit pattern (integer pipes)
    static __device__ __forceinline__ double abs(double x) {
        return __longlong_as_double(__double_as_longlong(x) & 0x7FFFFFFFFFFFFFFFll);
    }
    static __device__ __forceinline__ double flip(double x) {
        return __longlong_as_double(__double_as_longlong(x) ^ (long long)0x8000000000000000ull);
    }
    // min(floor(t), cap) for finite t >= 0, from the bit pattern
    static __device__ __forceinline__ int floor_index(double t, int cap) {
        const unsigned long long b = (unsigned long long)__double_as_longlong(t);
        const int e = (int)(b >> 52) - 1023;
        const int sh = min(max(52 - e, 0), 63);
        const unsigned long long v = ((b & 0xFFFFFFFFFFFFFull) | (1ull << 52)) >> sh;
        return (int)min(v, (unsigned long long)cap);
    }
    // t - k for finite t >= 0 and k = floor_index(t, cap) <= floor(t): the bits
    // below the binary point, plus floor(t) - k (non-zero beyond the last
    // bin), re-assembled in the integer pipes
    static __device__ __forceinline__ double frac(double t, int k) {
        const unsigned long long b = (unsigned long long)__double_as_longlong(t);
        const int e = (int)(b >> 52) - 1023;
        if (e > 30) return t - small_int_to_double(k);
        const int sh = 52 - max(e, 0);
        const unsigned long long M = (b & 0xFFFFFFFFFFFFFull) | (1ull << 52);
        const unsigned long long m = (((M >> sh) - (unsigned long long)k) << sh) + (M & ((1ull << sh) - 1ull));
        return e < 0 ? t : scaled_int((long long)m, -sh);
    }
    // l_c = -ln(1 - u) / Sigma_m, as -ln(1 - u) * (1 / Sigma_m), from the draw's words
    static __device__ __forceinline__ double collision(const CaseParams &c, int m, uint32_t hi, uint32_t lo) {
        return exp_variate_shared(k53(hi, lo)) * c.inv_sigma[m];
    }
    static __device__ __forceinline__ double interface(const CaseParams &c, int m, uint32_t hi, uint32_t lo) {
        return c.lambda[m] * exp_variate_shared(k53(hi, lo));
    }
    static __device__ __forceinline__ double inv_sigma(const CaseParams &c, int m) { return c.inv_sigma[m]; }
    static __device__ __forceinline__ double lambda(const CaseParams &c, int m) { return c.lambda[m]; }
    // -ln(1 - u) of two draws through one copy of the evaluation (the loop is
    // kept rolled: the instruction cache is one of the walk's limits)
    static __device__ __forceinline__ void exp_variates(uint32_t hi0, uint32_t lo0, uint32_t hi1, uint32_t lo1,
                                                        double *e0, double *e1) {
        unsigned long long ka = k53(hi0, lo0), kb = k53(hi1, lo1);
        double a = 0.0, b = 0.0;
#pragma unroll 1
        for (int t = 0; t < 2; ++t) {
            a = b;
            b = exp_variate_shared(ka);
            ka = kb;
        }
        *e0 = a;
        *e1 = b;
    }
    // 1/a in integer arithmetic (Newton-Raphson, cls_intmath.h)
    static __device__ __forceinline__ double recip(double a) { return recip_int(a); }
    // (sin, cos) of 2 pi u from the draw's words
    static __device__ __forceinline__ void sincos_2pi(uint32_t hi, uint32_t lo, double *s, double *co) {
        sincos_2pi_shared(k53(hi, lo), s, co);
    }
};

// FP32 tracking: position, direction and distances in float; the flights'
// deposits are summed exactly in a fixed-point difference array and the
// per-history statistics in FP64 (the tally regions below).
template <>
struct Real<float> {
    // the same draw truncated to its top 24 bits: u = k 2^-24
    static __device__ __forceinline__ float uniform(uint32_t hi, uint32_t) { return (float)(hi >> 8) * 0x1p-24f; }
    static __device__ __forceinline__ float two_u_minus_one(uint32_t hi, uint32_t lo) { return 2.0f * uniform(hi, lo) - 1.0f; }
    // FP32 tracking takes the hardware's approximate square root, reciprocal and
    // sine/cosine (a few FP32 ulps, below the FP32 walk's own rounding noise)
    static __device__ __forceinline__ float fast_sqrt(float x) {
        float r;
        asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
        return r;
    }
    static __device__ __forceinline__ float sqrt_uniform(uint32_t hi, uint32_t lo) { return fast_sqrt(uniform(hi, lo)); }
    static __device__ __forceinline__ void direction_cosines(uint32_t hi, uint32_t lo, bool cosine, float *mu,
                                                            float *st) {
        *mu = cosine ? sqrt_uniform(hi, lo) : two_u_minus_one(hi, lo);
        *st = fast_sqrt(1.0f - *mu * *mu);
    }
    static __device__ __forceinline__ float one_minus(uint32_t hi, uint32_t) {
        return (float)((1u << 24) - (hi >> 8)) * 0x1p-24f;
    }
    static __device__ __forceinline__ bool below(uint32_t hi, uint32_t, unsigned long long, uint32_t thr24) {
        return (hi >> 8) < thr24;
    }
    static __device__ __forceinline__ float inf() { return __int_as_float(0x7f800000); }
    static __device__ __forceinline__ bool pos(float w) { return w > 0.0f; }
    static __device__ __forceinline__ bool neg(float w) { return w < 0.0f; }
    static __device__ __forceinline__ float nonneg(float x) { return x > 0.0f ? x : 0.0f; }
    static __device__ __forceinline__ bool le(float a, float b) { return a <= b; }
    static __device__ __forceinline__ bool lt(float a, float b) { return a < b; }
    static __device__ __forceinline__ bool eq(float a, float b) { return a == b; }
    static __device__ __forceinline__ float sigma(const CaseParams &c, int m) { return c.sigma_f[m]; }
    static __device__ __forceinline__ unsigned long long thr_c53(const CaseParams &c, int m) { return c.thr_c53[m]; }
    static __device__ __forceinline__ uint32_t thr_c24(const CaseParams &c, int m) { return c.thr_c24[m]; }
    static __device__ __forceinline__ float L(const CaseParams &c) { return c.L_f; }
    static __device__ __forceinline__ float dx(const CaseParams &c) { return c.dx_f; }
    static __device__ __forceinline__ float inv_dx(const CaseParams &c) { return c.inv_dx_f; }
    static __device__ __forceinline__ bool is_zero(float x) { return x == 0.0f; }
    static __device__ __forceinline__ float abs(float x) { return fabsf(x); }
    static __device__ __forceinline__ float flip(float x) { return -x; }
    static __device__ __forceinline__ int floor_index(float t, int cap) { return min((int)t, cap); }
    static __device__ __forceinline__ float frac(float t, int k) { return t - (float)k; }
    static __device__ __forceinline__ float collision(const CaseParams &c, int m, uint32_t hi, uint32_t lo) {
        return -__logf(one_minus(hi, lo)) * c.inv_sigma_f[m];
    }
    static __device__ __forceinline__ float interface(const CaseParams &c, int m, uint32_t hi, uint32_t lo) {
        return -c.lambda_f[m] * __logf(one_minus(hi, lo));
    }
    static __device__ __forceinline__ float inv_sigma(const CaseParams &c, int m) { return c.inv_sigma_f[m]; }
    static __device__ __forceinline__ float lambda(const CaseParams &c, int m) { return c.lambda_f[m]; }
    static __device__ __forceinline__ void exp_variates(uint32_t hi0, uint32_t lo0, uint32_t hi1, uint32_t lo1, float *e0,
                                                        float *e1) {
        *e0 = -__logf(one_minus(hi0, lo0));
        *e1 = -__logf(one_minus(hi1, lo1));
    }
    static __device__ __forceinline__ float recip(float a) {
        float r;
        asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(a));
        return r;
    }
    // (sin, cos)(2 pi u) = -(sin, cos)(2 pi (u - 1/2)), the argument in [-pi, pi)
    static __device__ __forceinline__ void sincos_2pi(uint32_t hi, uint32_t lo, float *s, float *co) {
        float sn, cs;
        __sincosf(6.28318530717958647692f * (uniform(hi, lo) - 0.5f), &sn, &cs);
        *s = -sn;
        *co = -cs;
    }
};

// ----------------------------------------------------------- history state
template <typename P>
struct History {
    P r[3];
    P w[3];
    P iw[3];          // 1 / w (infinite when the component is 0)
    int m;
    uint32_t j;       // per-history draw index
    uint32_t c2, c3;  // words 2, 3 of the last Philox block (odd draws)
    uint32_t h_lo, h_hi, cid;
    uint32_t events, n_coll, n_int, n_refl;
    uint32_t pend;    // direction still to draw (DIR_*), 3D and extruded geometries
    P track0, track1; // per-history track length in material 0 / 1
};

// A new direction of the 3D or extruded walk is drawn by resolve_direction,
// which the history tracker runs once per step for every lane that needs one:
// the lanes born this step and those that scattered in the last one share one
// pass through the sqrt, sine/cosine and reciprocal arithmetic.
enum : uint32_t { DIR_NONE = 0, DIR_SCATTER = 1, DIR_SOURCE_COSINE = 2, DIR_SOURCE_ISOTROPIC = 3 };

// One flight's contribution to the mesh: a0 into bin k0, a1 into bin k1
// (k1 > k0) and c into each interior bin k0 < k < k1.  Empty when k1 < k0.
template <typename P>
struct Flight {
    int k0, k1;
    P a0, a1, c;
    bool tail;  // k1 is the mesh's last bin: the difference array's end marker falls past the mesh
};

// Output words (hi, lo) of draw j = s.j of the history; advances j.  Even
// draws compute a Philox block and keep its words 2, 3 for the odd draw.
template <typename P>
__device__ __forceinline__ void draw_words(History<P> &s, const RoundKeys &key, uint32_t &hi, uint32_t &lo) {
    if ((s.j & 1u) == 0u) {
        const uint4 o = philox4x32_10(make_uint4(s.j >> 1, s.h_lo, s.h_hi, s.cid), key);
        hi = o.x;
        lo = o.y;
        s.c2 = o.z;
        s.c3 = o.w;
    } else {
        hi = s.c2;
        lo = s.c3;
    }
    ++s.j;
}

// Output words of draws j and j + 1 (j = s.j); advances j by 2.  The pair
// always needs exactly one Philox block -- words (0,1), (2,3) of block j/2 for
// even j; the cached words of the last block and words (0,1) of block
// (j+1)/2 for odd j -- so a warp computes it once, whatever its lanes' parities.
template <typename P>
__device__ __forceinline__ void draw_pair(History<P> &s, const RoundKeys &key, uint32_t &hi0, uint32_t &lo0,
                                          uint32_t &hi1, uint32_t &lo1) {
    const bool odd = (s.j & 1u) != 0u;
    const uint4 o = philox4x32_10(make_uint4((s.j + 1u) >> 1, s.h_lo, s.h_hi, s.cid), key);
    hi0 = odd ? s.c2 : o.x;
    lo0 = odd ? s.c3 : o.y;
    hi1 = odd ? o.x : o.z;
    lo1 = odd ? o.y : o.w;
    s.c2 = o.z;  // read by draw j + 2 when it is odd
    s.c3 = o.w;
    s.j += 2u;
}

template <typename P>
__device__ __forceinline__ P draw(History<P> &s, const RoundKeys &key) {
    uint32_t hi, lo;
    draw_words(s, key, hi, lo);
    return Real<P>::uniform(hi, lo);
}

// 1 - u of the next draw, exactly
template <typename P>
__device__ __forceinline__ P draw_one_minus(History<P> &s, const RoundKeys &key) {
    uint32_t hi, lo;
    draw_words(s, key, hi, lo);
    return Real<P>::one_minus(hi, lo);
}

// 2u - 1 for the next draw u (isotropic direction cosine)
template <typename P>
__device__ __forceinline__ P draw_iso(History<P> &s, const RoundKeys &key) {
    uint32_t hi, lo;
    draw_words(s, key, hi, lo);
    return Real<P>::two_u_minus_one(hi, lo);
}

// whether the next draw is below the value whose thresholds are given
template <typename P>
__device__ __forceinline__ bool draw_below(History<P> &s, const RoundKeys &key, unsigned long long thr53, uint32_t thr24) {
    uint32_t hi, lo;
    draw_words(s, key, hi, lo);
    return Real<P>::below(hi, lo, thr53, thr24);
}


// Geometry of a case: G is a compile-time geometry code (1, 2, 3, 11, 13) for
// launches whose cases share one geometry, 0 to read it from the case.  A
// fixed G folds every geometry branch of the walk away.
template <int G>
__device__ __forceinline__ int geometry(const CaseParams &cp) {
    return G != 0 ? G : cp.d;
}

template <typename P>
__device__ __forceinline__ void set_direction(History<P> &s, P wx, P wy, P wz) {
    using R = Real<P>;
    s.w[0] = wx;
    s.w[1] = wy;
    s.w[2] = wz;
    if constexpr (sizeof(P) == 8) {  // one copy of the integer reciprocal, three passes
        P a = wx, b = wy, c = wz, r0 = P(0), r1 = P(0), r2 = P(0);
#pragma unroll 1
        for (int t = 0; t < 3; ++t) {
            r0 = r1;
            r1 = r2;
            r2 = R::is_zero(a) ? R::inf() : R::recip(a);
            a = b;
            b = c;
        }
        s.iw[0] = r0;
        s.iw[1] = r1;
        s.iw[2] = r2;
    } else {
        s.iw[0] = R::is_zero(wx) ? R::inf() : R::recip(wx);
        s.iw[1] = R::is_zero(wy) ? R::inf() : R::recip(wy);
        s.iw[2] = R::is_zero(wz) ? R::inf() : R::recip(wz);
    }
}

// Direction (wx, 0, 0) of the slab and the x-projected box: no reciprocal of
// the zero components
template <typename P>
__device__ __forceinline__ void set_direction_x(History<P> &s, P wx) {
    using R = Real<P>;
    s.w[0] = wx;
    s.w[1] = P(0);
    s.w[2] = P(0);
    s.iw[0] = R::is_zero(wx) ? R::inf() : R::recip(wx);
    s.iw[1] = R::inf();
    s.iw[2] = R::inf();
}

// Draw the pending direction of a 3D or extruded walk: mu, then the azimuth
// phi, then (at the source) the material label, in the order of the serial
// walk.  Cosine-law incidence (paper Sec. 4.3): mu = sqrt(xi) about +x,
// omega = (mu, st cos phi, st sin phi); isotropic (scattering, volume source):
// mu = 2 xi - 1, omega = (st cos phi, st sin phi, mu); st = sqrt(1 - mu^2).
template <typename P, int G = 0>
__device__ __forceinline__ void resolve_direction(History<P> &s, const CaseParams &cp, const RoundKeys &key) {
    if constexpr (G != 0 && G != 2 && G != 3) return;  // no pending directions in these geometries
    if (s.pend == DIR_NONE) return;
    const bool cosine = s.pend == DIR_SOURCE_COSINE;
    uint32_t hi, lo, phi_hi, phi_lo;
    draw_pair(s, key, hi, lo, phi_hi, phi_lo);  // mu, then phi
    P mu, st, sn, cs;
    Real<P>::direction_cosines(hi, lo, cosine, &mu, &st);
    Real<P>::sincos_2pi(phi_hi, phi_lo, &sn, &cs);
    const P a = st * cs, b = st * sn;
    set_direction(s, cosine ? mu : a, cosine ? a : b, cosine ? b : mu);
    if (s.pend != DIR_SCATTER) s.m = draw_below(s, key, cp.thr_p053, cp.thr_p024) ? 0 : 1;
    s.pend = DIR_NONE;
}

// Source: position and direction first, then the material label.  With
// DEFER, a 3D or extruded source leaves its direction and label pending for
// the caller's resolve_direction.
template <typename P, int G = 0, bool DEFER = false>
__device__ __forceinline__ void source(History<P> &s, const CaseParams &cp, const RoundKeys &key, uint64_t h) {
    using R = Real<P>;
    const int gd = geometry<G>(cp);
    s.h_lo = (uint32_t)h;
    s.h_hi = (uint32_t)(h >> 32);
    s.cid = cp.case_id;
    s.j = 0;
    s.events = s.n_coll = s.n_int = s.n_refl = 0;
    s.pend = DIR_NONE;
    s.track0 = s.track1 = P(0);
    s.r[0] = P(0);
    s.r[1] = P(0);
    s.r[2] = P(0);
    const P L = R::L(cp);
    if (gd == 3 || gd == 2) {
        if (cp.source == 1) s.r[0] = L * draw(s, key);  // suite II: uniform position, isotropic direction
        if (gd == 3) {  // y, then z
            uint32_t yh, yl, zh, zl;
            draw_pair(s, key, yh, yl, zh, zl);
            s.r[1] = L * R::uniform(yh, yl);
            s.r[2] = L * R::uniform(zh, zl);
        } else {
            s.r[1] = L * draw(s, key);
        }
        s.pend = (cp.source == 1) ? DIR_SOURCE_ISOTROPIC : DIR_SOURCE_COSINE;
        if (!DEFER) resolve_direction<P, G>(s, cp, key);
        return;
    }
    if (cp.source == 1) {
        s.r[0] = L * draw(s, key);
        if (gd == 11 || gd == 13) {
            set_direction_x(s, draw_iso(s, key));
        } else {
            uint32_t hi, lo;
            draw_words(s, key, hi, lo);
            const P w = (hi >> 31) == 0u ? P(1) : P(-1);  // u < 1/2
            s.w[0] = w;
            s.w[1] = P(0);
            s.w[2] = P(0);
            s.iw[0] = w;
            s.iw[1] = R::inf();
            s.iw[2] = R::inf();
        }
    } else if (gd == 11 || gd == 13) {
        uint32_t hi, lo;  // slab, projected box: mu = sqrt(xi)
        draw_words(s, key, hi, lo);
        set_direction_x(s, R::sqrt_uniform(hi, lo));
    } else {
        s.w[0] = P(1);
        s.w[1] = P(0);
        s.w[2] = P(0);
        s.iw[0] = P(1);
        s.iw[1] = R::inf();
        s.iw[2] = R::inf();
    }
    s.m = draw_below(s, key, cp.thr_p053, cp.thr_p024) ? 0 : 1;
}

// Trace sink (only instantiated by the trace kernel).
struct TraceSink {
    double *rows;
    int cap;
    int n;
};

template <typename P, bool TRACE>
__device__ __forceinline__ void trace_row(TraceSink *tr, int ev, const History<P> &s, double l) {
    if constexpr (TRACE) {
        if (tr->n < tr->cap) {
            double *row = tr->rows + 10 * (size_t)tr->n;
            row[0] = ev;
            row[1] = (double)s.j;
            row[2] = (double)s.r[0];
            row[3] = (double)s.r[1];
            row[4] = (double)s.r[2];
            row[5] = (double)s.w[0];
            row[6] = (double)s.w[1];
            row[7] = (double)s.w[2];
            row[8] = (double)s.m;
            row[9] = l;
        }
        tr->n++;
    }
}

// Track-length estimator: the flight x0 -> x1 (length l, direction cosine wx)
// scores in bin k the path length inside e_k <= x < e_k+1, the x-overlap times
// 1/|wx|; interior bins receive dx/|wx| each.  A flight inside one bin scores
// its length l itself, which stays exact for grazing flights (|wx| -> 0).  A
// flight with wx == 0 scores its whole length in the bin that contains x0.
template <typename P>
__device__ __forceinline__ void plan_flight(Flight<P> &f, History<P> &s, const CaseParams &cp, P x0, P x1, P l,
                                            int m) {
    using R = Real<P>;
    const P t = (m == 0 ? s.track0 : s.track1) + l;  // one add, the sum selected
    s.track0 = (m == 0) ? t : s.track0;
    s.track1 = (m == 0) ? s.track1 : t;
    f.k0 = 0;
    f.k1 = -1;
    if (!R::pos(l)) return;
    const int nb = cp.nbins;
    const P inv_dx = R::inv_dx(cp);
    // the x-extent clipped to [0, L]; every value below is >= 0, so min and
    // max are the integer comparisons of R::lt
    const P a = R::nonneg(x0), b = R::nonneg(x1);
    if (R::is_zero(s.w[0])) {
        const int k = R::floor_index(a * inv_dx, nb - 1);
        f.k0 = f.k1 = k;
        f.tail = k == nb - 1;
        f.a0 = l;
        return;
    }
    const P L = R::L(cp);
    const P lo = R::lt(a, b) ? a : b;
    P hi = R::lt(a, b) ? b : a;
    hi = R::lt(L, hi) ? L : hi;
    // bin coordinates x / dx: bin index = integer part; the end bins receive
    // (1 - frac) dx / |wx| and frac dx / |wx|
    const P ulo = lo * inv_dx, uhi = hi * inv_dx;
    const int k0 = R::floor_index(ulo, nb - 1);
    const int k1 = R::floor_index(uhi, nb - 1);
    f.k0 = k0;
    f.k1 = k1;
    f.tail = k1 == nb - 1;
    if (k0 == k1) {  // the flight lies inside one bin: its length itself
        f.a0 = l;
        return;
    }
    const P c = R::dx(cp) * R::abs(s.iw[0]);
    f.a0 = R::nonneg(fma(-R::frac(ulo, k0), c, c));
    f.a1 = R::frac(uhi, k1) * c;
    f.c = c;
}

// Distance along the flight to the face ahead on one axis: (L - r)/omega
// moving up, (0 - r)/omega moving down, clamped at 0; infinite when omega is
// +-0.  One multiply on every lane, no branch.
template <typename P>
__device__ __forceinline__ P face_distance(P r, P w, P iw, P L) {
    using R = Real<P>;
    const P target = R::pos(w) ? L : P(0);
    const P d = R::nonneg((target - r) * iw);
    return R::is_zero(w) ? R::inf() : d;
}

// One event of Algorithm A.  Fills the flight to score and returns -1 while
// the history continues, else the terminating event (EV_LEAK_X0, EV_LEAK_XL,
// EV_ABSORB, EV_CAPPED).
template <typename P, bool TRACE, int G = 0, bool DEFER = false>
__device__ __forceinline__ int step(History<P> &s, const CaseParams &cp, const RoundKeys &key, uint32_t max_events,
                                    Flight<P> &f, TraceSink *tr) {
    using R = Real<P>;
    const int gd = geometry<G>(cp);
    f.k0 = 0;
    f.k1 = -1;
    if (s.events == max_events) {
        trace_row<P, TRACE>(tr, EV_CAPPED, s, 0.0);
        return EV_CAPPED;
    }
    ++s.events;
    const int m = s.m;
    const P INF = R::inf();
    const P L = R::L(cp);

    // collision, then interface distance.  One Philox block serves both draws
    // (draw_pair), except in the FP32 x-projected walk, where holding the pair
    // spills registers (measured 10% slower there, 4-7% faster elsewhere).
    uint32_t hi, lo, ihi, ilo;
    P l_c, l_i;
    if constexpr (sizeof(P) == 4 && G == 13) {
        draw_words(s, key, hi, lo);
        l_c = R::pos(R::sigma(cp, m)) ? R::nonneg(R::collision(cp, m, hi, lo)) : INF;
        draw_words(s, key, ihi, ilo);
        l_i = R::interface(cp, m, ihi, ilo);
    } else {
        draw_pair(s, key, hi, lo, ihi, ilo);
        P e_c, e_i;
        R::exp_variates(hi, lo, ihi, ilo, &e_c, &e_i);
        l_c = R::pos(R::sigma(cp, m)) ? R::nonneg(e_c * R::inv_sigma(cp, m)) : INF;
        l_i = R::lambda(cp, m) * e_i;
    }
    if (gd == 11) l_i *= R::abs(s.iw[0]);  // slab: the chord projected on x, Lambda/|mu|
    else if (gd == 2) l_i /= sqrt(P(1) - s.w[2] * s.w[2]);  // extruded: in-plane chord along the flight
    l_i = R::nonneg(l_i);

    // boundary distance: x faces, then the lateral faces of the box
    // (the face ahead minus the position) / omega, on every lane; infinite for omega = 0
    int face = R::pos(s.w[0]) ? 1 : 0;  // 0: x = 0, 1: x = L, 2: lateral
    P l_b = face_distance(s.r[0], s.w[0], s.iw[0], L);
    P l_y = INF, l_z = INF;
    const bool box = gd == 3;
    const bool lateral = box || gd == 2;  // lateral faces: y (and z in the box; the extruded geometry has none)
    if (lateral) {
        l_y = face_distance(s.r[1], s.w[1], s.iw[1], L);
        if (R::lt(l_y, l_b)) {
            l_b = l_y;
            face = 2;
        }
        if (box) {
            l_z = face_distance(s.r[2], s.w[2], s.iw[2], L);
            if (R::lt(l_z, l_b)) {
                l_b = l_z;
                face = 2;
            }
        }
    }

    // the event: boundary, else collision, else interface.  Every lane then
    // moves and scores its flight on one converged path.
    const bool bnd = R::le(l_b, l_c) && R::le(l_b, l_i);
    const bool coll = !bnd && R::le(l_c, l_i);
    const bool leak = bnd && face != 2;
    const P l = bnd ? l_b : (coll ? l_c : l_i);
    const P x1 = leak ? ((face == 0) ? P(0) : L) : s.r[0] + l * s.w[0];
    plan_flight(f, s, cp, s.r[0], x1, l, m);
    s.r[0] = x1;
    if (lateral) {
        if (bnd && face == 2 && R::eq(l_y, l_b)) {  // specular reflection on a y face
            s.r[1] = R::pos(s.w[1]) ? L : P(0);
            s.w[1] = R::flip(s.w[1]);
            s.iw[1] = R::flip(s.iw[1]);
        } else {
            s.r[1] += l * s.w[1];
        }
    }
    if (box) {
        if (bnd && face == 2 && R::eq(l_z, l_b)) {  // and/or on a z face
            s.r[2] = R::pos(s.w[2]) ? L : P(0);
            s.w[2] = R::flip(s.w[2]);
            s.iw[2] = R::flip(s.iw[2]);
        } else {
            s.r[2] += l * s.w[2];
        }
    }
    if (leak) {
        const int ev = (face == 0) ? EV_LEAK_X0 : EV_LEAK_XL;
        trace_row<P, TRACE>(tr, ev, s, (double)l);
        return ev;
    }
    if (bnd) {
        ++s.n_refl;
        trace_row<P, TRACE>(tr, EV_REFLECT, s, (double)l);
        return -1;
    }
    if (coll) {
        ++s.n_coll;
        if (draw_below(s, key, R::thr_c53(cp, m), R::thr_c24(cp, m))) {
            if (gd == 1) {
                // u < 1/2 exactly when the top bit of the draw is clear
                draw_words(s, key, hi, lo);
                const P w = (hi >> 31) == 0u ? P(1) : P(-1);
                s.w[0] = w;
                s.iw[0] = w;
            } else if (gd == 11 || gd == 13) {
                set_direction_x(s, draw_iso(s, key));  // mu = 2 xi - 1
            } else {
                s.pend = DIR_SCATTER;  // mu = 2 xi - 1, then phi
                if (!DEFER) resolve_direction<P, G>(s, cp, key);
            }
            trace_row<P, TRACE>(tr, EV_SCATTER, s, (double)l);
            return -1;
        }
        trace_row<P, TRACE>(tr, EV_ABSORB, s, (double)l);
        return EV_ABSORB;
    }
    s.m = 1 - m;
    ++s.n_int;
    trace_row<P, TRACE>(tr, EV_INTERFACE, s, (double)l);
    return -1;
}

// ------------------------------------------------------- tally regions
// A warp-private shared-memory region (layout: region_bytes() in
// cls_internal.h): the bins, FP64 statistics, u64 counters and the lanes' own
// FP64 copies of the per-history statistics.  The FP64 walk's bins are
// doubles; the FP32 walk's are a fixed-point difference array (u64 with 32
// fraction bits), added with native integer atomics -- no retry loop when a
// warp's flights share an entry, as on thin slabs -- and prefix-summed exactly
// at the flush.
template <typename P>
constexpr bool kFixedBins = sizeof(P) == 4;

__device__ __forceinline__ unsigned long long *region_fixed(unsigned char *region) {
    return reinterpret_cast<unsigned long long *>(region);
}

// round(c 2^32), ties to even, for 0 <= c < 2^32, in two 32-bit halves: the
// integer part of c, and the fraction c - floor(c) (exact in float) scaled by
// 2^32 (exact) and rounded to the nearest integer, below 2^32 because a
// fraction of a float is at most 1 - 2^-24.  The halves add up to the one
// rounding of c 2^32, since its integer part shifts the rounded value by a
// multiple of 2^32.  Two 32-bit conversions instead of one to 64 bits: those
// run on the FP64 pipe, which the walk's history-end statistics already use
// (measured 1% faster on the sweep and the 3D box).
__device__ __forceinline__ unsigned long long fixed32(float c) {
    const uint32_t hi = __float2uint_rz(c);
    const float frac = c - __uint2float_rz(hi);
    return ((unsigned long long)hi << 32) | __float2uint_rn(frac * 0x1p32f);
}

// The lanes' own copies of the per-history statistics: FP64 in FP64 regions;
// in FP32 regions u64 fixed point -- t0, t1 with 32 fraction bits, t^2 with
// 24; the slot of t stays unused, its sum being that of t0 and t1 -- so that
// the FP32 walk sums them exactly.
template <typename P>
using LaneStat = typename std::conditional<kFixedBins<P>, unsigned long long, double>::type;

template <typename P>
__device__ __forceinline__ LaneStat<P> *region_lane_stats(unsigned char *region, int nbs) {
    return reinterpret_cast<LaneStat<P> *>(region + region_lane_stats_offset(kFixedBins<P>, nbs));
}

// A history longer than this (in track length) keeps its statistics out of the
// fixed-point lane copies: t <= 2^13 is below 2^45 with 32 fraction bits and
// t^2 below 2^50 with 24, so a lane's sums stay below 2^64 for up to 2^13
// histories between flushes (FP32 regions flush every 1024).
constexpr float kFixedTrackMax = 8192.0f;

template <typename P>
__device__ __forceinline__ double *region_stats(unsigned char *region, int nbs) {
    return reinterpret_cast<double *>(region + region_bins_bytes(kFixedBins<P>, nbs));
}

// The history's track length t and t^2 into this lane's own copy of the
// region's statistics (no atomics).  FP64 walk: in FP64.  FP32 walk: the
// history's float sums per material, t0 and t1, are rounded once to 32
// fraction bits and added exactly, t = t0 + t1 from those; t^2 is the square
// of the float t, rounded to 24 fraction bits.  Returns false, with nothing
// added, for a history the fixed-point copies cannot hold (track length
// beyond kFixedTrackMax): the caller adds it to the global FP64 statistics.
template <typename P>
__device__ __forceinline__ bool finish_history(unsigned char *region, int nbs, const History<P> &s, int lane) {
    LaneStat<P> *ls = region_lane_stats<P>(region, nbs) + lane;
    if constexpr (kFixedBins<P>) {
        const float t = s.track0 + s.track1;
        if (!(t <= kFixedTrackMax)) return false;
        const unsigned long long q0 = fixed32(s.track0), q1 = fixed32(s.track1);
        // the sum of t is that of t0 plus that of t1: the flush forms it
        ls[32 * S_T2] += __float2ull_rn(t * t * 0x1p24f);
        ls[32 * S_TRACK0] += q0;
        ls[32 * S_TRACK1] += q1;
    } else {
        const double t0 = (double)s.track0;
        const double t1 = (double)s.track1;
        const double t = t0 + t1;
        ls[32 * S_T] += t;
        ls[32 * S_T2] += t * t;
        ls[32 * S_TRACK0] += t0;
        ls[32 * S_TRACK1] += t1;
    }
    return true;
}

// Outcome and event counters of the lanes whose history ended this step
// (`ended`, scoring into region lreg < 2).  When several lanes ended they are
// summed over the warp per region (ballot counts, warp reductions of 16-bit
// halves) and one lane adds each to the region, else each lane adds its own:
// short histories that end together do not serialise on shared atomics.
__device__ __forceinline__ void count_one(unsigned long long *ct, int outcome, uint32_t n_coll, uint32_t n_int,
                                          uint32_t n_refl, uint32_t events) {
    const int c = (outcome == EV_LEAK_X0) ? C_R : (outcome == EV_LEAK_XL) ? C_T : (outcome == EV_ABSORB) ? C_A : C_CAPPED;
    atomicAdd(&ct[c], 1ull);
    if (n_coll) atomicAdd(&ct[C_COLL], (unsigned long long)n_coll);
    if (n_int) atomicAdd(&ct[C_INT], (unsigned long long)n_int);
    if (n_refl) atomicAdd(&ct[C_REFL], (unsigned long long)n_refl);
    atomicAdd(&ct[C_EVENTS], (unsigned long long)events);
    atomicMax(&ct[C_MAXEV], (unsigned long long)events);
}

__device__ __forceinline__ unsigned long long warp_sum32(bool mine, uint32_t x, bool small) {
    const uint32_t v = mine ? x : 0u;
    if (small) return __reduce_add_sync(CLS_FULL_MASK, v);  // 32 values below 2^27 sum below 2^32
    return (unsigned long long)__reduce_add_sync(CLS_FULL_MASK, v & 0xFFFFu) +
           ((unsigned long long)__reduce_add_sync(CLS_FULL_MASK, v >> 16) << 16);
}

template <typename P>
__device__ __forceinline__ void warp_count(unsigned char *regions, int rbytes, int nbs, bool ended, int lreg,
                                           const History<P> &s, int outcome, int lane, bool small) {
    const unsigned em = __ballot_sync(CLS_FULL_MASK, ended);
    if (em == 0u) return;
    if (__popc(em) < 4) {
        if (ended)
            count_one(reinterpret_cast<unsigned long long *>(region_stats<P>(regions + lreg * rbytes, nbs) + S_NUM),
                      outcome, s.n_coll, s.n_int, s.n_refl, s.events);
        return;
    }
#pragma unroll 1
    for (int r = 0; r < 2; ++r) {
        const bool mine = ended && lreg == r;
        const unsigned m = __ballot_sync(CLS_FULL_MASK, mine);
        if (m == 0u) continue;
        const unsigned nr = __popc(__ballot_sync(CLS_FULL_MASK, mine && outcome == EV_LEAK_X0));
        const unsigned nt = __popc(__ballot_sync(CLS_FULL_MASK, mine && outcome == EV_LEAK_XL));
        const unsigned na = __popc(__ballot_sync(CLS_FULL_MASK, mine && outcome == EV_ABSORB));
        const unsigned ncap = __popc(m) - nr - nt - na;
        const unsigned long long nc = warp_sum32(mine, s.n_coll, small), ni = warp_sum32(mine, s.n_int, small);
        const unsigned long long nf = warp_sum32(mine, s.n_refl, small), ne = warp_sum32(mine, s.events, small);
        const unsigned mx = __reduce_max_sync(CLS_FULL_MASK, mine ? s.events : 0u);
        if (lane == __ffs(m) - 1) {
            unsigned long long *ct = reinterpret_cast<unsigned long long *>(region_stats<P>(regions + r * rbytes, nbs) + S_NUM);
            if (nr) atomicAdd(&ct[C_R], (unsigned long long)nr);
            if (nt) atomicAdd(&ct[C_T], (unsigned long long)nt);
            if (na) atomicAdd(&ct[C_A], (unsigned long long)na);
            if (ncap) atomicAdd(&ct[C_CAPPED], (unsigned long long)ncap);
            if (nc) atomicAdd(&ct[C_COLL], nc);
            if (ni) atomicAdd(&ct[C_INT], ni);
            if (nf) atomicAdd(&ct[C_REFL], nf);
            atomicAdd(&ct[C_EVENTS], ne);
            atomicMax(&ct[C_MAXEV], (unsigned long long)mx);
        }
    }
}

// The interior bins of all lanes' flights, spread evenly over the 32 lanes:
// lane t of each round scores interior task base + t, found by a 5-step
// shuffle search over the warp's inclusive prefix sum of the interior counts.
// Lanes with lreg < 2 score into their FP64 region (FP64 walk only: the FP32
// walk's region lanes take the difference array and bring no tasks here);
// lanes with lreg == 2 into the FP64 global bins.
template <typename P>
__device__ __forceinline__ void spread_interior(unsigned char *regions, int rbytes, int lreg, double *gflux,
                                                uint64_t goff, int k0, P c, int ni, int lane) {
    int incl = ni;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(CLS_FULL_MASK, incl, o);
        if (lane >= o) incl += v;
    }
    const int total = __shfl_sync(CLS_FULL_MASK, incl, 31);
    if (total == 0) return;
    const bool any_global = __any_sync(CLS_FULL_MASK, lreg == 2 && ni > 0);
    const int base_bin = k0 + 1 - (incl - ni);  // interior task t of this lane goes to base_bin + t
    for (int base = 0; base < total; base += 32) {
        const int t = base + lane;
        int o = 0;
#pragma unroll
        for (int sft = 16; sft >= 1; sft >>= 1) {
            const int v = __shfl_sync(CLS_FULL_MASK, incl, o + sft - 1);
            if (v <= t) o += sft;
        }
        const int ob = __shfl_sync(CLS_FULL_MASK, base_bin, o);
        const P oc = __shfl_sync(CLS_FULL_MASK, c, o);
        const int oreg = __shfl_sync(CLS_FULL_MASK, lreg, o);
        uint64_t ogoff = 0;
        if (any_global) ogoff = __shfl_sync(CLS_FULL_MASK, goff, o);
        if (t < total) {
            if (!kFixedBins<P> && oreg < 2) {
                double *bins = reinterpret_cast<double *>(regions + oreg * rbytes);
                atomicAdd(&bins[ob + t], (double)oc);
            } else {
                atomicAdd(&gflux[ogoff + ob + t], (double)oc);
            }
        }
    }
}

// Score the warp's flights.
//   FP32 walk, region lanes: the flight's bins are a0 in k0, c in each interior
//   bin k0 < k < k1 and a1 in k1, each rounded once to 32 fraction bits (q0,
//   qc, q1; zero where the flight has no such bin); as a difference array D
//   (bin k = D[0] + ... + D[k]) that is D[k0] += q0, D[k0+1] += qc - q0 (or
//   q1 - q0 when k1 = k0 + 1), D[k1] += q1 - qc, D[k1+1] -= q1 -- two integer
//   atomics for a flight inside one bin, three when it spans two, four
//   otherwise -- and the flush's prefix sum returns exactly the rounded
//   deposits, whatever the order of the atomics.  With SKIP, an entry that
//   adds zero is left out (q0 = qc when the flight covers its first bin
//   whole, q1 = qc when it covers its last bin whole), and so is the end
//   marker D[k1+1] of a flight whose last bin is the mesh's (the flush never
//   reads past the last bin).
//   FP64 walk: each lane adds its two end bins, and the interior bins of all
//   lanes' flights are spread evenly over the 32 lanes (spread_interior), so
//   long flights do not serialise the warp; each interior bin is added
//   exactly (a difference array's prefix sums would cancel between near and
//   far bins, and FP64 parity holds to 1e-12 per bin).
// A lane with lreg == 2 scores straight into the FP64 global bins at
// gflux + goff, those of its (case, batch) (see the region eviction in the
// trackers).
template <typename P, bool SKIP = false>
__device__ __forceinline__ void warp_deposit(unsigned char *regions, int rbytes, int nbs, int lreg, double *gflux,
                                             uint64_t goff, const Flight<P> &f, int lane) {
    const bool has = f.k1 >= f.k0;
    if (has) {
        if (lreg < 2) {
            if constexpr (kFixedBins<P>) {
                // predicated, not branched: every lane with a flight runs the same code
                unsigned long long *D = region_fixed(regions + lreg * rbytes);
                const bool multi = f.k1 > f.k0, inter = f.k1 > f.k0 + 1;
                const unsigned long long q0 = fixed32((float)f.a0);
                const unsigned long long q1 = fixed32(multi ? (float)f.a1 : 0.0f);
                const unsigned long long qc = fixed32(inter ? (float)f.c : 0.0f);
                const unsigned long long d1 = (inter ? qc : q1) - q0;  // modulo 2^64: exact
                if constexpr (SKIP) {
                    if (q0 != 0ull) atomicAdd(&D[f.k0], q0);
                    if (d1 != 0ull && (multi || !f.tail)) atomicAdd(&D[f.k0 + 1], d1);
                    if (inter && q1 != qc) atomicAdd(&D[f.k1], q1 - qc);
                    if (multi && !f.tail) atomicAdd(&D[f.k1 + 1], 0ull - q1);
                } else {
                    atomicAdd(&D[f.k0], q0);
                    atomicAdd(&D[f.k0 + 1], d1);
                    if (inter) atomicAdd(&D[f.k1], q1 - qc);
                    if (multi) atomicAdd(&D[f.k1 + 1], 0ull - q1);
                }
            } else {
                double *bins = reinterpret_cast<double *>(regions + lreg * rbytes);
                atomicAdd(&bins[f.k0], (double)f.a0);
                if (f.k1 > f.k0) atomicAdd(&bins[f.k1], (double)f.a1);
            }
        } else {
            double *gbins = gflux + goff;
            atomicAdd(&gbins[f.k0], (double)f.a0);
            if (f.k1 > f.k0) atomicAdd(&gbins[f.k1], (double)f.a1);
        }
    }
    const int ni = (has && !(kFixedBins<P> && lreg < 2)) ? max(f.k1 - f.k0 - 1, 0) : 0;
    if (!__any_sync(CLS_FULL_MASK, ni > 0)) return;  // one vote instead of the scan when no lane has any
    spread_interior<P>(regions, rbytes, lreg, gflux, goff, f.k0, f.c, ni, lane);
}

// A finished history's outcome into the caller's record, when one is bound
// (OutcomeRecord): 0 reflected (left through x = 0), 1 transmitted (x = L),
// 2 absorbed, 3 capped.  One byte per history; the host has checked that the
// record holds the run's cases x histories.
__device__ __forceinline__ void record_outcome(const LaunchArgs &a, int case_index, uint32_t h_lo, uint32_t h_hi,
                                               int outcome) {
    if (a.outcomes == nullptr) return;
    const OutcomeRecord r = *a.outcomes;
    if (r.codes == nullptr) return;
    const uint64_t h = ((uint64_t)h_hi << 32) | h_lo;
    const uint8_t code = outcome == EV_LEAK_X0 ? 0 : outcome == EV_LEAK_XL ? 1 : outcome == EV_ABSORB ? 2 : 3;
    r.codes[(uint64_t)case_index * r.stride + (h - r.first)] = code;
}

// A history's track-length statistics added straight to the case's global
// FP64 tally block.
template <typename P>
__device__ __forceinline__ void add_history_stats_global(const LaunchArgs &a, int case_index, const History<P> &s) {
    double *st = a.t.stats + (size_t)case_index * S_NUM;
    const double t0 = (double)s.track0;
    const double t1 = (double)s.track1;
    const double t = t0 + t1;
    atomicAdd(&st[S_T], t);
    atomicAdd(&st[S_T2], t * t);
    if (__double_as_longlong(t0) != 0) atomicAdd(&st[S_TRACK0], t0);
    if (__double_as_longlong(t1) != 0) atomicAdd(&st[S_TRACK1], t1);
}

// History end for a lane that scores into global memory: the same statistics
// and counters as finish_history, added to the case's global tally block.
template <typename P>
__device__ __forceinline__ void finish_history_global(const LaunchArgs &a, int case_index, const History<P> &s,
                                                      int outcome, bool with_event_counts) {
    add_history_stats_global<P>(a, case_index, s);
    unsigned long long *ct = a.t.counters + (size_t)case_index * C_NUM;
    const int c = (outcome == EV_LEAK_X0) ? C_R : (outcome == EV_LEAK_XL) ? C_T : (outcome == EV_ABSORB) ? C_A : C_CAPPED;
    atomicAdd(&ct[c], 1ull);
    if (with_event_counts) {
        if (s.n_coll) atomicAdd(&ct[C_COLL], (unsigned long long)s.n_coll);
        if (s.n_int) atomicAdd(&ct[C_INT], (unsigned long long)s.n_int);
        if (s.n_refl) atomicAdd(&ct[C_REFL], (unsigned long long)s.n_refl);
        atomicAdd(&ct[C_EVENTS], (unsigned long long)s.events);
    }
    atomicMax(&ct[C_MAXEV], (unsigned long long)s.events);
}

// Flush a warp region into the global tally block of (case, batch): one global
// FP64 atomic per non-zero bin, statistic and counter; the region is zeroed.
template <typename P>
__device__ __forceinline__ void flush_region(unsigned char *region, const LaunchArgs &a, int case_index,
                                             uint32_t batch, int lane) {
    const int nbs = a.t.nbins_stride;
    const int nb = a.cases[case_index].nbins;
    double *g = a.t.flux + ((size_t)case_index * a.t.nbatch + batch) * (size_t)nbs;
    if constexpr (kFixedBins<P>) {
        // the exact prefix sum of the fixed-point difference array, 32 bins at a
        // time; its entry nb (past the last bin) sums to zero and is cleared
        unsigned long long *D = region_fixed(region);
        unsigned long long carry = 0ull;
        for (int base = 0; base <= nb; base += 32) {
            const int k = base + lane;
            unsigned long long d = (k <= nb) ? D[k] : 0ull;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned long long v = __shfl_up_sync(CLS_FULL_MASK, d, o);
                if (lane >= o) d += v;
            }
            const long long q = (long long)(carry + d);  // the bin's deposits, 2^-32 units
            carry += __shfl_sync(CLS_FULL_MASK, d, 31);
            if (k < nb && q != 0) atomicAdd(&g[k], (double)q * 0x1p-32);
            if (k <= nb) D[k] = 0ull;
        }
    } else {
        double *bins = reinterpret_cast<double *>(region);
        for (int k = lane; k < nb; k += 32) {
            const double v = bins[k];
            if (v != 0.0) {
                atomicAdd(&g[k], v);
                bins[k] = 0.0;
            }
        }
    }
    // the lanes' own copies of the per-history statistics, summed over the warp
    LaneStat<P> *ls = region_lane_stats<P>(region, nbs);
#pragma unroll
    for (int q = 0; q < S_NUM; ++q) {
        double v;
        if constexpr (kFixedBins<P>)
            v = (q == S_T) ? (double)(ls[32 * S_TRACK0 + lane] + ls[32 * S_TRACK1 + lane]) * 0x1p-32
                           : (double)ls[32 * q + lane] * (q == S_T2 ? 0x1p-24 : 0x1p-32);
        else v = ls[32 * q + lane];
        ls[32 * q + lane] = 0;
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) v += __shfl_xor_sync(CLS_FULL_MASK, v, o);
        if (lane == 0 && __double_as_longlong(v) != 0) atomicAdd(&a.t.stats[(size_t)case_index * S_NUM + q], v);
    }
    double *st = region_stats<P>(region, nbs);
    if (lane < S_NUM) {
        const double v = st[lane];
        if (v != 0.0) {
            atomicAdd(&a.t.stats[(size_t)case_index * S_NUM + lane], v);
            st[lane] = 0.0;
        }
    } else if (lane < S_NUM + C_NUM) {
        const int c = lane - S_NUM;
        unsigned long long *ct = reinterpret_cast<unsigned long long *>(st + S_NUM);
        const unsigned long long v = ct[c];
        if (v != 0ull) {
            unsigned long long *gc = &a.t.counters[(size_t)case_index * C_NUM + c];
            if (c == C_MAXEV) atomicMax(gc, v);
            else atomicAdd(gc, v);
            ct[c] = 0ull;
        }
    }
    __syncwarp();
}

// Global chunk index -> run entry (runs are in chunk order).
__device__ __forceinline__ int find_run(const LaunchArgs &a, uint64_t ch) {
    int lo = 0, hi = a.nruns - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (a.runs[mid].chunk_begin <= ch) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// ------------------------------------------------- history-based tracker
// Persistent kernel.  Each warp claims chunks of consecutive histories from a
// global counter; a lane whose history ends immediately takes the next history
// of the warp's current chunk (ballot + prefix popcount), so lanes stay busy
// across history and chunk boundaries.  Each warp owns two shared-memory tally
// regions keyed by (case, batch); a region is flushed to global memory when
// its key changes, after flush_every histories, or when the warp retires.
// When a new key arrives while both regions still serve live histories, the
// older region is flushed and re-keyed, and its remaining histories score
// straight into the FP64 global tallies: the warp never waits for a straggler
// of a heavy-tailed history-length distribution.
// Launch bounds: FP32 blocks of 256 threads, 4 per SM (64 registers); the 3D
// box takes 4 blocks of 224 threads (history_threads_fp32: 72 registers hold
// its state without spills).  FP64 blocks of at most kHistoryBlockFp64 = 128
// threads, 5 per SM (102 registers, 20 warps), 6 (85 registers, 24 warps) for
// the one-dimensional walks (rod, slab, x-projected box), whose state fits:
// the FP64 walk is latency-bound, and more resident warps hide its
// integer-arithmetic and shared-memory latencies (measured: 5% faster for the
// x-projected box at 6, no gain for the 3D box, which would spill).
template <typename P, int G>
struct HistoryBounds {
    static constexpr int threads = kHistoryBlockFp64, blocks = (G == 1 || G == 11 || G == 13) ? 6 : 5;
};
template <int G>
struct HistoryBounds<float, G> {
    static constexpr int threads = history_threads_fp32(G), blocks = 4;
};

// WC: the instance for launches of short histories, in which many histories
// end in the same step and many flights touch the slab's faces.  Its
// history-end counters are summed over the warp first (warp_count; otherwise
// each lane adds its own, count_one), and its deposits skip the difference
// array's zero entries and the end markers past the mesh (warp_deposit's
// SKIP): a flight from x = 0 or to x = L, over whole bins at that end, needs
// one or two shared atomics instead of four, and the lanes born at x = 0 no
// longer queue on the same entries.  The mixed-geometry kernel serves batch
// sweeps and always takes it.  Measured on the 256-case sweep: 10% faster
// (rods 12%) for the summed counters, 6.7% more for the skipped entries; on
// the 3D box's 47-event histories the first costs 1% and the second 2%, so
// the host picks the instance per launch.  A template parameter rather than a
// runtime switch: carrying both paths measured 1% slower on the 3D box.
template <typename P, int G, bool WC = (G == 0)>
__global__ void __launch_bounds__(HistoryBounds<P, G>::threads, HistoryBounds<P, G>::blocks) history_kernel(const LaunchArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int rb = a.region_bytes;
    unsigned char *regions = smem + (size_t)warp * 2 * rb;
    for (int i = lane; i < 2 * rb / 8; i += 32) reinterpret_cast<unsigned long long *>(regions)[i] = 0ull;
    load_math_tables<P>(threadIdx.x, blockDim.x);
    if constexpr (sizeof(P) == 8) __syncthreads();
    __syncwarp();

    // warp-uniform feeding state
    int key_run0 = -1, key_run1 = -1;
    uint32_t key_batch0 = 0, key_batch1 = 0;
    int fed0 = 0, fed1 = 0;
    uint64_t cursor = 0, end = 0;  // history ids of the chunk being fed
    int feed_reg = 0, feed_run = 0;
    uint32_t feed_batch = 0;
    bool exhausted = false;

    // lane state: lreg is the lane's tally region, or 2 once that region was
    // handed to a newer key (the lane then scores into global memory)
    History<P> s;
    Flight<P> f;
    bool alive = false;
    int lreg = 0, lcase = 0;
    uint32_t lbatch = 0;
    const RoundKeys &key = a.rk;
    const unsigned lt_mask = (1u << lane) - 1u;

    while (true) {
        unsigned need = __ballot_sync(CLS_FULL_MASK, !alive);
        while (need != 0u && !exhausted) {
            if (cursor == end) {
                unsigned long long ch;
                if (lane == 0) ch = atomicAdd(a.chunk_counter, 1ull);
                ch = __shfl_sync(CLS_FULL_MASK, ch, 0);
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
                if (key_run0 == run && key_batch0 == batch) r = 0;
                else if (key_run1 == run && key_batch1 == batch) r = 1;
                if (r < 0) {
                    const bool live0 = __any_sync(CLS_FULL_MASK, alive && lreg == 0);
                    const bool live1 = __any_sync(CLS_FULL_MASK, alive && lreg == 1);
                    const int other = feed_reg ^ 1;
                    if (!(other ? live1 : live0)) r = other;
                    else if (!(feed_reg ? live1 : live0)) r = feed_reg;
                    else r = other;  // both referenced: evict the older region
                    const int old_run = r ? key_run1 : key_run0;
                    const uint32_t old_batch = r ? key_batch1 : key_batch0;
                    if (old_run >= 0) {
                        flush_region<P>(regions + r * rb, a, a.runs[old_run].case_index, old_batch, lane);
                        // lanes still walking a history of the old key go on in global memory
                        if (alive && lreg == r) lreg = 2;
                    }
                    if (r == 0) {
                        key_run0 = run;
                        key_batch0 = batch;
                        fed0 = 0;
                    } else {
                        key_run1 = run;
                        key_batch1 = batch;
                        fed1 = 0;
                    }
                }
                feed_reg = r;
                feed_run = run;
                feed_batch = batch;
                cursor = rc.first + local0;
                end = cursor + cnt;
            }
            const uint64_t avail = end - cursor;
            const uint32_t nneed = __popc(need);
            const uint32_t take = (avail < nneed) ? (uint32_t)avail : nneed;
            const uint32_t rank = __popc(need & lt_mask);
            if (((need >> lane) & 1u) && rank < take) {
                lcase = a.runs[feed_run].case_index;
                lreg = feed_reg;
                lbatch = feed_batch;
                source<P, G, true>(s, a.cases[lcase], key, cursor + rank);
                alive = true;
            }
            if (feed_reg == 0) fed0 += (int)take;
            else fed1 += (int)take;
            cursor += take;
            need = __ballot_sync(CLS_FULL_MASK, !alive);
        }
        if (!__any_sync(CLS_FULL_MASK, alive)) break;
        f.k0 = 0;
        f.k1 = -1;
        int out = -1;
        if (alive) {
            // directions of the lanes born in this round and of those that scattered in the last
            resolve_direction<P, G>(s, a.cases[lcase], key);
            out = step<P, false, G, true>(s, a.cases[lcase], key, a.max_events, f, nullptr);
        }
        const uint64_t goff =
            (lreg == 2) ? ((uint64_t)lcase * (uint64_t)a.t.nbatch + lbatch) * (uint64_t)a.t.nbins_stride : 0ull;
        warp_deposit<P, WC>(regions, rb, a.t.nbins_stride, lreg, a.t.flux, goff, f, lane);
        if (out >= 0) {
            record_outcome(a, lcase, s.h_lo, s.h_hi, out);
            if (lreg < 2) {
                if (!finish_history<P>(regions + lreg * rb, a.t.nbins_stride, s, lane))
                    add_history_stats_global<P>(a, lcase, s);
                if constexpr (!(WC || G == 0))
                    count_one(reinterpret_cast<unsigned long long *>(region_stats<P>(regions + lreg * rb, a.t.nbins_stride) + S_NUM),
                              out, s.n_coll, s.n_int, s.n_refl, s.events);
            } else {
                finish_history_global<P>(a, lcase, s, out, true);
            }
        }
        // short histories often end together: their counters are then summed
        // over the warp first (the host asks for it when a launch's cases average
        // few events per history, and always for the mixed-geometry kernel)
        if constexpr (WC || G == 0)
            warp_count<P>(regions, rb, a.t.nbins_stride, out >= 0 && lreg < 2, lreg, s, out, lane,
                          a.max_events < (1u << 27));
        if (out >= 0) alive = false;
        // only FP32 regions flush early (their float partial sums stay short);
        // the host sets no flush interval for FP64 regions
        if (sizeof(P) == 4 && a.flush_every) {
            if (fed0 >= a.flush_every) {
                __syncwarp();
                flush_region<P>(regions, a, a.runs[key_run0].case_index, key_batch0, lane);
                fed0 = 0;
            }
            if (fed1 >= a.flush_every) {
                __syncwarp();
                flush_region<P>(regions + rb, a, a.runs[key_run1].case_index, key_batch1, lane);
                fed1 = 0;
            }
        }
    }
    __syncwarp();
    if (key_run0 >= 0) flush_region<P>(regions, a, a.runs[key_run0].case_index, key_batch0, lane);
    if (key_run1 >= 0) flush_region<P>(regions + rb, a, a.runs[key_run1].case_index, key_batch1, lane);
}

// ------------------------------------------------------------ trace kernel
template <typename P>
__global__ void trace_kernel(const TraceArgs a) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const CaseParams &cp = a.cases[a.case_index];
    const RoundKeys key = make_round_keys(a.seed);
    load_math_tables<P>(0, 1);
    History<P> s;
    Flight<P> f;
    source<P>(s, cp, key, a.history);
    TraceSink tr{a.rows, a.cap, 0};
    while (step<P, true>(s, cp, key, a.max_events, f, &tr) < 0) {
    }
    *a.n_rows = tr.n;
}

}  // namespace cls
