// cls_intmath.h -- the elementary functions of the FP64 walk's draws, in
// 64/128-bit integer arithmetic: the exponential variate -ln(1 - u) and the
// pair (sin, cos) of 2 pi u, for u = k 2^-53.
//
// The walk draws two distances per event, l_c = -ln(1 - u)/Sigma_m and
// l_i = -Lambda_m ln(1 - u) (paper Sec. 4), and the azimuth 2 pi u of every
// new 3D direction (Sec. 4.3).  On GB300 the FP64 pipe is the walk's
// bottleneck while the integer pipes idle, so these are evaluated in fixed
// point:
//  * the logarithm by the table-driven reduction of Tang (ACM TOMS 16, 1990)
//    with an exact 64-bit product for the reduced argument, the Taylor series
//    of ln(1 + r) by Horner's rule in Q31/Q63 (precision tapered to what each
//    term needs), the sum in 128-bit fixed point with 120 fraction bits, and
//    one rounding to the nearest double: within one ulp;
//  * sine and cosine by angle addition from the nearest of 256 tabulated
//    angles (|delta| <= pi/256) with the Taylor series of sin(delta) and
//    cos(delta) - 1, in Q62-Q69 fixed point: absolute error below 2^-60 before
//    the final rounding to double.
//
// Host and device compile the same code (the host build serves tests).
#pragma once

#include <stdint.h>
#include <math.h>
#include <string.h>

#include "cls_math_tables.h"

#ifdef __CUDACC__
#define CLS_HD __host__ __device__ __forceinline__
#else
#define CLS_HD static inline
#endif

namespace cls {

struct U128 {
    uint64_t lo, hi;
};

CLS_HD uint64_t umulhi64(uint64_t a, uint64_t b) {
#ifdef __CUDA_ARCH__
    return __umul64hi(a, b);
#else
    return (uint64_t)(((unsigned __int128)a * b) >> 64);
#endif
}

CLS_HD int64_t smulhi64(int64_t a, int64_t b) {
#ifdef __CUDA_ARCH__
    return __mul64hi(a, b);
#else
    return (int64_t)(((__int128)a * b) >> 64);
#endif
}

CLS_HD int clz64(uint64_t x) {  // x != 0
#ifdef __CUDA_ARCH__
    return __clzll((long long)x);
#else
    return __builtin_clzll(x);
#endif
}

CLS_HD double bits_to_double(uint64_t b) {
#ifdef __CUDA_ARCH__
    return __longlong_as_double((long long)b);
#else
    double d;
    memcpy(&d, &b, sizeof d);
    return d;
#endif
}

// floor(a b / 2^63) for signed Q63 operands
CLS_HD int64_t mulq63(int64_t a, int64_t b) {
    return (int64_t)(((uint64_t)smulhi64(a, b) << 1) | (((uint64_t)a * (uint64_t)b) >> 63));
}

// floor(a b / 2^63), unsigned
CLS_HD uint64_t umulq63(uint64_t a, uint64_t b) {
    return (umulhi64(a, b) << 1) | ((a * b) >> 63);
}

// m 2^-scale rounded to the nearest double (ties to even), for m != 0
CLS_HD double u128_to_double(U128 m, int scale) {
    const bool big = m.hi != 0;
    const int lz = big ? clz64(m.hi) : 64 + clz64(m.lo);
    // shift the leading one to bit 127
    const int sh = lz & 63;
    uint64_t hi = big ? m.hi : m.lo;
    uint64_t lo = big ? m.lo : 0ull;
    if (sh) {
        hi = (hi << sh) | (lo >> (64 - sh));
        lo <<= sh;
    }
    uint64_t mant = hi >> 11;  // 53 bits, leading one at bit 52
    const uint64_t round = (hi >> 10) & 1ull;
    const uint64_t sticky = (hi & 0x3FFull) | lo;
    mant += round & ((sticky != 0ull ? 1ull : 0ull) | (mant & 1ull));
    // value in [2^(127 - lz - scale), 2^(128 - lz - scale)); a carry out of
    // the rounding moves into the exponent field
    const uint64_t ex = (uint64_t)(127 - lz - scale + 1023 - 1);
    return bits_to_double((ex << 52) + mant);
}

// Tables in the memory the caller reads them from (shared memory on the GPU).
struct IntLogTables {
    const uint16_t *n;      // N_i
    const uint64_t (*t)[2]; // T_i 2^120, {low, high}
};

// -ln(1 - u) >= 0 for u = k 2^-53, 0 <= k < 2^53.
CLS_HD double exp_variate(uint64_t k, IntLogTables tab) {
    if (k == 0ull) return 0.0;
    if (k < (1ull << 44)) {
        // u < 2^-9: -ln(1 - u) = u (1 + v), v = u G(u),
        // G = 1/2 + u/3 + u^2/4 + u^3/5 + u^4/6 + u^5/7 (next term below 2^-66)
        const uint64_t U = k << 10;  // u 2^63, exact
        const uint32_t u31 = (uint32_t)(U >> 32);
        const uint32_t g4 = 0x15555555u + (uint32_t)(((uint64_t)u31 * 0x12492492u) >> 31);  // 1/6 + u/7
        const uint32_t g3 = 0x1999999Au + (uint32_t)(((uint64_t)u31 * g4) >> 31);          // 1/5 + u g4
        const uint64_t g2 = (1ull << 61) + umulq63(U, (uint64_t)g3 << 32);                 // 1/4 + u g3
        const uint64_t g1 = 0x2AAAAAAAAAAAAAABull + umulq63(U, g2);                        // 1/3 + u g2
        const uint64_t g = (1ull << 62) + umulq63(U, g1);                                  // 1/2 + u g1
        const uint64_t W = (1ull << 63) + umulq63(U, g);                                   // (1 + v) 2^63
        const U128 m = {k * W, umulhi64(k, W)};                                            // u (1 + v) 2^116
        return u128_to_double(m, 116);
    }
    // 1 - u = n 2^-53 = (1 + f) 2^(p - 53); N_i from the top 8 bits of f
    const uint64_t n = (1ull << 53) - k;
    const int lz = clz64(n);                  // 11 .. 63
    const uint64_t nn = n << (lz - 11);       // (1 + f) 2^52
    const int i = (int)(nn >> 44) & 255;
    const int E = lz - 10;                    // 53 - p >= 1
    // r = (1 + f) N_i / 2048 - 1, exactly, in Q63; |r| < 2^-8.6
    const int64_t R = (int64_t)(nn * (uint64_t)tab.n[i] - (1ull << 63));
    // ln(1 + r) = r + r^2 P(r), P = -1/2 + r/3 - r^2/4 + r^3/5 - r^4/6 + r^5/7
    // (next term below 2^-69), in Estrin's grouping (G. Estrin, Proc. Western
    // Joint Computer Conference, 1960): P = q0 + r^2 q1 + r^4 q2 with
    // q0 = -1/2 + r/3, q1 = -1/4 + r/5, q2 = -1/6 + r/7, so that the products
    // do not form one long dependent chain.  rq = R + R^2 P needs P to 2^-46
    // (|r| < 2^-8.6): q0 in Q63; q1 (times r^2 < 2^-17) and q2 (times
    // r^4 < 2^-34) in Q31, their products with r^2 2^47 and r^4 2^62 in 32 bits.
    const int32_t r31 = (int32_t)(R >> 32);
    const int64_t r2 = mulq63(R, R);                                                   // r^2 2^63
    const int64_t q0 = -(1ll << 62) + mulq63(R, 0x2AAAAAAAAAAAAAABll);                 // -1/2 + r/3
    const int32_t q1 = -0x20000000 + (int32_t)(((int64_t)r31 * 0x1999999A) >> 31);    // -1/4 + r/5
    const int32_t q2 = -0x15555555 + (int32_t)(((int64_t)r31 * 0x12492492) >> 31);    // -1/6 + r/7
    const int32_t r2s = (int32_t)(r2 >> 16);                                           // r^2 2^47
    const int32_t r4s = (int32_t)(((int64_t)r2s * r2s) >> 32);                         // r^4 2^62
    const int64_t P = q0 + (((int64_t)q1 * r2s) >> 15) + (((int64_t)q2 * r4s) >> 30);  // Q63
    const int64_t rq = R + mulq63(r2, P);                                              // ln(1 + r) 2^63
    // ln(1 - u) 2^120 = T_i - E ln2 + rq 2^57, two's complement (negative)
    const uint64_t t_lo = tab.t[i][0], t_hi = tab.t[i][1];
    const uint64_t e_lo = CLS_LN2_Q120_LO * (uint64_t)E;
    const uint64_t e_hi = CLS_LN2_Q120_HI * (uint64_t)E + umulhi64(CLS_LN2_Q120_LO, (uint64_t)E);
    uint64_t s_lo = t_lo - e_lo;
    uint64_t s_hi = t_hi - e_hi - (t_lo < e_lo ? 1ull : 0ull);
    const uint64_t a_lo = (uint64_t)rq << 57;
    const uint64_t a_hi = (uint64_t)(rq >> 7);
    const uint64_t x_lo = s_lo + a_lo;
    s_hi += a_hi + (x_lo < s_lo ? 1ull : 0ull);
    s_lo = x_lo;
    // magnitude -s
    const U128 m = {0ull - s_lo, ~s_hi + (s_lo == 0ull ? 1ull : 0ull)};
    return u128_to_double(m, 120);
}

// v 2^-62 rounded to the nearest double, for a signed Q62 value v
CLS_HD double q62_to_double(int64_t v) {
    if (v == 0) return 0.0;
    const uint64_t sgn = v < 0 ? (1ull << 63) : 0ull;
    const uint64_t a = v < 0 ? 0ull - (uint64_t)v : (uint64_t)v;
    const int lz = clz64(a);
    const uint64_t x = a << lz;  // leading one at bit 63
    uint64_t mant = x >> 11;
    const uint64_t round = (x >> 10) & 1ull;
    const uint64_t sticky = x & 0x3FFull;
    mant += round & ((sticky != 0ull ? 1ull : 0ull) | (mant & 1ull));
    const uint64_t ex = (uint64_t)(63 - lz - 62 + 1023 - 1);
    return bits_to_double(sgn | ((ex << 52) + mant));
}

// (sin, cos) of 2 pi u for u = k 2^-53, 0 <= k < 2^53; sc: {sin, cos} of
// 2 pi j/256 times 2^62.
CLS_HD void sincos_2pi_int(uint64_t k, const int64_t (*sc)[2], double *sn, double *cs) {
    const uint64_t j = (k + (1ull << 44)) >> 45;           // nearest tabulated angle, 0..256
    const int64_t t = (int64_t)k - (int64_t)(j << 45);     // in [-2^44, 2^44)
    const int64_t S = sc[j & 255ull][0], C = sc[j & 255ull][1];
    // delta = 2 pi t 2^-53 in Q69 (|delta| < 2^-6.3)
    const int64_t dh = smulhi64(t, CLS_TWO_PI_Q60);
    const uint64_t dl = (uint64_t)t * (uint64_t)CLS_TWO_PI_Q60;
    const int64_t d = (int64_t)(((uint64_t)dh << 20) | (dl >> 44));
    const int64_t d2 = smulhi64(d, d) >> 11;                               // delta^2, Q63
    // sin(delta) = delta - delta d2 (1/6 - d2 (1/120 - d2/5040))
    // cos(delta) - 1 = -d2 (1/2 - d2 (1/24 - d2/720))
    // The inner terms need only 32-bit operands: b = 1/120 - d2/5040 (used
    // times delta d2^2 < 2^-31) in Q31, and the products d2 b and d2/720
    // (used times delta d2 < 2^-18, and d2^2 < 2^-25) from d2 2^43 and
    // 32-bit coefficients, each within 2^-43.
    const int32_t d2h = (int32_t)(d2 >> 20);                                            // d2 2^43
    const int32_t b31 = 0x01111111 - (int32_t)(((int64_t)d2h * 0x00068068) >> 43);       // 1/120 - d2/5040, Q31
    const int64_t a = 0x1555555555555555ll - (((int64_t)d2h * b31) >> 11);              // 1/6 - d2 b
    const int64_t sd = d - mulq63(mulq63(d, d2), a);                                    // Q69
    const int64_t e = 0x0555555555555555ll - (((int64_t)d2h * 0x002D82D8) >> 11);       // 1/24 - d2/720
    const int64_t h = (1ll << 62) - mulq63(d2, e);                                      // 1/2 - d2 e
    const int64_t cm1 = -mulq63(d2, h);                                        // Q63
    // sin(a + delta) = S + S cm1 + C sin(delta); cos(a + delta) = C + C cm1 - S sin(delta)  (Q62)
    const int64_t s_cm1 = mulq63(S, cm1), c_cm1 = mulq63(C, cm1);
    const int64_t c_sd = smulhi64(C, sd) >> 5, s_sd = smulhi64(S, sd) >> 5;   // (Q62 Q69) >> 69
    *sn = q62_to_double(S + s_cm1 + c_sd);
    *cs = q62_to_double(C + c_cm1 - s_sd);
}

// floor(a d / 2^62) for a in (0, 2^62] and signed d
CLS_HD int64_t mulq62(int64_t a, int64_t d) {
    return (int64_t)(((uint64_t)smulhi64(a, d) << 2) | (((uint64_t)a * (uint64_t)d) >> 62));
}

// 1/a for a normal double a: Newton-Raphson iteration for the reciprocal,
// y <- y + y (1 - m y) (each step squares the relative error; P. Markstein,
// IBM J. Res. Dev. 34, 1990), on the significand m in [1, 2) from the FP32
// approximate reciprocal of its leading 24 bits (relative error below 2^-22):
// one step in 32-bit arithmetic (to about 2^-30), one in Q62 fixed point (to
// about 2^-59), then one rounding to the nearest double: within an ulp of 1/a.
// Zero, subnormal, infinite and NaN a take the division.
CLS_HD double recip_int(double a) {
    uint64_t b;
#ifdef __CUDA_ARCH__
    b = (uint64_t)__double_as_longlong(a);
#else
    memcpy(&b, &a, sizeof b);
#endif
    const int ex = (int)((b >> 52) & 0x7FF);
    if (ex == 0 || ex == 0x7FF) return 1.0 / a;
    const uint64_t M = (b & 0xFFFFFFFFFFFFFull) | (1ull << 52);  // m 2^52
    // seed: y0 ~ 1/m in (1/2, 1], from m's leading 24 bits
    const uint32_t fb = 0x3F800000u | (uint32_t)((b >> 29) & 0x7FFFFFu);
    float mf, rf;
#ifdef __CUDA_ARCH__
    mf = __uint_as_float(fb);
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(rf) : "f"(mf));
#else
    memcpy(&mf, &fb, sizeof mf);
    rf = 1.0f / mf;
#endif
    uint32_t rb;
    memcpy(&rb, &rf, sizeof rb);
    const int re = (int)((rb >> 23) & 0xFF) - 127;                    // -1, or 0 when y0 = 1
    // first step in 32-bit arithmetic (y0 and m to 31 fraction bits): y1
    // within about 2^-30 of 1/m
    const uint32_t y31 = ((rb & 0x7FFFFFu) | 0x800000u) << (8 + re);  // y0 2^31, at most 2^31
    const uint32_t m31 = (uint32_t)(M >> 21);                         // m 2^31, truncated
    const int64_t e0 = (int64_t)((1ull << 62) - (uint64_t)m31 * y31);  // (1 - m y0) 2^62, |.| < 2^41
    int64_t y = (int64_t)((uint64_t)y31 << 31) + (int64_t)y31 * (e0 >> 31);  // y1 2^62
    // second step in Q62
    {
        const uint64_t hi = umulhi64(M, (uint64_t)y), lo = M * (uint64_t)y;
        const int64_t t = (int64_t)((hi << 12) | (lo >> 52));         // m y 2^62
        y += mulq62(y, (1ll << 62) - t);
    }
    // 1/|a| = y 2^-62 2^(1023 - ex), rounded to 53 bits
    const uint64_t x = (uint64_t)y;
    const int lz = clz64(x);
    const uint64_t n = x << lz;
    uint64_t mant = n >> 11;
    mant += ((n >> 10) & 1ull) & (((n & 0x3FFull) != 0ull ? 1ull : 0ull) | (mant & 1ull));
    const uint64_t e = (uint64_t)(63 - lz - 62 + (1023 - ex) + 1023 - 1);
    return bits_to_double((b & (1ull << 63)) | ((e << 52) + mant));
}

// sqrt(X 2^-scale) rounded to the nearest double, for 0 <= X < 2^127 and even
// scale: Newton-Raphson iteration for the reciprocal square root,
// y <- y + y (1 - v y^2)/2, on v = X 2^-2t in [1/4, 1) from the FP32
// approximate reciprocal square root of v's leading 24 bits (relative error
// below 2^-22): one step in 32-bit arithmetic (to about 2^-29), one in Q61
// fixed point, then sqrt(v) = v y and one rounding: within an ulp.
CLS_HD double sqrt_int(U128 X, int scale) {
    if ((X.hi | X.lo) == 0ull) return 0.0;
    // normalise by an even shift: v = X' 2^-128 in [1/4, 1)
    const int lz = X.hi ? clz64(X.hi) : 64 + clz64(X.lo);
    const int sh = lz & ~1;
    uint64_t h = X.hi, l = X.lo;
    if (sh >= 64) {
        h = l << (sh - 64);
    } else if (sh > 0) {
        h = (h << sh) | (l >> (64 - sh));
    }
    const uint64_t v = h;  // v 2^64: the top 64 bits of X' (the rest is below the rounding)
    // seed y0 ~ 1/sqrt(v) in (1, 2], Q61
    float vf = (float)(uint32_t)(v >> 40) * 0x1p-24f, yf;  // v's leading 24 bits, exactly
#ifdef __CUDA_ARCH__
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(yf) : "f"(vf));
#else
    yf = 1.0f / sqrtf(vf);
#endif
    uint32_t yb;
    memcpy(&yb, &yf, sizeof yb);
    const int ye = (int)((yb >> 23) & 0xFF) - 127;  // 0, or 1 when y0 = 2
    // first step in 32-bit arithmetic (y0 and v to 30 fraction bits): y1
    // within about 2^-29 of 1/sqrt(v)
    const uint32_t y30 = ((yb & 0x7FFFFFu) | 0x800000u) << (7 + ye);  // y0 2^30, at most 2^31
    const uint32_t v32 = (uint32_t)(v >> 32);                          // v 2^32, truncated
    const uint32_t vy30 = (uint32_t)(((uint64_t)v32 * y30) >> 32);     // v y0 2^30
    const int64_t e0 = (int64_t)((1ull << 60) - (uint64_t)vy30 * y30);  // (1 - v y0^2) 2^60
    int64_t y = (int64_t)((uint64_t)y30 << 31) + (int64_t)y30 * (e0 >> 30);  // y1 2^61
    // second step in Q61
    {
        const uint64_t vy = umulhi64(v, (uint64_t)y);                 // v y, Q61
        const int64_t t = (int64_t)(umulhi64(vy, (uint64_t)y) << 4);  // v y^2, Q62
        y += mulq62(y, ((1ll << 62) - t) >> 1);                      // + y (1 - v y^2)/2
    }
    const uint64_t q = umulhi64(v, (uint64_t)y);  // sqrt(v) = v y, Q61, in [2^60, 2^61]
    const int qz = clz64(q);
    const uint64_t n = q << qz;
    uint64_t mant = n >> 11;
    mant += ((n >> 10) & 1ull) & (((n & 0x3FFull) != 0ull ? 1ull : 0ull) | (mant & 1ull));
    // sqrt(X 2^-scale) = sqrt(v) 2^((128 - sh - scale)/2)
    const int e2 = (128 - sh - scale) / 2;
    const uint64_t e = (uint64_t)(63 - qz - 61 + e2 + 1023 - 1);
    return bits_to_double((e << 52) + mant);
}

}  // namespace cls
