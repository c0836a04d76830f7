// cls_case.h -- host-side case set-up shared by every entry point that takes
// case parameters (cls_create / cls_batch_create and cls_run_noalloc): the
// parameter check and the derived quantities the kernels read (CaseParams).
#pragma once

#include <algorithm>
#include <cmath>
#include <cstring>

#include "../../include/cls.h"
#include "cls_internal.h"

namespace cls {

constexpr int kMaxBins = 4096;

// (sigma0, sigma1, lambda0, lambda1, c0, c1, L, d, nbins): Sigma_i >= 0 and
// finite, Lambda_i > 0 and finite, 0 <= c_i <= 1 (c_i = Sigma_s,i / Sigma_i,
// paper Sec. 2), L > 0, a known geometry code, 1 <= nbins <= kMaxBins.
inline int validate_case(const double *p) {
    const double s0 = p[0], s1 = p[1], l0 = p[2], l1 = p[3], c0 = p[4], c1 = p[5], L = p[6];
    const double d = p[7], nb = p[8];
    auto finite = [](double v) { return std::isfinite(v); };
    if (!(finite(s0) && s0 >= 0 && finite(s1) && s1 >= 0)) return CLS_E_INVAL;
    if (!(finite(l0) && l0 > 0 && finite(l1) && l1 > 0)) return CLS_E_INVAL;
    if (!(c0 >= 0 && c0 <= 1 && c1 >= 0 && c1 <= 1)) return CLS_E_INVAL;
    if (!(finite(L) && L > 0)) return CLS_E_INVAL;
    if (!(d == 1.0 || d == 2.0 || d == 3.0 || d == 11.0 || d == 13.0)) return CLS_E_INVAL;
    if (!(nb >= 1 && nb <= kMaxBins && nb == std::floor(nb))) return CLS_E_INVAL;
    return CLS_OK;
}

// Rough events-per-history estimate, used only to order cases largest first:
// flights per unit path length times an estimate of the path length, which
// grows with the number of scatterings ~ 1/(1 - c) and with the size L.
inline double cost_estimate(const CaseParams &c) {
    const double p0 = c.p0, p1 = 1.0 - c.p0;
    const double sig = p0 * c.sigma[0] + p1 * c.sigma[1];
    const double rate = sig + p0 / c.lambda[0] + p1 / c.lambda[1];
    const double cbar = sig > 0 ? (p0 * c.c[0] * c.sigma[0] + p1 * c.c[1] * c.sigma[1]) / sig : 0.0;
    const double tau = sig * c.L;
    const double ncol = std::min(1.0 / std::max(1.0 - cbar, 1e-6), 1.0 + tau * tau);
    const double path = std::min(c.L, 1.0 / std::max(sig, 1e-12)) * (1.0 + ncol * std::min(1.0, tau));
    return 1.0 + rate * path;
}

// The kernels' view of one validated case: p_0 = Lambda_0 / (Lambda_0 +
// Lambda_1) (paper Sec. 2), the mesh width, FP32 copies, reciprocals and the
// integer thresholds of the draw comparisons.  Case k of a launch draws with
// Philox counter word 3 = case_id.
inline CaseParams make_case(const double *p, uint32_t case_id) {
    CaseParams c;
    std::memset(&c, 0, sizeof(c));
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
    c.case_id = case_id;
    for (int i = 0; i < 2; ++i) {
        c.thr_c53[i] = unit_threshold(c.c[i], 53);
        c.thr_c24[i] = (uint32_t)unit_threshold((double)c.c_f[i], 24);
    }
    c.thr_p053 = unit_threshold(c.p0, 53);
    c.thr_p024 = (uint32_t)unit_threshold((double)c.p0_f, 24);
    c.cost = cost_estimate(c);
    return c;
}

}  // namespace cls
