// cls_debug.cu -- diagnostic entry points: the device Philox next to CUDA's
// curand_Philox4x32_10 (called from CUDA's header, not restated), the device
// draw-to-uniform mapping, the FP64 walk's elementary functions and the FP32
// walk's fixed-point conversion.
#include <curand_kernel.h>

#include <vector>

#include "../../include/cls.h"
#include "cls_device.cuh"

namespace {

__global__ void philox_pair_kernel(const uint32_t *in, int n, uint32_t *ours, uint32_t *theirs) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint4 c = make_uint4(in[6 * i + 0], in[6 * i + 1], in[6 * i + 2], in[6 * i + 3]);
    const uint2 k = make_uint2(in[6 * i + 4], in[6 * i + 5]);
    const cls::RoundKeys rk = cls::make_round_keys(((uint64_t)k.y << 32) | k.x);
    const uint4 a = cls::philox4x32_10(c, rk);
    const uint4 b = curand_Philox4x32_10(c, k);
    ours[4 * i + 0] = a.x;
    ours[4 * i + 1] = a.y;
    ours[4 * i + 2] = a.z;
    ours[4 * i + 3] = a.w;
    theirs[4 * i + 0] = b.x;
    theirs[4 * i + 1] = b.y;
    theirs[4 * i + 2] = b.z;
    theirs[4 * i + 3] = b.w;
}

__global__ void uniform_kernel(uint64_t seed, uint32_t case_id, const uint64_t *h, const uint64_t *j, int n,
                               double *o64, float *o32) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const cls::RoundKeys key = cls::make_round_keys(seed);
    cls::History<double> s64;
    cls::History<float> s32;
    s64.h_lo = s32.h_lo = (uint32_t)h[i];
    s64.h_hi = s32.h_hi = (uint32_t)(h[i] >> 32);
    s64.cid = s32.cid = case_id;
    // the cached odd words come from the even draw before them
    const uint32_t jj = (uint32_t)j[i];
    s64.j = s32.j = jj & ~1u;
    double u64 = cls::draw(s64, key);
    float u32 = cls::draw(s32, key);
    if (jj & 1u) {
        u64 = cls::draw(s64, key);
        u32 = cls::draw(s32, key);
    }
    o64[i] = u64;
    o32[i] = u32;
}

__global__ void math_kernel(const uint64_t *k, int n, double *out) {
    cls::load_math_tables<double>(threadIdx.x, blockDim.x);
    __syncthreads();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double sn, cs;
    cls::sincos_2pi_shared(k[i], &sn, &cs);
    const uint32_t hi = (uint32_t)(k[i] >> 21), lo = (uint32_t)(k[i] << 11);  // words whose top 53 bits are k
    const double mu = cls::Real<double>::two_u_minus_one(hi, lo);
    double *o = out + 6 * (size_t)i;
    o[0] = -cls::exp_variate_shared(k[i]);
    o[1] = sn;
    o[2] = cs;
    o[3] = cls::Real<double>::uniform(hi, lo);
    o[4] = mu;
    o[5] = cls::Real<double>::recip(mu);
}
__global__ void fixed32_kernel(const float *c, int n, unsigned long long *out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    out[i] = cls::fixed32(c[i]);
}
}  // namespace

extern "C" int cls_debug_philox(const uint32_t *in, int n, uint32_t *ours, uint32_t *theirs) {
    if (!in || n < 1 || !ours || !theirs) return CLS_E_INVAL;
    uint32_t *d = nullptr;
    const size_t bytes = (size_t)n * (6 + 4 + 4) * sizeof(uint32_t);
    if (cudaMalloc(&d, bytes) != cudaSuccess) return CLS_E_NOMEM;
    uint32_t *din = d, *dours = d + 6 * (size_t)n, *dtheirs = dours + 4 * (size_t)n;
    cudaError_t e = cudaMemcpy(din, in, 6 * (size_t)n * sizeof(uint32_t), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        philox_pair_kernel<<<(n + 255) / 256, 256>>>(din, n, dours, dtheirs);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(ours, dours, 4 * (size_t)n * sizeof(uint32_t), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(theirs, dtheirs, 4 * (size_t)n * sizeof(uint32_t), cudaMemcpyDeviceToHost);
    cudaFree(d);
    return e == cudaSuccess ? CLS_OK : CLS_E_CUDA;
}

extern "C" int cls_debug_uniform(uint64_t seed, uint32_t case_id, const uint64_t *h, const uint64_t *j, int n,
                                 double *out64, float *out32) {
    if (!h || !j || n < 1) return CLS_E_INVAL;
    for (int i = 0; i < n; ++i)
        if (j[i] >= (1ull << 32)) return CLS_E_INVAL;
    uint64_t *dh = nullptr;
    if (cudaMalloc(&dh, (size_t)n * (2 * sizeof(uint64_t) + sizeof(double) + sizeof(float))) != cudaSuccess)
        return CLS_E_NOMEM;
    uint64_t *dj = dh + n;
    double *d64 = reinterpret_cast<double *>(dj + n);
    float *d32 = reinterpret_cast<float *>(d64 + n);
    cudaError_t e = cudaMemcpy(dh, h, n * sizeof(uint64_t), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(dj, j, n * sizeof(uint64_t), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        uniform_kernel<<<(n + 255) / 256, 256>>>(seed, case_id, dh, dj, n, d64, d32);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess && out64) e = cudaMemcpy(out64, d64, n * sizeof(double), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && out32) e = cudaMemcpy(out32, d32, n * sizeof(float), cudaMemcpyDeviceToHost);
    cudaFree(dh);
    return e == cudaSuccess ? CLS_OK : CLS_E_CUDA;
}

extern "C" int cls_debug_math(const uint64_t *k, int n, double *ln1m, double *sin2pi, double *cos2pi, double *u,
                              double *mu, double *recip_mu) {
    if (!k || n < 1) return CLS_E_INVAL;
    for (int i = 0; i < n; ++i)
        if (k[i] >= (1ull << 53)) return CLS_E_INVAL;
    uint64_t *dk = nullptr;
    if (cudaMalloc(&dk, (size_t)n * (sizeof(uint64_t) + 6 * sizeof(double))) != cudaSuccess) return CLS_E_NOMEM;
    double *dout = reinterpret_cast<double *>(dk + n);
    cudaError_t e = cudaMemcpy(dk, k, n * sizeof(uint64_t), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        math_kernel<<<(n + 255) / 256, 256>>>(dk, n, dout);
        e = cudaGetLastError();
    }
    std::vector<double> host(6 * (size_t)n);
    if (e == cudaSuccess) e = cudaMemcpy(host.data(), dout, host.size() * sizeof(double), cudaMemcpyDeviceToHost);
    cudaFree(dk);
    if (e != cudaSuccess) return CLS_E_CUDA;
    double *outs[6] = {ln1m, sin2pi, cos2pi, u, mu, recip_mu};
    for (int c = 0; c < 6; ++c)
        if (outs[c])
            for (int i = 0; i < n; ++i) outs[c][i] = host[6 * (size_t)i + c];
    return CLS_OK;
}

extern "C" int cls_debug_fixed32(const float *c, int n, unsigned long long *out) {
    if (!c || !out || n < 1) return CLS_E_INVAL;
    for (int i = 0; i < n; ++i)
        if (!(c[i] >= 0.0f && c[i] < 0x1p32f)) return CLS_E_INVAL;
    float *dc = nullptr;
    if (cudaMalloc(&dc, (size_t)n * (sizeof(float) + sizeof(unsigned long long)) + 8) != cudaSuccess)
        return CLS_E_NOMEM;
    unsigned long long *dout = reinterpret_cast<unsigned long long *>(
        (reinterpret_cast<uintptr_t>(dc + n) + 7) & ~static_cast<uintptr_t>(7));
    cudaError_t e = cudaMemcpy(dc, c, n * sizeof(float), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        fixed32_kernel<<<(n + 255) / 256, 256>>>(dc, n, dout);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(out, dout, n * sizeof(unsigned long long), cudaMemcpyDeviceToHost);
    cudaFree(dc);
    return e == cudaSuccess ? CLS_OK : CLS_E_CUDA;
}
