// cls_fp64.cu -- double instantiations of the CLS kernels.  The FP64 walk makes
// the oracle's decisions draw for draw; its positions and distances agree with
// the oracle's to rounding (fused multiply-adds, reciprocals).
#include "cls_device.cuh"
#include "cls_event.cuh"

namespace cls {

// Internal linkage: the other precision's translation unit has a launcher of the
// same name and signature, and two external definitions would be merged by the
// linker into one (whichever it keeps, launching the other precision's kernel).
namespace {

template <int G>
cudaError_t launch_history_g(const LaunchArgs &a, int grid, int block, size_t smem, cudaStream_t s) {
    if (G != 0 && a.warp_counts) {
        static std::atomic<unsigned long long> optin_wc{0};
        const cudaError_t e = ensure_smem_optin(history_kernel<double, G, true>, optin_wc);
        if (e != cudaSuccess) return e;
        history_kernel<double, G, true><<<grid, block, smem, s>>>(a);
        return cudaGetLastError();
    }
    static std::atomic<unsigned long long> optin{0};
    const cudaError_t e = ensure_smem_optin(history_kernel<double, G>, optin);
    if (e != cudaSuccess) return e;
    history_kernel<double, G><<<grid, block, smem, s>>>(a);
    return cudaGetLastError();
}

}  // namespace

// One instantiation per geometry (compile-time branches) plus the mixed one.
cudaError_t launch_history_fp64(const LaunchArgs &a, int grid, int block, size_t smem, cudaStream_t s, int geom) {
    switch (geom) {
    case 1: return launch_history_g<1>(a, grid, block, smem, s);
    case 2: return launch_history_g<2>(a, grid, block, smem, s);
    case 3: return launch_history_g<3>(a, grid, block, smem, s);
    case 11: return launch_history_g<11>(a, grid, block, smem, s);
    case 13: return launch_history_g<13>(a, grid, block, smem, s);
    default: return launch_history_g<0>(a, grid, block, smem, s);
    }
}

cudaError_t launch_event_fp64(const LaunchArgs &a, int grid, int block, size_t smem, cudaStream_t s, int geom) {
    return launch_event_impl<double>(a, grid, block, smem, s, geom);
}

cudaError_t launch_trace_fp64(const TraceArgs &a, cudaStream_t s) {
    trace_kernel<double><<<1, 32, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t occupancy_history_fp64(int block, size_t smem, int *blocks_per_sm, int geom) {
    switch (geom) {
    case 1: return occupancy_with_smem(blocks_per_sm, history_kernel<double, 1>, block, smem);
    case 2: return occupancy_with_smem(blocks_per_sm, history_kernel<double, 2>, block, smem);
    case 3: return occupancy_with_smem(blocks_per_sm, history_kernel<double, 3>, block, smem);
    case 11: return occupancy_with_smem(blocks_per_sm, history_kernel<double, 11>, block, smem);
    case 13: return occupancy_with_smem(blocks_per_sm, history_kernel<double, 13>, block, smem);
    default: return occupancy_with_smem(blocks_per_sm, history_kernel<double, 0>, block, smem);
    }
}

int event_bank_fields(int precision) {
    return precision == 0 ? BankLayout<double>::kFields : BankLayout<float>::kFields;
}

cudaError_t occupancy_event_fp64(int block, size_t smem, int *blocks_per_sm, int geom) {
    return occupancy_event_impl<double>(block, smem, blocks_per_sm, geom);
}

}  // namespace cls
