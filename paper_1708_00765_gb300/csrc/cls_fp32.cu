// cls_fp32.cu -- float instantiations of the CLS kernels.
#include "cls_device.cuh"
#include "cls_event.cuh"

namespace cls {

template <int G, bool DIF>
cudaError_t launch_history_gd(const LaunchArgs &a, int grid, int block, size_t smem, cudaStream_t s) {
    static std::atomic<unsigned long long> optin{0};
    const cudaError_t e = ensure_smem_optin(history_kernel<float, G, DIF>, optin);
    if (e != cudaSuccess) return e;
    history_kernel<float, G, DIF><<<grid, block, smem, s>>>(a);
    return cudaGetLastError();
}

// with or without the interior-bin difference array (LaunchArgs::dif)
template <int G>
cudaError_t launch_history_g(const LaunchArgs &a, int grid, int block, size_t smem, cudaStream_t s) {
    return a.dif ? launch_history_gd<G, true>(a, grid, block, smem, s) : launch_history_gd<G, false>(a, grid, block, smem, s);
}

template <int G>
cudaError_t occupancy_history_g(int block, size_t smem, int *blocks_per_sm, bool dif) {
    return dif ? occupancy_with_smem(blocks_per_sm, history_kernel<float, G, true>, block, smem)
               : occupancy_with_smem(blocks_per_sm, history_kernel<float, G, false>, block, smem);
}

// One instantiation per geometry (compile-time branches) plus the mixed one.
cudaError_t launch_history_fp32(const LaunchArgs &a, int grid, int block, size_t smem, cudaStream_t s, int geom) {
    switch (geom) {
    case 1: return launch_history_g<1>(a, grid, block, smem, s);
    case 2: return launch_history_g<2>(a, grid, block, smem, s);
    case 3: return launch_history_g<3>(a, grid, block, smem, s);
    case 11: return launch_history_g<11>(a, grid, block, smem, s);
    case 13: return launch_history_g<13>(a, grid, block, smem, s);
    default: return launch_history_g<0>(a, grid, block, smem, s);
    }
}

cudaError_t launch_event_fp32(const LaunchArgs &a, int grid, int block, size_t smem, cudaStream_t s, int geom) {
    return launch_event_impl<float>(a, grid, block, smem, s, geom);
}

cudaError_t launch_trace_fp32(const TraceArgs &a, cudaStream_t s) {
    trace_kernel<float><<<1, 32, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t occupancy_history_fp32(int block, size_t smem, int *blocks_per_sm, int geom, bool dif) {
    switch (geom) {
    case 1: return occupancy_history_g<1>(block, smem, blocks_per_sm, dif);
    case 2: return occupancy_history_g<2>(block, smem, blocks_per_sm, dif);
    case 3: return occupancy_history_g<3>(block, smem, blocks_per_sm, dif);
    case 11: return occupancy_history_g<11>(block, smem, blocks_per_sm, dif);
    case 13: return occupancy_history_g<13>(block, smem, blocks_per_sm, dif);
    default: return occupancy_history_g<0>(block, smem, blocks_per_sm, dif);
    }
}

cudaError_t occupancy_event_fp32(int block, size_t smem, int *blocks_per_sm, int geom, bool dif) {
    return occupancy_event_impl<float>(block, smem, blocks_per_sm, geom, dif);
}

}  // namespace cls
