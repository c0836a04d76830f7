// cls_fp32.cu -- float instantiations of the CLS kernels.
#include "cls_device.cuh"
#include "cls_event.cuh"

namespace cls {

static bool g_history_attr_set = false;

cudaError_t launch_history_fp32(const LaunchArgs &a, int grid, int block, size_t smem, cudaStream_t s) {
    if (!g_history_attr_set) {
        cudaError_t e = cudaFuncSetAttribute(history_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        if (e != cudaSuccess) return e;
        g_history_attr_set = true;
    }
    history_kernel<float><<<grid, block, smem, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_event_fp32(const LaunchArgs &a, int grid, int block, size_t smem, cudaStream_t s) {
    return launch_event_impl<float>(a, grid, block, smem, s);
}

cudaError_t launch_trace_fp32(const TraceArgs &a, cudaStream_t s) {
    trace_kernel<float><<<1, 32, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t occupancy_history_fp32(int block, size_t smem, int *blocks_per_sm) {
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, history_kernel<float>, block, smem);
}

cudaError_t occupancy_event_fp32(int block, size_t smem, int *blocks_per_sm) {
    return occupancy_event_impl<float>(block, smem, blocks_per_sm);
}

}  // namespace cls
