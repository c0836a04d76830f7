// cls_fp64.cu -- double instantiations of the CLS kernels.  The FP64 walk makes
// the oracle's decisions draw for draw; its positions and distances agree with
// the oracle's to rounding (fused multiply-adds, reciprocals).
#include "cls_device.cuh"
#include "cls_event.cuh"

namespace cls {

static bool g_history_attr_set = false;

cudaError_t launch_history_fp64(const LaunchArgs &a, int grid, int block, size_t smem, cudaStream_t s) {
    if (!g_history_attr_set) {
        cudaError_t e = cudaFuncSetAttribute(history_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        if (e != cudaSuccess) return e;
        g_history_attr_set = true;
    }
    history_kernel<double><<<grid, block, smem, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_event_fp64(const LaunchArgs &a, int grid, int block, size_t smem, cudaStream_t s) {
    return launch_event_impl<double>(a, grid, block, smem, s);
}

cudaError_t launch_trace_fp64(const TraceArgs &a, cudaStream_t s) {
    trace_kernel<double><<<1, 32, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t occupancy_history_fp64(int block, size_t smem, int *blocks_per_sm) {
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, history_kernel<double>, block, smem);
}

size_t event_block_bytes() { return (sizeof(EventBlock) + 15) & ~(size_t)15; }

int event_bank_fields(int precision) {
    return precision == 0 ? BankLayout<double>::kFields : BankLayout<float>::kFields;
}

cudaError_t occupancy_event_fp64(int block, size_t smem, int *blocks_per_sm) {
    return occupancy_event_impl<double>(block, smem, blocks_per_sm);
}

}  // namespace cls
