// cls_event.cuh -- event-based tracker (structure-of-arrays particle bank).
#pragma once

#include "cls_device.cuh"

namespace cls {

template <typename P>
cudaError_t launch_event_impl(const LaunchArgs &, int, int, size_t, cudaStream_t) {
    return cudaErrorNotSupported;
}

}  // namespace cls
