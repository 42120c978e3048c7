// ccst_track_h128.cu -- the tracking kernel instantiated for frames 128 rows high.
#include "ccst_kernels.cuh"

namespace ccst {

template __global__ void track_kernel<128, 8>(Geom, Batch);
template __global__ void track_kernel<128, 16>(Geom, Batch);
template __global__ void track_kernel<128, 32>(Geom, Batch);
template __global__ void track_kernel<128, 64>(Geom, Batch);
template __global__ void track_kernel<128, 128>(Geom, Batch);
template __global__ void track_kernel<128, 128, true>(Geom, Batch);

const void* track_kernel_h128(int W) {
    switch (W) {
        case 8: return (const void*)track_kernel<128, 8>;
        case 16: return (const void*)track_kernel<128, 16>;
        case 32: return (const void*)track_kernel<128, 32>;
        case 64: return (const void*)track_kernel<128, 64>;
        case 128: return (const void*)track_kernel<128, 128>;
        default: return nullptr;
    }
}

const void* track_kernel_128_tc() { return (const void*)track_kernel<128, 128, true>; }

}  // namespace ccst
