// ccst_track_h64.cu -- the tracking kernel instantiated for frames 64 rows high.
#include "ccst_kernels.cuh"

namespace ccst {

template __global__ void track_kernel<64, 8>(Geom, Batch);
template __global__ void track_kernel<64, 16>(Geom, Batch);
template __global__ void track_kernel<64, 32>(Geom, Batch);
template __global__ void track_kernel<64, 64>(Geom, Batch);
template __global__ void track_kernel<64, 128>(Geom, Batch);

const void* track_kernel_h64(int W) {
    switch (W) {
        case 8: return (const void*)track_kernel<64, 8>;
        case 16: return (const void*)track_kernel<64, 16>;
        case 32: return (const void*)track_kernel<64, 32>;
        case 64: return (const void*)track_kernel<64, 64>;
        case 128: return (const void*)track_kernel<64, 128>;
        default: return nullptr;
    }
}

}  // namespace ccst
