// ccst_track_h32.cu -- the tracking kernel instantiated for frames 32 rows high.
#include "ccst_kernels.cuh"

namespace ccst {

template __global__ void track_kernel<32, 8>(Geom, Batch);
template __global__ void track_kernel<32, 16>(Geom, Batch);
template __global__ void track_kernel<32, 32>(Geom, Batch);
template __global__ void track_kernel<32, 64>(Geom, Batch);
template __global__ void track_kernel<32, 128>(Geom, Batch);

const void* track_kernel_h32(int W) {
    switch (W) {
        case 8: return (const void*)track_kernel<32, 8>;
        case 16: return (const void*)track_kernel<32, 16>;
        case 32: return (const void*)track_kernel<32, 32>;
        case 64: return (const void*)track_kernel<32, 64>;
        case 128: return (const void*)track_kernel<32, 128>;
        default: return nullptr;
    }
}

}  // namespace ccst
