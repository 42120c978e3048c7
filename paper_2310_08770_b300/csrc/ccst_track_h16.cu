// ccst_track_h16.cu -- the tracking kernel instantiated for frames 16 rows high.
#include "ccst_kernels.cuh"

namespace ccst {

template __global__ void track_kernel<16, 8>(Geom, Batch);
template __global__ void track_kernel<16, 16>(Geom, Batch);
template __global__ void track_kernel<16, 32>(Geom, Batch);
template __global__ void track_kernel<16, 64>(Geom, Batch);
template __global__ void track_kernel<16, 128>(Geom, Batch);

const void* track_kernel_h16(int W) {
    switch (W) {
        case 8: return (const void*)track_kernel<16, 8>;
        case 16: return (const void*)track_kernel<16, 16>;
        case 32: return (const void*)track_kernel<16, 32>;
        case 64: return (const void*)track_kernel<16, 64>;
        case 128: return (const void*)track_kernel<16, 128>;
        default: return nullptr;
    }
}

}  // namespace ccst
