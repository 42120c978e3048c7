// ccst_track_h8.cu -- the tracking kernel instantiated for frames 8 rows high.
#include "ccst_kernels.cuh"

namespace ccst {

template __global__ void track_kernel<8, 8>(Geom, Batch);
template __global__ void track_kernel<8, 16>(Geom, Batch);
template __global__ void track_kernel<8, 32>(Geom, Batch);
template __global__ void track_kernel<8, 64>(Geom, Batch);
template __global__ void track_kernel<8, 128>(Geom, Batch);

const void* track_kernel_h8(int W) {
    switch (W) {
        case 8: return (const void*)track_kernel<8, 8>;
        case 16: return (const void*)track_kernel<8, 16>;
        case 32: return (const void*)track_kernel<8, 32>;
        case 64: return (const void*)track_kernel<8, 64>;
        case 128: return (const void*)track_kernel<8, 128>;
        default: return nullptr;
    }
}

}  // namespace ccst
