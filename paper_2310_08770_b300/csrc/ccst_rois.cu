// ccst_rois.cu -- one persistent launch over ROIs of mixed sizes, each tracked against its
// own reference (a1-a7 per ROI, as in track_kernel).
//
// CTAs take work items from a counter. An item names its ROI's frame, its size class (a
// plan: tables and geometry for one square size) and its reference (resident spectra).
// When a CTA's next item has another size class, it re-carves shared memory for that size,
// rebuilds the twiddles and re-initialises its table barrier; items are ordered largest
// first, so a CTA changes size a few times at most. The per-frame work is track_frame, the
// body of the batched kernel.
#include "ccst_kernels.cuh"

namespace ccst {

__device__ __forceinline__ void bar_inval(const Smem& S) {
    if (threadIdx.x == 0) {
        const unsigned b = (unsigned)__cvta_generic_to_shared(S.bar);
        asm volatile("mbarrier.inval.shared::cta.b64 [%0];\n" ::"r"(b) : "memory");
    }
}

// kSmall: the instantiation for classes up to 64 x 64, with the CTA shape of
// track_kernel<64, 64> (so that its records equal ccst_track's at those sizes).
template <bool kSmall>
__global__ void __launch_bounds__(kSmall ? track_threads(64, 64) : kThreads, kSmall ? track_min_ctas(64, 64) : 1)
    track_rois_kernel(RoiBatch rb) {
    __shared__ Geom sg;
    __shared__ long long s_item;
    int cur = -1;                      // size class of the current set-up
    unsigned parity = 0;
    Smem S{};
    // Tensor Memory for the 128 x 128 class's tensor-core contraction; one CTA per SM (the
    // register file is full), so the allocation never waits on another CTA
    if constexpr (!kSmall) tc_setup();
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) s_item = (long long)atomicAdd(rb.next, 1u);
        __syncthreads();
        const long long i = s_item;
        if (i >= rb.n) break;
        const RoiItem it = rb.items[i];
        if (it.cls != cur) {
            if (cur >= 0) bar_inval(S);
            if (threadIdx.x == 0) sg = rb.geoms[it.cls];
            __syncthreads();
            S = carve(sg, ccst_smem);
            switch (sg.H) {
                case 16: track_setup<16, 16>(sg, S); break;
                case 32: track_setup<32, 32>(sg, S); break;
                case 64: track_setup<64, 64>(sg, S); break;
                default:
                    if constexpr (!kSmall) track_setup<128, 128>(sg, S);
                    break;
            }
            tables_bar_init(S);
            parity = 0;
            cur = it.cls;
        }
        if (threadIdx.x == 0) {
            const RefSpectra r = rb.refs[it.ref];
            sg.FE32 = r.FE32;
            sg.FE64 = r.FE64;
            sg.b64 = r.b64;
            sg.FEdf = r.FEdf;
        }
        __syncthreads();
        Batch b{};
        b.frames = it.frame;
        b.n = 1;
        b.pitch = it.pitch;
        b.vec_ok = it.vec_ok;
        b.out = rb.out;
        bool ok;
        const char* frame = (const char*)it.frame;
        switch (sg.H) {
            case 16: ok = track_frame<16, 16>(sg, b, S, it.out_index, frame, parity); break;
            case 32: ok = track_frame<32, 32>(sg, b, S, it.out_index, frame, parity); break;
            case 64: ok = track_frame<64, 64>(sg, b, S, it.out_index, frame, parity); break;
            default:
                if constexpr (!kSmall) ok = track_frame<128, 128>(sg, b, S, it.out_index, frame, parity);
                else ok = false;              // never given to this instantiation
                break;
        }
        if (!ok) break;
    }
    if constexpr (!kSmall) tc_teardown();
}

const void* track_rois_kernel_ptr(bool small) {
    return small ? (const void*)track_rois_kernel<true> : (const void*)track_rois_kernel<false>;
}

}  // namespace ccst
