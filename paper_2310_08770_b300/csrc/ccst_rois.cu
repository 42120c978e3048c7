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

// kClass: 0 for the size classes up to 64 x 64, with the CTA shape of track_kernel<64, 64>
// (so that its records equal ccst_track's at those sizes); 1 for the 128 x 128 class with
// both contraction forms; 2 for the 128 x 128 class whose plan contracts on tcgen05 (g.tc),
// compiled without the warp-MMA stages. Each instantiation holds only its own classes'
// bodies: a kernel that carried every size's body lost time to instruction fetch.
// g128: the 128 x 128 class's geometry (kClass 1 and 2), read from the parameter space as
// track_kernel reads its own; the small classes' geometries are copied to shared memory
// when a CTA changes class.
template <int kClass>
__global__ void __launch_bounds__(kClass == 0 ? track_threads(64, 64) : kThreads, kClass == 0 ? track_min_ctas(64, 64) : 1)
    track_rois_kernel(RoiBatch rb, Geom g128) {
    __shared__ long long s_item;
    __shared__ RefSpectra s_ref;       // the current item's reference
    auto next_item = [&](RoiItem* it) {
        __syncthreads();
        if (threadIdx.x == 0) s_item = (long long)atomicAdd(rb.next, 1u);
        __syncthreads();
        const long long i = s_item;
        // the last wave: every CTA takes at most one more item, so the kernel chained
        // behind this one may start filling the SMs that free up
        if (i >= rb.n - (long long)gridDim.x) pdl_trigger();
        if (i >= rb.n) return -1ll;
        *it = rb.items[i];
        return i;
    };
    auto item_ref = [&](const RoiItem& it, int H, int Wc) {
        if (threadIdx.x == 0) {
            s_ref = rb.refs[it.ref];
            // a per-ROI reference is cold in L2; the product step reads it after the row FFTs
            prefetch_l2(s_ref.FE32, (size_t)H * Wc * sizeof(float2));
        }
        __syncthreads();
    };
    auto item_batch = [&](const RoiItem& it) {
        Batch b{};
        b.frames = it.frame;
        b.n = 1;
        b.pitch = it.pitch;
        b.vec_ok = it.vec_ok;
        b.out = rb.out;
        return b;
    };
    unsigned parity = 0;
    if constexpr (kClass == 0) {
        __shared__ Geom sg;
        int cur = -1;                  // size class of the current set-up
        Smem S{};
        RoiItem it;
        while (next_item(&it) >= 0) {
            if (it.cls != cur) {
                if (cur >= 0) bar_inval(S);
                if (threadIdx.x == 0) sg = rb.geoms[it.cls];
                __syncthreads();
                S = carve(sg, ccst_smem);
                S.ref = &s_ref;
                switch (sg.H) {
                    case 16: track_setup<16, 16>(sg, S); break;
                    case 32: track_setup<32, 32>(sg, S); break;
                    default: track_setup<64, 64>(sg, S); break;
                }
                tables_bar_init(S);
                parity = 0;
                cur = it.cls;
            }
            item_ref(it, sg.H, sg.Wc);
            const Batch b = item_batch(it);
            const char* frame = (const char*)it.frame;
            bool ok;
            switch (sg.H) {
                case 16: ok = track_frame<16, 16>(sg, b, S, it.out_index, frame, parity); break;
                case 32: ok = track_frame<32, 32>(sg, b, S, it.out_index, frame, parity); break;
                default: ok = track_frame<64, 64>(sg, b, S, it.out_index, frame, parity); break;
            }
            if (!ok) break;
        }
    } else {
        // the one 128 x 128 class: set up once
        Smem S = carve(g128, ccst_smem);
        S.ref = &s_ref;
        track_setup<128, 128>(g128, S);
        tables_bar_init(S);
        // Tensor Memory for the tensor-core contraction; one CTA per SM (the register file
        // is full), so the allocation never waits on another CTA
        tc_setup();
        RoiItem it;
        while (next_item(&it) >= 0) {
            item_ref(it, 128, 65);
            if (!track_frame<128, 128, kClass == 2>(g128, item_batch(it), S, it.out_index, (const char*)it.frame,
                                                     parity))
                break;
        }
        tc_teardown();
    }
    pdl_wait();
}

const void* track_rois_kernel_ptr(int cls) {
    return cls == 0 ? (const void*)track_rois_kernel<0>
                    : cls == 1 ? (const void*)track_rois_kernel<1> : (const void*)track_rois_kernel<2>;
}

}  // namespace ccst
