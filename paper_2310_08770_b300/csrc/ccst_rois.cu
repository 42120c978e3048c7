// ccst_rois.cu -- persistent launches over ROIs of mixed sizes, each tracked against its
// own reference (a1-a7 per ROI, as in track_kernel).
//
// The host sorts the work items largest first and launches one kernel per side present
// (128, 64, 32, 16), each over its contiguous run of items. An item names its ROI's frame,
// its size class and its reference (resident spectra); CTAs take items from the launch's
// counter. The per-frame work is track_frame, the body of the batched kernel.
#include "ccst_kernels.cuh"

namespace ccst {

// CTAs per SM of a side's ROI kernel: track_kernel's count at 64 and 128 px. The 32 and
// 16 px bodies need far less shared memory, and with the registers capped at 80 and 64 a
// thread (a few hundred bytes of spills) three and four CTAs fit on an SM. Small frames are
// latency-bound and take the extra warps: 16 px ROIs alone 5.63 -> 6.66 M ROIs/s; 32 px
// alone unchanged, but the uneven mix, where its CTAs fill SMs beside the other sides'
// kernels, 4.72 -> 4.79 M. The arithmetic is unchanged, so the records are too.
constexpr int rois_min_ctas(int n) { return n == 32 ? 3 : n == 16 ? 4 : track_min_ctas(n, n); }

// kN: the side of every item of the launch, with the CTA size of track_kernel<kN, kN> (so
// that its records equal ccst_track's at that size); kTcOnly: the 128 x 128 class whose
// plan contracts on tcgen05 (g.tc), compiled without the warp-MMA stages. Each
// instantiation holds one side's body and reads that side's geometry g from the parameter
// space as track_kernel reads its own: a kernel that carried several sides' bodies, with
// the geometry in shared memory, lost time to instruction fetch.
template <int kN, bool kTcOnly>
__global__ void __launch_bounds__(track_threads(kN, kN), rois_min_ctas(kN)) track_rois_kernel(RoiBatch rb, Geom g) {
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
    Smem S = carve(g, ccst_smem);
    S.ref = &s_ref;
    track_setup<kN, kN>(g, S);
    tables_bar_init(S);
    if constexpr (kN == 128) {
        // Tensor Memory for the tensor-core contraction; one CTA per SM (the register file
        // is full), so the allocation never waits on another CTA
        tc_setup();
    }
    unsigned parity = 0;
    RoiItem it;
    while (next_item(&it) >= 0) {
        if (threadIdx.x == 0) {
            s_ref = rb.refs[it.ref];
            // a per-ROI reference is cold in L2; the product step reads it after the row FFTs
            prefetch_l2(s_ref.FE32, (size_t)kN * (kN / 2 + 1) * sizeof(float2));
        }
        __syncthreads();
        Batch b{};
        b.frames = it.frame;
        b.n = 1;
        b.pitch = it.pitch;
        b.vec_ok = it.vec_ok;
        b.out = rb.out;
        if (!track_frame<kN, kN, kTcOnly>(g, b, S, it.out_index, (const char*)it.frame, parity)) break;
    }
    if constexpr (kN == 128) tc_teardown();   // every exit path releases the columns
    pdl_wait();
}

const void* track_rois_kernel_ptr(int side, bool tc_only) {
    switch (side) {
        case 16: return (const void*)track_rois_kernel<16, false>;
        case 32: return (const void*)track_rois_kernel<32, false>;
        case 64: return (const void*)track_rois_kernel<64, false>;
        case 128: return tc_only ? (const void*)track_rois_kernel<128, true> : (const void*)track_rois_kernel<128, false>;
        default: return nullptr;
    }
}

}  // namespace ccst
