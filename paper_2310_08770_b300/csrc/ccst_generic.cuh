// ccst_generic.cuh -- data structures of the general-size kernel (ccst_generic.cu), which
// tracks every frame shape the power-of-two kernel does not take (H, W from 8 to 256).
#pragma once

#include "ccst_kernels.cuh"

namespace ccst {

struct GenPlan {
    int H, W, u, M, h0, method, in_dtype;
    float eps, sense;
    const dfc* wH;          // H:    e^{-2 pi i m / H}
    const dfc* wW;          // W:    e^{-2 pi i m / W}
    const dfc* uH;          // u H:  e^{+2 pi i m / (u H)}
    const dfc* uW;          // u W:  e^{+2 pi i m / (u W)}
};

struct GenItem {
    const void* frame;
    long long pitch;
    long long out_index;
    int plan;
    int ref;
};

// Scratch of one CTA of the general-size kernel, in complex double-floats: X (H x Wh), the
// work array (max(H, M) x Wh) and the operand plane (H x W double-floats), Wh = W/2 + 1.
inline long long gen_scratch_stride(int H, int W, int M) {
    const long long Wh = W / 2 + 1;
    return (long long)H * Wh + (long long)(H > M ? H : M) * Wh + ((long long)H * W + 1) / 2;
}

struct GenBatch {
    const GenItem* items;    // the work list, or null: item i is frame i of a uniform batch
    long long n;
    const GenPlan* plans;
    const dfc* const* refs;  // per reference: the half spectrum F[b], H x (W/2 + 1) double-floats
    Result* out;
    unsigned* next;
    dfc* scratch;            // per CTA: scratch_stride complex double-floats
    long long scratch_stride;
    // uniform batch (items == null): frame i at frames + i * frame_bytes, row pitch `pitch`
    // elements, plan `plan`, reference `ref`, record i
    const void* frames;
    long long frame_bytes;
    long long pitch;
    int plan, ref;
};

// Kernel addresses (ccst_generic.cu).
const void* track_generic_kernel_ptr();
const void* gen_init_tables_ptr();
const void* gen_frame_to_f32_ptr();
const void* gen_ref_rows_ptr();
const void* gen_ref_cols_ptr();

}  // namespace ccst
