// ccst_generic.cuh -- data structures of the general-size kernel (ccst_generic.cu), which
// tracks every frame shape the power-of-two kernel does not take (H, W from 8 to 256).
#pragma once

#include "ccst_kernels.cuh"

namespace ccst {

struct GenPlan {
    int H, W, u, M, h0, method, in_dtype;
    int H1, H2, W1, W2;     // H = H1 H2, W = W1 W2: the two levels of each DFT
    float eps, sense;
    int exhaustive;         // 1: the whole upsampled grid in double-float (verification)
    const dfc* wH;          // H:    e^{-2 pi i m / H}
    const dfc* wW;          // W:    e^{-2 pi i m / W}
    const dfc* uH;          // u H:  e^{+2 pi i m / (u H)}
    const dfc* uW;          // u W:  e^{+2 pi i m / (u W)}
    const float2* EY;       // H x M, FP32: e^{2 pi i ky' (jy - h0) / (uH)}, fftfreq-signed ky'
    const float2* EX;       // (W/2 + 1) x M, FP32: e^{2 pi i kx' (jx - h0) / (uW)} (kx = W/2: -W/2)
};

struct GenItem {
    const void* frame;
    long long pitch;
    long long out_index;
    int plan;
    int ref;
};

// Upsampled grids of at most this many points keep their FP32 values between the two passes.
constexpr int kGenGridKeep = 65536;

// Scratch of one CTA of the general-size kernel, in complex double-floats: X (H x Wh), the
// work array (max(H, M) x Wh), the operand plane (H x W double-floats), the inner DFT
// levels (H x W) and the FP32 grid values (M x M floats, if kept), Wh = W/2 + 1.
inline long long gen_scratch_stride(int H, int W, int M) {
    const long long Wh = W / 2 + 1, MM = (long long)M * M;
    return (long long)H * Wh + (long long)(H > M ? H : M) * Wh + ((long long)H * W + 1) / 2 + (long long)H * W +
           (MM <= kGenGridKeep ? (MM + 3) / 4 : 0);
}

// The two levels of an N-point DFT: N1 the largest divisor of N not above sqrt(N).
inline int gen_split(int N) {
    int n1 = 1;
    for (int d = 1; d * d <= N; ++d)
        if (N % d == 0) n1 = d;
    return n1;
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
    // frames the FP32 general-size kernel (ccst_mixed.cu) could not certify: items n ..
    // n + *fb_count - 1 of this launch are fb_items[0 ..] (null: none)
    const GenItem* fb_items;
    const unsigned* fb_count;
};

// Kernel addresses (ccst_generic.cu).
const void* track_generic_kernel_ptr();
const void* gen_init_tables_ptr();
const void* gen_frame_to_f32_ptr();
const void* gen_ref_rows_ptr();
const void* gen_ref_cols_ptr();
const void* gen_fill_synthetic_ptr();
const void* gen_init_grid_tables_ptr();

}  // namespace ccst
