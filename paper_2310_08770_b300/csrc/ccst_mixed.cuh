// ccst_mixed.cuh -- plan and launch arguments of the general-size FP32 kernel
// (ccst_mixed.cu): square sides 48, 96, 192 and 256, whose FFT lengths factor into 2s and
// 3s. One frame per cluster of CL CTAs (1 for 48 and 96, 2 for 192, 4 for 256): each CTA
// owns H/CL rows for the row transforms and a band of about (W/2 + 1)/CL spectrum columns
// for everything after them, and the CTAs exchange rows and columns through distributed
// shared memory. Frames whose FP32 decisions the guard levels cannot certify are appended
// to a fallback list that the double-float general-size kernel (ccst_generic.cu) then
// tracks, so every record is either certified FP32 or the double-float path's own.
#pragma once

#include "ccst_generic.cuh"

namespace ccst {

constexpr unsigned kRMixed = 0x100u;   // record flag: tracked by the general-size FP32 kernel

struct MixPlan {
    int H, W, L, Wc, Hh;        // L = W/2, Wc = W/2 + 1, Hh = H/2
    int CL, KB;                 // CTAs per frame, spectrum columns per CTA (the last may have fewer)
    int NT;                     // threads per CTA
    int u, M, h0, pmax, TX;     // grid offsets t in [-h0, pmax]; TX = h0 + 1 (tx = 0..h0)
    int method, in_dtype;
    float eps, sense;
    float tau_int, tau0, tau1;  // guard thresholds, relative to sum w|X|
    int RSX, RSG, G;            // row strides (float2) of the band and staging buffers; staged rows
    int TC;                     // t rows per contraction chunk
    int TAp, TXp;               // row lengths of the stage-A (t) and stage-B (tx) tables
    int tbs;                    // one-CTA sides: the stage-B table is copied into shared memory
                                //   each frame, beside a t chunk small enough that the work
                                //   area keeps its size
    int off_w, off_small, smem; // shared-memory carve: band, work area, small arrays (bytes)
    const float2* t4h;          // H: W_H^{n2 k1} [k1][n2] (column FFT)
    const float2* t4r;          // L: W_L^{n2 k1} [k1][n2] (half-length row FFT)
    const float2* rtw;          // L/2 + 1: e^{-2 pi i k / W}
    const float2* phH;          // H: e^{2 pi i m / H}
    const float2* phW;          // W: e^{2 pi i m / W}
    const float2* tA;           // [Hh][TAp]: (cos(2 pi m t/(uH)) - 1, sin(2 pi m t/(uH))), m = i + 1, t = t' + 1
    const float2* tB;           // [Wc][TXp]: (g cos(2 pi kx' tx/(uW)), g sin(.)), g = fold weight
    const float* tG;            // [Wc][TXp]: g (cos(2 pi kx' tx/(uW)) - 1)
    // the double-float level: twiddles as double-floats, the phase tables e^{+2 pi i m/(uH)}
    // (m < uH) and e^{+2 pi i m/(uW)} (m < uW) of the double-float kernel's plan, staged rows
    // per group, and its shared-memory carve (spectrum band at 0, staging, candidate sums)
    const dfc* t4h_d;
    const dfc* t4r_d;
    const dfc* rtw_d;
    const dfc* uHd;
    const dfc* uWd;
    int G2, off_l2s, off_l2c;
};

struct MixArgs {
    const GenItem* items;       // the work list (device), or null: a uniform batch
    long long first, n;         // items[first, first + n), or frames 0 .. n-1 of the uniform batch
    const void* frames;         // uniform batch: frame i at frames + i * frame_bytes
    long long frame_bytes, pitch;
    int plan, ref;              // uniform batch: plan and reference ids (general-size numbering)
    MixPlan p;
    const dfc* const* refs;     // per reference: the half spectrum F[b], H x Wc double-floats
    Result* out;
    unsigned* next;             // item counter, zero at launch
    GenItem* fb;                // fallback list (capacity >= n) and its count
    unsigned* fb_count;
    float* dbg_int;             // optional: n x H x W integer surfaces (unnormalised)
    float* dbg_sub;             // optional: n x M x M peak-relative upsampled surfaces (unnormalised)
    const int* dbg_pairs;       // optional: n x 2 grid indices (ja, jb): only v(jb) - v(ja) by the
    float* dbg_d32;             //   pair-difference level is computed, into dbg_d32 (no record)
};

// Diagnostic outputs of a general-size launch (tests only).
struct MixDbg {
    float* dbg_int;
    float* dbg_sub;
    const int* pairs;
    float* d32;
};

// Shapes with an FP32 kernel (H x W: the squares 48, 96, 192, 256 and the paper's Table I
// shape 256 x 128 both ways), and their CTAs per frame.
inline bool mix_shape_ok(int H, int W) {
    return (H == W && (H == 48 || H == 96 || H == 192 || H == 256)) || (H == 256 && W == 128) ||
           (H == 128 && W == 256);
}
__host__ __device__ constexpr int mix_cluster(int H, int W) { return H * W <= 96 * 96 ? 1 : H * W <= 192 * 192 ? 2 : 4; }

// Kernel address for an H x W plan (null if none), and the plan's tables and layout: fills
// every field of *p from (H, W, u, method, in_dtype, eps) and uploads the tables into one
// device block that the caller owns (*mem). Returns 0, or -1 if the shape or u has no FP32
// kernel (the caller keeps the double-float path alone), or a CUDA error code.
const void* mix_kernel_ptr(int H, int W);
int mix_plan_create(int H, int W, int u, int method, int in_dtype, float eps, float tau_int, float tau0,
                    float tau1, int smem_optin, MixPlan* p, void** mem);

}  // namespace ccst
