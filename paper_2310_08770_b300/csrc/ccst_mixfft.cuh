// ccst_mixfft.cuh -- mixed-radix (2, 3) FFT building blocks for the general-size FP32
// kernel (ccst_mixed.cu): register DFTs of 2, 3, 4, 6, 8, 12 and 16 points and in-place
// four-step passes over shared memory, in both directions.
//
// A length N = N1 N2 transform (Cooley-Tukey four-step):
//   forward, natural input x[N2 n1 + n2]:
//     pass S (strided): for each n2, the N1-point DFT over n1, result k1 times W_N^{n2 k1},
//       stored back at slot N2 k1 + n2;
//     pass C (contiguous): for each k1, the N2-point DFT over the slots N2 k1 + n2; output
//       X[k1 + N1 k2] lands at slot N2 k1 + k2, i.e. X[k] sits at mix_pos(k).
//   inverse, input X[k] at slot mix_pos(k) (the forward's output order):
//     pass C: for each k1, the N2-point inverse DFT over k2 (slots N2 k1 + k2); result n2
//       times W_N^{-n2 k1}, stored back at slot N2 k1 + n2;
//     pass S: for each n2, the N1-point inverse DFT over k1 (slots N2 k1 + n2); output
//       x[n2 + N2 n1] lands at slot N2 n1 + n2, the natural position.
// Both directions run in place and neither scales. Loads and stores go through functors,
// so that packing, products and scans fuse into the passes.
#pragma once

#include "ccst_fft.cuh"

namespace ccst {
namespace mix {

// Four-step factorisation of each supported length (N2 = 1: one register DFT, no pass C).
template <int N> struct MSplit;
template <> struct MSplit<3> { static constexpr int N1 = 3, N2 = 1; };
template <> struct MSplit<4> { static constexpr int N1 = 4, N2 = 1; };
template <> struct MSplit<6> { static constexpr int N1 = 6, N2 = 1; };
template <> struct MSplit<8> { static constexpr int N1 = 8, N2 = 1; };
template <> struct MSplit<12> { static constexpr int N1 = 12, N2 = 1; };
template <> struct MSplit<16> { static constexpr int N1 = 16, N2 = 1; };
template <> struct MSplit<24> { static constexpr int N1 = 8, N2 = 3; };
template <> struct MSplit<32> { static constexpr int N1 = 8, N2 = 4; };
template <> struct MSplit<48> { static constexpr int N1 = 12, N2 = 4; };
template <> struct MSplit<64> { static constexpr int N1 = 8, N2 = 8; };
template <> struct MSplit<96> { static constexpr int N1 = 12, N2 = 8; };
template <> struct MSplit<128> { static constexpr int N1 = 16, N2 = 8; };
template <> struct MSplit<192> { static constexpr int N1 = 16, N2 = 12; };
template <> struct MSplit<256> { static constexpr int N1 = 16, N2 = 16; };

template <int N>
__host__ __device__ constexpr int mix_pos(int k) {
    return MSplit<N>::N2 * (k % MSplit<N>::N1) + k / MSplit<N>::N1;
}
// padded physical slot of logical slot i in a shared-memory sequence: one gap after every
// N2 slots, so that the contiguous groups of pass C start on distinct banks
template <int N>
__host__ __device__ constexpr int mix_phys(int i) {
    return MSplit<N>::N2 > 1 ? i + i / MSplit<N>::N2 : i;
}
template <int N>
__host__ __device__ constexpr int mix_padded_len() {
    return MSplit<N>::N2 > 1 ? N + MSplit<N>::N1 : N;
}

// cos / sin of 2 pi k / 12, k = 0..5
__device__ __forceinline__ float c12(int k) {
    return k == 0 ? 1.0f : k == 1 ? 0.866025403784438647f : k == 2 ? 0.5f : k == 3 ? 0.0f
         : k == 4 ? -0.5f : -0.866025403784438647f;
}
__device__ __forceinline__ float s12(int k) {
    return k == 0 ? 0.0f : k == 1 ? 0.5f : k == 2 ? 0.866025403784438647f : k == 3 ? 1.0f
         : k == 4 ? 0.866025403784438647f : 0.5f;
}
// x * exp(-+ 2 pi i idx / 12) (forward: minus sign), idx a compile-time constant after unrolling
template <bool INV>
__device__ __forceinline__ float2 mul_w12(float2 x, int idx) {
    idx %= 12;
    if (idx >= 6) { x = make_float2(-x.x, -x.y); idx -= 6; }      // W^6 = -1
    if (idx == 0) return x;
    if (idx == 3) return INV ? make_float2(-x.y, x.x) : make_float2(x.y, -x.x);
    const float c = c12(idx), s = INV ? s12(idx) : -s12(idx);
    return make_float2(fmaf(x.x, c, -x.y * s), fmaf(x.x, s, x.y * c));
}

// 3-point DFT in place: X1,2 = a - (b + c)/2 -+ i (sqrt(3)/2)(b - c) (forward)
template <bool INV>
__device__ __forceinline__ void dft3(float2& a, float2& b, float2& c) {
    constexpr float kS3 = 0.866025403784438647f;
    const float2 s = cadd(b, c), d = csub(b, c);
    const float2 t = make_float2(fmaf(-0.5f, s.x, a.x), fmaf(-0.5f, s.y, a.y));
    const float2 r = INV ? make_float2(-kS3 * d.y, kS3 * d.x) : make_float2(kS3 * d.y, -kS3 * d.x);   // -+ i s3 d
    a = cadd(a, s);
    b = cadd(t, r);
    c = csub(t, r);
}

// In-register DFT of R points, natural order in and out (FP32; the double-float overload
// follows). 6 = 3 x 2 and 12 = 3 x 4 use the
// four-step split R = R1 R2 (R1-point DFTs over v[R2 n1 + n2], twiddles W_R^{n2 k1},
// R2-point DFTs, X[k1 + R1 k2] read from slot R2 k1 + k2); the powers of two are the
// radix-2/4 register DFTs of ccst_fft.cuh.
template <int R, bool INV>
__device__ __forceinline__ void mdft(float2 (&v)[R]) {
    if constexpr (R == 1) {
    } else if constexpr (R == 3) {
        dft3<INV>(v[0], v[1], v[2]);
    } else if constexpr (R == 6 || R == 12) {
        constexpr int R1 = 3, R2 = R / 3;
#pragma unroll
        for (int n2 = 0; n2 < R2; ++n2) dft3<INV>(v[n2], v[R2 + n2], v[2 * R2 + n2]);
#pragma unroll
        for (int k1 = 1; k1 < R1; ++k1)
#pragma unroll
            for (int n2 = 1; n2 < R2; ++n2) v[R2 * k1 + n2] = mul_w12<INV>(v[R2 * k1 + n2], n2 * k1 * (12 / R));
#pragma unroll
        for (int k1 = 0; k1 < R1; ++k1) {
            if constexpr (R2 == 2) dft2<INV>(v[R2 * k1], v[R2 * k1 + 1]);
            else dft4<INV>(v[R2 * k1], v[R2 * k1 + 1], v[R2 * k1 + 2], v[R2 * k1 + 3]);
        }
        float2 t[R];
#pragma unroll
        for (int i = 0; i < R; ++i) t[i] = v[i];
#pragma unroll
        for (int k1 = 0; k1 < R1; ++k1)
#pragma unroll
            for (int k2 = 0; k2 < R2; ++k2) v[k1 + R1 * k2] = t[R2 * k1 + k2];
    } else {
        dft_reg<R, INV>(v);
    }
}

// ------------------------------------------------------------------ double-float
// The same register DFTs over double-float complex values (the last guard level): the
// radix-2/4 butterflies of ccst_fft.cuh and a 3-point DFT, all constants as double-floats.
template <bool INV>
__device__ __forceinline__ dfc mul_w12_df(dfc x, int idx) {
    constexpr double kS3 = 0.86602540378443864676;      // sqrt(3)/2
    idx %= 12;
    if (idx >= 6) { x = {df_neg(x.re), df_neg(x.im)}; idx -= 6; }
    if (idx == 0) return x;
    if (idx == 3) return INV ? dfc{df_neg(x.im), x.re} : dfc{x.im, df_neg(x.re)};
    const double c = idx == 1 ? kS3 : idx == 2 ? 0.5 : idx == 4 ? -0.5 : -kS3;
    const double sn = idx == 1 ? 0.5 : idx == 2 ? kS3 : idx == 4 ? kS3 : 0.5;
    return cmul(x, dfc{df_const(c), df_const(INV ? sn : -sn)});
}
template <bool INV>
__device__ __forceinline__ void dft3_df(dfc& a, dfc& b, dfc& c) {
    const df k3 = df_const(0.86602540378443864676);
    const dfc s = cadd(b, c), d = csub(b, c);
    const dfc t = csub(a, dfc{df_scale(s.re, 0.5f), df_scale(s.im, 0.5f)});
    const dfc sd = {df_mul(k3, d.re), df_mul(k3, d.im)};
    const dfc r = INV ? dfc{df_neg(sd.im), sd.re} : dfc{sd.im, df_neg(sd.re)};   // -+ i s3 d
    a = cadd(a, s);
    b = cadd(t, r);
    c = csub(t, r);
}
template <int R, bool INV>
__device__ __forceinline__ void mdft(dfc (&v)[R]) {
    if constexpr (R == 1) {
    } else if constexpr (R == 3) {
        dft3_df<INV>(v[0], v[1], v[2]);
    } else if constexpr (R == 6 || R == 12) {
        constexpr int R1 = 3, R2 = R / 3;
#pragma unroll
        for (int n2 = 0; n2 < R2; ++n2) dft3_df<INV>(v[n2], v[R2 + n2], v[2 * R2 + n2]);
#pragma unroll
        for (int k1 = 1; k1 < R1; ++k1)
#pragma unroll
            for (int n2 = 1; n2 < R2; ++n2) v[R2 * k1 + n2] = mul_w12_df<INV>(v[R2 * k1 + n2], n2 * k1 * (12 / R));
#pragma unroll
        for (int k1 = 0; k1 < R1; ++k1) {
            if constexpr (R2 == 2) dft2_df<INV>(v[R2 * k1], v[R2 * k1 + 1]);
            else dft4_df<INV>(v[R2 * k1], v[R2 * k1 + 1], v[R2 * k1 + 2], v[R2 * k1 + 3]);
        }
        dfc t[R];
#pragma unroll
        for (int i = 0; i < R; ++i) t[i] = v[i];
#pragma unroll
        for (int k1 = 0; k1 < R1; ++k1)
#pragma unroll
            for (int k2 = 0; k2 < R2; ++k2) v[k1 + R1 * k2] = t[R2 * k1 + k2];
    } else {
        dft_reg_df<R, INV>(v);
    }
}

// Forward pass S over nseq sequences. kSeqFast: consecutive tasks take consecutive
// sequences (column data); otherwise consecutive n2 of one sequence (row data).
// t4: W_N^{n2 k1} laid out [k1][n2]; ld(s, n2, n1) -> sample N2 n1 + n2; st(s, n2, k1, v)
// stores the result for slot N2 k1 + n2.
template <int N1, int N2, bool kSeqFast, int NT, class T, class LD, class ST>
__device__ __forceinline__ void fwd_pass_s(int nseq, const T* t4, LD ld, ST st) {
    const int ntask = nseq * N2;
    for (int task = threadIdx.x; task < ntask; task += NT) {
        int s, n2;
        if (kSeqFast) { n2 = task / nseq; s = task - n2 * nseq; }
        else { s = task / N2; n2 = task - s * N2; }
        T v[N1];
#pragma unroll
        for (int n1 = 0; n1 < N1; ++n1) v[n1] = ld(s, n2, n1);
        mdft<N1, false>(v);
        if (N2 > 1) {
#pragma unroll
            for (int k1 = 1; k1 < N1; ++k1) v[k1] = cmul(v[k1], t4[k1 * N2 + n2]);
        }
#pragma unroll
        for (int k1 = 0; k1 < N1; ++k1) st(s, n2, k1, v[k1]);
    }
}
// Forward pass C: ld(s, k1, n2) -> slot N2 k1 + n2; st(s, k1, k2, v) receives X[k1 + N1 k2]
// (slot N2 k1 + k2).
template <int N1, int N2, bool kSeqFast, int NT, class LD, class ST>
__device__ __forceinline__ void fwd_pass_c(int nseq, LD ld, ST st) {
    const int ntask = nseq * N1;
    for (int task = threadIdx.x; task < ntask; task += NT) {
        int s, k1;
        if (kSeqFast) { k1 = task / nseq; s = task - k1 * nseq; }
        else { s = task / N1; k1 = task - s * N1; }
        decltype(ld(0, 0, 0)) w[N2];
#pragma unroll
        for (int n2 = 0; n2 < N2; ++n2) w[n2] = ld(s, k1, n2);
        mdft<N2, false>(w);
#pragma unroll
        for (int k2 = 0; k2 < N2; ++k2) st(s, k1, k2, w[k2]);
    }
}
// Inverse pass C: ld(s, k1, k2) -> X[k1 + N1 k2] (slot N2 k1 + k2); st(s, k1, n2, v) stores
// the twiddled result for slot N2 k1 + n2.
template <int N1, int N2, bool kSeqFast, int NT, class LD, class ST>
__device__ __forceinline__ void inv_pass_c(int nseq, const float2* t4, LD ld, ST st) {
    const int ntask = nseq * N1;
    for (int task = threadIdx.x; task < ntask; task += NT) {
        int s, k1;
        if (kSeqFast) { k1 = task / nseq; s = task - k1 * nseq; }
        else { s = task / N1; k1 = task - s * N1; }
        float2 w[N2];
#pragma unroll
        for (int k2 = 0; k2 < N2; ++k2) w[k2] = ld(s, k1, k2);
        mdft<N2, true>(w);
        if (k1 > 0) {
#pragma unroll
            for (int n2 = 1; n2 < N2; ++n2) w[n2] = cmul(w[n2], cconj(t4[k1 * N2 + n2]));
        }
#pragma unroll
        for (int n2 = 0; n2 < N2; ++n2) st(s, k1, n2, w[n2]);
    }
}
// Inverse pass S: ld(s, n2, k1) -> slot N2 k1 + n2; st(s, n2, n1, v) receives x[n2 + N2 n1]
// (slot N2 n1 + n2).
template <int N1, int N2, bool kSeqFast, int NT, class LD, class ST>
__device__ __forceinline__ void inv_pass_s(int nseq, LD ld, ST st) {
    const int ntask = nseq * N2;
    for (int task = threadIdx.x; task < ntask; task += NT) {
        int s, n2;
        if (kSeqFast) { n2 = task / nseq; s = task - n2 * nseq; }
        else { s = task / N2; n2 = task - s * N2; }
        float2 v[N1];
#pragma unroll
        for (int k1 = 0; k1 < N1; ++k1) v[k1] = ld(s, n2, k1);
        mdft<N1, true>(v);
#pragma unroll
        for (int n1 = 0; n1 < N1; ++n1) st(s, n2, n1, v[n1]);
    }
}

}  // namespace mix
}  // namespace ccst
