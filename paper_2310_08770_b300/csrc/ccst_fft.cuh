// ccst_fft.cuh -- four-step FFT passes over shared memory with the small DFTs in registers.
//
// A length N = N1*N2 DFT (Cooley-Tukey, "four-step" form):
//   X[k1 + N1 k2] = sum_{n2} W_{N2}^{n2 k2} W_N^{n2 k1} sum_{n1} x[N2 n1 + n2] W_{N1}^{n1 k1}.
// Pass 1: each task (sequence s, n2) gathers the N1 samples x[N2 n1 + n2], does an
// N1-point DFT in registers, applies the twiddles W_N^{n2 k1} and stores result k1 at
// index N2 k1 + n2 (the slots it read). Pass 2: each task (s, k1) reads the N2
// contiguous indices N2 k1 + n2, does an N2-point DFT and hands X[k1 + N1 k2] to its
// store functor; the natural in-place position of that output is N2 k1 + k2, i.e.
// X[k] ends at fft_pos(k) = N2 (k mod N1) + k div N1. Loads and stores go through
// functors so that reordering, the real/complex split, the spectral product and
// padding are fused into the passes instead of extra sweeps over shared memory.
#pragma once

#include "ccst_device.cuh"

namespace ccst {

// Factorisation N = N1 * N2 used for each supported length (N2 = 1: one pass).
template <int N> struct Split;
template <> struct Split<8> { static constexpr int N1 = 8, N2 = 1; };
template <> struct Split<16> { static constexpr int N1 = 4, N2 = 4; };
template <> struct Split<32> { static constexpr int N1 = 8, N2 = 4; };
template <> struct Split<64> { static constexpr int N1 = 8, N2 = 8; };
template <> struct Split<128> { static constexpr int N1 = 16, N2 = 8; };

__host__ __device__ constexpr int split_n2(int N) { return N <= 8 ? 1 : (N <= 32 ? 4 : 8); }
__host__ __device__ constexpr int split_n1(int N) { return N / split_n2(N); }

// Position of X[k] after both passes, and its inverse.
__device__ __forceinline__ int fft_pos(int k, int N1, int N2) { return N2 * (k % N1) + k / N1; }
__device__ __forceinline__ int fft_unpos(int q, int N1, int N2) { return (q % N2) * N1 + q / N2; }

// cos / sin of 2 pi k / 16, k = 0..7
__device__ __forceinline__ float c16(int k) {
    return k == 0 ? 1.0f : k == 1 ? 0.923879532511286756f : k == 2 ? 0.707106781186547524f
         : k == 3 ? 0.382683432365089772f : k == 4 ? 0.0f : k == 5 ? -0.382683432365089772f
         : k == 6 ? -0.707106781186547524f : -0.923879532511286756f;
}
__device__ __forceinline__ float s16(int k) {
    return k == 0 ? 0.0f : k == 1 ? 0.382683432365089772f : k == 2 ? 0.707106781186547524f
         : k == 3 ? 0.923879532511286756f : k == 4 ? 1.0f : k == 5 ? 0.923879532511286756f
         : k == 6 ? 0.707106781186547524f : 0.382683432365089772f;
}

// x * exp(-+ 2 pi i idx / 16) (forward: minus sign), idx a compile-time constant after unrolling.
template <bool INV>
__device__ __forceinline__ float2 mul_w16(float2 x, int idx) {
    if (idx == 0) return x;
    if (idx == 4) return INV ? make_float2(-x.y, x.x) : make_float2(x.y, -x.x);
    const float c = c16(idx), s = INV ? s16(idx) : -s16(idx);
    return make_float2(fmaf(x.x, c, -x.y * s), fmaf(x.x, s, x.y * c));
}

__host__ __device__ constexpr int brev_c(int i, int bits) {
    int r = 0;
    for (int b = 0; b < bits; ++b) r |= ((i >> b) & 1) << (bits - 1 - b);
    return r;
}
__host__ __device__ constexpr int log2_c(int n) { return n <= 1 ? 0 : 1 + log2_c(n / 2); }

// In-register DFT of R = 1, 2, 4, 8 or 16 points, natural order in and out.
template <int R, bool INV>
__device__ __forceinline__ void dft_reg(float2 (&v)[R]) {
    if (R == 1) return;
    constexpr int bits = log2_c(R);
#pragma unroll
    for (int i = 0; i < R; ++i) {
        const int j = brev_c(i, bits);
        if (j > i) { const float2 t = v[i]; v[i] = v[j]; v[j] = t; }
    }
#pragma unroll
    for (int span = 2; span <= R; span <<= 1) {
        const int half = span >> 1;
#pragma unroll
        for (int st = 0; st < R; st += span) {
#pragma unroll
            for (int j = 0; j < half; ++j) {
                const float2 b = mul_w16<INV>(v[st + j + half], j * (16 / span));
                const float2 a = v[st + j];
                v[st + j] = make_float2(a.x + b.x, a.y + b.y);
                v[st + j + half] = make_float2(a.x - b.x, a.y - b.y);
            }
        }
    }
}

// W_N^{e} = exp(-+ 2 pi i e / N), 0 <= e < N, from the shared table tw[k] = exp(-2 pi i k / Ntw).
template <int N, bool INV>
__device__ __forceinline__ float2 tw_n(const float2* tw, int logNtw, int e) {
    constexpr int lg = log2_c(N);
    const int sh = logNtw - lg;
    float2 t;
    if (e < (N >> 1)) t = tw[e << sh];
    else { t = tw[(e - (N >> 1)) << sh]; t = make_float2(-t.x, -t.y); }
    if (INV) t.y = -t.y;
    return t;
}

// Pass 1 over nseq sequences. kSeqFast: consecutive tasks take consecutive sequences
// (column-like data); otherwise consecutive n2 of one sequence (row-like data).
template <int N1, int N2, bool INV, bool kSeqFast, class LD, class ST>
__device__ __forceinline__ void fft_pass1(int nseq, const float2* tw, int logNtw, LD ld, ST st) {
    constexpr int N = N1 * N2;
    const int ntask = nseq * N2;
    for (int task = threadIdx.x; task < ntask; task += blockDim.x) {
        int s, n2;
        if (kSeqFast) { n2 = task / nseq; s = task - n2 * nseq; }
        else { s = task / N2; n2 = task - s * N2; }
        float2 v[N1];
#pragma unroll
        for (int n1 = 0; n1 < N1; ++n1) v[n1] = ld(s, N2 * n1 + n2);
        dft_reg<N1, INV>(v);
        if (N2 > 1) {
#pragma unroll
            for (int k1 = 1; k1 < N1; ++k1) v[k1] = cmul(v[k1], tw_n<N, INV>(tw, logNtw, n2 * k1));
        }
#pragma unroll
        for (int k1 = 0; k1 < N1; ++k1) st(s, N2 * k1 + n2, v[k1]);
    }
}

// Pass 2: st(s, k, q, value) receives X[k] (k = k1 + N1 k2) and its in-place position q.
template <int N1, int N2, bool INV, bool kSeqFast, class LD, class ST>
__device__ __forceinline__ void fft_pass2(int nseq, LD ld, ST st) {
    const int ntask = nseq * N1;
    for (int task = threadIdx.x; task < ntask; task += blockDim.x) {
        int s, k1;
        if (kSeqFast) { k1 = task / nseq; s = task - k1 * nseq; }
        else { s = task / N1; k1 = task - s * N1; }
        float2 w[N2];
#pragma unroll
        for (int n2 = 0; n2 < N2; ++n2) w[n2] = ld(s, N2 * k1 + n2);
        dft_reg<N2, INV>(w);
#pragma unroll
        for (int k2 = 0; k2 < N2; ++k2) st(s, k1 + N1 * k2, N2 * k1 + k2, w[k2]);
    }
}

}  // namespace ccst
