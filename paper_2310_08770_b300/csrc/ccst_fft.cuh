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
    idx &= 15;
    if (idx >= 8) { x = make_float2(-x.x, -x.y); idx -= 8; }      // W^8 = -1
    if (idx == 0) return x;
    if (idx == 4) return INV ? make_float2(-x.y, x.x) : make_float2(x.y, -x.x);
    const float c = c16(idx), s = INV ? s16(idx) : -s16(idx);
    return make_float2(fmaf(x.x, c, -x.y * s), fmaf(x.x, s, x.y * c));
}

template <bool INV>
__device__ __forceinline__ void dft2(float2& a, float2& b) {
    const float2 t = a;
    a = cadd(t, b);
    b = csub(t, b);
}
// 4-point DFT in place: (a, b, c, d) <- X[0..3].
template <bool INV>
__device__ __forceinline__ void dft4(float2& a, float2& b, float2& c, float2& d) {
    const float2 s0 = cadd(a, c), d0 = csub(a, c), s1 = cadd(b, d), d1 = csub(b, d);
    const float2 r = INV ? make_float2(-d1.y, d1.x) : make_float2(d1.y, -d1.x);   // -+ i d1
    a = cadd(s0, s1);
    c = csub(s0, s1);
    b = cadd(d0, r);
    d = csub(d0, r);
}

// In-register DFT of R = 1, 2, 4, 8 or 16 points, natural order in and out. 8 = 2 x 4 and
// 16 = 4 x 4 use the same four-step split as the shared-memory passes: R1-point DFTs over
// the samples R2 n1 + n2, twiddles W_R^{n2 k1}, R2-point DFTs, then X[k1 + R1 k2] is read
// from slot R2 k1 + k2. Every loop has constant bounds so all indices and twiddles fold.
template <int R, bool INV>
__device__ __forceinline__ void dft_reg(float2 (&v)[R]) {
    if constexpr (R == 2) {
        dft2<INV>(v[0], v[1]);
    } else if constexpr (R == 4) {
        dft4<INV>(v[0], v[1], v[2], v[3]);
    } else if constexpr (R == 8 || R == 16) {
        constexpr int R1 = R / 4, R2 = 4;
#pragma unroll
        for (int n2 = 0; n2 < R2; ++n2) {
            if constexpr (R1 == 2) dft2<INV>(v[n2], v[R2 + n2]);
            else dft4<INV>(v[n2], v[R2 + n2], v[2 * R2 + n2], v[3 * R2 + n2]);
        }
#pragma unroll
        for (int k1 = 1; k1 < R1; ++k1)
#pragma unroll
            for (int n2 = 1; n2 < R2; ++n2)
                v[R2 * k1 + n2] = mul_w16<INV>(v[R2 * k1 + n2], n2 * k1 * (16 / R));
#pragma unroll
        for (int k1 = 0; k1 < R1; ++k1) dft4<INV>(v[R2 * k1], v[R2 * k1 + 1], v[R2 * k1 + 2], v[R2 * k1 + 3]);
        float2 t[R];
#pragma unroll
        for (int i = 0; i < R; ++i) t[i] = v[i];
#pragma unroll
        for (int k1 = 0; k1 < R1; ++k1)
#pragma unroll
            for (int k2 = 0; k2 < R2; ++k2) v[k1 + R1 * k2] = t[R2 * k1 + k2];
    }
}

__host__ __device__ constexpr int log2_c(int n) { return n <= 1 ? 0 : 1 + log2_c(n / 2); }

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

// Inter-pass twiddles W_N^{n2 k1} laid out [k1][n2] (N1 x N2 entries), so that the
// lanes of a warp, which differ in n2 or share it, read distinct banks or broadcast.
template <int N>
__device__ __forceinline__ void build_pass_twiddles(float2* t4, const float2* tw, int logNtw) {
    constexpr int N2 = Split<N>::N2;
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
        const int k1 = i / N2, n2 = i - k1 * N2;
        t4[i] = tw_n<N, false>(tw, logNtw, n2 * k1);
    }
}

// Pass 1 over nseq sequences. kSeqFast: consecutive tasks take consecutive sequences
// (column-like data); otherwise consecutive n2 of one sequence (row-like data).
// t4: the [k1][n2] twiddle table of this length (build_pass_twiddles).
// ld(s, n2, n1) returns sample N2 n1 + n2 of sequence s; st(s, n2, k1, v) stores the
// pass result k1 at index N2 k1 + n2. The index parts are passed separately so that
// the functors' addresses are linear in the unrolled n1 / k1.
template <int N1, int N2, bool INV, bool kSeqFast, class LD, class ST>
__device__ __forceinline__ void fft_pass1(int nseq, const float2* t4, LD ld, ST st) {
    const int ntask = nseq * N2;
    for (int task = threadIdx.x; task < ntask; task += blockDim.x) {
        int s, n2;
        if (kSeqFast) { n2 = task / nseq; s = task - n2 * nseq; }
        else { s = task / N2; n2 = task - s * N2; }
        float2 v[N1];
#pragma unroll
        for (int n1 = 0; n1 < N1; ++n1) v[n1] = ld(s, n2, n1);
        dft_reg<N1, INV>(v);
        if (N2 > 1) {
#pragma unroll
            for (int k1 = 1; k1 < N1; ++k1) {
                float2 w = t4[k1 * N2 + n2];
                if (INV) w.y = -w.y;
                v[k1] = cmul(v[k1], w);
            }
        }
#pragma unroll
        for (int k1 = 0; k1 < N1; ++k1) st(s, n2, k1, v[k1]);
    }
}

// Pass 2: ld(s, k1, n2) returns the pass-1 result at index N2 k1 + n2; st(s, k1, k2, v)
// receives X[k1 + N1 k2], whose in-place position is N2 k1 + k2.
template <int N1, int N2, bool INV, bool kSeqFast, class LD, class ST>
__device__ __forceinline__ void fft_pass2(int nseq, LD ld, ST st) {
    const int ntask = nseq * N1;
    for (int task = threadIdx.x; task < ntask; task += blockDim.x) {
        int s, k1;
        if (kSeqFast) { k1 = task / nseq; s = task - k1 * nseq; }
        else { s = task / N1; k1 = task - s * N1; }
        float2 w[N2];
#pragma unroll
        for (int n2 = 0; n2 < N2; ++n2) w[n2] = ld(s, k1, n2);
        dft_reg<N2, INV>(w);
#pragma unroll
        for (int k2 = 0; k2 < N2; ++k2) st(s, k1, k2, w[k2]);
    }
}


// ------------------------------------------------------------------ double-float passes
// The same four-step passes over double-float complex values (the last guard level):
// register DFTs built from 2- and 4-point butterflies, twiddles W_N^{n2 k1} from a
// [k1][n2] table. Sums use the absolute-error double-word addition (an FFT's error bound).
namespace dfconst {
constexpr double kC1 = 0.92387953251128675613;      // cos(pi/8)
constexpr double kS1 = 0.38268343236508977173;      // sin(pi/8)
constexpr double kR2 = 0.70710678118654752440;      // sqrt(1/2)
}  // namespace dfconst

__device__ __forceinline__ df df_const(double x) {
    const float h = (float)x;
    return {h, (float)(x - (double)h)};
}
// cos / sin of 2 pi k / 16, k = 0..7
__device__ __forceinline__ df df_c16(int k) {
    return k == 0 ? df_const(1.0) : k == 1 ? df_const(dfconst::kC1) : k == 2 ? df_const(dfconst::kR2)
         : k == 3 ? df_const(dfconst::kS1) : k == 4 ? df_const(0.0) : k == 5 ? df_const(-dfconst::kS1)
         : k == 6 ? df_const(-dfconst::kR2) : df_const(-dfconst::kC1);
}
__device__ __forceinline__ df df_s16(int k) {
    return k == 0 ? df_const(0.0) : k == 1 ? df_const(dfconst::kS1) : k == 2 ? df_const(dfconst::kR2)
         : k == 3 ? df_const(dfconst::kC1) : k == 4 ? df_const(1.0) : k == 5 ? df_const(dfconst::kC1)
         : k == 6 ? df_const(dfconst::kR2) : df_const(dfconst::kS1);
}
// x * exp(-+ 2 pi i idx / 16), idx a compile-time constant after unrolling
template <bool INV>
__device__ __forceinline__ dfc mul_w16_df(dfc x, int idx) {
    idx &= 15;
    if (idx >= 8) { x = {df_neg(x.re), df_neg(x.im)}; idx -= 8; }
    if (idx == 0) return x;
    if (idx == 4) return INV ? dfc{df_neg(x.im), x.re} : dfc{x.im, df_neg(x.re)};
    const df c = df_c16(idx), s = INV ? df_s16(idx) : df_neg(df_s16(idx));
    return cmul(x, dfc{c, s});
}
template <bool INV>
__device__ __forceinline__ void dft2_df(dfc& a, dfc& b) {
    const dfc t = a;
    a = cadd(t, b);
    b = csub(t, b);
}
template <bool INV>
__device__ __forceinline__ void dft4_df(dfc& a, dfc& b, dfc& c, dfc& d) {
    const dfc s0 = cadd(a, c), d0 = csub(a, c), s1 = cadd(b, d), d1 = csub(b, d);
    const dfc r = INV ? dfc{df_neg(d1.im), d1.re} : dfc{d1.im, df_neg(d1.re)};     // -+ i d1
    a = cadd(s0, s1);
    c = csub(s0, s1);
    b = cadd(d0, r);
    d = csub(d0, r);
}
// In-register DFT of R = 1, 2, 4, 8 or 16 points (the splits of dft_reg)
template <int R, bool INV>
__device__ __forceinline__ void dft_reg_df(dfc (&v)[R]) {
    if constexpr (R == 2) {
        dft2_df<INV>(v[0], v[1]);
    } else if constexpr (R == 4) {
        dft4_df<INV>(v[0], v[1], v[2], v[3]);
    } else if constexpr (R == 8 || R == 16) {
        constexpr int R1 = R / 4, R2 = 4;
#pragma unroll
        for (int n2 = 0; n2 < R2; ++n2) {
            if constexpr (R1 == 2) dft2_df<INV>(v[n2], v[R2 + n2]);
            else dft4_df<INV>(v[n2], v[R2 + n2], v[2 * R2 + n2], v[3 * R2 + n2]);
        }
#pragma unroll
        for (int k1 = 1; k1 < R1; ++k1)
#pragma unroll
            for (int n2 = 1; n2 < R2; ++n2)
                v[R2 * k1 + n2] = mul_w16_df<INV>(v[R2 * k1 + n2], n2 * k1 * (16 / R));
#pragma unroll
        for (int k1 = 0; k1 < R1; ++k1) dft4_df<INV>(v[R2 * k1], v[R2 * k1 + 1], v[R2 * k1 + 2], v[R2 * k1 + 3]);
        dfc t[R];
#pragma unroll
        for (int i = 0; i < R; ++i) t[i] = v[i];
#pragma unroll
        for (int k1 = 0; k1 < R1; ++k1)
#pragma unroll
            for (int k2 = 0; k2 < R2; ++k2) v[k1 + R1 * k2] = t[R2 * k1 + k2];
    }
}
// W_N^{n2 k1} (forward) laid out [k1][n2], from twd[k] = exp(-2 pi i k / Ntw), k < Ntw/2
template <int N>
__device__ __forceinline__ void build_pass_twiddles_df(dfc* t4, const dfc* twd, int logNtw) {
    constexpr int N2 = Split<N>::N2, lg = log2_c(N);
    const int sh = logNtw - lg;
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
        const int k1 = i / N2, n2 = i - k1 * N2, e = (n2 * k1) & (N - 1);
        dfc t = e < (N >> 1) ? twd[e << sh] : twd[(e - (N >> 1)) << sh];
        if (e >= (N >> 1)) t = {df_neg(t.re), df_neg(t.im)};
        t4[i] = t;
    }
}
template <int N1, int N2, bool kSeqFast, class LD, class ST>
__device__ __forceinline__ void fft_pass1_df(int nseq, const dfc* t4, LD ld, ST st) {
    const int ntask = nseq * N2;
    for (int task = threadIdx.x; task < ntask; task += blockDim.x) {
        int s, n2;
        if (kSeqFast) { n2 = task / nseq; s = task - n2 * nseq; }
        else { s = task / N2; n2 = task - s * N2; }
        dfc v[N1];
#pragma unroll
        for (int n1 = 0; n1 < N1; ++n1) v[n1] = ld(s, n2, n1);
        dft_reg_df<N1, false>(v);
        if (N2 > 1) {
#pragma unroll
            for (int k1 = 1; k1 < N1; ++k1) v[k1] = cmul(v[k1], t4[k1 * N2 + n2]);
        }
#pragma unroll
        for (int k1 = 0; k1 < N1; ++k1) st(s, n2, k1, v[k1]);
    }
}
template <int N1, int N2, bool kSeqFast, class LD, class ST>
__device__ __forceinline__ void fft_pass2_df(int nseq, LD ld, ST st) {
    const int ntask = nseq * N1;
    for (int task = threadIdx.x; task < ntask; task += blockDim.x) {
        int s, k1;
        if (kSeqFast) { k1 = task / nseq; s = task - k1 * nseq; }
        else { s = task / N1; k1 = task - s * N1; }
        dfc w[N2];
#pragma unroll
        for (int n2 = 0; n2 < N2; ++n2) w[n2] = ld(s, k1, n2);
        dft_reg_df<N2, false>(w);
#pragma unroll
        for (int k2 = 0; k2 < N2; ++k2) st(s, k1, k2, w[k2]);
    }
}

}  // namespace ccst
