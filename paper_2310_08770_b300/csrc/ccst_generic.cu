// ccst_generic.cu -- the tracking path of Secs. II-III for every frame shape the
// power-of-two kernel does not take: H and W from 8 to 256, any factors (48, 96, 192, 256,
// 256 x 128, ...). Two-level DFTs over the Hermitian half of the real-input spectrum and
// the full-grid upsampled sum, in double-float on the FP32 pipes (about 2^-46 per term):
// its decisions are those of an FP64 evaluation except on genuine ties. The integer
// surface and the upsampled grid are first evaluated in FP32 with a rounding bound, and
// only the points the bound cannot rule out are evaluated in double-float, by the same
// operations as the exhaustive double-float evaluation (CCST_FLAG_EXHAUSTIVE), so the
// records are the ones that evaluation gives.
//
// Per frame (one CTA of 512 threads; a CTA takes frames from a counter), Wh = W/2 + 1,
// g(kx) = 1 at kx = 0 and kx = W/2, 2 elsewhere (the fold of the Hermitian pair):
//   a = I (CC-U) or (I + eps)^2 (CC-SN), as double-floats                   (Eqs. 4, 7)
//   R[y][kx]  = sum_x a(y, x) wW^(x kx)                                     kx < Wh
//   X[ky][kx] = (sum_y R[y][kx] wH^(y ky)) conj F[b](ky, kx)               (Eq. 4)
//   Q[y][kx]  = sum_ky X[ky][kx] wH^-(ky y)
//   c(y, x)   = sum_kx g(kx) Re Q[y][kx] wW^-(kx x)                         (HW x the surface)
//   p = the extremum of c (lowest flat index on ties), wrapped to (-N/2, N/2]
//   V[jy][kx] = sum_ky X[ky][kx] e^{2 pi i ky' (py u + jy - h0) / (uH)}
//   cu(jy, jx) = sum_kx g(kx) Re V[jy][kx] e^{2 pi i kx' (px u + jx - h0) / (uW)}
// (wN = e^{-2 pi i / N}; k' the fftfreq-signed frequency, Nyquist at -N/2; every angle
// index reduced exactly in integers modulo N or uN), then the extremum of cu (lowest flat
// index on ties) and the 24-byte record.
//
// The fold is exact for the interpolant's definition (the real part of the full
// signed-frequency sum), with one rule: in the columns 0 < kx < W/2 the y-Nyquist row
// (ky = H/2, H even) pairs with itself at -kx, so its y-phase enters only through its
// real part cos(pi sy).
#include "ccst_generic.cuh"

namespace ccst {

constexpr unsigned kRGeneric = 0x80u;   // record flag: tracked by this path
constexpr unsigned kRNonFinite = 0x10u; // record flag: the surface was not finite
constexpr int kGridCap = 8192;          // most upsampled-grid candidates re-evaluated in double-float
constexpr int kRowCap = 256;            // most distinct grid rows among them
constexpr int kRowWords = 769;          // row bitmap words: M = ceil(1.5 u) <= 24577 for u <= 16384
constexpr int kIntCand = 8;             // most integer-surface candidates re-evaluated in double-float

// Block extremum of (value, index): the largest value, the lowest index on ties.
__device__ void gen_block_best(double& v, long long& j, double* sv, long long* sj) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const double ov = __shfl_xor_sync(0xffffffffu, v, o);
        const long long oj = __shfl_xor_sync(0xffffffffu, j, o);
        if (ov > v || (ov == v && oj < j)) { v = ov; j = oj; }
    }
    if (lane == 0) { sv[wid] = v; sj[wid] = j; }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < nw; ++w)
            if (sv[w] > v || (sv[w] == v && sj[w] < j)) { v = sv[w]; j = sj[w]; }
        sv[0] = v;
        sj[0] = j;
    }
    __syncthreads();
    v = sv[0];
    j = sj[0];
    __syncthreads();
}

__device__ __forceinline__ long long gen_mod(long long a, long long m) {
    a %= m;
    return a < 0 ? a + m : a;
}
// 16- and 8-byte vector accesses: every complex double-float array of this kernel starts on
// a 16-byte boundary (allocation bases and offsets in whole complex elements), so one access
// moves one element instead of four (two).
__device__ __forceinline__ dfc ldc(const dfc* p) {
    const float4 v = *reinterpret_cast<const float4*>(p);
    return dfc{df{v.x, v.y}, df{v.z, v.w}};
}
__device__ __forceinline__ void stc(dfc* p, dfc v) {
    *reinterpret_cast<float4*>(p) = make_float4(v.re.hi, v.re.lo, v.im.hi, v.im.lo);
}
__device__ __forceinline__ df ldd(const df* p) {
    const float2 v = *reinterpret_cast<const float2*>(p);
    return df{v.x, v.y};
}
__device__ __forceinline__ void std_(df* p, df v) { *reinterpret_cast<float2*>(p) = make_float2(v.hi, v.lo); }

// Re(a b) in double-float
__device__ __forceinline__ df gen_re_mul(dfc a, dfc b) {
    return df_add_abs(df_mul(a.re, b.re), df_neg(df_mul(a.im, b.im)));
}

// Block sum and maximum of one double per thread (sv: 32 doubles of shared memory).
__device__ double gen_block_sum(double v, double* sv) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();
    if (lane == 0) sv[wid] = v;
    __syncthreads();
    double s = 0.0;
    for (int w = 0; w < nw; ++w) s += sv[w];
    __syncthreads();
    return s;
}
__device__ double gen_block_max(double v, double* sv) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    __syncthreads();
    if (lane == 0) sv[wid] = v;
    __syncthreads();
    double s = sv[0];
    for (int w = 1; w < nw; ++w) s = fmax(s, sv[w]);
    __syncthreads();
    return s;
}

// One point of the upsampled grid in FP32: sum_kx Re V32[kx] EX[kx][jx], V32 carrying the
// fold weight g(kx) and the x-phase of the integer shift; ex = EX + jx, rows M apart (the
// lanes of a warp read consecutive jx: coalesced).
__device__ __forceinline__ float gen_cu32(const float2* V, const float2* ex, int Wh, int M) {
    float acc = 0.f;
    for (int kx = 0; kx < Wh; ++kx) {
        const float2 v = V[kx], e = ex[(size_t)kx * M];
        acc = __fmaf_rn(v.x, e.x, acc);
        acc = __fmaf_rn(-v.y, e.y, acc);
    }
    return acc;
}

__global__ void __launch_bounds__(512) track_generic_kernel(GenBatch gb) {
    __shared__ double sv[32];
    __shared__ long long sj[32];
    __shared__ long long s_item;
    __shared__ __align__(16) dfc s_wH[256], s_wW[256];                       // e^{-2 pi i m / H}, e^{-2 pi i m / W}
    __shared__ int s_nc, s_nrows;                              // upsampled-grid candidates and their rows
    __shared__ unsigned s_rowbits[kRowWords];
    __shared__ int s_rowpre[kRowWords], s_rowof[kRowCap];
    __shared__ float2 s_wH32[256], s_wW32[256];                // the same twiddles in FP32
    __shared__ int s_nci, s_candi[kIntCand];                   // integer-surface candidates
    __shared__ double s_cvali[kIntCand];
    dfc* const X = gb.scratch + (size_t)blockIdx.x * gb.scratch_stride;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) s_item = (long long)atomicAdd(gb.next, 1u);
        __syncthreads();
        const long long item = s_item;
        const long long nfb = gb.fb_count ? (long long)*gb.fb_count : 0;
        if (item >= gb.n + nfb) break;
        GenItem it;
        if (item >= gb.n) {
            it = gb.fb_items[item - gb.n];
        } else if (gb.items) {
            it = gb.items[item];
        } else {
            it.frame = (const char*)gb.frames + item * gb.frame_bytes;
            it.pitch = gb.pitch;
            it.out_index = item;
            it.plan = gb.plan;
            it.ref = gb.ref;
        }
        const GenPlan pl = gb.plans[it.plan];
        const int H = pl.H, W = pl.W, Wh = W / 2 + 1, u = pl.u, M = pl.M, h0 = pl.h0;
        const long long DH = (long long)u * H, DW = (long long)u * W;
        const int nyq_y = (H % 2 == 0) ? H / 2 : -1;              // the y-Nyquist row, if any
        const dfc* Fb = gb.refs[it.ref];                           // H x Wh
        const int H1 = pl.H1, H2 = pl.H2, W1 = pl.W1, W2 = pl.W2;
        dfc* B = X + (size_t)H * Wh;                               // R, then Q, then V
        df* a = (df*)(B + (size_t)(H > M ? H : M) * Wh);           // operand plane, H x W
        dfc* T = (dfc*)a + ((size_t)H * W + 1) / 2;                // inner DFT levels, H x W
        const dfc zero = dfc{df{0.f, 0.f}, df{0.f, 0.f}};
        const df epsd = df_from_double((double)pl.eps);
        for (int m = threadIdx.x; m < H; m += blockDim.x) stc(s_wH + m, ldc(pl.wH + m));
        for (int m = threadIdx.x; m < W; m += blockDim.x) stc(s_wW + m, ldc(pl.wW + m));
        for (int o = threadIdx.x; o < H * W; o += blockDim.x) {
            const int y = o / W, x = o - y * W;
            const df I = df_make(pixel_f32(it.frame, pl.in_dtype, (long long)y * it.pitch + x));
            if (pl.method == 0) {
                std_(a + o, I);
            } else {
                const df ip = df_add(I, epsd);
                std_(a + o, df_mul(ip, ip));
            }
        }
        __syncthreads();
        // The four DFTs, each in two levels N = N1 N2 (k = k1 + N1 k2, n = N2 n1 + n2):
        // sum_n f(n) w^(n k) = sum_n2 w^(n2 k) [sum_n1 f(N2 n1 + n2) w^(N2 n1 k1)], the inner
        // sums being N1-point DFTs and the outer twiddle w^(n2 k) the product of the
        // classic twiddle and the N2-point kernel.
        // R[y][kx] = sum_x a(y, x) wW^(x kx); first T[y][n2][k1], then kx < Wh
        for (int o = threadIdx.x; o < H * W; o += blockDim.x) {
            const int y = o / W, r = o - y * W, n2 = r / W1, k1 = r - n2 * W1;
            const int step = (W2 * k1) % W;
            dfc acc = zero;
            int m = 0;
            for (int n1 = 0; n1 < W1; ++n1) {
                const df v = ldd(a + y * W + W2 * n1 + n2);
                const dfc t = ldc(s_wW + m);
                acc = cadd(acc, dfc{df_mul(v, t.re), df_mul(v, t.im)});
                m += step;
                if (m >= W) m -= W;
            }
            stc(T + o, acc);
        }
        __syncthreads();
        for (int o = threadIdx.x; o < H * Wh; o += blockDim.x) {
            const int y = o / Wh, kx = o - y * Wh, k1 = kx % W1;
            dfc acc = zero;
            int m = 0;
            for (int n2 = 0; n2 < W2; ++n2) {
                acc = cadd(acc, cmul(ldc(T + (y * W + n2 * W1 + k1)), ldc(s_wW + m)));
                m += kx;
                if (m >= W) m -= W;
            }
            stc(B + o, acc);
        }
        __syncthreads();
        // X[ky][kx] = (sum_y R[y][kx] wH^(y ky)) conj F[b](ky, kx); T[n2][k1][kx] first
        for (int o = threadIdx.x; o < H * Wh; o += blockDim.x) {
            const int r = o / Wh, kx = o - r * Wh, n2 = r / H1, k1 = r - n2 * H1;
            const int step = (H2 * k1) % H;
            dfc acc = zero;
            int m = 0;
            for (int n1 = 0; n1 < H1; ++n1) {
                acc = cadd(acc, cmul(ldc(B + ((H2 * n1 + n2) * Wh + kx)), ldc(s_wH + m)));
                m += step;
                if (m >= H) m -= H;
            }
            stc(T + o, acc);
        }
        __syncthreads();
        for (int o = threadIdx.x; o < H * Wh; o += blockDim.x) {
            const int ky = o / Wh, kx = o - ky * Wh, k1 = ky % H1;
            dfc acc = zero;
            int m = 0;
            for (int n2 = 0; n2 < H2; ++n2) {
                acc = cadd(acc, cmul(ldc(T + ((n2 * H1 + k1) * Wh + kx)), ldc(s_wH + m)));
                m += ky;
                if (m >= H) m -= H;
            }
            stc(X + o, cmul(acc, cconj(ldc(Fb + o))));
        }
        __syncthreads();
        // The integer surface. Without the exhaustive flag it is first evaluated in FP32 (X
        // rounded once, the same two-level inverses) with a rounding bound Bi; the points within
        // 2 Bi of the FP32 best are then evaluated in double-float by the exhaustive
        // evaluation's own operations, in its order (at most icap of them; more, none, or the
        // flag: the exhaustive evaluation over the whole surface).
        float2* X32 = (float2*)a;                                  // X rounded to FP32, H x Wh
        double sumA = 0.0;                                         // sum_k |X32(k)|_1, full spectrum
        double best = -INFINITY;
        long long bj = 0x7fffffffffffffffLL;
        bool int_full = pl.exhaustive != 0;
        if (!int_full) {
            for (int o = threadIdx.x; o < H * Wh; o += blockDim.x) {
                const dfc xv = ldc(X + o);
                X32[o] = make_float2(xv.re.hi, xv.im.hi);
            }
            for (int m = threadIdx.x; m < H; m += blockDim.x) s_wH32[m] = make_float2(s_wH[m].re.hi, s_wH[m].im.hi);
            for (int m = threadIdx.x; m < W; m += blockDim.x) s_wW32[m] = make_float2(s_wW[m].re.hi, s_wW[m].im.hi);
            __syncthreads();
            double sA = 0.0;
            for (int kx = threadIdx.x; kx < Wh; kx += blockDim.x) {
                double s = 0.0;
                for (int ky = 0; ky < H; ++ky) s += fabs((double)X32[ky * Wh + kx].x) + fabs((double)X32[ky * Wh + kx].y);
                sA += (kx != 0 && 2 * kx != W) ? 2.0 * s : s;
            }
            sumA = gen_block_sum(sA, sv);
            float2* T32 = (float2*)T;                              // column level H x Wh, then row level H x W
            float2* Q32 = (float2*)B;                              // H x Wh
            // columns: T32[n2][y1][kx] = sum_n1 X32[H2 n1 + n2][kx] wH^-(H2 n1 y1), then Q32
            for (int o = threadIdx.x; o < H * Wh; o += blockDim.x) {
                const int r = o / Wh, kx = o - r * Wh, n2 = r / H1, y1 = r - n2 * H1;
                const int step = (H2 * y1) % H;
                float ar = 0.f, ai = 0.f;
                int m = 0;
                for (int n1 = 0; n1 < H1; ++n1) {
                    const float2 x = X32[(H2 * n1 + n2) * Wh + kx], w = s_wH32[m];
                    ar = __fmaf_rn(x.x, w.x, ar);
                    ar = __fmaf_rn(x.y, w.y, ar);
                    ai = __fmaf_rn(x.y, w.x, ai);
                    ai = __fmaf_rn(-x.x, w.y, ai);
                    m += step;
                    if (m >= H) m -= H;
                }
                T32[o] = make_float2(ar, ai);
            }
            __syncthreads();
            for (int o = threadIdx.x; o < H * Wh; o += blockDim.x) {
                const int y = o / Wh, kx = o - y * Wh, y1 = y % H1;
                float ar = 0.f, ai = 0.f;
                int m = 0;
                for (int n2 = 0; n2 < H2; ++n2) {
                    const float2 t = T32[(n2 * H1 + y1) * Wh + kx], w = s_wH32[m];
                    ar = __fmaf_rn(t.x, w.x, ar);
                    ar = __fmaf_rn(t.y, w.y, ar);
                    ai = __fmaf_rn(t.y, w.x, ai);
                    ai = __fmaf_rn(-t.x, w.y, ai);
                    m += y;
                    if (m >= H) m -= H;
                }
                Q32[o] = make_float2(ar, ai);
            }
            __syncthreads();
            // rows, Hermitian-completed: T32[y][n2][x1] = sum_n1 Q(y, W2 n1 + n2) wW^-(W2 n1 x1)
            for (int o = threadIdx.x; o < H * W; o += blockDim.x) {
                const int y = o / W, r = o - y * W, n2 = r / W1, x1 = r - n2 * W1;
                const int step = (W2 * x1) % W;
                float ar = 0.f, ai = 0.f;
                int m = 0;
                for (int n1 = 0; n1 < W1; ++n1) {
                    const int k = W2 * n1 + n2;
                    float2 q = k < Wh ? Q32[y * Wh + k] : Q32[y * Wh + W - k];
                    if (k >= Wh) q.y = -q.y;
                    const float2 w = s_wW32[m];
                    ar = __fmaf_rn(q.x, w.x, ar);
                    ar = __fmaf_rn(q.y, w.y, ar);
                    ai = __fmaf_rn(q.y, w.x, ai);
                    ai = __fmaf_rn(-q.x, w.y, ai);
                    m += step;
                    if (m >= W) m -= W;
                }
                T32[o] = make_float2(ar, ai);
            }
            __syncthreads();
            // c32(y, x) = Re sum_n2 T32[y][n2][x mod W1] wW^-(n2 x), one fixed FMA chain (both passes)
            auto c32 = [&](int o) -> float {
                const int y = o / W, x = o - y * W, x1 = x % W1;
                float acc = 0.f;
                int m = 0;
                for (int n2 = 0; n2 < W2; ++n2) {
                    const float2 t = T32[y * W + n2 * W1 + x1], w = s_wW32[m];
                    acc = __fmaf_rn(t.x, w.x, acc);
                    acc = __fmaf_rn(t.y, w.y, acc);
                    m += x;
                    if (m >= W) m -= W;
                }
                return pl.sense * acc;
            };
            float b32 = -INFINITY;
            for (int o = threadIdx.x; o < H * W; o += blockDim.x) b32 = fmaxf(b32, c32(o));
            // |c32 - c| <= Bi: rounding of X and the tables, gamma_n per FMA chain, sqrt(2) per
            // complex product in the 1-norm, through both levels of both inverses
            const double Bi = 1.1 * (8.0 * (W1 + W2) + 16.0 + 9.0 * (H1 + H2) + 22.0) * 0x1p-24 * sumA + 0x1p-30 * sumA;
            const double thr_i = gen_block_max((double)b32, sv) - 2.0 * Bi;
            if (threadIdx.x == 0) s_nci = 0;
            __syncthreads();
            const int icap_raw = (H * W) / (H2 * Wh + W2);
            const int icap = icap_raw < 1 ? 1 : (icap_raw > kIntCand ? kIntCand : icap_raw);
            for (int o = threadIdx.x; o < H * W; o += blockDim.x)
                if ((double)c32(o) >= thr_i) {
                    const int k = atomicAdd(&s_nci, 1);
                    if (k < icap) s_candi[k] = o;
                }
            __syncthreads();
            const int nci = s_nci;
            if (nci == 0 || nci > icap) {
                int_full = true;
            } else {
                dfc* P1 = T;                                       // nci x H2 x Wh: column level 1
                dfc* P3 = T + (size_t)nci * H2 * Wh;               // nci x W2: row level 1
                dfc* P2 = B;                                       // nci x Wh: the candidate's row of Q
                for (int t = threadIdx.x; t < nci * H2 * Wh; t += blockDim.x) {
                    const int cidx = t / (H2 * Wh), r = t - cidx * H2 * Wh, n2 = r / Wh, kx = r - n2 * Wh;
                    const int y1 = (s_candi[cidx] / W) % H1, step = (H2 * y1) % H;
                    dfc acc = zero;
                    int m = 0;
                    for (int n1 = 0; n1 < H1; ++n1) {
                        acc = cadd(acc, cmul(ldc(X + ((H2 * n1 + n2) * Wh + kx)), cconj(ldc(s_wH + m))));
                        m += step;
                        if (m >= H) m -= H;
                    }
                    stc(P1 + t, acc);
                }
                __syncthreads();
                for (int t = threadIdx.x; t < nci * Wh; t += blockDim.x) {
                    const int cidx = t / Wh, kx = t - cidx * Wh, y = s_candi[cidx] / W;
                    dfc acc = zero;
                    int m = 0;
                    for (int n2 = 0; n2 < H2; ++n2) {
                        acc = cadd(acc, cmul(ldc(P1 + ((size_t)(cidx * H2 + n2) * Wh + kx)), cconj(ldc(s_wH + m))));
                        m += y;
                        if (m >= H) m -= H;
                    }
                    stc(P2 + t, acc);
                }
                __syncthreads();
                for (int t = threadIdx.x; t < nci * W2; t += blockDim.x) {
                    const int cidx = t / W2, n2 = t - cidx * W2, x1 = (s_candi[cidx] % W) % W1;
                    const int step = (W2 * x1) % W;
                    const dfc* q = P2 + (size_t)cidx * Wh;
                    dfc acc = zero;
                    int m = 0;
                    for (int n1 = 0; n1 < W1; ++n1) {
                        const int k = W2 * n1 + n2;
                        const dfc qv = k < Wh ? ldc(q + k) : cconj(ldc(q + (W - k)));
                        acc = cadd(acc, cmul(qv, cconj(ldc(s_wW + m))));
                        m += step;
                        if (m >= W) m -= W;
                    }
                    stc(P3 + t, acc);
                }
                __syncthreads();
                if (threadIdx.x < nci) {
                    const int x = s_candi[threadIdx.x] % W;
                    df acc = df{0.f, 0.f};
                    int m = 0;
                    for (int n2 = 0; n2 < W2; ++n2) {
                        acc = df_add_abs(acc, gen_re_mul(ldc(P3 + (size_t)threadIdx.x * W2 + n2), cconj(ldc(s_wW + m))));
                        m += x;
                        if (m >= W) m -= W;
                    }
                    s_cvali[threadIdx.x] = pl.sense * df_to_double(acc);
                }
                __syncthreads();
                for (int k = 0; k < nci; ++k) {
                    const double v = s_cvali[k];
                    const long long j = s_candi[k];
                    if (v > best || (v == best && j < bj)) { best = v; bj = j; }
                }
                __syncthreads();
            }
        }
        if (int_full) {
            // Q[y][kx] = sum_ky X[ky][kx] wH^-(ky y); T[n2][y1][kx] first
            for (int o = threadIdx.x; o < H * Wh; o += blockDim.x) {
                const int r = o / Wh, kx = o - r * Wh, n2 = r / H1, y1 = r - n2 * H1;
                const int step = (H2 * y1) % H;
                dfc acc = zero;
                int m = 0;
                for (int n1 = 0; n1 < H1; ++n1) {
                    acc = cadd(acc, cmul(ldc(X + ((H2 * n1 + n2) * Wh + kx)), cconj(ldc(s_wH + m))));
                    m += step;
                    if (m >= H) m -= H;
                }
                stc(T + o, acc);
            }
            __syncthreads();
            for (int o = threadIdx.x; o < H * Wh; o += blockDim.x) {
                const int y = o / Wh, kx = o - y * Wh, y1 = y % H1;
                dfc acc = zero;
                int m = 0;
                for (int n2 = 0; n2 < H2; ++n2) {
                    acc = cadd(acc, cmul(ldc(T + ((n2 * H1 + y1) * Wh + kx)), cconj(ldc(s_wH + m))));
                    m += y;
                    if (m >= H) m -= H;
                }
                stc(B + o, acc);
            }
            __syncthreads();
            // c(y, x) = Re sum_{k < W} Q[y][k] wW^-(k x), the row completed by Q[y][W - k] =
            // conj Q[y][k] (X is the spectrum of a real surface); T[y][n2][x1] first. The
            // extremum, lowest flat index on ties
            for (int o = threadIdx.x; o < H * W; o += blockDim.x) {
                const int y = o / W, r = o - y * W, n2 = r / W1, x1 = r - n2 * W1;
                const int step = (W2 * x1) % W;
                dfc acc = zero;
                int m = 0;
                for (int n1 = 0; n1 < W1; ++n1) {
                    const int k = W2 * n1 + n2;
                    const dfc qv = k < Wh ? ldc(B + (y * Wh + k)) : cconj(ldc(B + (y * Wh + W - k)));
                    acc = cadd(acc, cmul(qv, cconj(ldc(s_wW + m))));
                    m += step;
                    if (m >= W) m -= W;
                }
                stc(T + o, acc);
            }
            __syncthreads();
            for (int o = threadIdx.x; o < H * W; o += blockDim.x) {
                const int y = o / W, x = o - y * W, x1 = x % W1;
                df acc = df{0.f, 0.f};
                int m = 0;
                for (int n2 = 0; n2 < W2; ++n2) {
                    acc = df_add_abs(acc, gen_re_mul(ldc(T + (y * W + n2 * W1 + x1)), cconj(ldc(s_wW + m))));
                    m += x;
                    if (m >= W) m -= W;
                }
                const double v = pl.sense * df_to_double(acc);
                if (v > best || (v == best && o < bj)) { best = v; bj = o; }
            }
            gen_block_best(best, bj, sv, sj);
        }
        const int iy = (int)(bj / W), ix = (int)(bj % W);
        const int py = iy > H / 2 ? iy - H : iy;
        const int px = ix > W / 2 ? ix - W : ix;
        // The upsampled grid. First in FP32 with a rounding bound Bnd: every point whose FP32
        // value is within 2 Bnd of the FP32 best is a candidate, and only the candidates are
        // evaluated in double-float, by the same operations and order as the exhaustive
        // evaluation below (so the record is the one that evaluation gives). Too many
        // candidates, or the exhaustive flag: the whole grid in double-float.
        bool full = pl.exhaustive != 0;
        if (!full) {
            float2* V32 = (float2*)B;                              // M x Wh (X32, sumA: from the integer stage)
            // X32 <- X32 e^{2 pi i (ky py / H + kx px / W)}: the integer shift's phase (periodic in
            // k, so unsigned k serves; real (+-1) on the Nyquist row and column), leaving the
            // frame-independent tables EY, EX for the grid offsets
            {
                const int pyy = ((py % H) + H) % H, pxx = ((px % W) + W) % W;
                for (int o = threadIdx.x; o < H * Wh; o += blockDim.x) {
                    const int ky = o / Wh, kx = o - ky * Wh;
                    const float2 a = s_wH32[(int)(((long long)ky * pyy) % H)], b = s_wW32[(int)(((long long)kx * pxx) % W)];
                    const float2 ph = make_float2(a.x * b.x - a.y * b.y, -(a.x * b.y + a.y * b.x));   // conj(a b)
                    const float2 x = X32[o];
                    X32[o] = make_float2(x.x * ph.x - x.y * ph.y, x.x * ph.y + x.y * ph.x);
                }
                __syncthreads();
            }
            // V32[jy][kx] = g(kx) sum_ky X32[ky][kx] EY[ky][jy]; in the weight-2 columns the
            // y-Nyquist row (H even) takes the real part of EY only
            for (int o = threadIdx.x; o < M * Wh; o += blockDim.x) {
                const int jy = o / Wh, kx = o - jy * Wh;
                const bool folded = kx != 0 && 2 * kx != W;
                const float2* xc = X32 + kx;
                const float2* ey = pl.EY + jy;
                const int k1 = nyq_y >= 0 ? nyq_y : H;                 // rows before the Nyquist row
                float ar = 0.f, ai = 0.f;
                for (int ky = 0; ky < k1; ++ky) {
                    const float2 e = ey[(size_t)ky * M], x = xc[ky * Wh];
                    ar = __fmaf_rn(x.x, e.x, ar);
                    ar = __fmaf_rn(-x.y, e.y, ar);
                    ai = __fmaf_rn(x.x, e.y, ai);
                    ai = __fmaf_rn(x.y, e.x, ai);
                }
                if (nyq_y >= 0) {
                    float2 e = ey[(size_t)nyq_y * M];
                    if (folded) e.y = 0.f;
                    const float2 x = xc[nyq_y * Wh];
                    ar = __fmaf_rn(x.x, e.x, ar);
                    ar = __fmaf_rn(-x.y, e.y, ar);
                    ai = __fmaf_rn(x.x, e.y, ai);
                    ai = __fmaf_rn(x.y, e.x, ai);
                    for (int ky = nyq_y + 1; ky < H; ++ky) {
                        const float2 e2 = ey[(size_t)ky * M], x2 = xc[ky * Wh];
                        ar = __fmaf_rn(x2.x, e2.x, ar);
                        ar = __fmaf_rn(-x2.y, e2.y, ar);
                        ai = __fmaf_rn(x2.x, e2.y, ai);
                        ai = __fmaf_rn(x2.y, e2.x, ai);
                    }
                }
                const float gw = folded ? 2.f : 1.f;               // the fold weight, exact
                V32[o] = make_float2(gw * ar, gw * ai);
            }
            // bound ingredients: sumA (above) and max_jy S(jy), S(jy) = sum_kx |V32(jy, kx)|_1
            // (V32 carries the fold weight)
            double sS = 0.0;
            __syncthreads();
            for (int jy = threadIdx.x; jy < M; jy += blockDim.x) {
                double s = 0.0;
                for (int kx = 0; kx < Wh; ++kx) s += fabs((double)V32[jy * Wh + kx].x) + fabs((double)V32[jy * Wh + kx].y);
                sS = fmax(sS, s);
            }
            const double maxS = gen_block_max(sS, sv);
            const double u32 = 0x1p-24;
            // (sumA was taken before the phase rotation, which can grow a 1-norm by sqrt(2))
            const double Bnd = 1.01 * ((2.0 * Wh + 3.0) * u32 * maxS + 1.42 * (4.0 * H + 16.0) * u32 * sumA) +
                               0x1p-30 * (maxS + sumA);
            // pass 1: the FP32 best (the values kept when the grid is small enough); pass 2:
            // the candidates
            float* G = (float*)(T + (size_t)H * W);
            const bool keep = M * M <= kGenGridKeep;
            float b32 = -INFINITY;
            for (int o = threadIdx.x; o < M * M; o += blockDim.x) {
                const int jy = o / M, jx = o - jy * M;
                const float v = pl.sense * gen_cu32(V32 + jy * Wh, pl.EX + jx, Wh, M);
                if (keep) G[o] = v;
                b32 = fmaxf(b32, v);
            }
            const double thr = gen_block_max((double)b32, sv) - 2.0 * Bnd;
            // pass 2: the candidates, listed in the T region (free by now: ints, gcap of them)
            int* cand = (int*)T;
            const int gcap = kGridCap < 4 * H * W ? kGridCap : 4 * H * W;
            if (threadIdx.x == 0) s_nc = 0;
            __syncthreads();
            for (int o = threadIdx.x; o < M * M; o += blockDim.x) {
                const int jy = o / M, jx = o - jy * M;
                const float v = keep ? G[o] : pl.sense * gen_cu32(V32 + jy * Wh, pl.EX + jx, Wh, M);
                if ((double)v >= thr) {
                    const int k = atomicAdd(&s_nc, 1);
                    if (k < gcap) cand[k] = o;
                }
            }
            __syncthreads();
            const int nc = s_nc;
            const int nwords = (M + 31) >> 5;
            if (nc == 0 || nc > gcap || nwords > kRowWords) {      // none: a non-finite grid
                full = true;
            } else {
                // the candidates' rows: a bitmap over jy, then slot(jy) = rows below jy (in
                // order, so the slots do not depend on the order the candidates were listed)
                for (int w = threadIdx.x; w < nwords; w += blockDim.x) s_rowbits[w] = 0u;
                __syncthreads();
                for (int k = threadIdx.x; k < nc; k += blockDim.x) {
                    const int jy = cand[k] / M;
                    atomicOr(&s_rowbits[jy >> 5], 1u << (jy & 31));
                }
                __syncthreads();
                if (threadIdx.x == 0) {
                    int sum = 0;
                    for (int w = 0; w < nwords; ++w) {
                        s_rowpre[w] = sum;
                        sum += __popc(s_rowbits[w]);
                    }
                    s_nrows = sum;
                }
                __syncthreads();
                const int nrows = s_nrows;
                if (nrows > kRowCap) {
                    full = true;
                } else {
                    for (int w = threadIdx.x; w < nwords; w += blockDim.x) {
                        unsigned bits = s_rowbits[w];
                        int slot = s_rowpre[w];
                        while (bits) {
                            s_rowof[slot++] = 32 * w + __ffs(bits) - 1;
                            bits &= bits - 1;
                        }
                    }
                    __syncthreads();
                    // V(jy, kx) in double-float for the candidates' rows, by the exhaustive
                    // evaluation's operations (V32 is no longer read)
                    for (int t = threadIdx.x; t < nrows * Wh; t += blockDim.x) {
                        const int slot = t / Wh, kx = t - slot * Wh, jy = s_rowof[slot];
                        const long long q = gen_mod((long long)py * u + jy - h0, DH), nq = gen_mod((long long)H * q, DH);
                        const bool folded = kx != 0 && 2 * kx != W;
                        // the operands of row ky + 1 are loaded while row ky is accumulated (the
                        // table and X live in L2); the arithmetic is the exhaustive loop's
                        auto table_index = [&](int ky, long long mm) {
                            if (2 * ky >= H) { mm -= nq; if (mm < 0) mm += DH; }
                            return mm;
                        };
                        dfc acc = zero;
                        long long m = 0;
                        dfc en = ldc(pl.uH + table_index(0, 0)), xn = ldc(X + kx);
                        for (int ky = 0; ky < H; ++ky) {
                            dfc e = en;
                            const dfc x = xn;
                            m += q;
                            if (m >= DH) m -= DH;
                            if (ky + 1 < H) {
                                en = ldc(pl.uH + table_index(ky + 1, m));
                                xn = ldc(X + ((ky + 1) * Wh + kx));
                            }
                            if (ky == nyq_y && folded) e.im = df{0.f, 0.f};
                            acc = cadd(acc, cmul(x, e));
                        }
                        stc(B + t, acc);
                    }
                    __syncthreads();
                    // each candidate: the exhaustive evaluation's sum over kx of its row
                    best = -INFINITY;
                    bj = 0x7fffffffffffffffLL;
                    for (int k = threadIdx.x; k < nc; k += blockDim.x) {
                        const int o = cand[k], jy = o / M, jx = o - jy * M;
                        const int w = jy >> 5;
                        const int slot = s_rowpre[w] + __popc(s_rowbits[w] & ((1u << (jy & 31)) - 1u));
                        const long long q = gen_mod((long long)px * u + jx - h0, DW), nq = gen_mod((long long)W * q, DW);
                        const dfc* vrow = B + (size_t)slot * Wh;
                        df acc = df{0.f, 0.f};
                        long long m = 0;
                        for (int kx = 0; kx < Wh; ++kx) {
                            long long ms = m;
                            if (2 * kx >= W) { ms -= nq; if (ms < 0) ms += DW; }
                            df t = gen_re_mul(ldc(vrow + kx), ldc(pl.uW + ms));
                            if (kx != 0 && 2 * kx != W) t = df_scale(t, 2.f);
                            acc = df_add_abs(acc, t);
                            m += q;
                            if (m >= DW) m -= DW;
                        }
                        const double v = pl.sense * df_to_double(acc);
                        if (v > best || (v == best && o < bj)) { best = v; bj = o; }
                    }
                    gen_block_best(best, bj, sv, sj);
                }
            }
        }
        if (full) {
            // V[jy][kx] = sum_ky X[ky][kx] e^{2 pi i ky' q / (uH)}, q = py u + jy - h0: the index
            // ky q mod uH advances by q per row, and the negative rows subtract H q mod uH
            for (int o = threadIdx.x; o < M * Wh; o += blockDim.x) {
                const int jy = o / Wh, kx = o - jy * Wh;
                const long long q = gen_mod((long long)py * u + jy - h0, DH), nq = gen_mod((long long)H * q, DH);
                const bool folded = kx != 0 && 2 * kx != W;
                dfc acc = zero;
                long long m = 0;
                for (int ky = 0; ky < H; ++ky) {
                    long long ms = m;
                    if (2 * ky >= H) { ms -= nq; if (ms < 0) ms += DH; }
                    dfc e = ldc(pl.uH + ms);
                    if (ky == nyq_y && folded) e.im = df{0.f, 0.f};
                    acc = cadd(acc, cmul(ldc(X + (ky * Wh + kx)), e));
                    m += q;
                    if (m >= DH) m -= DH;
                }
                stc(B + o, acc);
            }
            __syncthreads();
            // cu(jy, jx) = sum_kx g(kx) Re V[jy][kx] e^{2 pi i kx' q / (uW)}, q = px u + jx - h0
            best = -INFINITY;
            bj = 0x7fffffffffffffffLL;
            for (int o = threadIdx.x; o < M * M; o += blockDim.x) {
                const int jy = o / M, jx = o - jy * M;
                const long long q = gen_mod((long long)px * u + jx - h0, DW), nq = gen_mod((long long)W * q, DW);
                df acc = df{0.f, 0.f};
                long long m = 0;
                for (int kx = 0; kx < Wh; ++kx) {
                    long long ms = m;
                    if (2 * kx >= W) { ms -= nq; if (ms < 0) ms += DW; }
                    df t = gen_re_mul(ldc(B + (jy * Wh + kx)), ldc(pl.uW + ms));
                    if (kx != 0 && 2 * kx != W) t = df_scale(t, 2.f);
                    acc = df_add_abs(acc, t);
                    m += q;
                    if (m >= DW) m -= DW;
                }
                const double v = pl.sense * df_to_double(acc);
                if (v > best || (v == best && o < bj)) { best = v; bj = o; }
            }
            gen_block_best(best, bj, sv, sj);
        }
        if (threadIdx.x == 0) {
            const int jy = (int)(bj / M), jx = (int)(bj % M);
            Result r;
            r.dy = (float)(((double)py * u + jy - h0) / u);
            r.dx = (float)(((double)px * u + jx - h0) / u);
            r.peak = (float)(pl.sense * best / ((double)H * W));
            r.ipy = py;
            r.ipx = px;
            r.flags = kRGeneric | (best > -INFINITY && best < INFINITY ? 0u : kRNonFinite);
            gb.out[it.out_index] = r;
        }
    }
}

// The FP32 grid tables of one general shape: EY[ky][jy] = e^{2 pi i ky' (jy - h0) / (uH)} and
// EX[kx][jx] = e^{2 pi i kx' (jx - h0) / (uW)}, k' the fftfreq-signed frequency (the x-Nyquist
// column kx = W/2 is -W/2), every angle index reduced exactly in integers.
__global__ void gen_init_grid_tables(int H, int W, int u, int M, int h0, float2* EY, float2* EX) {
    const int Wh = W / 2 + 1;
    const long long DH = (long long)u * H, DW = (long long)u * W, ny = (long long)H * M;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < ny + (long long)Wh * M;
         i += (long long)gridDim.x * blockDim.x) {
        const bool y = i < ny;
        const long long r = y ? i : i - ny;
        const int k = (int)(r / M), j = (int)(r - (long long)k * M);
        const int N = y ? H : W;
        const long long D = y ? DH : DW;
        const long long ks = 2 * k >= N ? k - N : k;
        long long m = (ks * (j - h0)) % D;
        if (m < 0) m += D;
        double s, c;
        sincospi(2.0 * (double)m / (double)D, &s, &c);
        (y ? EY : EX)[r] = make_float2((float)c, (float)s);
    }
}

// Tables of one general shape: e^{-2 pi i m / H} (m < H), e^{-2 pi i m / W} (m < W),
// e^{+2 pi i m / (uH)} (m < uH) and e^{+2 pi i m / (uW)} (m < uW), one block of
// H + W + uH + uW double-floats.
__global__ void gen_init_tables(int H, int W, int u, dfc* tab) {
    const long long DH = (long long)u * H, DW = (long long)u * W, n = H + W + DH + DW;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        double s, c;
        if (i < H) {
            sincospi(-2.0 * (double)i / (double)H, &s, &c);
        } else if (i < H + W) {
            sincospi(-2.0 * (double)(i - H) / (double)W, &s, &c);
        } else if (i < H + W + DH) {
            sincospi(2.0 * (double)(i - H - W) / (double)DH, &s, &c);
        } else {
            sincospi(2.0 * (double)(i - H - W - DH) / (double)DW, &s, &c);
        }
        tab[i] = dfc{df_from_double(c), df_from_double(s)};
    }
}

// The half spectrum F[b] (kx <= W/2) of one reference, in FP64 by direct DFTs (b = E, or
// 1/(E + eps) for CC-SN): rows, then columns, one thread per output.
__global__ void gen_ref_rows(int H, int W, int method, float eps, const float* ref, double2* R) {
    __shared__ double2 tw[256];
    for (int m = threadIdx.x; m < W; m += blockDim.x) {
        double s, c;
        sincospi(-2.0 * (double)m / (double)W, &s, &c);
        tw[m] = make_double2(c, s);
    }
    __syncthreads();
    const int Wh = W / 2 + 1;
    for (int o = blockIdx.x * blockDim.x + threadIdx.x; o < H * Wh; o += gridDim.x * blockDim.x) {
        const int y = o / Wh, kx = o - y * Wh;
        double re = 0.0, im = 0.0;
        int m = 0;
        for (int x = 0; x < W; ++x) {
            const double e = (double)ref[y * W + x];
            const double b = method == 0 ? e : 1.0 / (e + (double)eps);
            re += b * tw[m].x;
            im += b * tw[m].y;
            m += kx;
            if (m >= W) m -= W;
        }
        R[o] = make_double2(re, im);
    }
}

__global__ void gen_ref_cols(int H, int W, const double2* R, dfc* Fb) {
    __shared__ double2 tw[256];
    for (int m = threadIdx.x; m < H; m += blockDim.x) {
        double s, c;
        sincospi(-2.0 * (double)m / (double)H, &s, &c);
        tw[m] = make_double2(c, s);
    }
    __syncthreads();
    const int Wh = W / 2 + 1;
    for (int o = blockIdx.x * blockDim.x + threadIdx.x; o < H * Wh; o += gridDim.x * blockDim.x) {
        const int ky = o / Wh, kx = o - ky * Wh;
        double re = 0.0, im = 0.0;
        int m = 0;
        for (int y = 0; y < H; ++y) {
            const double2 r = R[y * Wh + kx], t = tw[m];
            re += r.x * t.x - r.y * t.y;
            im += r.x * t.y + r.y * t.x;
            m += ky;
            if (m >= H) m -= H;
        }
        Fb[o] = dfc{df_from_double(re), df_from_double(im)};
    }
}

// A frame already on the device (u16 or f32, row pitch in elements) as the FP32 reference
// image the two kernels above read.
__global__ void gen_frame_to_f32(int H, int W, int in_dtype, const void* frame, long long pitch, float* out) {
    for (int o = blockIdx.x * blockDim.x + threadIdx.x; o < H * W; o += gridDim.x * blockDim.x) {
        const int y = o / W, x = o - y * W;
        out[o] = pixel_f32(frame, in_dtype, (long long)y * pitch + x);
    }
}

// Synthetic frames for timing (the autotuner): a spot of sigma 3 on a background, moved per
// frame, plus a hash-based pseudo-noise, in the context's input type. The kernel's work per
// frame does not depend on the values.
__global__ void gen_fill_synthetic(int H, int W, int in_dtype, long long n, void* frames) {
    const long long total = n * H * W;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
        const long long f = i / ((long long)H * W);
        const int r = (int)(i - f * H * W), y = r / W, x = r - y * W;
        const float cy = 0.5f * H + (float)(f % 7) * 0.37f - 1.1f, cx = 0.5f * W - (float)(f % 5) * 0.29f + 0.6f;
        const float d2 = (y - cy) * (y - cy) + (x - cx) * (x - cx);
        unsigned h = (unsigned)i * 2654435761u;
        h ^= h >> 15;
        h *= 2246822519u;
        h ^= h >> 13;
        const float v = 20.f + 1500.f * __expf(-d2 / 18.f) + (float)(h & 15u);
        if (in_dtype == 0) ((unsigned short*)frames)[i] = (unsigned short)v;
        else ((float*)frames)[i] = v;
    }
}

const void* gen_fill_synthetic_ptr() { return (const void*)gen_fill_synthetic; }
const void* gen_init_grid_tables_ptr() { return (const void*)gen_init_grid_tables; }
const void* gen_ref_rows_ptr() { return (const void*)gen_ref_rows; }
const void* gen_ref_cols_ptr() { return (const void*)gen_ref_cols; }
const void* track_generic_kernel_ptr() { return (const void*)track_generic_kernel; }
const void* gen_init_tables_ptr() { return (const void*)gen_init_tables; }
const void* gen_frame_to_f32_ptr() { return (const void*)gen_frame_to_f32; }

}  // namespace ccst
