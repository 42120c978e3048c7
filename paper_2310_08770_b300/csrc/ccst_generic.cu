// ccst_generic.cu -- the tracking path of Secs. II-III for every frame shape the
// power-of-two kernel does not take: H and W from 8 to 256, any factors (48, 96, 192, 256,
// 256 x 128, ...). Direct DFTs over the Hermitian half of the real-input spectrum and the
// full-grid upsampled sum, all in double-float on the FP32 pipes. Slower than the
// power-of-two kernel, but general, and precise enough (about 2^-46 per term) that no
// near-tie guard is needed: its decisions are those of an FP64 evaluation except on
// genuine ties.
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
// Re(a b) in double-float
__device__ __forceinline__ df gen_re_mul(dfc a, dfc b) {
    return df_add_abs(df_mul(a.re, b.re), df_neg(df_mul(a.im, b.im)));
}

__global__ void __launch_bounds__(512) track_generic_kernel(GenBatch gb) {
    __shared__ double sv[32];
    __shared__ long long sj[32];
    __shared__ long long s_item;
    __shared__ dfc s_wH[256], s_wW[256];                       // e^{-2 pi i m / H}, e^{-2 pi i m / W}
    dfc* const X = gb.scratch + (size_t)blockIdx.x * gb.scratch_stride;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) s_item = (long long)atomicAdd(gb.next, 1u);
        __syncthreads();
        const long long item = s_item;
        if (item >= gb.n) break;
        GenItem it;
        if (gb.items) {
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
        dfc* B = X + (size_t)H * Wh;                               // R, then Q, then V
        df* a = (df*)(B + (size_t)(H > M ? H : M) * Wh);           // operand plane, H x W
        const dfc zero = dfc{df{0.f, 0.f}, df{0.f, 0.f}};
        const df epsd = df_from_double((double)pl.eps);
        for (int m = threadIdx.x; m < H; m += blockDim.x) s_wH[m] = pl.wH[m];
        for (int m = threadIdx.x; m < W; m += blockDim.x) s_wW[m] = pl.wW[m];
        for (int o = threadIdx.x; o < H * W; o += blockDim.x) {
            const int y = o / W, x = o - y * W;
            const df I = df_make(pixel_f32(it.frame, pl.in_dtype, (long long)y * it.pitch + x));
            if (pl.method == 0) {
                a[o] = I;
            } else {
                const df ip = df_add(I, epsd);
                a[o] = df_mul(ip, ip);
            }
        }
        __syncthreads();
        // R[y][kx] = sum_x a(y, x) wW^(x kx)
        for (int o = threadIdx.x; o < H * Wh; o += blockDim.x) {
            const int y = o / Wh, kx = o - y * Wh;
            dfc acc = zero;
            int m = 0;
            for (int x = 0; x < W; ++x) {
                const df v = a[y * W + x];
                const dfc t = s_wW[m];
                acc = cadd(acc, dfc{df_mul(v, t.re), df_mul(v, t.im)});
                m += kx;
                if (m >= W) m -= W;
            }
            B[o] = acc;
        }
        __syncthreads();
        // X[ky][kx] = (sum_y R[y][kx] wH^(y ky)) conj F[b](ky, kx)
        for (int o = threadIdx.x; o < H * Wh; o += blockDim.x) {
            const int ky = o / Wh, kx = o - ky * Wh;
            dfc acc = zero;
            int m = 0;
            for (int y = 0; y < H; ++y) {
                acc = cadd(acc, cmul(B[y * Wh + kx], s_wH[m]));
                m += ky;
                if (m >= H) m -= H;
            }
            X[o] = cmul(acc, cconj(Fb[o]));
        }
        __syncthreads();
        // Q[y][kx] = sum_ky X[ky][kx] wH^-(ky y)
        for (int o = threadIdx.x; o < H * Wh; o += blockDim.x) {
            const int y = o / Wh, kx = o - y * Wh;
            dfc acc = zero;
            int m = 0;
            for (int ky = 0; ky < H; ++ky) {
                acc = cadd(acc, cmul(X[ky * Wh + kx], cconj(s_wH[m])));
                m += y;
                if (m >= H) m -= H;
            }
            B[o] = acc;
        }
        __syncthreads();
        // c(y, x) = sum_kx g(kx) Re Q[y][kx] wW^-(kx x); the extremum, lowest flat index on ties
        double best = -INFINITY;
        long long bj = 0x7fffffffffffffffLL;
        for (int o = threadIdx.x; o < H * W; o += blockDim.x) {
            const int y = o / W, x = o - y * W;
            df acc = df{0.f, 0.f};
            int m = 0;
            for (int kx = 0; kx < Wh; ++kx) {
                df t = gen_re_mul(B[y * Wh + kx], cconj(s_wW[m]));
                if (kx != 0 && 2 * kx != W) t = df_scale(t, 2.f);
                acc = df_add_abs(acc, t);
                m += x;
                if (m >= W) m -= W;
            }
            const double v = pl.sense * df_to_double(acc);
            if (v > best || (v == best && o < bj)) { best = v; bj = o; }
        }
        gen_block_best(best, bj, sv, sj);
        const int iy = (int)(bj / W), ix = (int)(bj % W);
        const int py = iy > H / 2 ? iy - H : iy;
        const int px = ix > W / 2 ? ix - W : ix;
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
                dfc e = pl.uH[ms];
                if (ky == nyq_y && folded) e.im = df{0.f, 0.f};
                acc = cadd(acc, cmul(X[ky * Wh + kx], e));
                m += q;
                if (m >= DH) m -= DH;
            }
            B[o] = acc;
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
                df t = gen_re_mul(B[jy * Wh + kx], pl.uW[ms]);
                if (kx != 0 && 2 * kx != W) t = df_scale(t, 2.f);
                acc = df_add_abs(acc, t);
                m += q;
                if (m >= DW) m -= DW;
            }
            const double v = pl.sense * df_to_double(acc);
            if (v > best || (v == best && o < bj)) { best = v; bj = o; }
        }
        gen_block_best(best, bj, sv, sj);
        if (threadIdx.x == 0) {
            const int jy = (int)(bj / M), jx = (int)(bj % M);
            Result r;
            r.dy = (float)(((double)py * u + jy - h0) / u);
            r.dx = (float)(((double)px * u + jx - h0) / u);
            r.peak = (float)(pl.sense * best / ((double)H * W));
            r.ipy = py;
            r.ipx = px;
            r.flags = kRGeneric;
            gb.out[it.out_index] = r;
        }
    }
}

// Tables of one general shape: e^{-2 pi i m / H} (m < H), e^{-2 pi i m / W} (m < W),
// e^{+2 pi i m / (uH)} (m < uH) and e^{+2 pi i m / (uW)} (m < uW), one block of
// H + W + uH + uW entries.
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

const void* gen_ref_rows_ptr() { return (const void*)gen_ref_rows; }
const void* gen_ref_cols_ptr() { return (const void*)gen_ref_cols; }
const void* track_generic_kernel_ptr() { return (const void*)track_generic_kernel; }
const void* gen_init_tables_ptr() { return (const void*)gen_init_tables; }
const void* gen_frame_to_f32_ptr() { return (const void*)gen_frame_to_f32; }

}  // namespace ccst
