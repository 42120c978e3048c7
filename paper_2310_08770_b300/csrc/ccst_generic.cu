// ccst_generic.cu -- the tracking path of Secs. II-III for square ROIs whose side is not a
// power of two up to 128 (48, 96, 192, 256, ...): direct DFTs and the full-grid upsampled
// sum, all in double-float on the FP32 pipes. Slower than the power-of-two kernel, but
// general, and precise enough (about 2^-46 per term) that no near-tie guard is needed:
// its decisions are those of an FP64 evaluation except on genuine ties.
//
// Per ROI (one CTA of 512 threads; a CTA takes ROIs from a counter):
//   a  = I (CC-U) or (I + eps)^2 (CC-SN), as double-floats
//   R[y][kx]   = sum_x a(y, x) w^(x kx)                     (w = e^{-2 pi i / N})
//   X[ky][kx]  = (sum_y R[y][kx] w^(y ky)) conj F[b](ky, kx)   (Eq. 4 / 7)
//   T[ky][x]   = sum_kx X[ky][kx] w^-(kx x)
//   c(y, x)    = Re sum_ky T[ky][x] w^-(ky y)               (N^2 c, the integer surface)
//   p = the extremum of c (lowest flat index on ties), wrapped to (-N/2, N/2]
//   U[ky][jx]  = sum_kx X[ky][kx] e^{2 pi i kx' (px u + jx - h0) / (uN)}
//   cu(jy, jx) = Re sum_ky U[ky][jx] e^{2 pi i ky' (py u + jy - h0) / (uN)}
// with fftfreq-signed k' and every angle index reduced exactly in integers modulo N or uN,
// then the extremum of cu (lowest flat index on ties) and the 24-byte record.
#include "ccst_kernels.cuh"

namespace ccst {

constexpr unsigned kRGeneric = 0x80u;   // record flag: tracked by this path

// Block extremum of (value, index): the largest sense * value, the lowest index on ties.
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

__device__ __forceinline__ dfc gen_mac(dfc acc, dfc a, dfc b) { return cadd(acc, cmul(a, b)); }
__device__ __forceinline__ dfc gen_conj_mul(dfc a, dfc b) { return cmul(a, cconj(b)); }
__device__ __forceinline__ long long gen_mod(long long a, long long m) {
    a %= m;
    return a < 0 ? a + m : a;
}

__global__ void __launch_bounds__(512) track_generic_kernel(GenBatch gb) {
    __shared__ double sv[32];
    __shared__ long long sj[32];
    __shared__ long long s_item;
    dfc* A = gb.scratch + (size_t)blockIdx.x * gb.scratch_stride;        // R, then T, then U
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) s_item = (long long)atomicAdd(gb.next, 1u);
        __syncthreads();
        const long long item = s_item;
        if (item >= gb.n) break;
        const GenItem it = gb.items[item];
        const GenPlan pl = gb.plans[it.plan];
        const int N = pl.N, NN = N * N, u = pl.u, M = pl.M, h0 = pl.h0;
        const long long D = (long long)u * N;
        const dfc* w = pl.wN;                                      // e^{-2 pi i m / N}
        const dfc* wu = pl.wU;                                     // e^{+2 pi i m / (uN)}
        const dfc* Fb = gb.refs[it.ref];
        dfc* X = A + (size_t)NN + (size_t)N * M;                  // [ky][kx]
        const df epsd = df_from_double((double)pl.eps);
        const dfc zero = dfc{df{0.f, 0.f}, df{0.f, 0.f}};
        auto operand = [&](int y, int x) {
            const df I = df_make(pixel_f32(it.frame, pl.in_dtype, (long long)y * it.pitch + x));
            if (pl.method == 0) return I;
            const df ip = df_add(I, epsd);
            return df_mul(ip, ip);
        };
        // R[y][kx] = sum_x a(y, x) w^(x kx)
        for (int o = threadIdx.x; o < NN; o += blockDim.x) {
            const int y = o / N, kx = o - y * N;
            dfc acc = zero;
            int m = 0;
            for (int x = 0; x < N; ++x) {
                const df a = operand(y, x);
                const dfc t = w[m];
                acc = cadd(acc, dfc{df_mul(a, t.re), df_mul(a, t.im)});
                m += kx;
                if (m >= N) m -= N;
            }
            A[o] = acc;
        }
        __syncthreads();
        // X[ky][kx] = (sum_y R[y][kx] w^(y ky)) conj F[b]
        for (int o = threadIdx.x; o < NN; o += blockDim.x) {
            const int ky = o / N, kx = o - ky * N;
            dfc acc = zero;
            int m = 0;
            for (int y = 0; y < N; ++y) {
                acc = gen_mac(acc, A[y * N + kx], w[m]);
                m += ky;
                if (m >= N) m -= N;
            }
            X[o] = gen_conj_mul(acc, Fb[o]);
        }
        __syncthreads();
        // T[ky][x] = sum_kx X[ky][kx] w^-(kx x)
        for (int o = threadIdx.x; o < NN; o += blockDim.x) {
            const int ky = o / N, x = o - ky * N;
            dfc acc = zero;
            int m = 0;
            for (int kx = 0; kx < N; ++kx) {
                acc = gen_mac(acc, X[ky * N + kx], cconj(w[m]));
                m += x;
                if (m >= N) m -= N;
            }
            A[o] = acc;
        }
        __syncthreads();
        // c(y, x) = Re sum_ky T[ky][x] w^-(ky y); the extremum, lowest flat index on ties
        double best = -INFINITY;
        long long bj = 0x7fffffffffffffffLL;
        for (int o = threadIdx.x; o < NN; o += blockDim.x) {
            const int y = o / N, x = o - y * N;
            df acc = df{0.f, 0.f};
            int m = 0;
            for (int ky = 0; ky < N; ++ky) {
                const dfc t = A[ky * N + x], c = cconj(w[m]);
                acc = df_add_abs(acc, df_add_abs(df_mul(t.re, c.re), df_neg(df_mul(t.im, c.im))));
                m += y;
                if (m >= N) m -= N;
            }
            const double v = pl.sense * df_to_double(acc);
            if (v > best || (v == best && o < bj)) { best = v; bj = o; }
        }
        gen_block_best(best, bj, sv, sj);
        const int py = (int)(bj / N) > N / 2 ? (int)(bj / N) - N : (int)(bj / N);
        const int px = (int)(bj % N) > N / 2 ? (int)(bj % N) - N : (int)(bj % N);
        // U[ky][jx] = sum_kx X[ky][kx] e^{2 pi i kx' (px u + jx - h0) / (uN)}; the index k' q mod uN
        // advances by q mod uN per bin, and the negative frequencies subtract N q mod uN
        for (int o = threadIdx.x; o < N * M; o += blockDim.x) {
            const int ky = o / M, jx = o - ky * M;
            const long long q = gen_mod((long long)px * u + jx - h0, D), nq = gen_mod((long long)N * q, D);
            dfc acc = zero;
            long long m = 0;
            for (int kx = 0; kx < N; ++kx) {
                long long ms = m;
                if (2 * kx >= N) { ms -= nq; if (ms < 0) ms += D; }
                acc = gen_mac(acc, X[ky * N + kx], wu[ms]);
                m += q;
                if (m >= D) m -= D;
            }
            A[o] = acc;
        }
        __syncthreads();
        // cu(jy, jx) = Re sum_ky U[ky][jx] e^{2 pi i ky' (py u + jy - h0) / (uN)}
        best = -INFINITY;
        bj = 0x7fffffffffffffffLL;
        for (int o = threadIdx.x; o < M * M; o += blockDim.x) {
            const int jy = o / M, jx = o - jy * M;
            const long long q = gen_mod((long long)py * u + jy - h0, D), nq = gen_mod((long long)N * q, D);
            df acc = df{0.f, 0.f};
            long long m = 0;
            for (int ky = 0; ky < N; ++ky) {
                long long ms = m;
                if (2 * ky >= N) { ms -= nq; if (ms < 0) ms += D; }
                const dfc t = A[ky * M + jx], c = wu[ms];
                acc = df_add_abs(acc, df_add_abs(df_mul(t.re, c.re), df_neg(df_mul(t.im, c.im))));
                m += q;
                if (m >= D) m -= D;
            }
            const double val = df_to_double(acc);
            const double v = pl.sense * val;
            if (v > best || (v == best && o < bj)) { best = v; bj = o; }
        }
        gen_block_best(best, bj, sv, sj);
        if (threadIdx.x == 0) {
            const int jy = (int)(bj / M), jx = (int)(bj % M);
            Result r;
            r.dy = (float)(((double)py * u + jy - h0) / u);
            r.dx = (float)(((double)px * u + jx - h0) / u);
            r.peak = (float)(pl.sense * best / ((double)N * N));
            r.ipy = py;
            r.ipx = px;
            r.flags = kRGeneric;
            gb.out[it.out_index] = r;
        }
    }
}

// Tables of one general size: w[m] = e^{-2 pi i m / N}, m < N, and e^{+2 pi i m / (uN)}, m < uN.
__global__ void gen_init_tables(int N, int u, dfc* wN, dfc* wU) {
    const long long D = (long long)u * N;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N + D; i += (long long)gridDim.x * blockDim.x) {
        double s, c;
        if (i < N) {
            sincospi(-2.0 * (double)i / (double)N, &s, &c);
            wN[i] = dfc{df_from_double(c), df_from_double(s)};
        } else {
            const long long m = i - N;
            sincospi(2.0 * (double)m / (double)D, &s, &c);
            wU[m] = dfc{df_from_double(c), df_from_double(s)};
        }
    }
}

// F[b] of one reference, full N x N, in FP64 by direct DFTs (b = E, or 1/(E + eps) for
// CC-SN): rows, then columns, one thread per output; the block keeps e^{-2 pi i m / N}.
__global__ void gen_ref_rows(int N, int method, float eps, const float* ref, double2* R) {
    __shared__ double2 tw[256];
    for (int m = threadIdx.x; m < N; m += blockDim.x) {
        double s, c;
        sincospi(-2.0 * (double)m / (double)N, &s, &c);
        tw[m] = make_double2(c, s);
    }
    __syncthreads();
    for (int o = blockIdx.x * blockDim.x + threadIdx.x; o < N * N; o += gridDim.x * blockDim.x) {
        const int y = o / N, kx = o - y * N;
        double re = 0.0, im = 0.0;
        int m = 0;
        for (int x = 0; x < N; ++x) {
            const double e = (double)ref[y * N + x];
            const double b = method == 0 ? e : 1.0 / (e + (double)eps);
            re += b * tw[m].x;
            im += b * tw[m].y;
            m += kx;
            if (m >= N) m -= N;
        }
        R[o] = make_double2(re, im);
    }
}

__global__ void gen_ref_cols(int N, const double2* R, dfc* Fb) {
    __shared__ double2 tw[256];
    for (int m = threadIdx.x; m < N; m += blockDim.x) {
        double s, c;
        sincospi(-2.0 * (double)m / (double)N, &s, &c);
        tw[m] = make_double2(c, s);
    }
    __syncthreads();
    for (int o = blockIdx.x * blockDim.x + threadIdx.x; o < N * N; o += gridDim.x * blockDim.x) {
        const int ky = o / N, kx = o - ky * N;
        double re = 0.0, im = 0.0;
        int m = 0;
        for (int y = 0; y < N; ++y) {
            const double2 r = R[y * N + kx], t = tw[m];
            re += r.x * t.x - r.y * t.y;
            im += r.x * t.y + r.y * t.x;
            m += ky;
            if (m >= N) m -= N;
        }
        Fb[o] = dfc{df_from_double(re), df_from_double(im)};
    }
}

const void* gen_ref_rows_ptr() { return (const void*)gen_ref_rows; }
const void* gen_ref_cols_ptr() { return (const void*)gen_ref_cols; }
const void* track_generic_kernel_ptr() { return (const void*)track_generic_kernel; }
const void* gen_init_tables_ptr() { return (const void*)gen_init_tables; }

}  // namespace ccst
