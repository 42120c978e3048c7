// ccst_adjoint.cuh -- the continuous peak of the cross-correlation interpolant and its
// vector-Jacobian product (the adjoint of the displacement). The 2-D transforms, Newton's
// row sums, the product spectrum and the VJP spectra run in double-float on the FP32 pipes
// (B300's FP64 rate is about 1/64 of its FP32 rate); the phases, Newton's moments and the
// partial-sum accumulation are FP64.
//
// The tracker's estimate is the extremum of the interpolant of Sec. III on the 1/u grid,
// a piecewise-constant function of the pixels. The differentiable quantity is the
// stationary point s* of the same interpolant without the grid,
//   f(s) = (1/HW) Re sum_k X(k) e^{2 pi i (ky' sy / H + kx' sx / W)},  X = F[a] conj F[b]
// (all H x W frequencies, fftfreq-signed; (a, b) the operands of Eq. (4) or (7)), found by
// Newton's method from the grid peak. With the Hessian Hf at s* and an upstream gradient
// g = dL/ds*, w = -Hf^{-1} g and
//   dL/da(r) = (1/HW) Re sum_k (2 pi i w.k'/N) conj F[b](k) e^{2 pi i k.(s* - r)/N}
//   dL/db(r) = (1/HW) Re sum_k (2 pi i w.k'/N) F[a](k)      e^{2 pi i k.(s* + r)/N}
// then the chain rule to the pixels of I and E.
//
// On the half spectrum (kx = 0 .. W/2) the sums fold in Hermitian pairs. The pair of bin
// (ky, kx) is (-ky, -kx); at a Nyquist index the pair keeps the same signed frequency, so a
// spectrum Q that is not Hermitian there enters a real sum as its symmetrised form
// (Q(k) + conj Q(pair)) / 2, which is Hermitian and can go through a complex-to-real
// transform. In f itself this makes the y-Nyquist row of the columns 0 < kx < W/2 enter
// through cos(pi sy) alone.
#pragma once

#include <math_constants.h>

#include "ccst_kernels.cuh"

namespace ccst {

struct AdjArgs {
    const void* frames;     // n frames (in_dtype), rows `pitch` elements apart
    long long n, pitch;
    const Result* rec;      // the tracker's records: Newton starts at their grid peaks
    const float* g;         // n x 2 upstream gradient (dL/ddx, dL/ddy), or null (peak only)
    double* peak;           // n x 2 (dx, dy) of s*, or null
    int* status;            // n status words, or null
    float* g_frames;        // n x H x W dL/dI, or null
    double2* scratch;       // [gridDim.x][H][Wc] per-CTA work spectrum
    double2* part;          // [gridDim.x][H][Wc] per-CTA sum of the dL/db spectra, or null
};

constexpr int kAdjNotConverged = 1;   // Newton did not settle within the iteration limit
constexpr int kAdjNotExtremum = 2;    // s* is not a maximum (CC-U) / minimum (CC-SN)
constexpr int kAdjFar = 4;            // s* is more than one pixel from the grid peak
constexpr int kAdjIters = 50;

__device__ __forceinline__ int adj_freq(int k, int N) { return k < (N >> 1) ? k : k - N; }   // N/2 -> -N/2

__device__ __forceinline__ double2 adj_i_times(double kappa, double2 z) {   // i kappa z
    return make_double2(-kappa * z.y, kappa * z.x);
}

__device__ __forceinline__ double2 dfc_double(dfc v) { return make_double2(df_to_double(v.re), df_to_double(v.im)); }

__device__ __forceinline__ dfc shfl_xor_dfc(dfc v, int o) {
    return dfc{df{__shfl_xor_sync(0xffffffffu, v.re.hi, o), __shfl_xor_sync(0xffffffffu, v.re.lo, o)},
               df{__shfl_xor_sync(0xffffffffu, v.im.hi, o), __shfl_xor_sync(0xffffffffu, v.im.lo, o)}};
}

// Deterministic block sum of 6 doubles; the result is valid in thread 0.
__device__ void adj_block_sum6(double v[6], double* red) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int j = 0; j < 6; ++j) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[j] += __shfl_xor_sync(0xffffffffu, v[j], o);
    }
    if (lane == 0)
        for (int j = 0; j < 6; ++j) red[wid * 6 + j] = v[j];
    __syncthreads();
    if (threadIdx.x == 0)
        for (int j = 0; j < 6; ++j) {
            double s = 0.0;
            for (int w = 0; w < nw; ++w) s += red[w * 6 + j];
            v[j] = s;
        }
    __syncthreads();
}

// Shared memory of adj_kernel, in double2: the transform buffer (then X as double-floats),
// Ay[H], Bx[Wc], the row sums R[H][3] (+3 for the y-Nyquist row's middle columns), 6
// doubles per warp, the double-float column phases and factors BxF, kap, -kap^2 [Wc], and
// the double-float row phases and factors AyF, kapy [H].
__host__ __device__ inline int adj_nbuf(int H, int W) {
    const int a = (H / 2) * W, b = (W / 2 + 1) * (H + 1);
    return a > b ? a : b;
}
__host__ __device__ inline size_t adj_smem_bytes(int H, int W) {
    return (size_t)(adj_nbuf(H, W) + H + (W / 2 + 1) + 3 * H + 3 + 3 * 16 + 8 + 2 * (W / 2 + 1) + 2 + 2 * H) *
           sizeof(double2);
}

// One CTA per frame f = blockIdx.x, blockIdx.x + gridDim.x, ... (blockDim.x = 512).
__global__ void __launch_bounds__(512) adj_kernel(Geom g, AdjArgs a) {
    extern __shared__ double2 adj_smem[];
    const int H = g.H, W = g.W, Wc = g.Wc, Hp = H / 2, HWc = H * Wc, t = threadIdx.x;
    const int CS = H + 1;                      // column stride of the buffer, padded against bank conflicts
    dfc* buf = (dfc*)adj_smem;                 // transforms in double-float, then X (weighted)
    double2* Ay = adj_smem + adj_nbuf(H, W);
    double2* Bx = Ay + H;
    double2* R = Bx + Wc;                      // [H][3], then the y-Nyquist middle part [3]
    double* red = (double*)(R + 3 * H + 3);    // [16 warps][6]
    dfc* BxF = (dfc*)(red + 6 * 16 + 16);      // [Wc] Bx as double-floats
    df* kapd = (df*)(BxF + Wc);                // [Wc] 2 pi kx' / W
    df* kap2d = kapd + Wc;                     // [Wc] -(2 pi kx' / W)^2
    dfc* AyF = (dfc*)(kap2d + Wc);             // [H] Ay as double-floats
    df* kapyd = (df*)(AyF + H);                // [H] 2 pi ky' / H
    __shared__ double st[8];                   // sy, sx, hyy, hxy, hxx, step, f
    __shared__ int sflag;
    const double eps = (double)g.eps, inv_hw = 1.0 / ((double)H * W);
    const dfc* FbD = g.FEdf;                   // F[b] as double-floats (H x Wc)
    double2* S = a.scratch + (size_t)blockIdx.x * HWc;
    dfc* Sd = (dfc*)S;                         // S as double-float scratch between the passes
    double2* P = a.part ? a.part + (size_t)blockIdx.x * HWc : nullptr;
    if (P)
        for (int i = t; i < HWc; i += blockDim.x) P[i] = make_double2(0.0, 0.0);
    const size_t fbytes = (size_t)H * a.pitch * (g.in_dtype == 0 ? 2 : 4);
    const df eps_d = df_from_double(eps);
    auto operand = [&](const void* fr, int y, int x) {
        const df I = df_make(pixel_f32(fr, g.in_dtype, (long long)y * a.pitch + x));
        if (g.method == 0) return I;
        const df ip = df_add(I, eps_d);
        return df_mul(ip, ip);
    };
    const df half = {0.5f, 0.f};
    // rows of tpr consecutive lanes each, for the per-row sums over kx
    const int tpr = (int)(blockDim.x / H) < 32 ? (int)(blockDim.x / H) : 32;
    for (long long f = blockIdx.x; f < a.n; f += gridDim.x) {
        const void* fr = (const char*)a.frames + (size_t)f * fbytes;
        // ---- F[a]: row pairs in buf, unpacked to S, columns in buf (column-major [Wc][H])
        for (int i = t; i < Hp * W; i += blockDim.x) {
            const int r = i / W, x = i - r * W;
            buf[r * W + brev(x, g.logW)] = dfc{operand(fr, 2 * r, x), operand(fr, 2 * r + 1, x)};
        }
        __syncthreads();
        fft_r2_passes(buf, g.logW, Hp, W, 1, g.twdf, g.logNtw, false);
        for (int i = t; i < Hp * Wc; i += blockDim.x) {
            const int r = i / Wc, kx = i - r * Wc;
            const dfc zk = buf[r * W + kx], zc = cconj(buf[r * W + ((W - kx) & (W - 1))]);
            Sd[(2 * r) * Wc + kx] = dfc{df_mul(df_add_abs(zk.re, zc.re), half), df_mul(df_add_abs(zk.im, zc.im), half)};
            Sd[(2 * r + 1) * Wc + kx] = dfc{df_mul(df_add_abs(zk.im, df_neg(zc.im)), half),
                                            df_neg(df_mul(df_add_abs(zk.re, df_neg(zc.re)), half))};
        }
        __syncthreads();
        for (int i = t; i < HWc; i += blockDim.x) {
            const int ky = i / Wc, kx = i - ky * Wc;
            buf[kx * CS + brev(ky, g.logH)] = Sd[i];
        }
        __syncthreads();
        fft_r2_passes(buf, g.logH, Wc, CS, 1, g.twdf, g.logNtw, false);
        // Sd keeps F[a] (row-major); the buffer takes X = F[a] conj F[b] with the fold weight
        // (1 at kx = 0 and W/2, 2 elsewhere: exact), all in double-float; each thread
        // rewrites the slot it read
        for (int i = t; i < HWc; i += blockDim.x) {
            const int ky = i / Wc, kx = i - ky * Wc;
            const dfc fd = buf[kx * CS + ky];
            Sd[i] = fd;
            const dfc x = cmul(fd, cconj(FbD[i]));
            buf[kx * CS + ky] = (kx == 0 || 2 * kx == W) ? x : dfc{df_scale(x.re, 2.f), df_scale(x.im, 2.f)};
        }
        for (int k = t; k < Wc; k += blockDim.x) {
            const double kap = 2.0 * CUDART_PI * adj_freq(k, W) / W;
            kapd[k] = df_from_double(kap);
            kap2d[k] = df_from_double(-kap * kap);
        }
        for (int k = t; k < H; k += blockDim.x) kapyd[k] = df_from_double(2.0 * CUDART_PI * adj_freq(k, H) / H);
        if (t == 0) {
            const Result q = a.rec[f];
            st[0] = ((double)q.ipy * g.u + rint((double)q.dy * g.u - (double)q.ipy * g.u)) / g.u;
            st[1] = ((double)q.ipx * g.u + rint((double)q.dx * g.u - (double)q.ipx * g.u)) / g.u;
            sflag = 0;
        }
        __syncthreads();
        const double sy0 = st[0], sx0 = st[1];
        // ---- Newton on grad f = 0
        int iters = 0;
        bool done = false;
        double hyy = 0.0, hxy = 0.0, hxx = 0.0;
        for (;;) {
            const double sy = st[0], sx = st[1];
            for (int k = t; k < H; k += blockDim.x) {
                double sn, cs;
                sincospi(2.0 * adj_freq(k, H) * sy / H, &sn, &cs);
                Ay[k] = make_double2(cs, sn);
                AyF[k] = dfc{df_from_double(cs), df_from_double(sn)};
            }
            for (int k = t; k < Wc; k += blockDim.x) {
                double sn, cs;
                sincospi(2.0 * adj_freq(k, W) * sx / W, &sn, &cs);
                Bx[k] = make_double2(cs, sn);
                BxF[k] = dfc{df_from_double(cs), df_from_double(sn)};
            }
            __syncthreads();
            if (done) break;                                    // Ay, Bx now at s*
            // row sums R0 = sum c X B, R1 = sum c X (i kx) B, R2 = sum c X (-kx^2) B, in
            // double-float (about 2^-46 a term; s* settles to about 1e-13 px)
            const int row = t / tpr, j = t - row * tpr;
            if (row < H) {
                const dfc z0 = dfc{df{0.f, 0.f}, df{0.f, 0.f}};
                dfc r0 = z0, r1 = z0, r2 = z0, m0 = z0, m1 = z0, m2 = z0;
                const bool nyq_row = 2 * row == H;
                for (int kx = j; kx < Wc; kx += tpr) {
                    const dfc xb = cmul(buf[kx * CS + row], BxF[kx]);
                    const df kap = kapd[kx], kap2 = kap2d[kx];
                    const dfc x1 = dfc{df_neg(df_mul(kap, xb.im)), df_mul(kap, xb.re)};
                    const dfc x2 = dfc{df_mul(kap2, xb.re), df_mul(kap2, xb.im)};
                    if (nyq_row && kx != 0 && 2 * kx != W) {
                        m0 = cadd(m0, xb); m1 = cadd(m1, x1); m2 = cadd(m2, x2);
                    } else {
                        r0 = cadd(r0, xb); r1 = cadd(r1, x1); r2 = cadd(r2, x2);
                    }
                }
                for (int o = tpr >> 1; o > 0; o >>= 1) {
                    r0 = cadd(r0, shfl_xor_dfc(r0, o)); r1 = cadd(r1, shfl_xor_dfc(r1, o));
                    r2 = cadd(r2, shfl_xor_dfc(r2, o)); m0 = cadd(m0, shfl_xor_dfc(m0, o));
                    m1 = cadd(m1, shfl_xor_dfc(m1, o)); m2 = cadd(m2, shfl_xor_dfc(m2, o));
                }
                if (j == 0) {
                    R[3 * row] = dfc_double(r0); R[3 * row + 1] = dfc_double(r1); R[3 * row + 2] = dfc_double(r2);
                    if (nyq_row) { R[3 * H] = dfc_double(m0); R[3 * H + 1] = dfc_double(m1); R[3 * H + 2] = dfc_double(m2); }
                }
            }
            __syncthreads();
            double v[6] = {0, 0, 0, 0, 0, 0};                   // f, fy, fx, fyy, fxy, fxx
            for (int ky = t; ky < H; ky += blockDim.x) {
                const double kap = 2.0 * CUDART_PI * adj_freq(ky, H) / H;
                const double2 A = Ay[ky], A1 = adj_i_times(kap, A);
                const double2 A2 = make_double2(-kap * kap * A.x, -kap * kap * A.y);
                const double2 r0 = R[3 * ky], r1 = R[3 * ky + 1], r2 = R[3 * ky + 2];
                v[0] += cmul(A, r0).x;  v[1] += cmul(A1, r0).x; v[2] += cmul(A, r1).x;
                v[3] += cmul(A2, r0).x; v[4] += cmul(A1, r1).x; v[5] += cmul(A, r2).x;
                if (2 * ky == H) {                              // middle columns: cos(pi sy) alone
                    double sn, cs;
                    sincospi(sy, &sn, &cs);
                    const double c0 = cs, c1 = -CUDART_PI * sn, c2 = -CUDART_PI * CUDART_PI * cs;
                    const double2 m0 = R[3 * H], m1 = R[3 * H + 1], m2 = R[3 * H + 2];
                    v[0] += c0 * m0.x; v[1] += c1 * m0.x; v[2] += c0 * m1.x;
                    v[3] += c2 * m0.x; v[4] += c1 * m1.x; v[5] += c0 * m2.x;
                }
            }
            adj_block_sum6(v, red);
            if (t == 0) {
                const double fy = v[1] * inv_hw, fx = v[2] * inv_hw;
                hyy = v[3] * inv_hw; hxy = v[4] * inv_hw; hxx = v[5] * inv_hw;
                const double det = hyy * hxx - hxy * hxy;
                const double dy = (hxx * fy - hxy * fx) / det, dx = (hyy * fx - hxy * fy) / det;
                st[0] = sy - dy;
                st[1] = sx - dx;
                st[2] = hyy; st[3] = hxy; st[4] = hxx;
                ++iters;
                const double step = fmax(fabs(dy), fabs(dx));
                if (!(step >= 1e-11)) {
                    sflag = 1;                                             // settled (or NaN: stop)
                } else if (iters >= kAdjIters) {
                    sflag = 2;
                }
            }
            __syncthreads();
            done = sflag != 0;
        }
        hyy = st[2]; hxy = st[3]; hxx = st[4];
        const double sy = st[0], sx = st[1];
        int status = 0;
        if (sflag != 1) status |= kAdjNotConverged;
        const double det = hyy * hxx - hxy * hxy;
        const bool kind = det > 0.0 && (g.method == 0 ? hyy < 0.0 : hyy > 0.0);
        if (!kind) status |= kAdjNotExtremum;
        if (!(fabs(sy - sy0) <= 1.0 && fabs(sx - sx0) <= 1.0)) status |= kAdjFar;
        if (t == 0) {
            if (a.peak) { a.peak[2 * f] = sx; a.peak[2 * f + 1] = sy; }
            if (a.status) a.status[f] = status;
        }
        if (!a.g) { __syncthreads(); continue; }
        // ---- the VJP: w = -Hf^{-1} g (zero for a frame without a valid s*)
        double wy = 0.0, wx = 0.0;
        if (status == 0) {
            const double gx = a.g[2 * f], gy = a.g[2 * f + 1];
            wy = -(hxx * gy - hxy * gx) / det;
            wx = -(hyy * gx - hxy * gy) / det;
        }
        // dL/db spectra, symmetrised, into this CTA's partial sum
        // (in double-float: the phases AyF, BxF, the frequencies kapy, kap, F[a] and F[b])
        const df wyd = df_from_double(wy), wxd = df_from_double(wx);
        // k' and the pair's k' (negated, except on a Nyquist index), each weighted by w, and
        // the phase at k and at the pair
        auto wdot = [&](int ky, int kx, df* kw, df* kwp, dfc* ph, dfc* pph) {
            const bool ny = 2 * ky == H, nx = 2 * kx == W;
            const df my = kapyd[ky], mx = kapd[kx];
            *kw = df_add(df_mul(wyd, my), df_mul(wxd, mx));
            *kwp = df_add(df_mul(wyd, ny ? my : df_neg(my)), df_mul(wxd, (nx || kx == 0) ? mx : df_neg(mx)));
            const dfc ay = AyF[ky], bx = BxF[kx];
            *ph = cmul(ay, bx);
            *pph = cmul(ny ? ay : cconj(ay), nx ? bx : cconj(bx));
        };
        if (P) {
            for (int i = t; i < HWc; i += blockDim.x) {
                const int ky = i / Wc, kx = i - ky * Wc;
                df kw, kwp;
                dfc ph, pph;
                wdot(ky, kx, &kw, &kwp, &ph, &pph);
                const dfc fa = Sd[i];
                const dfc q = cmul(ph, fa), qp = cmul(pph, cconj(fa));
                // z = i kw q, zp = i kwp qp; the partial sum takes (z + conj-free pair) / 2
                const df sx = df_add(df_neg(df_mul(kw, q.im)), df_neg(df_mul(kwp, qp.im)));   // z.x + zp.x
                const df sy = df_add(df_mul(kw, q.re), df_neg(df_mul(kwp, qp.re)));          // z.y - zp.y
                const double2 p = P[i];
                P[i] = make_double2(p.x + 0.5 * df_to_double(sx), p.y + 0.5 * df_to_double(sy));
            }
        }
        // dL/da: V(k) = conj of (2 pi i w.k') conj F[b](k) e^{2 pi i k'.s}, symmetrised, then
        // (1/HW) sum_k V_h(k) e^{+2 pi i k.r} through a complex-to-real transform
        if (a.g_frames) {
            for (int i = t; i < HWc; i += blockDim.x) {
                const int ky = i / Wc, kx = i - ky * Wc;
                df kw, kwp;
                dfc ph, pph;
                wdot(ky, kx, &kw, &kwp, &ph, &pph);
                const dfc fb = FbD[i];
                const dfc q = cmul(ph, cconj(fb)), qp = cmul(pph, fb);
                // Z(k) = i kw q, Z(pair) = i kwp qp; V = conj Z; V_h = (V(k) + conj V(pair)) / 2
                // = (conj Z(k) + Z(pair)) / 2
                const df vx = df_add(df_neg(df_mul(kw, q.im)), df_neg(df_mul(kwp, qp.im)));   // Z.x + Zp.x
                const df vy = df_add(df_neg(df_mul(kw, q.re)), df_mul(kwp, qp.re));          // -Z.y + Zp.y
                buf[kx * CS + brev(ky, g.logH)] = dfc{df_scale(vx, 0.5f), df_scale(vy, 0.5f)};
            }
            __syncthreads();
            fft_r2_passes(buf, g.logH, Wc, CS, 1, g.twdf, g.logNtw, true);
            for (int i = t; i < HWc; i += blockDim.x) {
                const int ky = i / Wc, kx = i - ky * Wc;
                Sd[i] = buf[kx * CS + ky];
            }
            __syncthreads();
            for (int i = t; i < Hp * W; i += blockDim.x) {
                const int r = i / W, kx = i - r * W;
                dfc ye, yo;
                if (kx < Wc) { ye = Sd[(2 * r) * Wc + kx]; yo = Sd[(2 * r + 1) * Wc + kx]; }
                else { ye = cconj(Sd[(2 * r) * Wc + W - kx]); yo = cconj(Sd[(2 * r + 1) * Wc + W - kx]); }
                buf[r * W + brev(kx, g.logW)] = dfc{df_add_abs(ye.re, df_neg(yo.im)), df_add_abs(ye.im, yo.re)};
            }
            __syncthreads();
            fft_r2_passes(buf, g.logW, Hp, W, 1, g.twdf, g.logNtw, true);
            float* gI = a.g_frames + (size_t)f * H * W;
            for (int i = t; i < Hp * W; i += blockDim.x) {
                const int r = i / W, x = i - r * W;
                double d0 = df_to_double(buf[r * W + x].re) * inv_hw, d1 = df_to_double(buf[r * W + x].im) * inv_hw;
                if (g.method != 0) {
                    d0 *= 2.0 * ((double)pixel_f32(fr, g.in_dtype, (long long)(2 * r) * a.pitch + x) + eps);
                    d1 *= 2.0 * ((double)pixel_f32(fr, g.in_dtype, (long long)(2 * r + 1) * a.pitch + x) + eps);
                }
                gI[(2 * r) * W + x] = (float)d0;
                gI[(2 * r + 1) * W + x] = (float)d1;
            }
        }
        __syncthreads();
    }
}

// dL/dE, columns: sum the CTAs' partial spectra in order, inverse over y. One CTA per column.
__global__ void __launch_bounds__(128) adj_ref_cols(Geom g, const double2* part, int nparts, double2* Y) {
    __shared__ double2 z[128];
    __shared__ double2 tw[64];
    const int H = g.H, Wc = g.Wc, HWc = H * Wc, kx = blockIdx.x, t = threadIdx.x;
    for (int k = t; k < g.Ntw / 2; k += blockDim.x) tw[k] = g.tw64[k];
    double2 s = make_double2(0.0, 0.0);
    if (t < H)
        for (int b = 0; b < nparts; ++b) {
            const double2 v = part[(size_t)b * HWc + t * Wc + kx];
            s.x += v.x;
            s.y += v.y;
        }
    if (t < H) z[brev(t, g.logH)] = s;
    __syncthreads();
    fft_r2_passes(z, g.logH, 1, H, 1, tw, g.logNtw, true);
    if (t < H) Y[t * Wc + kx] = z[t];
}

// dL/dE, rows: inverse over x of two rows at once (Hermitian in kx), scale 1/(HW), chain
// rule (CC-SN: b = 1/(E + eps), dL/dE = -b^2 dL/db). One CTA per row pair.
__global__ void __launch_bounds__(128) adj_ref_rows(Geom g, const double2* Y, float* g_ref) {
    __shared__ double2 z[128];
    __shared__ double2 tw[64];
    const int W = g.W, Wc = g.Wc, r = blockIdx.x, t = threadIdx.x;
    for (int k = t; k < g.Ntw / 2; k += blockDim.x) tw[k] = g.tw64[k];
    if (t < W) {
        double2 ye, yo;
        if (t < Wc) { ye = Y[(2 * r) * Wc + t]; yo = Y[(2 * r + 1) * Wc + t]; }
        else { ye = cconj(Y[(2 * r) * Wc + W - t]); yo = cconj(Y[(2 * r + 1) * Wc + W - t]); }
        z[brev(t, g.logW)] = make_double2(ye.x - yo.y, ye.y + yo.x);
    }
    __syncthreads();
    fft_r2_passes(z, g.logW, 1, W, 1, tw, g.logNtw, true);
    if (t < W) {
        const double s = 1.0 / ((double)g.H * W);
        double d0 = z[t].x * s, d1 = z[t].y * s;
        if (g.method != 0) {
            const double b0 = g.b64[(2 * r) * W + t], b1 = g.b64[(2 * r + 1) * W + t];
            d0 *= -b0 * b0;
            d1 *= -b1 * b1;
        }
        g_ref[(2 * r) * W + t] = (float)d0;
        g_ref[(2 * r + 1) * W + t] = (float)d1;
    }
}

}  // namespace ccst
