// ccst.cu -- the C ABI of libccst (declared in include/ccst.h): context set-up,
// launches, CUDA-graph replay of batches and the serving tickets.
#include <algorithm>
#include <condition_variable>
#include <deque>
#include <random>
#include <unordered_map>
#include <atomic>
#include <chrono>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <cmath>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <tuple>
#include <vector>

#include <cuda_runtime.h>

#include "ccst.h"
#include "ccst_kernels.cuh"
#include "ccst_adjoint.cuh"
#include "ccst_generic.cuh"
#include "ccst_mixed.cuh"

using namespace ccst;

static_assert(sizeof(ccst_result) == sizeof(Result), "result record layout");
static_assert(sizeof(ccst_result) == 24, "result record is 24 bytes");

namespace {

constexpr int kTickets = 64;      // in-flight submissions per context
constexpr int kHostSlots = 4;     // staging slots of the pipelined host path
constexpr size_t kMaxGraphs = 512;
// static shared memory beside the dynamic plan: the tensor-core state of the 128 x 128
// kernels (TcShared), and in the ROI kernel also its Geom and work-item index
constexpr int kTcStaticSmem = 64;
constexpr int kRoisStaticSmem = (int)sizeof(Geom) + 128;

// Guard thresholds, in units of the FP32 unit roundoff eps32 times sum w|X|. Each is a
// multiple of the largest surface error measured against the FP64 oracle at that level:
// the integer surface errs by at most 2.2 eps32 sum|X| (threshold 32), the peak-relative
// upsampled surface by under 0.125 (threshold 1), the FP32 pair differences by under
// 0.0026 (threshold 0.02). Points the threshold cannot separate go to the next level.
constexpr float kEps32 = 1.1920929e-07f;
constexpr float kTauInt = 32.0f * kEps32;
constexpr float kTau0 = 1.0f * kEps32;
constexpr float kTau1 = 0.02f * kEps32;
// The same three levels for the FP32 general-size kernel (ccst_mixed.cu), which re-decides
// what they leave open from a double-float spectrum and otherwise falls back to the double-
// float kernel. Largest errors measured against the FP64 oracle (u = 100, in eps32 sum w|X|):
//   integer surface                 4.1 (all sides, both methods)
//   peak-relative surface, CC-U     0.056 (sides 48 to 256)
//   the same, CC-SN                 0.0083 at 48, 0.0068 at 96, 0.0030 at 192, 0.0013 at 256
//   pair differences                0.0014 (CC-U), 0.0003 (CC-SN)
// Each threshold keeps an 8x margin or more; a level-1 winner must lead by 2 tau1 (two
// differences, each within tau1). CC-SN gets its own because its sum w|X| is dominated by
// the DC term, which the peak-relative sums never see; and the larger its side, the more
// that term dominates, so its tau0 falls with the side.
constexpr float kMixTauInt = 32.0f * kEps32;
constexpr float kMixTau0 = 1.0f * kEps32;
constexpr float kMixTau1 = 0.02f * kEps32;
constexpr float kMixTau1Sn = 0.005f * kEps32;
static float mix_tau0_sn(int N) { return (N <= 96 ? 0.125f : N <= 192 ? 0.06f : 0.03f) * kEps32; }
constexpr int kMixCounters = 8;     // per lane: [0] fallback count, [1 + s] item counter of FP32 segment s

std::mutex g_create_err_mu;
std::string g_create_err = "no error";

// ------------------------------------------------------------ init kernels
__global__ void init_twiddles(int Ntw, double2* tw64, float2* tw32) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < Ntw / 2; k += gridDim.x * blockDim.x) {
        double s, c;
        sincospi(-2.0 * (double)k / (double)Ntw, &s, &c);
        tw64[k] = make_double2(c, s);
        tw32[k] = make_float2((float)c, (float)s);
    }
}

__global__ void init_tables(Geom g, float* cm1, float* sA, float* wc, float* ws, float* gc, uint2* tah, uint2* tbh) {
    const long long Dy = (long long)g.u * g.H, Dx = (long long)g.u * g.W;
    const int nA = g.Hh * g.T1p, nB = g.Wc * g.T1p;
    const int Hq = g.Hh / 2, SAq = g.SA / 2, T1 = g.T1p, T8 = g.T1p8;
    // the tensor-core tables: uint2 fp16 pairs (warp-level form), or with g.tc single fp16
    // values of four 128-byte-swizzled K-major matrices each (stage A: [cos - 1, sin] x
    // [hi, lo], RA rows t - 1, K = m - 1; stage B: [w cos, w sin] x [hi, lo], T1p8 rows tx,
    // K = kx)
    const int nAh = g.tc ? 4 * g.RA * 64 : 2 * g.TAB * Hq, nBh = g.tc ? 4 * T8 * 64 : 2 * T1 * SAq, nBn = 2 * T8;
    const float s13 = 8192.f;                                // 2^13: table scale of the fp16 pairs
    float* bn = g.tc ? (float*)((unsigned char*)tbh + (size_t)4 * T8 * 128) : (float*)(tbh + nBh);
    // w cos, w sin and w (cos - 1) of 2 pi kx' t/(uW), kx' the signed frequency (W/2 -> -W/2)
    auto wcs = [&](int kx, int t, float* a, float* b, float* c) {
        const int kxs = (kx < g.W / 2) ? kx : kx - g.W;
        const double w = (kx == 0 || 2 * kx == g.W) ? 1.0 : 2.0;
        *a = 0.f; *b = 0.f; *c = 0.f;
        if (t <= g.h0) {
            long long r = ((long long)kxs * t) % Dx;
            if (r < 0) r += Dx;
            double s, co;
            sincospi(2.0 * (double)r / (double)Dx, &s, &co);
            const double h = sinpi((double)r / (double)Dx);
            *a = (float)(w * co);
            *b = (float)(w * s);
            *c = (float)(w * (-2.0 * h * h));
        }
    };
    auto cm1_s = [&](int m, int t, float* c1, float* s1) {
        *c1 = 0.f;
        *s1 = 0.f;
        if (t >= 0 && t <= g.h0) {
            const long long r = ((long long)m * t) % Dy;     // angle 2 pi r / (uH)
            const double h = sinpi((double)r / (double)Dy);
            *c1 = (float)(-2.0 * h * h);                     // cos - 1 without cancellation
            *s1 = (float)sinpi(2.0 * (double)r / (double)Dy);
        }
    };
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nA + nB + nAh + nBh + nBn; i += gridDim.x * blockDim.x) {
        if (i < nA) {
            const int m = i / g.T1p + 1, t = i % g.T1p;
            cm1_s(m, t, &cm1[i], &sA[i]);
        } else if (i < nA + nB) {
            const int k = i - nA;
            const int kx = k / g.T1p, t = k % g.T1p;
            wcs(kx, t, &wc[k], &ws[k], &gc[k]);
        } else if (g.tc && i < nA + nB + nAh) {
            const int k = i - nA - nB;
            const int mat = k / (g.RA * 64), rem = k - mat * g.RA * 64, ta = rem / 64, kk = rem - ta * 64;
            float c1, s1;
            cm1_s(kk + 1, ta + 1, &c1, &s1);
            const float v = s13 * (mat < 2 ? c1 : s1);
            const __half hi = __float2half_rn(v);
            const __half out = (mat & 1) ? __float2half_rn(v - __half2float(hi)) : hi;
            *(__half*)((unsigned char*)tah + (size_t)mat * g.RA * 128 + sw128_off(ta, kk)) = out;
        } else if (g.tc && i < nA + nB + nAh + nBh) {
            const int k = i - nA - nB - nAh;
            const int mat = k / (T8 * 64), rem = k - mat * T8 * 64, tx = rem / 64, kx = rem - tx * 64;
            float a, b, d;
            wcs(kx, tx, &a, &b, &d);
            const float v = s13 * (mat < 2 ? a : b);
            const __half hi = __float2half_rn(v);
            const __half out = (mat & 1) ? __float2half_rn(v - __half2float(hi)) : hi;
            *(__half*)((unsigned char*)tbh + (size_t)mat * T8 * 128 + sw128_off(tx, kx)) = out;
        } else if (i < nA + nB + nAh) {
            // stage-A pairs: [cm1 | s][t - 1][pair p of m = 2p+1, 2p+2], pairs swizzled by row
            const int k = i - nA - nB;
            const int which = k / (g.TAB * Hq), rem = k - which * g.TAB * Hq;
            const int ta = rem / Hq, p = (rem - ta * Hq) ^ pswz(ta, Hq);
            float a, b, cc, d;
            cm1_s(2 * p + 1, ta + 1, &a, &b);
            cm1_s(2 * p + 2, ta + 1, &cc, &d);
            tah[k] = which ? split_pair(s13 * b, s13 * d) : split_pair(s13 * a, s13 * cc);
        } else if (i < nA + nB + nAh + nBh) {
            // stage-B pairs: [w cos | w sin][tx][pair p of kx = 2p, 2p+1], pairs swizzled by row
            const int k = i - nA - nB - nAh;
            const int which = k / (T1 * SAq), rem = k - which * T1 * SAq;
            const int tx = rem / SAq, p = (rem - tx * SAq) ^ pswz(tx, SAq);
            float a0, b0, c0, a1, b1, c1;
            wcs(2 * p, tx, &a0, &b0, &c0);
            wcs(2 * p + 1, tx, &a1, &b1, &c1);
            tbh[k] = which ? split_pair(s13 * b0, s13 * b1) : split_pair(s13 * a0, s13 * a1);
        } else {
            // kx = W/2 column in FP32: [w cos | w sin][tx], tx < T1p8
            const int k = i - nA - nB - nAh - nBh;
            const int which = k / T8, tx = k - which * T8;
            float a, b, d;
            wcs(g.W / 2, tx, &a, &b, &d);
            bn[k] = which ? b : a;
        }
    }
}

// Double-float copies: FFT twiddles, the reference spectrum, and the two-level tables of
// exp(2 pi i n / D) for D = uH and uW (coarse steps of B, fine steps of 1).
__global__ void init_dfloat(Geom g, const double2* tw64, const double2* FE64, dfc* twdf, dfc* FEdf,
                            dfc* eyc, dfc* eyf, dfc* exc, dfc* exf, int ncy, int ncx) {
    const long long Dy = (long long)g.u * g.H, Dx = (long long)g.u * g.W;
    const int nFE = g.H * g.Wc, ntw = g.Ntw / 2;
    const int total = ntw + nFE + ncy + g.By + ncx + g.Bx;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
        int k = i;
        if (k < ntw) {
            twdf[k] = {df_from_double(tw64[k].x), df_from_double(tw64[k].y)};
            continue;
        }
        k -= ntw;
        if (k < nFE) {
            FEdf[k] = {df_from_double(FE64[k].x), df_from_double(FE64[k].y)};
            continue;
        }
        k -= nFE;
        long long n;
        long long D;
        dfc* dst;
        if (k < ncy) { n = (long long)k * g.By; D = Dy; dst = eyc + k; }
        else if ((k -= ncy) < g.By) { n = k; D = Dy; dst = eyf + k; }
        else if ((k -= g.By) < ncx) { n = (long long)k * g.Bx; D = Dx; dst = exc + k; }
        else { k -= ncx; n = k; D = Dx; dst = exf + k; }
        double s, c;
        sincospi(2.0 * (double)(n % D) / (double)D, &s, &c);
        *dst = {df_from_double(c), df_from_double(s)};
    }
}

__global__ void init_ref_operand(Geom g, const float* ref, double* b64) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < g.H * g.W; i += gridDim.x * blockDim.x) {
        const double e = (double)ref[i];
        b64[i] = (g.method == 0) ? e : 1.0 / (e + (double)g.eps);
    }
}

__global__ void __launch_bounds__(256) init_ref_spectrum(Geom g, double2* work, double2* FE64, float2* FE32) {
    __shared__ double red[32];
    double2* Z = work;
    double2* Xh = work + (size_t)(g.H / 2) * g.W;
    fft_r2c_f64_global(g, g.b64, nullptr, 0, Z, Xh, red);
    for (int idx = threadIdx.x; idx < g.H * g.Wc; idx += blockDim.x) {
        const int ky = idx / g.Wc, kx = idx - ky * g.Wc;
        const double2 v = Xh[ky * g.Wcp + kx];
        FE64[idx] = v;
        FE32[idx] = make_float2((float)v.x, (float)v.y);
    }
}

bool is_pow2(int x) { return x > 0 && (x & (x - 1)) == 0; }
int ilog2(int x) { int l = 0; while ((1 << l) < x) ++l; return l; }

// Sizes, layout choices and the shared-memory plan for H x W frames and params p.
// Returns false if no plan fits in smem_limit bytes.
bool plan_geometry(int H, int W, const ccst_params& p, size_t smem_limit, Geom* out) {
    Geom g{};
    g.H = H; g.W = W; g.logH = ilog2(H); g.logW = ilog2(W); g.Hh = H / 2;
    g.Wc = W / 2 + 1; g.Wcp = (g.Wc + 1) & ~1;
    g.SA = W / 2;
    g.SZ = packed_row_stride(W);                         // the stride the kernels assume
    g.u = p.upsample; g.M = (3 * p.upsample + 1) / 2; g.h0 = g.M / 2; g.pmax = g.M - 1 - g.h0;
    g.T1p = (g.h0 + 1 + 3) & ~3;
    g.T1p8 = (g.h0 + 1 + 7) & ~7;
    g.Ntw = H > W ? H : W; g.logNtw = ilog2(g.Ntw);
    g.lN1h = ilog2(split_n1(H)); g.lN2h = ilog2(split_n2(H));
    g.lN1w = ilog2(split_n1(W)); g.lN2w = ilog2(split_n2(W));
    g.method = p.method; g.in_dtype = p.in_dtype; g.eps = p.eps;
    g.sense = p.method == CCST_CC_U ? 1.f : -1.f;
    g.tau_int = kTauInt; g.tau0 = kTau0; g.tau1 = kTau1;
    g.guard = (p.flags & CCST_FLAG_TIE_GUARD) ? 1 : 0;
    // the 128 x 128 kernels hold the tensor-core state in static shared memory
    if (H == 128 && W == 128) smem_limit -= kTcStaticSmem;
    const int h15 = ((g.h0 + 14) / 15) * 15;
    for (int smem_tables = 1; smem_tables >= 0; --smem_tables) {
        for (int tc = h15; tc >= 15; tc -= 15) {
            g.TC = tc;
            g.nchunk = (g.h0 + tc - 1) / tc;
            g.TAB = g.nchunk * tc;
            g.tables_smem = smem_tables;
            g.tc = 0;
            // the 5th-generation tensor-core contraction: 128 x 128 frames (K = 64 in both
            // stages), one chunk, tables in shared memory, every operand and accumulator
            // within 128 rows / lanes
            if (H == 128 && W == 128 && smem_tables && g.nchunk == 1 && tc <= 128 && g.T1p8 <= 128) {
                Geom t = g;
                t.tc = 1;
                t.RA = (t.TAB + 7) & ~7;
                t.NB = (t.TC + 15) & ~15;
                if (t.RA <= 128 && t.NB <= 128 && smem_plan(t).total <= smem_limit) { *out = t; return true; }
            }
            if (smem_plan(g).total <= smem_limit) { *out = g; return true; }
        }
    }
    return false;
}


// ------------------------------------------------- real-time reference (Sec. III B)
// One cooperative launch sets the reference spectrum E and refreshes the reference from
// it: FP64 2-D transforms over the H x (W/2+1) half spectrum, row pairs and columns
// spread over the CTAs, with three grid barriers between the phases:
//   rows:    Y = F_x[frame + off], two real rows packed into one complex row
//            (mean mode: E = the sum of the partial spectra / the frame count, Eq. 8)
//   columns: F = F_y Y; E = a0 F(k) e^{+2 pi i (ky' dy/H + kx' dx/W)} + b1 E (Eq. 9), or
//            E = F when starting (mean mode: E as it is); Y = F_y^-1 E
//   rows:    b64 = F_x^-1 Y / (HW) (CC-SN: 1 / that); Y = F_x b64
//   columns: FE64 / FE32 / FEdf = F_y Y
// Buffers written by other CTAs in the launch are read with L2-only loads. One thread per
// element of a row or column: blockDim (128) >= H, W.
struct RtArgs {
    const void* frame;          // device frame (in_dtype), rows `pitch` elements apart
    long long pitch;
    double off;                 // added to every pixel (CC-SN: eps)
    int mode;                   // kRtStart: E = F[frame]; kRtUpdate: Eq. 9 with *rec; kRtMean: Eq. 8
    double a0, b1;
    Result* rec;                // record of the frame (upd): flags gain 0x40 when the update fails
    double2* E;                 // [H][Wc] filtered spectrum (filter state)
    double2* Y;                 // [H][Wc] work spectrum
    double* b64;                // [H][W]  reference operand
    double2* FE64;
    float2* FE32;
    dfc* FEdf;
    unsigned* sync;             // [0] arrivals, [1] generation, [2] sticky error
    unsigned base;              // 3 G s: arrivals before this launch (s launches since the reset)
    unsigned extra;             // arrivals the barriers wait for beyond the grid (0; tests: 1)
    unsigned limit;             // polls before a barrier gives up
    const double2* part;        // kRtMean: nparts partial sums [nparts][H][Wc] ...
    int nparts;
    const unsigned* count;      // ... over *count frames
    unsigned* next;             // frame counter of the tracking kernel, zeroed here (or null)
    int frame_f64;              // kRtStart: `frame` is an FP64 image (pitch in doubles), not in_dtype
};

constexpr int kRtStart = 0, kRtUpdate = 1, kRtMean = 2;

constexpr unsigned kRtStale = 0x40u;     // the reference update after this frame did not run

// Grid barrier with a bounded wait: a count-up barrier on sync[0]. Barrier k (1, 2, 3) of
// the launch numbered s since the counter was zeroed completes when the counter reaches
// 3 s G + k G (+ extra), G = gridDim.x: each CTA adds one arrival with release semantics
// and polls with acquire loads. Returns false (and sets the sticky error sync[2]) when the
// others do not arrive within the limit; the CTA must then leave the kernel.
__device__ bool rt_grid_barrier(unsigned* sync, unsigned target, unsigned limit) {
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(sync) : "memory");
        bool good = true;
        unsigned v, it = 0;
        for (;;) {
            asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(sync) : "memory");
            if ((int)(v - target) >= 0) break;
            if (++it > limit) { good = false; atomicOr(sync + 2, 1u); break; }
        }
        ok = good;
    }
    __syncthreads();
    return ok != 0;
}

// A launch that leaves before its barriers still counts its three arrivals.
__device__ inline void rt_skip_barriers(unsigned* sync) {
    if (threadIdx.x == 0) atomicAdd(sync, 3u);
}

// The displacement a record carries is d = (p u + t) / u exactly; this is p u + t.
__device__ inline long long rt_grid_index(float d, int p, int u) {
    return (long long)p * u + llrint((double)d * u - (double)p * u);
}

// e^{+2 pi i k' d / N} on one axis of length N as a complex double-float, d = q / u
// (q = p u + t), from the context's two-level table of e^{2 pi i n / D}, D = u N, with
// n = k' q mod D reduced exactly in integers. The Nyquist bin of an even N takes the real
// part, cos(pi d).
__device__ inline dfc rt_axis_phase_df(int k, int N, long long q, long long D, const dfc* coarse, const dfc* fine,
                                       int B) {
    const bool nyq = 2 * k == N;
    const long long ks = (nyq || k < (N >> 1)) ? k : k - N;
    long long n = (ks * q) % D;
    if (n < 0) n += D;
    dfc e = df_twiddle(coarse, fine, B, n);
    if (nyq) e.im = df{0.f, 0.f};
    return e;
}

// Y (work spectrum) holds complex double-floats in its 16-byte slots, read and written
// around L1.
__device__ __forceinline__ dfc ld_dfc_cg(const double2* p) {
    const float4 v = __ldcg((const float4*)p);
    return dfc{df{v.x, v.y}, df{v.z, v.w}};
}
__device__ __forceinline__ void st_dfc_cg(double2* p, dfc v) {
    __stcg((float4*)p, make_float4(v.re.hi, v.re.lo, v.im.hi, v.im.lo));
}
__device__ __forceinline__ dfc dfc_from(double2 v) { return dfc{df_from_double(v.x), df_from_double(v.y)}; }
__device__ __forceinline__ double2 dfc_to(dfc v) { return make_double2(df_to_double(v.re), df_to_double(v.im)); }

// the two real rows held in z = Y[2r] + i Y[2r+1] after a row transform, split and stored
__device__ __forceinline__ void rt_store_row_pair(const RtArgs& a, int W, int Wc, int r, const dfc* z, int kx) {
    const df half = {0.5f, 0.f};
    const dfc zk = z[kx], zc = cconj(z[(W - kx) & (W - 1)]);
    st_dfc_cg(a.Y + (2 * r) * Wc + kx, dfc{df_mul(df_add_abs(zk.re, zc.re), half), df_mul(df_add_abs(zk.im, zc.im), half)});
    st_dfc_cg(a.Y + (2 * r + 1) * Wc + kx, dfc{df_mul(df_add_abs(zk.im, df_neg(zc.im)), half),
                                                df_neg(df_mul(df_add_abs(zk.re, df_neg(zc.re)), half))});
}

// forward transform of the frame's real row pair (2r, 2r+1) into Y
__device__ void rt_row_pair_fwd(const Geom& g, const RtArgs& a, int r, dfc* z, const dfc* tw) {
    const int W = g.W, Wc = g.Wc;
    const df off = df_from_double(a.off);
    for (int x = threadIdx.x; x < W; x += blockDim.x) {
        const long long i0 = (long long)(2 * r) * a.pitch + x, i1 = i0 + a.pitch;
        const df p0 = a.frame_f64 ? df_from_double(((const double*)a.frame)[i0]) : df_make(pixel_f32(a.frame, g.in_dtype, i0));
        const df p1 = a.frame_f64 ? df_from_double(((const double*)a.frame)[i1]) : df_make(pixel_f32(a.frame, g.in_dtype, i1));
        z[brev(x, g.logW)] = dfc{df_add(p0, off), df_add(p1, off)};
    }
    __syncthreads();
    fft_r2_passes(z, g.logW, 1, W, 1, tw, g.logNtw, false);
    for (int kx = threadIdx.x; kx < Wc; kx += blockDim.x) rt_store_row_pair(a, W, Wc, r, z, kx);
    __syncthreads();
}

// column kx of Y, transformed over y (in natural order in z)
__device__ void rt_col_fwd(const Geom& g, const RtArgs& a, int kx, dfc* z, const dfc* tw) {
    for (int ky = threadIdx.x; ky < g.H; ky += blockDim.x) z[brev(ky, g.logH)] = ld_dfc_cg(a.Y + ky * g.Wc + kx);
    __syncthreads();
    fft_r2_passes(z, g.logH, 1, g.H, 1, tw, g.logNtw, false);
}

// The transforms run in double-float on the FP32 pipes (FP64 chains in two warps were the
// update's latency); the filter state E and the operand b64 stay FP64.
__global__ void __launch_bounds__(128) rt_update(Geom g, RtArgs a) {
    __shared__ dfc z[128];
    __shared__ dfc tw[64];                                 // FFT twiddles, Ntw/2 <= 64
    const int H = g.H, W = g.W, Wc = g.Wc, Hp = H / 2, HWc = H * Wc;
    const bool upd = a.mode == kRtUpdate;
    if (a.next && blockIdx.x == 0 && threadIdx.x == 0) *a.next = 0;   // frame counter of the next tracking launch
    if (__ldcg(a.sync + 2) != 0) {                         // an earlier update failed: E is stale
        if (upd && blockIdx.x == 0 && threadIdx.x == 0) atomicOr(&a.rec->flags, kRtStale);
        return rt_skip_barriers(a.sync);
    }
    long long qy = 0, qx = 0;
    if (upd) {
        const Result q = *a.rec;
        if (q.flags & 0x20u) return rt_skip_barriers(a.sync);   // no displacement: E stays
        qy = rt_grid_index(q.dy, q.ipy, g.u);
        qx = rt_grid_index(q.dx, q.ipx, g.u);
    }
    const long long Dy = (long long)g.u * H, Dx = (long long)g.u * W;
    for (int k = threadIdx.x; k < g.Ntw / 2; k += blockDim.x) tw[k] = g.twdf[k];
    __syncthreads();
    const unsigned G = gridDim.x, b1t = a.base + G + a.extra, b2t = b1t + G, b3t = b2t + G;
    auto failed = [&]() {
        if (upd && threadIdx.x == 0) atomicOr(&a.rec->flags, kRtStale);
    };
    if (a.mode == kRtMean) {
        // E = (1/N) sum of the partial spectra, in a fixed order; no frames: E stays
        const unsigned cnt = __ldcg(a.count);
        if (cnt == 0) return rt_skip_barriers(a.sync);
        const double inv = 1.0 / (double)cnt;
        for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < HWc; i += gridDim.x * blockDim.x) {
            double2 s = make_double2(0.0, 0.0);
            for (int b = 0; b < a.nparts; ++b) {
                const double2 v = __ldcg(a.part + (size_t)b * HWc + i);
                s.x += v.x;
                s.y += v.y;
            }
            __stcg(a.E + i, make_double2(s.x * inv, s.y * inv));
        }
    } else {
        for (int r = blockIdx.x; r < Hp; r += gridDim.x) rt_row_pair_fwd(g, a, r, z, tw);
    }
    if (!rt_grid_barrier(a.sync, b1t, a.limit)) return failed();
    const int t = threadIdx.x;
    for (int kx = blockIdx.x; kx < Wc; kx += gridDim.x) {
        dfc e = dfc{df{0.f, 0.f}, df{0.f, 0.f}};
        if (a.mode == kRtMean) {
            if (t < H) e = dfc_from(__ldcg(a.E + t * Wc + kx));
        } else {
            rt_col_fwd(g, a, kx, z, tw);
            if (t < H) {
                e = z[t];
                double2 ed = dfc_to(e);
                if (upd) {
                    const double2 s = dfc_to(cmul(e, cmul(rt_axis_phase_df(t, H, qy, Dy, g.eyc, g.eyf, g.By),
                                                          rt_axis_phase_df(kx, W, qx, Dx, g.exc, g.exf, g.Bx))));
                    const double2 p = __ldcg(a.E + t * Wc + kx);
                    ed = make_double2(a.a0 * s.x + a.b1 * p.x, a.a0 * s.y + a.b1 * p.y);
                    e = dfc_from(ed);
                }
                __stcg(a.E + t * Wc + kx, ed);
            }
        }
        __syncthreads();
        if (t < H) z[brev(t, g.logH)] = e;
        __syncthreads();
        fft_r2_passes(z, g.logH, 1, H, 1, tw, g.logNtw, true);
        if (t < H) st_dfc_cg(a.Y + t * Wc + kx, z[t]);
        __syncthreads();
    }
    if (!rt_grid_barrier(a.sync, b2t, a.limit)) return failed();
    const float sc = 1.0f / ((float)H * W);                // a power of two: exact on a double-float
    for (int r = blockIdx.x; r < Hp; r += gridDim.x) {
        // Y rows 2r, 2r+1 are Hermitian in kx: one complex inverse gives both real rows
        if (t < W) {
            dfc ye, yo;
            if (t < Wc) {
                ye = ld_dfc_cg(a.Y + (2 * r) * Wc + t);
                yo = ld_dfc_cg(a.Y + (2 * r + 1) * Wc + t);
            } else {
                ye = cconj(ld_dfc_cg(a.Y + (2 * r) * Wc + W - t));
                yo = cconj(ld_dfc_cg(a.Y + (2 * r + 1) * Wc + W - t));
            }
            z[brev(t, g.logW)] = dfc{df_add_abs(ye.re, df_neg(yo.im)), df_add_abs(ye.im, yo.re)};   // ye + i yo
        }
        __syncthreads();
        fft_r2_passes(z, g.logW, 1, W, 1, tw, g.logNtw, true);
        dfc bz = dfc{df{0.f, 0.f}, df{0.f, 0.f}};
        if (t < W) {
            const double e0 = df_to_double(df_scale(z[t].re, sc)), e1 = df_to_double(df_scale(z[t].im, sc));
            const double b0 = g.method == 0 ? e0 : 1.0 / e0, b1v = g.method == 0 ? e1 : 1.0 / e1;
            __stcg(a.b64 + (2 * r) * W + t, b0);
            __stcg(a.b64 + (2 * r + 1) * W + t, b1v);
            bz = dfc{df_from_double(b0), df_from_double(b1v)};
        }
        __syncthreads();
        if (t < W) z[brev(t, g.logW)] = bz;
        __syncthreads();
        fft_r2_passes(z, g.logW, 1, W, 1, tw, g.logNtw, false);
        if (t < Wc) rt_store_row_pair(a, W, Wc, r, z, t);
        __syncthreads();
    }
    if (!rt_grid_barrier(a.sync, b3t, a.limit)) return failed();
    for (int kx = blockIdx.x; kx < Wc; kx += gridDim.x) {
        rt_col_fwd(g, a, kx, z, tw);
        if (t < H) {
            const dfc e = z[t];
            a.FE64[t * Wc + kx] = dfc_to(e);
            a.FE32[t * Wc + kx] = make_float2(e.re.hi, e.im.hi);
            a.FEdf[t * Wc + kx] = e;
        }
        __syncthreads();
    }
}

// Eq. 8, the sum: CTA b adds F[I_f + off](k) e^{+2 pi i (ky' dy_f/H + kx' dx_f/W)} over its
// frames f = b, b + gridDim.x, ... into its own partial spectrum part[b] ([H][Wc], FP64),
// d_f the displacement of record f taken exactly. Records flagged CCST_R_TIMEOUT are left
// out; *count gains the number of frames taken. scratch[b] holds the row transforms of the
// frame in flight. The transforms and phase products run in double-float on the FP32
// pipes (about 2^-46 per butterfly, against magnitudes), the accumulation in FP64.
// Shared memory: max(H/2 * W, Wc * (H + 1)) + H + Wc complex double-floats (16 bytes each).
__global__ void __launch_bounds__(512) off_accumulate(Geom g, const void* frames, long long n, long long pitch,
                                                      double off, const Result* rec, double2* scratch,
                                                      double2* part, unsigned* count) {
    extern __shared__ double2 ccst_rt_smem[];
    const int H = g.H, W = g.W, Wc = g.Wc, Hp = H / 2, HWc = H * Wc;
    const int CS = H + 1;                               // column stride, padded against bank conflicts
    const int nbuf = Hp * W > Wc * CS ? Hp * W : Wc * CS;
    dfc* buf = (dfc*)ccst_rt_smem;
    dfc* py = buf + nbuf;
    dfc* px = py + H;
    dfc* S = (dfc*)(scratch + (size_t)blockIdx.x * HWc);
    double2* P = part + (size_t)blockIdx.x * HWc;
    for (int i = threadIdx.x; i < HWc; i += blockDim.x) P[i] = make_double2(0.0, 0.0);
    const size_t fbytes = (size_t)H * pitch * (g.in_dtype == 0 ? 2 : 4);
    const df offd = df_from_double(off);
    const df half = {0.5f, 0.f};
    unsigned taken = 0;
    for (long long f = blockIdx.x; f < n; f += gridDim.x) {
        const Result q = rec[f];
        if (q.flags & 0x20u) continue;
        ++taken;
        const long long qy = rt_grid_index(q.dy, q.ipy, g.u), qx = rt_grid_index(q.dx, q.ipx, g.u);
        const void* fr = (const char*)frames + (size_t)f * fbytes;
        for (int k = threadIdx.x; k < H; k += blockDim.x)
            py[k] = rt_axis_phase_df(k, H, qy, (long long)g.u * H, g.eyc, g.eyf, g.By);
        for (int k = threadIdx.x; k < Wc; k += blockDim.x)
            px[k] = rt_axis_phase_df(k, W, qx, (long long)g.u * W, g.exc, g.exf, g.Bx);
        for (int i = threadIdx.x; i < Hp * W; i += blockDim.x) {
            const int r = i / W, x = i - r * W;
            const df v0 = df_add(df_make(pixel_f32(fr, g.in_dtype, (long long)(2 * r) * pitch + x)), offd);
            const df v1 = df_add(df_make(pixel_f32(fr, g.in_dtype, (long long)(2 * r + 1) * pitch + x)), offd);
            buf[r * W + brev(x, g.logW)] = dfc{v0, v1};
        }
        __syncthreads();
        fft_r2_passes(buf, g.logW, Hp, W, 1, g.twdf, g.logNtw, false);
        for (int i = threadIdx.x; i < Hp * Wc; i += blockDim.x) {
            const int r = i / Wc, kx = i - r * Wc;
            const dfc zk = buf[r * W + kx], zc = cconj(buf[r * W + ((W - kx) & (W - 1))]);
            // rows 2r and 2r+1: (zk + zc) / 2 and (zk - zc) / (2i)
            S[(2 * r) * Wc + kx] = dfc{df_mul(df_add_abs(zk.re, zc.re), half), df_mul(df_add_abs(zk.im, zc.im), half)};
            S[(2 * r + 1) * Wc + kx] = dfc{df_mul(df_add_abs(zk.im, df_neg(zc.im)), half),
                                           df_neg(df_mul(df_add_abs(zk.re, df_neg(zc.re)), half))};
        }
        __syncthreads();
        for (int i = threadIdx.x; i < HWc; i += blockDim.x) {
            const int ky = i / Wc, kx = i - ky * Wc;
            buf[kx * CS + brev(ky, g.logH)] = S[i];
        }
        __syncthreads();
        fft_r2_passes(buf, g.logH, Wc, CS, 1, g.twdf, g.logNtw, false);
        for (int i = threadIdx.x; i < HWc; i += blockDim.x) {      // element i is this thread's in every frame
            const int ky = i / Wc, kx = i - ky * Wc;
            const dfc v = cmul(buf[kx * CS + ky], cmul(py[ky], px[kx]));
            const double2 p = P[i];
            P[i] = make_double2(p.x + df_to_double(v.re), p.y + df_to_double(v.im));
        }
        __syncthreads();
    }
    if (threadIdx.x == 0 && taken) atomicAdd(count, taken);
}

// Drift removal over n records (Sec. III B). The recurrence is sequential, so one thread
// runs it: Eq. 10 when lim <= 0, else Eqs. 11-12 with each step of R cut to length lim.
// R_0 = a0 r_0 in both forms; out[2i], out[2i+1] = r_i - R_i for r = (dx, dy).
__global__ void rt_drift(const Result* rec, long long n, double a0, double b1, double lim, double* out) {
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    double Rx = 0.0, Ry = 0.0;
    for (long long i = 0; i < n; ++i) {
        const double rx = rec[i].dx, ry = rec[i].dy;
        if (i == 0) {
            Rx = a0 * rx;
            Ry = a0 * ry;
        } else if (lim <= 0.0) {
            Rx = a0 * rx + b1 * Rx;
            Ry = a0 * ry + b1 * Ry;
        } else {
            const double sx = a0 * rx + (b1 - 1.0) * Rx, sy = a0 * ry + (b1 - 1.0) * Ry;
            const double len = hypot(sx, sy);
            const double f = len > lim ? lim / len : 1.0;
            Rx += f * sx;
            Ry += f * sy;
        }
        out[2 * i] = rx - Rx;
        out[2 * i + 1] = ry - Ry;
    }
}

}  // namespace

// ---------------------------------------------------------------- context
// Scratch of the general-size kernel for one stream of launches: launches that share a
// lane must run one after another (their CTAs reuse the same scratch).
struct GenLane {
    dfc* scratch = nullptr;
    size_t scratch_elems = 0;
    GenItem* d_items = nullptr;
    size_t items_cap = 0;
    GenItem* d_fb = nullptr;        // the FP32 kernel's fallback list
    size_t fb_cap = 0;
    unsigned* d_mixc = nullptr;     // kMixCounters counters of the FP32 kernel's launches
};

static void lane_free(GenLane& l) {
    if (l.scratch) cudaFree(l.scratch);
    if (l.d_items) cudaFree(l.d_items);
    if (l.d_fb) cudaFree(l.d_fb);
    if (l.d_mixc) cudaFree(l.d_mixc);
    l = GenLane{};
}

// The uneven-ROI kernel of one power-of-two side (ccst_rois.cu): its address (null until a
// plan of that side exists), the side's geometry (a parameter of the kernel), its dynamic
// shared memory and its grid (CTAs per SM x SMs).
struct RoiKernel {
    const void* fn = nullptr;
    Geom g{};
    size_t smem = 0;
    int grid = 0;
};
static int roi_side_slot(int side) { return side == 16 ? 0 : side == 32 ? 1 : side == 64 ? 2 : 3; }
// Item counters of an uneven-ROI batch's power-of-two part: one per side's launch.
constexpr int kRoiCounters = 4;

// A second stream with its fork and join events, made on first use: the general-size part
// of an uneven-ROI batch runs on it beside the power-of-two part.
struct SideStream {
    cudaStream_t st = nullptr;
    cudaEvent_t fork = nullptr, join = nullptr;
};

static cudaError_t side_make(SideStream& s) {
    cudaError_t e = cudaSuccess;
    if (!s.st && (e = cudaStreamCreateWithFlags(&s.st, cudaStreamNonBlocking)) != cudaSuccess) return e;
    if (!s.fork && (e = cudaEventCreateWithFlags(&s.fork, cudaEventDisableTiming)) != cudaSuccess) return e;
    if (!s.join && (e = cudaEventCreateWithFlags(&s.join, cudaEventDisableTiming)) != cudaSuccess) return e;
    return e;
}

static void side_free(SideStream& s) {
    if (s.st) cudaStreamSynchronize(s.st);
    if (s.st) cudaStreamDestroy(s.st);
    if (s.fork) cudaEventDestroy(s.fork);
    if (s.join) cudaEventDestroy(s.join);
    s = SideStream{};
}

struct ccst_ctx {
    Geom g{};
    ccst_params p{};
    cudaStream_t stream = nullptr;
    int device = 0;
    int grid_main = 1;
    int threads = kThreads;            // CTA size of track_kernel<H, W> (track_threads)
    size_t smem = 0;
    const void* kernel = nullptr;      // track_kernel<H, W>
    bool dead = false;
    std::string err = "no error";
    // device allocations
    void* d_ref32 = nullptr;
    double* d_b64 = nullptr;
    double2* d_FE64 = nullptr;
    float2* d_FE32 = nullptr;
    double2* d_tw64 = nullptr;
    float2* d_tw32 = nullptr;
    float* d_tab = nullptr;       // all stage tables in one block
    dfc* d_df = nullptr;          // double-float tables in one block
    void* d_frames = nullptr;     // host-path staging
    Result* d_out = nullptr;      // host-path staging
    unsigned* d_next = nullptr;   // frame counter of the tracking launches
    // real-time reference (Sec. III B): the filtered spectrum F[E] (CC-SN: F[E + eps]) and a
    // work spectrum, [H][W/2+1] double2 each; the filter's a0, b1
    double2* d_rtE = nullptr;
    double2* d_rtY = nullptr;
    unsigned* d_rtSync = nullptr;     // grid barrier of the update: arrivals, generation, error
    int rt_grid = 0;
    unsigned rt_seq = 0;              // update launches since the barrier counter was zeroed
    // offline reference (Sec. III A): per-CTA partial sums and row scratch, [off_parts][H][Wc]
    double2* d_offPart = nullptr;
    double2* d_offScratch = nullptr;
    int off_parts = 0;                // partial sums written by the last accumulation
    int off_max_parts = 0;
    double2* d_adjY = nullptr;        // adjoint: [H][Wc] column-inverse of the summed dL/db spectra
    // reference refinement by the adjoint (ccst_refine_reference): workspace for `cap` frames
    struct RefineWs {
        int64_t cap = 0;
        Result* rec = nullptr;        // [cap] records of the calibration frames
        double* peak = nullptr;       // [cap][2] continuous peaks (dx, dy)
        int32_t* status = nullptr;    // [cap]
        float* g = nullptr;           // [cap][2] dL/ds*
        double* E = nullptr;          // [H][W] the template being refined
        double* Eprev = nullptr;      // [H][W] the last accepted template
        float* gE = nullptr;          // [H][W] dL/dE at E
        float* gEprev = nullptr;      // [H][W] dL/dE at Eprev
        double* scal = nullptr;       // [0] loss at E, [1] step, [2] loss at Eprev, [3] Eprev valid
    } rf;
    double rt_a0 = 0.0, rt_b1 = 1.0;
    bool rt_on = false;               // ccst_rt_begin has run
    // uneven-ROI batches: size classes (plan 0 = this context's size) and references
    // (ref 0 = this context's reference), their device copies, and the work-item buffer
    struct SizePlan {
        Geom g;
        int ncy = 0, ncx = 0;         // double-float table lengths
        std::vector<void*> mem;       // owned allocations (none for plan 0)
    };
    struct RefEntry {
        int cls = -1;                 // power-of-two size class, -1 if none
        int gcls = -1;                // general size class (ccst_generic.cu), -1 if none
        RefSpectra r{};
        const dfc* gFb = nullptr;     // general size: the half spectrum F[b], H x (W/2 + 1)
        std::vector<void*> mem;       // owned allocations (none for ref 0)
    };
    struct GenPlanH {
        GenPlan p;
        std::vector<void*> mem;
        MixPlan mp{};                 // the FP32 general-size kernel's plan, if `mix`
        bool mix = false;
        int mix_grid = 0;             // resident CTAs of that kernel (whole clusters)
    };
    std::vector<SizePlan> plans;
    std::vector<RefEntry> refs;
    std::vector<GenPlanH> gplans;
    GenPlan* d_gplans = nullptr;
    const dfc** d_grefs = nullptr;
    size_t gplans_cap = 0, grefs_cap = 0;
    std::vector<GenItem> h_gitems;
    // lane 0: ccst_track and ccst_track_rois (ordered through the context's stream);
    // lanes 1 and 2: the two streams of the pipelined host path
    GenLane glane[3];
    int gen_grid = 0;
    int gen_threads = 512;            // CTA size of the general-size kernel (ccst_autotune may lower it)
    bool gen_dirty = true;            // plans or references changed since the last upload
    bool mix_off = false;             // ccst_autotune: the FP32 general-size kernel is bypassed
    bool general = false;             // every frame of this context takes the general-size kernel
    RefSpectra* d_refs = nullptr;
    size_t refs_cap = 0;
    RoiItem* d_items = nullptr;
    size_t items_cap = 0;
    std::vector<RoiItem> h_items;
    // ROI batches captured as CUDA graphs (CCST_FLAG_GRAPHS): one per (stream, out, work
    // list), each with its own uploaded work items and frame counters; the general-size
    // kernel's scratch is one lane per stream (graphs on one stream run in order). Dropped
    // (after their last replay) whenever plans, references or schedules change.
    struct RoiGraph {
        std::vector<ccst_roi> rois;   // the work list it was captured for
        cudaGraphExec_t exec = nullptr;
        cudaEvent_t done = nullptr;
        RoiItem* d_items = nullptr;
        GenItem* d_gitems = nullptr;
        unsigned* counters = nullptr; // [0], [1] power-of-two kernels (128 px; up to 64 px), [2] general-size
    };
    std::map<std::tuple<cudaStream_t, void*, int64_t, uint64_t>, RoiGraph> roi_graphs;
    std::map<cudaStream_t, GenLane> roi_lanes;
    int64_t roi_graph_instantiations = 0, roi_graph_replays = 0;
    SideStream rside;                 // ROI batches' general-size part (direct and captured)
    bool rois_dirty = true;
    RoiKernel rois_k[4];              // the ROI kernel of each side 16, 32, 64, 128 (roi_side_slot)
    void* d_addref_tmp = nullptr;     // ccst_add_reference: reference copy and FFT workspace
    size_t addref_tmp_bytes = 0;
    // graphs keyed by (stream, frames, n, pitch, out). Each owns a profiling event pair, a
    // completion event and a frame counter that no other graph uses, so graphs of different
    // batches can run at once on different streams. Replays of one graph are ordered by CUDA
    // (a graph exec runs after its own previous launch), so its counter is never shared.
    // A counter goes back to the pool only after the graph's last replay has finished
    // (drop_graphs waits on the completion events first).
    struct GraphEntry {
        cudaGraphExec_t exec = nullptr;
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        cudaEvent_t done = nullptr;    // recorded after every replay
        unsigned counter = 0;          // index into d_graph_counters
    };
    unsigned* d_graph_counters = nullptr;   // kMaxGraphs counters, one per cached graph
    std::vector<unsigned> free_graph_counters;
    int64_t graph_instantiations = 0, graph_replays = 0;
    // direct launches take counters from a ring of kTickets; before a counter is reused,
    // the new launch's stream waits for the previous launch that used it (ring_ev), so
    // launches on different streams never share a counter (d_next stays the real-time
    // path's counter)
    unsigned* d_launch_counters = nullptr;
    unsigned launch_seq = 0;
    cudaEvent_t ring_ev[kTickets] = {};
    bool ring_used[kTickets] = {};
    // the ROI path and a general-shape context's ccst_track share per-context device
    // buffers (work-item lists, the general kernel's lane-0 scratch, fixed counters): each
    // such call waits for the previous one, whichever stream it ran on (shared_ev)
    cudaEvent_t shared_ev = nullptr;
    bool shared_used = false;
    std::map<std::tuple<cudaStream_t, const void*, long long, long long, void*>, GraphEntry> graphs;
    // profiling ring for direct launches
    std::vector<cudaEvent_t> prof0, prof1;
    int prof_next = 0, prof_used = 0;
    bool capturing = false;
    cudaEvent_t cap_e0 = nullptr, cap_e1 = nullptr;   // event pair of the graph being captured
    // serving tickets
    cudaEvent_t ev[kTickets] = {};
    bool busy[kTickets] = {};
    uint64_t ticket_of[kTickets] = {};
    uint64_t next_ticket = 1;
    // pipelined host path: per slot a device staging area, a frame counter and the ticket
    // using it; slots alternate between two streams
    cudaStream_t hstream[2] = {nullptr, nullptr};
    void* h_frames[kHostSlots] = {};
    Result* h_out[kHostSlots] = {};
    unsigned* h_next = nullptr;
    uint64_t h_ticket[kHostSlots] = {};
    uint64_t h_count = 0;
};

static int fail(ccst_ctx* c, int code, const std::string& msg) {
    if (c) {
        c->err = msg;
        if (code == CCST_E_CUDA) c->dead = true;
    } else {
        std::lock_guard<std::mutex> lk(g_create_err_mu);
        g_create_err = msg;
    }
    return code;
}

#define CK(ctx, call)                                                                              \
    do {                                                                                           \
        cudaError_t e_ = (call);                                                                   \
        if (e_ != cudaSuccess)                                                                     \
            return fail((ctx), e_ == cudaErrorMemoryAllocation ? CCST_E_NOMEM : CCST_E_CUDA,       \
                        std::string(#call) + ": " + cudaGetErrorString(e_));                      \
    } while (0)

// Destroy every cached graph after its last replay has finished, and return the frame
// counters to the pool: no counter is handed out again while a launch may still use it.
static void drop_graphs(ccst_ctx* c) {
    for (auto& kv : c->graphs)
        if (kv.second.done) cudaEventSynchronize(kv.second.done);
    for (auto& kv : c->graphs) {
        if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
        if (kv.second.e0) cudaEventDestroy(kv.second.e0);
        if (kv.second.e1) cudaEventDestroy(kv.second.e1);
        if (kv.second.done) cudaEventDestroy(kv.second.done);
    }
    c->graphs.clear();
    c->free_graph_counters.clear();
    for (unsigned i = 0; i < (unsigned)kMaxGraphs; ++i) c->free_graph_counters.push_back((unsigned)kMaxGraphs - 1 - i);
}

static void free_roi_graph(ccst_ctx::RoiGraph& e) {
    if (e.done) cudaEventSynchronize(e.done);
    if (e.exec) cudaGraphExecDestroy(e.exec);
    if (e.done) cudaEventDestroy(e.done);
    if (e.d_items) cudaFree(e.d_items);
    if (e.d_gitems) cudaFree(e.d_gitems);
    if (e.counters) cudaFree(e.counters);
    e = ccst_ctx::RoiGraph{};
}

// Destroy every captured ROI graph after its last replay has finished.
static void drop_roi_graphs(ccst_ctx* c) {
    for (auto& kv : c->roi_graphs) free_roi_graph(kv.second);
    c->roi_graphs.clear();
}

// A frame counter of the direct-launch ring for a launch on `stream`: the stream first
// waits for the previous launch that used the same counter (a no-op when it ran on the
// same stream or has finished). Call ring_release after the launch has been issued.
static unsigned ring_acquire(ccst_ctx* c, cudaStream_t stream, cudaError_t* err) {
    const unsigned k = c->launch_seq++ % kTickets;
    *err = cudaSuccess;
    if (c->ring_used[k]) {
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        *err = cudaStreamIsCapturing(stream, &cs);
        // inside a caller's stream capture the wait would join an outside event into the
        // graph; the caller's graph then orders its own launches
        if (*err == cudaSuccess && cs == cudaStreamCaptureStatusNone)
            *err = cudaStreamWaitEvent(stream, c->ring_ev[k], 0);
    }
    return k;
}

// Order a call that uses the context's shared buffers after the previous such call.
static cudaError_t shared_acquire(ccst_ctx* c, cudaStream_t stream) {
    if (!c->shared_ev) {
        const cudaError_t e = cudaEventCreateWithFlags(&c->shared_ev, cudaEventDisableTiming);
        if (e != cudaSuccess) return e;
    }
    if (!c->shared_used) return cudaSuccess;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaError_t e = cudaStreamIsCapturing(stream, &cs);
    if (e == cudaSuccess && cs == cudaStreamCaptureStatusNone) e = cudaStreamWaitEvent(stream, c->shared_ev, 0);
    return e;
}

static cudaError_t shared_release(ccst_ctx* c, cudaStream_t stream) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaError_t e = cudaStreamIsCapturing(stream, &cs);
    if (e != cudaSuccess || cs != cudaStreamCaptureStatusNone) return e;
    e = cudaEventRecord(c->shared_ev, stream);
    if (e == cudaSuccess) c->shared_used = true;
    return e;
}

static cudaError_t ring_release(ccst_ctx* c, unsigned k, cudaStream_t stream) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaError_t e = cudaStreamIsCapturing(stream, &cs);
    if (e != cudaSuccess || cs != cudaStreamCaptureStatusNone) return e;
    e = cudaEventRecord(c->ring_ev[k], stream);
    if (e == cudaSuccess) c->ring_used[k] = true;
    return e;
}

static void free_all(ccst_ctx* c) {
    drop_graphs(c);
    drop_roi_graphs(c);
    for (auto& kv : c->roi_lanes) lane_free(kv.second);
    c->roi_lanes.clear();
    side_free(c->rside);
    for (size_t i = 0; i < c->prof0.size(); ++i) {
        cudaEventDestroy(c->prof0[i]);
        cudaEventDestroy(c->prof1[i]);
    }
    c->prof0.clear();
    c->prof1.clear();
    for (int i = 0; i < kTickets; ++i) {
        if (c->ev[i]) cudaEventDestroy(c->ev[i]);
        if (c->ring_ev[i]) cudaEventDestroy(c->ring_ev[i]);
    }
    for (int i = 0; i < kHostSlots; ++i) {
        if (c->h_frames[i]) cudaFree(c->h_frames[i]);
        if (c->h_out[i]) cudaFree(c->h_out[i]);
    }
    if (c->h_next) cudaFree(c->h_next);
    for (int i = 0; i < 2; ++i)
        if (c->hstream[i]) cudaStreamDestroy(c->hstream[i]);
    for (auto& pl : c->plans)
        for (void* p : pl.mem) cudaFree(p);
    for (auto& re : c->refs)
        for (void* p : re.mem) cudaFree(p);
    for (auto& gp : c->gplans)
        for (void* p : gp.mem) cudaFree(p);
    c->plans.clear();
    c->refs.clear();
    c->gplans.clear();
    if (c->shared_ev) cudaEventDestroy(c->shared_ev);
    void* ptrs[] = {c->d_ref32, c->d_b64, c->d_FE64, c->d_FE32, c->d_tw64, c->d_tw32,
                    c->d_tab,   c->d_df,  c->d_frames, c->d_out, c->d_next, c->d_rtE, c->d_rtY, c->d_rtSync,
                    c->d_offPart, c->d_offScratch, c->d_adjY, c->d_refs, c->d_items, c->d_addref_tmp,
                    c->d_graph_counters, c->d_launch_counters, c->d_gplans, c->d_grefs};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    for (auto& l : c->glane) lane_free(l);
    void* rfp[] = {c->rf.rec, c->rf.peak, c->rf.status, c->rf.g, c->rf.E, c->rf.Eprev, c->rf.gE, c->rf.gEprev,
                   c->rf.scal};
    for (void* p : rfp)
        if (p) cudaFree(p);
}

static int gen_track(ccst_ctx* c, const Batch& b, cudaStream_t stream, GenLane& lane, unsigned* counter,
                     const MixDbg* dbg = nullptr);
static int gen_ref_spectrum(ccst_ctx* c, int H, int W, const void* src, int frame_kind, long long pitch, dfc* Fb);
static int add_generic_reference(ccst_ctx* c, const float* ref, int H, int W, int* ref_id);
static int not_general(ccst_ctx* c, const char* who);

extern "C" int ccst_version(void) { return CCST_VERSION; }

extern "C" int ccst_default_params(ccst_params* p) {
    if (!p) return CCST_E_INVALID;
    std::memset(p, 0, sizeof(*p));
    p->upsample = 100;
    p->method = CCST_CC_U;
    p->eps = 200.0f;
    p->in_dtype = CCST_U16;
    p->max_batch = 256;
    p->stream = nullptr;
    p->flags = CCST_FLAG_TIE_GUARD;
    return CCST_OK;
}

// A general-shape context (H, W in [8, 256], not both powers of two up to 128): plan 0 is
// its shape, ref 0 its reference as a half spectrum for the general-size kernel, which
// every batch of the context runs on.
static int create_general(const float* ref, int H, int W, const ccst_params& p, ccst_ctx** out) {
    ccst_ctx* c = new (std::nothrow) ccst_ctx();
    if (!c) return fail(nullptr, CCST_E_NOMEM, "ccst_create: host allocation failed");
    c->p = p;
    c->stream = (cudaStream_t)p.stream;
    c->general = true;
    auto bail = [&](int code) {
        fail(nullptr, code, "ccst_create: " + c->err);
        free_all(c);
        delete c;
        return code;
    };
    cudaError_t e = cudaGetDevice(&c->device);
    if (e != cudaSuccess) {
        c->err = std::string("cudaGetDevice: ") + cudaGetErrorString(e);
        return bail(CCST_E_CUDA);
    }
    Geom& g = c->g;
    g.H = H; g.W = W; g.Wc = W / 2 + 1;
    g.u = p.upsample; g.M = (3 * p.upsample + 1) / 2; g.h0 = g.M / 2; g.pmax = g.M - 1 - g.h0;
    g.method = p.method; g.in_dtype = p.in_dtype; g.eps = p.eps;
    g.sense = p.method == CCST_CC_U ? 1.f : -1.f;
    const size_t elem = p.in_dtype == CCST_U16 ? 2 : 4;
    struct { void** ptr; size_t bytes; } allocs[] = {
        {(void**)&c->d_frames, (size_t)p.max_batch * H * W * elem},
        {(void**)&c->d_out, (size_t)p.max_batch * sizeof(Result)},
        {(void**)&c->d_next, 256},
        {(void**)&c->d_launch_counters, kTickets * sizeof(unsigned)},
    };
    for (auto& a : allocs)
        if ((e = cudaMalloc(a.ptr, a.bytes)) != cudaSuccess) {
            c->err = std::string("cudaMalloc: ") + cudaGetErrorString(e);
            return bail(e == cudaErrorMemoryAllocation ? CCST_E_NOMEM : CCST_E_CUDA);
        }
    for (int i = 0; i < kTickets; ++i)
        if ((e = cudaEventCreateWithFlags(&c->ev[i], cudaEventDisableTiming)) != cudaSuccess ||
            (e = cudaEventCreateWithFlags(&c->ring_ev[i], cudaEventDisableTiming)) != cudaSuccess) {
            c->err = std::string("event: ") + cudaGetErrorString(e);
            return bail(CCST_E_CUDA);
        }
    ccst_ctx::SizePlan p0;
    p0.g = g;
    c->plans.push_back(p0);
    int id = -1;
    const int rc = add_generic_reference(c, ref, H, W, &id);
    if (rc) return bail(rc);
    *out = c;
    return CCST_OK;
}

extern "C" int ccst_create(const float* ref, int H, int W, const ccst_params* pin, ccst_ctx** out) {
    if (!ref || !out) return fail(nullptr, CCST_E_INVALID, "ccst_create: null ref or out");
    *out = nullptr;
    ccst_params p;
    if (pin) p = *pin; else ccst_default_params(&p);
    const bool fast = is_pow2(H) && is_pow2(W) && H >= 8 && W >= 8 && H <= 128 && W <= 128;
    if (H < 8 || W < 8 || H > 256 || W > 256)
        return fail(nullptr, CCST_E_SHAPE, "ccst_create: H and W must be in [8, 256]");
    if (p.upsample < 1 || p.upsample > 16384)
        return fail(nullptr, CCST_E_INVALID, "ccst_create: upsample must be in [1, 16384]");
    if (p.method != CCST_CC_U && p.method != CCST_CC_SN)
        return fail(nullptr, CCST_E_INVALID, "ccst_create: unknown method");
    if (p.in_dtype != CCST_U16 && p.in_dtype != CCST_F32)
        return fail(nullptr, CCST_E_INVALID, "ccst_create: unknown in_dtype");
    if (p.max_batch < 1) return fail(nullptr, CCST_E_INVALID, "ccst_create: max_batch must be > 0");
    if (p.method == CCST_CC_SN && !(p.eps == p.eps))
        return fail(nullptr, CCST_E_INVALID, "ccst_create: eps is NaN");
    if (!fast) return create_general(ref, H, W, p, out);

    ccst_ctx* c = new (std::nothrow) ccst_ctx();
    if (!c) return fail(nullptr, CCST_E_NOMEM, "ccst_create: host allocation failed");
    c->p = p;
    c->stream = (cudaStream_t)p.stream;
    Geom& g = c->g;
    auto bail = [&](int code) { free_all(c); delete c; return code; };
    cudaError_t e;
    int dev = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) {
        fail(nullptr, CCST_E_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
        return bail(CCST_E_CUDA);
    }
    c->device = dev;
    cudaDeviceProp prop;
    if ((e = cudaGetDeviceProperties(&prop, dev)) != cudaSuccess) {
        fail(nullptr, CCST_E_CUDA, std::string("cudaGetDeviceProperties: ") + cudaGetErrorString(e));
        return bail(CCST_E_CUDA);
    }
    const size_t limit = prop.sharedMemPerBlockOptin;
    if (!plan_geometry(H, W, p, limit, &g)) {
        fail(nullptr, CCST_E_SHAPE, "ccst_create: frame too large for shared memory");
        return bail(CCST_E_SHAPE);
    }
    c->smem = smem_plan(g).total;

    const size_t HW = (size_t)H * W, HWc = (size_t)H * g.Wc;
    const size_t tabA = (size_t)g.Hh * g.T1p, tabB = (size_t)g.Wc * g.T1p;
    const size_t l2per = (size_t)(H / 2) * W + (size_t)H * g.Wcp;   // FP64 FFT workspace at create
    const size_t elem = p.in_dtype == CCST_U16 ? 2 : 4;
    const long long Dy = (long long)g.u * H, Dx = (long long)g.u * W;
    g.By = 1; while ((long long)g.By * g.By < Dy) ++g.By;
    g.Bx = 1; while ((long long)g.Bx * g.Bx < Dx) ++g.Bx;
    const int ncy = (int)((Dy + g.By - 1) / g.By), ncx = (int)((Dx + g.Bx - 1) / g.Bx);
    const size_t ndf = (size_t)(g.Ntw / 2) + HWc + ncy + g.By + ncx + g.Bx;
    double2* d_work = nullptr;
    struct { void** ptr; size_t bytes; } allocs[] = {
        {(void**)&c->d_ref32, HW * sizeof(float)},
        {(void**)&c->d_b64, HW * sizeof(double)},
        {(void**)&c->d_FE64, HWc * sizeof(double2)},
        {(void**)&c->d_FE32, HWc * sizeof(float2)},
        {(void**)&c->d_tw64, (size_t)(g.Ntw / 2) * sizeof(double2)},
        {(void**)&c->d_tw32, (size_t)(g.Ntw / 2) * sizeof(float2)},
        {(void**)&c->d_tab, (2 * tabA + 3 * tabB) * sizeof(float) + table_bytes(g)},
        {(void**)&c->d_df, ndf * sizeof(dfc)},
        {(void**)&d_work, l2per * sizeof(double2)},
        {(void**)&c->d_frames, (size_t)p.max_batch * HW * elem},
        {(void**)&c->d_out, (size_t)p.max_batch * sizeof(Result)},
        {(void**)&c->d_next, 256},
        {(void**)&c->d_launch_counters, kTickets * sizeof(unsigned)},
    };
    for (auto& a : allocs) {
        if ((e = cudaMalloc(a.ptr, a.bytes)) != cudaSuccess) {
            fail(nullptr, e == cudaErrorMemoryAllocation ? CCST_E_NOMEM : CCST_E_CUDA,
                 std::string("cudaMalloc: ") + cudaGetErrorString(e));
            return bail(e == cudaErrorMemoryAllocation ? CCST_E_NOMEM : CCST_E_CUDA);
        }
    }
    g.FE32 = c->d_FE32; g.FE64 = c->d_FE64; g.b64 = c->d_b64; g.tw32 = c->d_tw32; g.tw64 = c->d_tw64;
    g.tA_cm1 = c->d_tab; g.tA_s = c->d_tab + tabA;
    g.tB_wc = c->d_tab + 2 * tabA; g.tB_ws = g.tB_wc + tabB; g.tB_gc = g.tB_ws + tabB;
    g.tAh = (const uint2*)(g.tB_gc + tabB);           // 16-byte aligned: the block sizes above are multiples of 4
    g.tBh = (const uint2*)((const char*)g.tAh + ta_bytes(g));
    dfc* twdf = c->d_df;
    dfc* FEdf = twdf + g.Ntw / 2;
    dfc* eyc = FEdf + HWc;
    dfc* eyf = eyc + ncy;
    dfc* exc = eyf + g.By;
    dfc* exf = exc + ncx;
    g.twdf = twdf; g.FEdf = FEdf; g.eyc = eyc; g.eyf = eyf; g.exc = exc; g.exf = exf;

    auto step = [&](cudaError_t e2, const char* what) {
        if (e2 != cudaSuccess) fail(nullptr, CCST_E_CUDA, std::string(what) + ": " + cudaGetErrorString(e2));
        return e2 == cudaSuccess;
    };
    auto bail_work = [&](int code) { cudaFree(d_work); return bail(code); };
    if (!step(cudaMemcpyAsync(c->d_ref32, ref, HW * sizeof(float), cudaMemcpyDefault, c->stream), "copy ref"))
        return bail_work(CCST_E_CUDA);
    init_twiddles<<<1, 256, 0, c->stream>>>(g.Ntw, c->d_tw64, c->d_tw32);
    init_tables<<<64, 256, 0, c->stream>>>(g, (float*)g.tA_cm1, (float*)g.tA_s, (float*)g.tB_wc,
                                           (float*)g.tB_ws, (float*)g.tB_gc, (uint2*)g.tAh, (uint2*)g.tBh);
    init_ref_operand<<<32, 256, 0, c->stream>>>(g, (const float*)c->d_ref32, c->d_b64);
    init_ref_spectrum<<<1, 256, 0, c->stream>>>(g, d_work, c->d_FE64, c->d_FE32);
    init_dfloat<<<32, 256, 0, c->stream>>>(g, c->d_tw64, c->d_FE64, twdf, FEdf, eyc, eyf, exc, exf, ncy, ncx);
    if (!step(cudaGetLastError(), "init kernels") || !step(cudaStreamSynchronize(c->stream), "init sync"))
        return bail_work(CCST_E_CUDA);
    cudaFree(d_work);
    d_work = nullptr;
    c->kernel = (H == 128 && W == 128 && g.tc) ? track_kernel_128_tc() : track_kernel_for(H, W);
    c->threads = track_threads(H, W);
    // the attribute is per function: set it to the device limit so contexts of any size coexist
    if (!step(cudaFuncSetAttribute(c->kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)limit - ((H == 128 && W == 128) ? kTcStaticSmem : 0)),
              "smem attribute"))
        return bail(CCST_E_CUDA);
    int occ = 0;
    if (!step(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, c->kernel, c->threads, c->smem), "occupancy"))
        return bail(CCST_E_CUDA);
    if (occ < 1) {
        fail(nullptr, CCST_E_SHAPE, "ccst_create: tracking kernel does not fit on an SM");
        return bail(CCST_E_SHAPE);
    }
    c->grid_main = prop.multiProcessorCount * occ;
    for (int i = 0; i < kTickets; ++i)
        if (!step(cudaEventCreateWithFlags(&c->ev[i], cudaEventDisableTiming), "event") ||
            !step(cudaEventCreateWithFlags(&c->ring_ev[i], cudaEventDisableTiming), "event"))
            return bail(CCST_E_CUDA);
    if (p.flags & CCST_FLAG_PROFILE) {
        c->prof0.resize(1024);
        c->prof1.resize(1024);
        for (int i = 0; i < 1024; ++i)
            if (!step(cudaEventCreate(&c->prof0[i]), "event") || !step(cudaEventCreate(&c->prof1[i]), "event"))
                return bail(CCST_E_CUDA);
    }
    *out = c;
    return CCST_OK;
}

static int launch(ccst_ctx* c, const Batch& b, bool reset_counter = true, unsigned* counter = nullptr) {
    if (b.n == 0) return CCST_OK;
    const int grid = (int)(b.n < c->grid_main ? b.n : c->grid_main);
    const bool prof = (c->p.flags & CCST_FLAG_PROFILE) != 0;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (prof) {
        if (c->capturing) {
            e0 = c->cap_e0;
            e1 = c->cap_e1;
        } else {
            e0 = c->prof0[c->prof_next];
            e1 = c->prof1[c->prof_next];
            c->prof_next = (c->prof_next + 1) % (int)c->prof0.size();
            if (c->prof_used < (int)c->prof0.size()) ++c->prof_used;
        }
        CK(c, cudaEventRecordWithFlags(e0, c->stream, c->capturing ? cudaEventRecordExternal : 0));
    }
    {
        Geom gk = c->g;
        Batch bk = b;
        int ring = -1;
        if (!counter) {
            cudaError_t e;
            ring = (int)ring_acquire(c, c->stream, &e);
            CK(c, e);
            counter = c->d_launch_counters + ring;
        }
        bk.next = counter;
        if (reset_counter) CK(c, cudaMemsetAsync(bk.next, 0, sizeof(unsigned), c->stream));
        void* args[] = {&gk, &bk};
        CK(c, cudaLaunchKernel(c->kernel, dim3(grid), dim3(c->threads), args, c->smem, c->stream));
        if (ring >= 0) CK(c, ring_release(c, (unsigned)ring, c->stream));
    }
    if (prof) CK(c, cudaEventRecordWithFlags(e1, c->stream, c->capturing ? cudaEventRecordExternal : 0));
    CK(c, cudaGetLastError());
    return CCST_OK;
}

// Plain launch on `stream` with its own frame counter (the pipelined host path).
static int launch_on(ccst_ctx* c, const Batch& b, cudaStream_t stream, unsigned* counter) {
    if (b.n == 0) return CCST_OK;
    const int grid = (int)(b.n < c->grid_main ? b.n : c->grid_main);
    Geom gk = c->g;
    Batch bk = b;
    bk.next = counter;
    CK(c, cudaMemsetAsync(counter, 0, sizeof(unsigned), stream));
    void* args[] = {&gk, &bk};
    CK(c, cudaLaunchKernel(c->kernel, dim3(grid), dim3(c->threads), args, c->smem, stream));
    CK(c, cudaGetLastError());
    return CCST_OK;
}

static int check_ctx(ccst_ctx* c) {
    if (!c) return CCST_E_INVALID;
    if (c->dead) return CCST_E_CUDA;
    return CCST_OK;
}

static int make_batch(ccst_ctx* c, const void* frames, int64_t n, int64_t pitch, ccst_result* out, Batch* b) {
    if (n < 0 || n > c->p.max_batch) return fail(c, CCST_E_INVALID, "n outside [0, max_batch]");
    if (n > 0 && (!frames || !out)) return fail(c, CCST_E_INVALID, "null frames or out");
    if (pitch == 0) pitch = c->g.W;
    if (pitch < c->g.W) return fail(c, CCST_E_INVALID, "pitch_elems < W");
    b->frames = frames;
    b->n = n;
    b->pitch = pitch;
    b->out = (Result*)out;
    const size_t el = c->p.in_dtype == CCST_U16 ? 2 : 4;
    b->vec_ok = ((uintptr_t)frames % 16 == 0) && ((size_t)pitch * el % 16 == 0) ? 1 : 0;
    b->dbg_int = nullptr;
    b->dbg_sub = nullptr;
    b->dbg_pairs = nullptr;
    b->dbg_d32 = nullptr;
    b->dbg_d64 = nullptr;
    b->next = nullptr;
    b->dbg_no_copy = 0;
    return CCST_OK;
}

extern "C" int ccst_track(ccst_ctx* c, const void* frames_dev, int64_t n, int64_t pitch_elems,
                          ccst_result* out_dev) {
    int rc = check_ctx(c);
    if (rc) return rc;
    Batch b;
    if ((rc = make_batch(c, frames_dev, n, pitch_elems, out_dev, &b))) return rc;
    if (n == 0) return CCST_OK;
    if (c->general) {
        cudaError_t e;
        const unsigned k = ring_acquire(c, c->stream, &e);
        CK(c, e);
        CK(c, shared_acquire(c, c->stream));
        if ((rc = gen_track(c, b, c->stream, c->glane[0], c->d_launch_counters + k))) return rc;
        CK(c, ring_release(c, k, c->stream));
        CK(c, shared_release(c, c->stream));
        return CCST_OK;
    }
    const bool graphs = (c->p.flags & CCST_FLAG_GRAPHS) && c->stream != nullptr;
    if (!graphs) return launch(c, b);
    auto key = std::make_tuple(c->stream, frames_dev, (long long)n, (long long)b.pitch, (void*)out_dev);
    auto it = c->graphs.find(key);
    if (it == c->graphs.end()) {
        if (c->graphs.size() >= kMaxGraphs || c->free_graph_counters.empty()) drop_graphs(c);
        if (!c->d_graph_counters) CK(c, cudaMalloc(&c->d_graph_counters, kMaxGraphs * sizeof(unsigned)));
        ccst_ctx::GraphEntry ent;
        CK(c, cudaEventCreateWithFlags(&ent.done, cudaEventDisableTiming));
        ent.counter = c->free_graph_counters.back();
        c->free_graph_counters.pop_back();
        unsigned* counter = c->d_graph_counters + ent.counter;
        if (c->p.flags & CCST_FLAG_PROFILE) {
            CK(c, cudaEventCreate(&ent.e0));
            CK(c, cudaEventCreate(&ent.e1));
        }
        cudaGraph_t graph;
        CK(c, cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
        c->capturing = true;
        c->cap_e0 = ent.e0;
        c->cap_e1 = ent.e1;
        const int lrc = launch(c, b, true, counter);
        c->capturing = false;
        cudaError_t e = cudaStreamEndCapture(c->stream, &graph);
        if (lrc) return lrc;
        CK(c, e);
        e = cudaGraphInstantiate(&ent.exec, graph, 0);
        cudaGraphDestroy(graph);
        CK(c, e);
        ++c->graph_instantiations;
        it = c->graphs.emplace(key, ent).first;
    }
    CK(c, cudaGraphLaunch(it->second.exec, c->stream));
    CK(c, cudaEventRecord(it->second.done, c->stream));
    ++c->graph_replays;
    return CCST_OK;
}

extern "C" int ccst_track_host(ccst_ctx* c, const void* frames_host, int64_t n, int64_t pitch_elems,
                               ccst_result* out_host) {
    int rc = check_ctx(c);
    if (rc) return rc;
    if (n < 0 || n > c->p.max_batch) return fail(c, CCST_E_INVALID, "n outside [0, max_batch]");
    if (n == 0) return CCST_OK;
    if (!frames_host || !out_host) return fail(c, CCST_E_INVALID, "null frames or out");
    if (pitch_elems == 0) pitch_elems = c->g.W;
    if (pitch_elems < c->g.W) return fail(c, CCST_E_INVALID, "pitch_elems < W");
    const size_t elem = c->p.in_dtype == CCST_U16 ? 2 : 4;
    const size_t row = (size_t)c->g.W * elem;
    CK(c, cudaMemcpy2DAsync(c->d_frames, row, frames_host, (size_t)pitch_elems * elem, row,
                            (size_t)n * c->g.H, cudaMemcpyHostToDevice, c->stream));
    if ((rc = ccst_track(c, c->d_frames, n, 0, (ccst_result*)c->d_out))) return rc;
    CK(c, cudaMemcpyAsync(out_host, c->d_out, (size_t)n * sizeof(Result), cudaMemcpyDeviceToHost, c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
    return CCST_OK;
}

extern "C" int ccst_submit_host(ccst_ctx* c, const void* frames_host, int64_t n, int64_t pitch_elems,
                                ccst_result* out_host, uint64_t* ticket) {
    int rc = check_ctx(c);
    if (rc) return rc;
    if (!ticket) return fail(c, CCST_E_INVALID, "null ticket");
    if (n < 0 || n > c->p.max_batch) return fail(c, CCST_E_INVALID, "n outside [0, max_batch]");
    if (n > 0 && (!frames_host || !out_host)) return fail(c, CCST_E_INVALID, "null frames or out");
    if (pitch_elems == 0) pitch_elems = c->g.W;
    if (pitch_elems < c->g.W) return fail(c, CCST_E_INVALID, "pitch_elems < W");
    const size_t elem = c->p.in_dtype == CCST_U16 ? 2 : 4;
    const size_t row = (size_t)c->g.W * elem;
    if (!c->h_next) {                    // first use: streams and staging areas
        for (int i = 0; i < 2; ++i) CK(c, cudaStreamCreateWithFlags(&c->hstream[i], cudaStreamNonBlocking));
        for (int i = 0; i < kHostSlots; ++i) {
            cudaError_t e = cudaMalloc(&c->h_frames[i], (size_t)c->p.max_batch * c->g.H * row);
            if (e == cudaSuccess) e = cudaMalloc((void**)&c->h_out[i], (size_t)c->p.max_batch * sizeof(Result));
            if (e != cudaSuccess)
                return fail(c, e == cudaErrorMemoryAllocation ? CCST_E_NOMEM : CCST_E_CUDA,
                            std::string("cudaMalloc: ") + cudaGetErrorString(e));
        }
        CK(c, cudaMalloc((void**)&c->h_next, 256 * kHostSlots));
        // the work on the internal streams follows everything issued on the context's stream
        cudaEvent_t e0;
        CK(c, cudaEventCreateWithFlags(&e0, cudaEventDisableTiming));
        CK(c, cudaEventRecord(e0, c->stream));
        for (int i = 0; i < 2; ++i) CK(c, cudaStreamWaitEvent(c->hstream[i], e0, 0));
        CK(c, cudaEventDestroy(e0));
    }
    const int hs = (int)(c->h_count % kHostSlots);
    // the slot's previous submission must be finished before its staging area is reused
    if (c->h_ticket[hs]) {
        const int ts = (int)(c->h_ticket[hs] % kTickets);
        if (c->busy[ts] && c->ticket_of[ts] == c->h_ticket[hs]) CK(c, cudaEventSynchronize(c->ev[ts]));
    }
    const uint64_t t = c->next_ticket;
    const int slot = (int)(t % kTickets);
    if (c->busy[slot]) return fail(c, CCST_E_BUSY, "all submission slots in flight");
    cudaStream_t st = c->hstream[hs & 1];
    if (n > 0) {
        CK(c, cudaMemcpy2DAsync(c->h_frames[hs], row, frames_host, (size_t)pitch_elems * elem, row,
                                (size_t)n * c->g.H, cudaMemcpyHostToDevice, st));
        Batch b;
        if ((rc = make_batch(c, c->h_frames[hs], n, 0, (ccst_result*)c->h_out[hs], &b))) return rc;
        rc = c->general ? gen_track(c, b, st, c->glane[1 + (hs & 1)], c->h_next + 64 * hs)
                        : launch_on(c, b, st, c->h_next + 64 * hs);
        if (rc) return rc;
        CK(c, cudaMemcpyAsync(out_host, c->h_out[hs], (size_t)n * sizeof(Result), cudaMemcpyDeviceToHost, st));
    }
    CK(c, cudaEventRecord(c->ev[slot], st));
    c->busy[slot] = true;
    c->ticket_of[slot] = t;
    c->next_ticket = t + 1;
    c->h_ticket[hs] = t;
    ++c->h_count;
    *ticket = t;
    return CCST_OK;
}

extern "C" int ccst_set_stream(ccst_ctx* c, void* stream) {
    int rc = check_ctx(c);
    if (rc) return rc;
    c->stream = (cudaStream_t)stream;      // cached graphs are keyed by stream: none is dropped
    return CCST_OK;
}

extern "C" int ccst_graph_stats(ccst_ctx* c, int64_t* instantiations, int64_t* replays, int64_t* cached) {
    int rc = check_ctx(c);
    if (rc) return rc;
    if (!instantiations || !replays || !cached) return fail(c, CCST_E_INVALID, "ccst_graph_stats: null output");
    *instantiations = c->graph_instantiations + c->roi_graph_instantiations;
    *replays = c->graph_replays + c->roi_graph_replays;
    *cached = (int64_t)(c->graphs.size() + c->roi_graphs.size());
    return CCST_OK;
}

extern "C" int ccst_sync(ccst_ctx* c) {
    int rc = check_ctx(c);
    if (rc) return rc;
    CK(c, cudaStreamSynchronize(c->stream));
    return CCST_OK;
}

extern "C" int ccst_submit(ccst_ctx* c, const void* frames_dev, int64_t n, ccst_result* out_dev,
                           uint64_t* ticket) {
    int rc = check_ctx(c);
    if (rc) return rc;
    if (!ticket) return fail(c, CCST_E_INVALID, "null ticket");
    const uint64_t t = c->next_ticket;
    const int slot = (int)(t % kTickets);
    if (c->busy[slot]) return fail(c, CCST_E_BUSY, "all submission slots in flight");
    if ((rc = ccst_track(c, frames_dev, n, 0, out_dev))) return rc;
    CK(c, cudaEventRecord(c->ev[slot], c->stream));
    c->busy[slot] = true;
    c->ticket_of[slot] = t;
    c->next_ticket = t + 1;
    *ticket = t;
    return CCST_OK;
}

extern "C" int ccst_poll(ccst_ctx* c, uint64_t ticket, int timeout_us, int* done) {
    int rc = check_ctx(c);
    if (rc) return rc;
    if (!done) return fail(c, CCST_E_INVALID, "null done");
    *done = 0;
    const int slot = (int)(ticket % kTickets);
    if (!c->busy[slot] || c->ticket_of[slot] != ticket) return fail(c, CCST_E_INVALID, "unknown ticket");
    const auto t_end = std::chrono::steady_clock::now() + std::chrono::microseconds(timeout_us < 0 ? 0 : timeout_us);
    for (;;) {
        const cudaError_t e = cudaEventQuery(c->ev[slot]);
        if (e == cudaSuccess) {
            c->busy[slot] = false;
            *done = 1;
            return CCST_OK;
        }
        if (e != cudaErrorNotReady) CK(c, e);
        if (std::chrono::steady_clock::now() >= t_end) return CCST_E_TIMEOUT;
        std::this_thread::sleep_for(std::chrono::microseconds(20));
    }
}

// ------------------------------------------------------------ continuous peak and adjoint
static int off_prepare(ccst_ctx* c);

static int adj_run(ccst_ctx* c, const void* frames, int64_t n, int64_t pitch, const ccst_result* rec,
                   const float* gdxdy, double* peak, int32_t* status, float* g_frames, float* g_ref,
                   const char* who) {
    int rc = check_ctx(c);
    if (rc) return rc;
    if ((rc = not_general(c, who))) return rc;
    if (n < 0) return fail(c, CCST_E_INVALID, std::string(who) + ": n < 0");
    if (n > 0 && (!rec || !frames)) return fail(c, CCST_E_INVALID, std::string(who) + ": null frames or records");
    if (pitch == 0) pitch = c->g.W;
    if (pitch < c->g.W) return fail(c, CCST_E_INVALID, std::string(who) + ": pitch_elems < W");
    const Geom& g = c->g;
    if (g_ref) CK(c, cudaMemsetAsync(g_ref, 0, (size_t)g.H * g.W * sizeof(float), c->stream));
    if (n == 0) return CCST_OK;
    if ((rc = off_prepare(c))) return rc;
    const size_t smem = adj_smem_bytes(g.H, g.W);
    if (!c->d_adjY) {
        CK(c, cudaFuncSetAttribute(adj_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        CK(c, cudaMalloc(&c->d_adjY, (size_t)g.H * g.Wc * sizeof(double2)));
    }
    const int grid = (int)(n < c->off_max_parts ? n : c->off_max_parts);
    AdjArgs a;
    a.frames = frames;
    a.n = n;
    a.pitch = pitch;
    a.rec = (const Result*)rec;
    a.g = gdxdy;
    a.peak = peak;
    a.status = status;
    a.g_frames = g_frames;
    a.scratch = c->d_offScratch;
    a.part = g_ref ? c->d_offPart : nullptr;
    adj_kernel<<<grid, 512, smem, c->stream>>>(g, a);
    CK(c, cudaGetLastError());
    if (g_ref) {
        adj_ref_cols<<<g.Wc, 128, 0, c->stream>>>(g, c->d_offPart, grid, c->d_adjY);
        adj_ref_rows<<<g.H / 2, 128, 0, c->stream>>>(g, c->d_adjY, g_ref);
        CK(c, cudaGetLastError());
    }
    return CCST_OK;
}

extern "C" int ccst_peak_continuous(ccst_ctx* c, const void* frames_dev, int64_t n, int64_t pitch_elems,
                                    const ccst_result* rec_dev, double* peak_dev, int32_t* status_dev) {
    if (c && n > 0 && !peak_dev && !status_dev)
        return fail(c, CCST_E_INVALID, "ccst_peak_continuous: no output");
    return adj_run(c, frames_dev, n, pitch_elems, rec_dev, nullptr, peak_dev, status_dev, nullptr, nullptr,
                   "ccst_peak_continuous");
}

extern "C" int ccst_backward(ccst_ctx* c, const void* frames_dev, int64_t n, int64_t pitch_elems,
                             const ccst_result* rec_dev, const float* g_dxdy_dev, float* g_frames_dev,
                             float* g_ref_dev) {
    if (c && n > 0 && !g_dxdy_dev) return fail(c, CCST_E_INVALID, "ccst_backward: null upstream gradient");
    return adj_run(c, frames_dev, n, pitch_elems, rec_dev, g_dxdy_dev, nullptr, nullptr, g_frames_dev, g_ref_dev,
                   "ccst_backward");
}

extern "C" void ccst_destroy(ccst_ctx* c) {
    if (!c) return;
    cudaStreamSynchronize(c->stream);
    free_all(c);
    delete c;
}

extern "C" const char* ccst_last_error(ccst_ctx* c) {
    if (c) return c->err.c_str();
    std::lock_guard<std::mutex> lk(g_create_err_mu);
    return g_create_err.c_str();
}

// Diagnostic entry (tests only): runs ccst_track without graphs and also writes the
// FP32 integer surfaces (n x H x W, unnormalised) and the FP32 delta surfaces
// (n x M x M, unnormalised, relative to the integer peak) when the pointers are non-null.
extern "C" int ccst_debug_surfaces(ccst_ctx* c, const void* frames_dev, int64_t n, int64_t pitch_elems,
                                   ccst_result* out_dev, float* int_surf_dev, float* sub_surf_dev) {
    int rc = check_ctx(c);
    if (rc) return rc;
    if (c->general && !c->gplans[c->refs[0].gcls].mix) return not_general(c, "ccst_debug_surfaces");
    Batch b;
    if ((rc = make_batch(c, frames_dev, n, pitch_elems, out_dev, &b))) return rc;
    if (c->general) {
        // the FP32 general-size kernel's surfaces; frames it cannot certify still get their
        // records from the double-float kernel
        if (n == 0) return CCST_OK;
        cudaError_t e;
        const unsigned k = ring_acquire(c, c->stream, &e);
        CK(c, e);
        CK(c, shared_acquire(c, c->stream));
        const MixDbg dbg{int_surf_dev, sub_surf_dev, nullptr, nullptr};
        if ((rc = gen_track(c, b, c->stream, c->glane[0], c->d_launch_counters + k, &dbg))) return rc;
        CK(c, ring_release(c, k, c->stream));
        CK(c, shared_release(c, c->stream));
        return CCST_OK;
    }
    b.dbg_int = int_surf_dev;
    b.dbg_sub = sub_surf_dev;
    return launch(c, b);
}

extern "C" int ccst_profile_kernel_ms(ccst_ctx* c, double* sum_ms, int64_t* launches) {
    int rc = check_ctx(c);
    if (rc) return rc;
    if ((rc = not_general(c, "ccst_profile_kernel_ms"))) return rc;
    if (!(c->p.flags & CCST_FLAG_PROFILE) || !sum_ms || !launches)
        return fail(c, CCST_E_INVALID, "profiling is off or null output");
    CK(c, cudaStreamSynchronize(c->stream));
    double total = 0.0;
    int64_t cnt = 0;
    float ms = 0.f;
    for (auto& kv : c->graphs) {
        if (cudaEventElapsedTime(&ms, kv.second.e0, kv.second.e1) == cudaSuccess) { total += ms; ++cnt; }
    }
    cudaGetLastError();   // a graph that never replayed leaves its events unrecorded
    for (int i = 0; i < c->prof_used; ++i) {
        CK(c, cudaEventElapsedTime(&ms, c->prof0[i], c->prof1[i]));
        total += ms;
        ++cnt;
    }
    *sum_ms = total;
    *launches = cnt;
    return CCST_OK;
}

extern "C" int ccst_profile_reset(ccst_ctx* c) {
    int rc = check_ctx(c);
    if (rc) return rc;
    if ((rc = not_general(c, "ccst_profile_reset"))) return rc;
    c->prof_used = 0;
    c->prof_next = 0;
    return CCST_OK;
}

// Diagnostic entry (tests only): for frame f, v(jb) - v(ja) of the upsampled surface for the
// grid pair pairs_dev[2f], pairs_dev[2f+1], by the FP32 pair-difference guard (d32) and by
// FP64 accumulation over the FP32 spectrum (d64). Unnormalised units. Results only: no tracking.
extern "C" int ccst_debug_pairs(ccst_ctx* c, const void* frames_dev, int64_t n, int64_t pitch_elems,
                                const int32_t* pairs_dev, float* d32_dev, double* d64_dev) {
    int rc = check_ctx(c);
    if (rc) return rc;
    if (c->general && !c->gplans[c->refs[0].gcls].mix) return not_general(c, "ccst_debug_pairs");
    if (!pairs_dev || !d32_dev || !d64_dev) return fail(c, CCST_E_INVALID, "null pair buffers");
    Batch b;
    if ((rc = make_batch(c, frames_dev, n, pitch_elems, (ccst_result*)c->d_out, &b))) return rc;
    if (c->general) {
        // the FP32 general-size kernel's pair-difference level; it has no FP64 variant (NaN)
        if (n == 0) return CCST_OK;
        CK(c, cudaMemsetAsync(d64_dev, 0xFF, (size_t)n * sizeof(double), c->stream));
        cudaError_t e;
        const unsigned k = ring_acquire(c, c->stream, &e);
        CK(c, e);
        CK(c, shared_acquire(c, c->stream));
        const MixDbg dbg{nullptr, nullptr, pairs_dev, d32_dev};
        if ((rc = gen_track(c, b, c->stream, c->glane[0], c->d_launch_counters + k, &dbg))) return rc;
        CK(c, ring_release(c, k, c->stream));
        CK(c, shared_release(c, c->stream));
        return CCST_OK;
    }
    b.dbg_pairs = pairs_dev;
    b.dbg_d32 = d32_dev;
    b.dbg_d64 = d64_dev;
    if (n == 0) return CCST_OK;
    const int grid = (int)(n < c->grid_main ? n : c->grid_main);
    Geom gk = c->g;
    void* args[] = {&gk, &b};
    CK(c, cudaLaunchKernel(c->kernel, dim3(grid), dim3(c->threads), args, c->smem, c->stream));
    return CCST_OK;
}

// Diagnostic entry (tests only): tracks with the table copies withheld, so that the first
// bounded wait of every CTA runs out; the frames reached report CCST_R_TIMEOUT.
extern "C" int ccst_debug_timeout(ccst_ctx* c, const void* frames_dev, int64_t n, int64_t pitch_elems,
                                  ccst_result* out_dev) {
    int rc = check_ctx(c);
    if (rc) return rc;
    if ((rc = not_general(c, "ccst_debug_timeout"))) return rc;
    Batch b;
    if ((rc = make_batch(c, frames_dev, n, pitch_elems, out_dev, &b))) return rc;
    b.dbg_no_copy = 1;
    if (n == 0) return CCST_OK;
    const int grid = (int)(n < c->grid_main ? n : c->grid_main);
    Geom gk = c->g;
    void* args[] = {&gk, &b};
    CK(c, cudaLaunchKernel(c->kernel, dim3(grid), dim3(c->threads), args, c->smem, c->stream));
    return CCST_OK;
}

// ------------------------------------------------------- real-time reference (Sec. III B)
// One reference update (rt_update) on the context's stream; rec null when starting.
static int rt_launch(ccst_ctx* c, int mode, const void* frame, long long pitch, ccst_result* rec,
                     unsigned extra = 0, int frame_f64 = 0) {
    const Geom& g = c->g;
    RtArgs a;
    a.frame = frame;
    a.frame_f64 = frame_f64;
    a.pitch = pitch;
    a.off = g.method == CCST_CC_SN ? (double)g.eps : 0.0;
    a.mode = mode;
    a.a0 = c->rt_a0;
    a.b1 = c->rt_b1;
    a.rec = (Result*)rec;
    a.E = c->d_rtE;
    a.Y = c->d_rtY;
    a.b64 = c->d_b64;
    a.FE64 = c->d_FE64;
    a.FE32 = c->d_FE32;
    a.FEdf = const_cast<dfc*>(g.FEdf);
    a.sync = c->d_rtSync;
    a.extra = extra;
    a.base = 3u * (unsigned)c->rt_grid * c->rt_seq++;
    a.limit = extra ? (1u << 12) : (1u << 22);
    a.part = c->d_offPart;
    a.nparts = c->off_parts;
    a.count = c->d_rtSync + 3;
    a.next = c->d_next;
    Geom gk = g;
    void* args[] = {&gk, &a};
    CK(c, cudaLaunchCooperativeKernel((const void*)rt_update, dim3(c->rt_grid), dim3(128), args, 0, c->stream));
    return CCST_OK;
}

// Filter state and grid-barrier words of the reference updates, on first use.
static int rt_prepare(ccst_ctx* c) {
    if (c->d_rtE) return CCST_OK;
    const Geom& g = c->g;
    const size_t HWc = (size_t)g.H * g.Wc;
    int coop = 0, per_sm = 0, sms = 0;
    CK(c, cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, c->device));
    CK(c, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device));
    CK(c, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, rt_update, 128, 0));
    if (!coop || per_sm < 1) return fail(c, CCST_E_UNSUPPORTED, "reference update: no cooperative launch");
    const int want = g.Wc > g.H / 2 ? g.Wc : g.H / 2;
    c->rt_grid = want < per_sm * sms ? want : per_sm * sms;
    CK(c, cudaMalloc(&c->d_rtSync, 4 * sizeof(unsigned)));
    CK(c, cudaMemsetAsync(c->d_rtSync, 0, 4 * sizeof(unsigned), c->stream));
    c->rt_seq = 0;
    CK(c, cudaMalloc(&c->d_rtY, HWc * sizeof(double2)));
    CK(c, cudaMalloc(&c->d_rtE, HWc * sizeof(double2)));
    return CCST_OK;
}

static int check_frame(ccst_ctx* c, const void* frame, int64_t* pitch, const char* who) {
    if (!frame) return fail(c, CCST_E_INVALID, std::string(who) + ": null frame");
    if (*pitch == 0) *pitch = c->g.W;
    if (*pitch < c->g.W) return fail(c, CCST_E_INVALID, std::string(who) + ": pitch_elems < W");
    return CCST_OK;
}

extern "C" int ccst_set_reference_frame(ccst_ctx* c, const void* frame_dev, int64_t pitch_elems) {
    int rc = check_ctx(c);
    if (rc) return rc;
    if ((rc = check_frame(c, frame_dev, &pitch_elems, "ccst_set_reference_frame"))) return rc;
    if (c->general)
        return gen_ref_spectrum(c, c->g.H, c->g.W, frame_dev, 1, pitch_elems, (dfc*)c->refs[0].gFb);
    if ((rc = rt_prepare(c))) return rc;
    CK(c, cudaMemsetAsync(c->d_rtSync, 0, 4 * sizeof(unsigned), c->stream));
    c->rt_seq = 0;
    return rt_launch(c, kRtStart, frame_dev, pitch_elems, nullptr);
}

extern "C" int ccst_set_reference_image(ccst_ctx* c, const double* image_dev) {
    int rc = check_ctx(c);
    if (rc) return rc;
    if ((rc = not_general(c, "ccst_set_reference_image"))) return rc;
    if (!image_dev) return fail(c, CCST_E_INVALID, "ccst_set_reference_image: null image");
    if ((rc = rt_prepare(c))) return rc;
    CK(c, cudaMemsetAsync(c->d_rtSync, 0, 4 * sizeof(unsigned), c->stream));
    c->rt_seq = 0;
    return rt_launch(c, kRtStart, image_dev, c->g.W, nullptr, 0, 1);
}

// ------------------------------------------- reference refinement by the adjoint
// The template E is refined by gradient steps on the mean squared error of the continuous
// peaks of calibration frames with known displacements d_i:
//   L(E) = (1/n) sum_{i: status 0} |s*_i(E) - d_i|^2,   dL/ds*_i = 2 (s*_i - d_i) / n,
// dL/dE from the adjoint (ccst_backward). A step is E <- E - h |E| / |dL/dE| dL/dE (2-norms
// over the pixels). A step whose loss exceeds the last accepted one is undone and h halved.

// Block-wide sum of one double per thread in a fixed order (a shuffle tree per warp, then
// the warps' sums in warp order); the result is returned to every thread.
__device__ double refine_block_sum(double v, double* red) {
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = (int)(blockDim.x >> 5);
    __syncthreads();
    if (l == 0) red[w] = v;
    __syncthreads();
    if (w == 0) {
        v = l < nw ? red[l] : 0.0;
        for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (l == 0) red[32] = v;
    }
    __syncthreads();
    return red[32];
}

// E from the reference operand b: CC-U E = b, CC-SN E = 1/b - eps.
__global__ void refine_init(Geom g, const double* b64, double* E, double* scal, double step) {
    const int n = g.H * g.W;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        E[i] = g.method == 0 ? b64[i] : 1.0 / b64[i] - (double)g.eps;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        scal[0] = 0.0;
        scal[1] = step;
        scal[2] = 0.0;
        scal[3] = 0.0;
    }
}

// Loss at the current template and the upstream gradient of every frame.
__global__ void __launch_bounds__(256) refine_seed(const double* peak, const int32_t* status, const double* target,
                                                   long long n, float* g, double* scal) {
    __shared__ double red[33];
    double acc = 0.0;
    const double inv = 1.0 / (double)n;
    for (long long i = threadIdx.x; i < n; i += blockDim.x) {
        float gx = 0.f, gy = 0.f;
        if (status[i] == 0) {
            const double ex = peak[2 * i] - target[2 * i], ey = peak[2 * i + 1] - target[2 * i + 1];
            acc += ex * ex + ey * ey;
            gx = (float)(2.0 * ex * inv);
            gy = (float)(2.0 * ey * inv);
        }
        g[2 * i] = gx;
        g[2 * i + 1] = gy;
    }
    acc = refine_block_sum(acc, red);
    if (threadIdx.x == 0) scal[0] = acc * inv;
}

// Accept the evaluated template (or undo the step and halve it), record the loss and the
// step that produced it, and take the next step unless this is the last evaluation.
__global__ void __launch_bounds__(1024) refine_step(int nel, double* E, double* Eprev, const float* gE, float* gEprev,
                                                    double* scal, double* hist, int k, int last) {
    __shared__ double red[33];
    __shared__ int revert;
    __shared__ double coef;
    if (threadIdx.x == 0) {
        const double L = scal[0];
        hist[2 * k] = L;
        hist[2 * k + 1] = scal[1];
        revert = scal[3] != 0.0 && L > scal[2];
        if (revert) scal[1] *= 0.5;
        else scal[2] = L;
        scal[3] = 1.0;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < nel; i += blockDim.x) {
        if (revert) E[i] = Eprev[i];
        else { Eprev[i] = E[i]; gEprev[i] = gE[i]; }
    }
    if (last) return;
    double se = 0.0, sg = 0.0;
    for (int i = threadIdx.x; i < nel; i += blockDim.x) {
        const double gv = (double)gEprev[i];
        se += E[i] * E[i];
        sg += gv * gv;
    }
    se = refine_block_sum(se, red);
    sg = refine_block_sum(sg, red);
    if (threadIdx.x == 0) coef = sg > 0.0 ? scal[1] * sqrt(se) / sqrt(sg) : 0.0;
    __syncthreads();
    for (int i = threadIdx.x; i < nel; i += blockDim.x) E[i] -= coef * (double)gEprev[i];
}

extern "C" int ccst_refine_reference(ccst_ctx* c, const void* frames_dev, int64_t n, int64_t pitch_elems,
                                     const double* target_dev, int steps, double step_rel, double* hist_dev,
                                     double* ref_out_dev) {
    int rc = check_ctx(c);
    if (rc) return rc;
    if ((rc = not_general(c, "ccst_refine_reference"))) return rc;
    if (n < 1 || steps < 0 || !(step_rel > 0.0) || !std::isfinite(step_rel))
        return fail(c, CCST_E_INVALID, "ccst_refine_reference: need n >= 1, steps >= 0, finite step_rel > 0");
    if (!target_dev || !hist_dev) return fail(c, CCST_E_INVALID, "ccst_refine_reference: null target or hist");
    if ((rc = check_frame(c, frames_dev, &pitch_elems, "ccst_refine_reference"))) return rc;
    const Geom& g = c->g;
    const int nel = g.H * g.W;
    auto& w = c->rf;
    if (!w.E) {
        CK(c, cudaMalloc(&w.E, nel * sizeof(double)));
        CK(c, cudaMalloc(&w.Eprev, nel * sizeof(double)));
        CK(c, cudaMalloc(&w.gE, nel * sizeof(float)));
        CK(c, cudaMalloc(&w.gEprev, nel * sizeof(float)));
        CK(c, cudaMalloc(&w.scal, 4 * sizeof(double)));
    }
    if (w.cap < n) {
        CK(c, cudaStreamSynchronize(c->stream));          // the old buffers may still be in use
        void* old[] = {w.rec, w.peak, w.status, w.g};
        for (void* p : old)
            if (p) cudaFree(p);
        w.rec = nullptr; w.peak = nullptr; w.status = nullptr; w.g = nullptr;
        w.cap = 0;
        CK(c, cudaMalloc(&w.rec, (size_t)n * sizeof(Result)));
        CK(c, cudaMalloc(&w.peak, (size_t)n * 2 * sizeof(double)));
        CK(c, cudaMalloc(&w.status, (size_t)n * sizeof(int32_t)));
        CK(c, cudaMalloc(&w.g, (size_t)n * 2 * sizeof(float)));
        w.cap = n;
    }
    const size_t elem = c->p.in_dtype == CCST_U16 ? 2 : 4;
    refine_init<<<32, 256, 0, c->stream>>>(g, c->d_b64, w.E, w.scal, step_rel);
    CK(c, cudaGetLastError());
    for (int k = 0; k <= steps; ++k) {
        for (int64_t s = 0; s < n; s += c->p.max_batch) {          // records against the current E
            const int64_t m = n - s < c->p.max_batch ? n - s : c->p.max_batch;
            Batch b;
            const char* f = (const char*)frames_dev + (size_t)s * g.H * pitch_elems * elem;
            if ((rc = make_batch(c, f, m, pitch_elems, (ccst_result*)(w.rec + s), &b))) return rc;
            if ((rc = launch(c, b))) return rc;
        }
        if ((rc = ccst_peak_continuous(c, frames_dev, n, pitch_elems, (const ccst_result*)w.rec, w.peak, w.status)))
            return rc;
        refine_seed<<<1, 256, 0, c->stream>>>(w.peak, w.status, target_dev, (long long)n, w.g, w.scal);
        CK(c, cudaGetLastError());
        if ((rc = ccst_backward(c, frames_dev, n, pitch_elems, (const ccst_result*)w.rec, w.g, nullptr, w.gE)))
            return rc;
        refine_step<<<1, 1024, 0, c->stream>>>(nel, w.E, w.Eprev, w.gE, w.gEprev, w.scal, hist_dev, k, k == steps);
        CK(c, cudaGetLastError());
        if ((rc = ccst_set_reference_image(c, w.E))) return rc;
    }
    if (ref_out_dev) CK(c, cudaMemcpyAsync(ref_out_dev, w.E, nel * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
    return CCST_OK;
}

extern "C" int ccst_rt_begin(ccst_ctx* c, const void* frame0_dev, int64_t pitch_elems, double a0, double b1) {
    int rc = check_ctx(c);
    if (rc) return rc;
    if ((rc = not_general(c, "ccst_rt_begin"))) return rc;
    if (!std::isfinite(a0) || !std::isfinite(b1)) return fail(c, CCST_E_INVALID, "ccst_rt_begin: a0, b1 not finite");
    if ((rc = check_frame(c, frame0_dev, &pitch_elems, "ccst_rt_begin"))) return rc;
    if ((rc = ccst_set_reference_frame(c, frame0_dev, pitch_elems))) return rc;
    c->rt_a0 = a0;
    c->rt_b1 = b1;
    c->rt_on = true;
    return CCST_OK;
}

extern "C" int ccst_rt_track(ccst_ctx* c, const void* frames_dev, int64_t n, int64_t pitch_elems,
                             ccst_result* out_dev) {
    int rc = check_ctx(c);
    if (rc) return rc;
    if ((rc = not_general(c, "ccst_rt_track"))) return rc;
    if (!c->rt_on) return fail(c, CCST_E_INVALID, "ccst_rt_track: no real-time reference (ccst_rt_begin)");
    if (n < 0) return fail(c, CCST_E_INVALID, "ccst_rt_track: n < 0");
    if (n == 0) return CCST_OK;
    if (!frames_dev || !out_dev) return fail(c, CCST_E_INVALID, "ccst_rt_track: null frames or out");
    if (pitch_elems == 0) pitch_elems = c->g.W;
    if (pitch_elems < c->g.W) return fail(c, CCST_E_INVALID, "ccst_rt_track: pitch_elems < W");
    const Geom& g = c->g;
    const size_t fbytes = (size_t)g.H * pitch_elems * (c->p.in_dtype == CCST_U16 ? 2 : 4);
    for (int64_t i = 0; i < n; ++i) {
        const void* frame = (const char*)frames_dev + (size_t)i * fbytes;
        Batch b;
        if ((rc = make_batch(c, frame, 1, pitch_elems, out_dev + i, &b))) return rc;
        if ((rc = launch(c, b, i == 0, c->d_next))) return rc;   // frame i against E_{i-1}; the update
                                                                 // zeroes d_next for the next frame
        if ((rc = rt_launch(c, kRtUpdate, frame, pitch_elems, out_dev + i))) return rc;   // E_i
    }
    return CCST_OK;
}

// ---------------------------------------------------------- offline reference (Sec. III A)
static size_t off_smem_bytes(const Geom& g) {
    const int nbuf = (g.H / 2) * g.W > g.Wc * (g.H + 1) ? (g.H / 2) * g.W : g.Wc * (g.H + 1);
    return (size_t)(nbuf + g.H + g.Wc) * sizeof(double2);
}

static int off_prepare(ccst_ctx* c) {
    if (c->d_offPart) return CCST_OK;
    const Geom& g = c->g;
    const size_t smem = off_smem_bytes(g);
    CK(c, cudaFuncSetAttribute(off_accumulate, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0, sms = 0;
    CK(c, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device));
    CK(c, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, off_accumulate, 512, smem));
    if (per_sm < 1) return fail(c, CCST_E_SHAPE, "ccst_offline_update: the frame transform does not fit on an SM");
    c->off_max_parts = per_sm * sms;
    const size_t bytes = (size_t)c->off_max_parts * g.H * g.Wc * sizeof(double2);
    CK(c, cudaMalloc(&c->d_offPart, bytes));
    CK(c, cudaMalloc(&c->d_offScratch, bytes));
    return CCST_OK;
}

extern "C" int ccst_offline_update(ccst_ctx* c, const void* frames_dev, int64_t n, int64_t pitch_elems,
                                   const ccst_result* rec_dev) {
    int rc = check_ctx(c);
    if (rc) return rc;
    if ((rc = not_general(c, "ccst_offline_update"))) return rc;
    if (n < 0) return fail(c, CCST_E_INVALID, "ccst_offline_update: n < 0");
    if (n == 0) return CCST_OK;
    if (!rec_dev) return fail(c, CCST_E_INVALID, "ccst_offline_update: null records");
    if ((rc = check_frame(c, frames_dev, &pitch_elems, "ccst_offline_update"))) return rc;
    if ((rc = rt_prepare(c)) || (rc = off_prepare(c))) return rc;
    const Geom& g = c->g;
    const int grid = (int)(n < c->off_max_parts ? n : c->off_max_parts);
    c->off_parts = grid;
    const double off = g.method == CCST_CC_SN ? (double)g.eps : 0.0;
    CK(c, cudaMemsetAsync(c->d_rtSync + 3, 0, sizeof(unsigned), c->stream));
    off_accumulate<<<grid, 512, off_smem_bytes(g), c->stream>>>(g, frames_dev, (long long)n, (long long)pitch_elems,
                                                                 off, (const Result*)rec_dev, c->d_offScratch,
                                                                 c->d_offPart, c->d_rtSync + 3);
    CK(c, cudaGetLastError());
    return rt_launch(c, kRtMean, nullptr, 0, nullptr);
}

extern "C" int ccst_offline_track(ccst_ctx* c, const void* frames_dev, int64_t n, int64_t pitch_elems, int passes,
                                  ccst_result* out_dev) {
    int rc = check_ctx(c);
    if (rc) return rc;
    if ((rc = not_general(c, "ccst_offline_track"))) return rc;
    if (n < 1 || passes < 0) return fail(c, CCST_E_INVALID, "ccst_offline_track: n < 1 or passes < 0");
    if (!out_dev) return fail(c, CCST_E_INVALID, "ccst_offline_track: null out");
    if ((rc = check_frame(c, frames_dev, &pitch_elems, "ccst_offline_track"))) return rc;
    if ((rc = ccst_set_reference_frame(c, frames_dev, pitch_elems))) return rc;          // E_0 = I_0
    const size_t fbytes = (size_t)c->g.H * pitch_elems * (c->p.in_dtype == CCST_U16 ? 2 : 4);
    for (int p = 0; p <= passes; ++p) {
        for (int64_t s = 0; s < n; s += c->p.max_batch) {                           // every frame against E_p
            const int64_t m = n - s < c->p.max_batch ? n - s : c->p.max_batch;
            Batch b;
            if ((rc = make_batch(c, (const char*)frames_dev + (size_t)s * fbytes, m, pitch_elems, out_dev + s, &b)))
                return rc;
            if ((rc = launch(c, b))) return rc;
        }
        if (p < passes && (rc = ccst_offline_update(c, frames_dev, n, pitch_elems, out_dev))) return rc;   // E_{p+1}
    }
    return CCST_OK;
}

extern "C" int ccst_reference_status(ccst_ctx* c, int* stale) {
    int rc = check_ctx(c);
    if (rc) return rc;
    if (!stale) return fail(c, CCST_E_INVALID, "ccst_reference_status: null stale");
    *stale = 0;
    if (!c->d_rtSync) return CCST_OK;
    unsigned err = 0;
    CK(c, cudaStreamSynchronize(c->stream));
    CK(c, cudaMemcpy(&err, c->d_rtSync + 2, sizeof(unsigned), cudaMemcpyDeviceToHost));
    *stale = err != 0;
    return CCST_OK;
}

extern "C" int ccst_debug_reference(ccst_ctx* c, double* ref_dev) {
    int rc = check_ctx(c);
    if (rc) return rc;
    if ((rc = not_general(c, "ccst_debug_reference"))) return rc;
    if (!ref_dev) return fail(c, CCST_E_INVALID, "ccst_debug_reference: null buffer");
    CK(c, cudaMemcpyAsync(ref_dev, c->d_b64, (size_t)c->g.H * c->g.W * sizeof(double), cudaMemcpyDeviceToDevice,
                          c->stream));
    return CCST_OK;
}

extern "C" int ccst_debug_rt_timeout(ccst_ctx* c, const void* frame_dev, int64_t pitch_elems,
                                     ccst_result* rec_dev) {
    int rc = check_ctx(c);
    if (rc) return rc;
    if ((rc = not_general(c, "ccst_debug_rt_timeout"))) return rc;
    if (!c->rt_on) return fail(c, CCST_E_INVALID, "ccst_debug_rt_timeout: no real-time reference (ccst_rt_begin)");
    if (!frame_dev || !rec_dev) return fail(c, CCST_E_INVALID, "ccst_debug_rt_timeout: null frame or record");
    if (pitch_elems == 0) pitch_elems = c->g.W;
    if (pitch_elems < c->g.W) return fail(c, CCST_E_INVALID, "ccst_debug_rt_timeout: pitch_elems < W");
    return rt_launch(c, kRtUpdate, frame_dev, pitch_elems, rec_dev, 1);
}

extern "C" int ccst_drift_correct(const ccst_result* rec_dev, int64_t n, double a0, double b1, double alpha,
                                  int u, double* out_dev, void* stream) {
    if (n < 0 || (n > 0 && (!rec_dev || !out_dev))) return CCST_E_INVALID;
    if (!std::isfinite(a0) || !std::isfinite(b1) || !(alpha == alpha) || (alpha > 0.0 && u < 1))
        return CCST_E_INVALID;
    if (n == 0) return CCST_OK;
    const double lim = alpha > 0.0 ? alpha / u : 0.0;
    rt_drift<<<1, 32, 0, (cudaStream_t)stream>>>((const Result*)rec_dev, (long long)n, a0, b1, lim, out_dev);
    return cudaGetLastError() == cudaSuccess ? CCST_OK : CCST_E_CUDA;
}

// ------------------------------------------------------------------ uneven-ROI batches
static bool rois_size_ok(int H, int W) { return H == W && (H == 16 || H == 32 || H == 64 || H == 128); }

static void df_lengths(const Geom& g, int* ncy, int* ncx) {
    const long long Dy = (long long)g.u * g.H, Dx = (long long)g.u * g.W;
    *ncy = (int)((Dy + g.By - 1) / g.By);
    *ncx = (int)((Dx + g.Bx - 1) / g.Bx);
}

// Plan 0 and ref 0 are the context's own size and reference.
static void rois_init(ccst_ctx* c) {
    if (!c->plans.empty()) return;
    ccst_ctx::SizePlan p0;
    p0.g = c->g;
    df_lengths(c->g, &p0.ncy, &p0.ncx);
    c->plans.push_back(p0);
    ccst_ctx::RefEntry r0;
    r0.cls = rois_size_ok(c->g.H, c->g.W) ? 0 : -1;
    r0.r = RefSpectra{c->d_FE32, c->d_FE64, c->d_b64, c->g.FEdf};
    c->refs.push_back(r0);
}

// The size class of H x W, made on first use: geometry, twiddles, stage tables and the
// double-float tables, as ccst_create makes them for the context's own size.
static int rois_plan(ccst_ctx* c, int H, int W, int* cls) {
    for (size_t i = 0; i < c->plans.size(); ++i)
        if (c->plans[i].g.H == H && c->plans[i].g.W == W) {
            *cls = (int)i;
            return CCST_OK;
        }
    int limit = 0;
    CK(c, cudaDeviceGetAttribute(&limit, cudaDevAttrMaxSharedMemoryPerBlockOptin, c->device));
    ccst_ctx::SizePlan sp;
    Geom& g = sp.g;
    // the ROI kernel keeps its Geom, work-item index and tensor-core state in static shared memory
    if (!plan_geometry(H, W, c->p, (size_t)(limit - kRoisStaticSmem), &g))
        return fail(c, CCST_E_SHAPE, "ccst_add_reference: frame too large");
    const long long Dy = (long long)g.u * H, Dx = (long long)g.u * W;
    g.By = 1; while ((long long)g.By * g.By < Dy) ++g.By;
    g.Bx = 1; while ((long long)g.Bx * g.Bx < Dx) ++g.Bx;
    df_lengths(g, &sp.ncy, &sp.ncx);
    const size_t HWc = (size_t)H * g.Wc;
    const size_t tabA = (size_t)g.Hh * g.T1p, tabB = (size_t)g.Wc * g.T1p;
    const size_t ndf = (size_t)(g.Ntw / 2) + HWc + sp.ncy + g.By + sp.ncx + g.Bx;
    double2* tw64 = nullptr;
    float2* tw32 = nullptr;
    float* tab = nullptr;
    dfc* df = nullptr;
    struct { void** ptr; size_t bytes; } allocs[] = {
        {(void**)&tw64, (size_t)(g.Ntw / 2) * sizeof(double2)},
        {(void**)&tw32, (size_t)(g.Ntw / 2) * sizeof(float2)},
        {(void**)&tab, (2 * tabA + 3 * tabB) * sizeof(float) + table_bytes(g)},
        {(void**)&df, ndf * sizeof(dfc)},
    };
    for (auto& a : allocs) {
        const cudaError_t e = cudaMalloc(a.ptr, a.bytes);
        if (e != cudaSuccess) {
            for (void* p : sp.mem) cudaFree(p);
            return fail(c, e == cudaErrorMemoryAllocation ? CCST_E_NOMEM : CCST_E_CUDA,
                        std::string("cudaMalloc: ") + cudaGetErrorString(e));
        }
        sp.mem.push_back(*a.ptr);
    }
    g.tw64 = tw64; g.tw32 = tw32;
    g.tA_cm1 = tab; g.tA_s = tab + tabA;
    g.tB_wc = tab + 2 * tabA; g.tB_ws = g.tB_wc + tabB; g.tB_gc = g.tB_ws + tabB;
    g.tAh = (const uint2*)(g.tB_gc + tabB);
    g.tBh = (const uint2*)((const char*)g.tAh + ta_bytes(g));
    g.twdf = df;
    g.FEdf = df + g.Ntw / 2;                               // the first reference's slot (unused)
    g.eyc = g.FEdf + HWc; g.eyf = g.eyc + sp.ncy; g.exc = g.eyf + g.By; g.exf = g.exc + sp.ncx;
    init_twiddles<<<1, 256, 0, c->stream>>>(g.Ntw, tw64, tw32);
    init_tables<<<64, 256, 0, c->stream>>>(g, (float*)g.tA_cm1, (float*)g.tA_s, (float*)g.tB_wc, (float*)g.tB_ws,
                                           (float*)g.tB_gc, (uint2*)g.tAh, (uint2*)g.tBh);
    CK(c, cudaGetLastError());
    c->plans.push_back(sp);
    *cls = (int)c->plans.size() - 1;
    c->rois_dirty = true;
    return CCST_OK;
}

static bool generic_size_ok(int H, int W) { return H == W && H >= 8 && H <= 256 && !rois_size_ok(H, W); }

extern "C" int ccst_add_reference(ccst_ctx* c, const float* ref, int H, int W, int* ref_id) {
    int rc = check_ctx(c);
    if (rc) return rc;
    if (!ref || !ref_id) return fail(c, CCST_E_INVALID, "ccst_add_reference: null ref or ref_id");
    if (generic_size_ok(H, W)) {
        rois_init(c);
        return add_generic_reference(c, ref, H, W, ref_id);
    }
    if (!rois_size_ok(H, W))
        return fail(c, CCST_E_SHAPE, "ccst_add_reference: ROIs are square, 8 to 256 pixels a side");
    rois_init(c);
    int cls = 0;
    if ((rc = rois_plan(c, H, W, &cls))) return rc;
    const Geom pg = c->plans[cls].g;
    const size_t HW = (size_t)H * W, HWc = (size_t)H * pg.Wc;
    const size_t l2per = (size_t)(H / 2) * W + (size_t)H * pg.Wcp;
    ccst_ctx::RefEntry re;
    re.cls = cls;
    // one block per reference: b64 | FE64 | FE32 | FEdf (each size a multiple of 16 bytes);
    // the reference copy and the FFT workspace live in a scratch block the context keeps
    const size_t nb64 = HW * sizeof(double), nFE64 = HWc * sizeof(double2), nFE32 = (HWc * sizeof(float2) + 15) & ~(size_t)15;
    const size_t ntmp = HW * sizeof(float) + l2per * sizeof(double2);
    char* blk = nullptr;
    cudaError_t e = cudaMalloc(&blk, nb64 + nFE64 + nFE32 + HWc * sizeof(dfc));
    if (e != cudaSuccess)
        return fail(c, e == cudaErrorMemoryAllocation ? CCST_E_NOMEM : CCST_E_CUDA, std::string("cudaMalloc: ") + cudaGetErrorString(e));
    re.mem.push_back(blk);
    double* b64 = (double*)blk;
    double2* FE64 = (double2*)(blk + nb64);
    float2* FE32 = (float2*)(blk + nb64 + nFE64);
    dfc* FEdf = (dfc*)(blk + nb64 + nFE64 + nFE32);
    auto undo = [&]() { for (void* p : re.mem) cudaFree(p); };
    if (c->addref_tmp_bytes < ntmp) {
        if (c->d_addref_tmp) cudaFree(c->d_addref_tmp);
        c->d_addref_tmp = nullptr;
        c->addref_tmp_bytes = 0;
        e = cudaMalloc(&c->d_addref_tmp, ntmp);
        if (e != cudaSuccess) {
            undo();
            return fail(c, e == cudaErrorMemoryAllocation ? CCST_E_NOMEM : CCST_E_CUDA, std::string("cudaMalloc: ") + cudaGetErrorString(e));
        }
        c->addref_tmp_bytes = ntmp;
    }
    double2* work = (double2*)c->d_addref_tmp;
    float* ref32 = (float*)((char*)c->d_addref_tmp + l2per * sizeof(double2));
    Geom gt = pg;
    gt.b64 = b64;
    e = cudaMemcpyAsync(ref32, ref, HW * sizeof(float), cudaMemcpyDefault, c->stream);
    if (e == cudaSuccess) {
        init_ref_operand<<<32, 256, 0, c->stream>>>(gt, ref32, b64);
        init_ref_spectrum<<<1, 256, 0, c->stream>>>(gt, work, FE64, FE32);
        const int ncy = c->plans[cls].ncy, ncx = c->plans[cls].ncx;
        init_dfloat<<<32, 256, 0, c->stream>>>(gt, pg.tw64, FE64, (dfc*)pg.twdf, FEdf, (dfc*)pg.eyc, (dfc*)pg.eyf,
                                               (dfc*)pg.exc, (dfc*)pg.exf, ncy, ncx);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    }
    if (e != cudaSuccess) {
        undo();
        return fail(c, CCST_E_CUDA, std::string("ccst_add_reference: ") + cudaGetErrorString(e));
    }
    re.r = RefSpectra{FE32, FE64, b64, FEdf};
    c->refs.push_back(re);
    c->rois_dirty = true;
    c->gen_dirty = true;
    *ref_id = (int)c->refs.size() - 1;
    return CCST_OK;
}

// Device copies of the references; each side's ROI kernel, shared-memory size and grid.
static int rois_upload(ccst_ctx* c) {
    if (!c->rois_dirty) return CCST_OK;
    if (c->refs_cap < c->refs.size()) {
        if (c->d_refs) cudaFree(c->d_refs);
        c->d_refs = nullptr;
        c->refs_cap = 0;
        CK(c, cudaMalloc(&c->d_refs, 2 * c->refs.size() * sizeof(RefSpectra)));
        c->refs_cap = 2 * c->refs.size();
    }
    std::vector<RefSpectra> rs;
    for (auto& re : c->refs) rs.push_back(re.r);
    CK(c, cudaMemcpy(c->d_refs, rs.data(), rs.size() * sizeof(RefSpectra), cudaMemcpyHostToDevice));
    int limit = 0, occ = 0, sms = 0;
    CK(c, cudaDeviceGetAttribute(&limit, cudaDevAttrMaxSharedMemoryPerBlockOptin, c->device));
    CK(c, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device));
    for (auto& pl : c->plans) {
        if (!rois_size_ok(pl.g.H, pl.g.W)) continue;
        RoiKernel& rk = c->rois_k[roi_side_slot(pl.g.H)];
        rk.fn = track_rois_kernel_ptr(pl.g.H, pl.g.tc != 0);
        rk.g = pl.g;
        rk.smem = smem_plan(pl.g).total;
        const int threads = track_threads(pl.g.H, pl.g.W);
        CK(c, cudaFuncSetAttribute(rk.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, limit - kRoisStaticSmem));
        CK(c, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, rk.fn, threads, rk.smem));
        if (occ < 1) return fail(c, CCST_E_SHAPE, "ccst_track_rois: the ROI kernel does not fit on an SM");
        rk.grid = occ * sms;
    }
    c->rois_dirty = false;
    return CCST_OK;
}

// ------------------------------------------------------------------- general sizes
// A shape outside the power-of-two kernel (48, 96, 192, 256, 256 x 128, ...) gets a plan
// of the double-float path: e^{-2 pi i m / H}, e^{-2 pi i m / W}, e^{+2 pi i m / (uH)} and
// e^{+2 pi i m / (uW)} in one table block.
static int gen_plan(ccst_ctx* c, int H, int W, int* gcls) {
    for (size_t i = 0; i < c->gplans.size(); ++i)
        if (c->gplans[i].p.H == H && c->gplans[i].p.W == W) {
            *gcls = (int)i;
            return CCST_OK;
        }
    int u = c->p.upsample;
    const long long DH = (long long)u * H, DW = (long long)u * W;
    if (DH > (1LL << 22) || DW > (1LL << 22))
        return fail(c, CCST_E_SHAPE, "general size: u x N above 2^22");
    ccst_ctx::GenPlanH gp;
    GenPlan& pl = gp.p;
    pl.H = H;
    pl.W = W;
    pl.u = u;
    pl.M = (3 * u + 1) / 2;
    pl.h0 = pl.M / 2;
    pl.method = c->p.method;
    pl.in_dtype = c->p.in_dtype;
    pl.eps = c->p.eps;
    pl.sense = c->p.method == CCST_CC_SN ? -1.f : 1.f;
    pl.exhaustive = (c->p.flags & CCST_FLAG_EXHAUSTIVE) ? 1 : 0;
    pl.H1 = gen_split(H);
    pl.H2 = H / pl.H1;
    pl.W1 = gen_split(W);
    pl.W2 = W / pl.W1;
    dfc* tab = nullptr;
    const size_t ntab = (size_t)(H + W + DH + DW);
    int M = pl.M, h0 = pl.h0;
    const size_t ngrid = (size_t)(H + W / 2 + 1) * M;
    CK(c, cudaMalloc(&tab, ntab * sizeof(dfc) + ngrid * sizeof(float2)));
    gp.mem.push_back(tab);
    pl.wH = tab;
    pl.wW = tab + H;
    pl.uH = tab + H + W;
    pl.uW = tab + H + W + DH;
    float2* EY = (float2*)(tab + ntab);
    float2* EX = EY + (size_t)H * M;
    pl.EY = EY;
    pl.EX = EX;
    void* a2[] = {&H, &W, &u, &tab};
    void* a3[] = {&H, &W, &u, &M, &h0, &EY, &EX};
    cudaError_t e = cudaLaunchKernel(gen_init_tables_ptr(), dim3(64), dim3(256), a2, 0, c->stream);
    if (e == cudaSuccess) e = cudaLaunchKernel(gen_init_grid_tables_ptr(), dim3(128), dim3(256), a3, 0, c->stream);
    if (e != cudaSuccess) {
        cudaFree(tab);
        return fail(c, CCST_E_CUDA, std::string("gen_init_tables: ") + cudaGetErrorString(e));
    }
    if (!pl.exhaustive && mix_shape_ok(H, W)) {
        // the FP32 kernel for this side, with this kernel as its fallback
        int optin = 0;
        CK(c, cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, c->device));
        void* mm = nullptr;
        const bool sn = c->p.method == CCST_CC_SN;
        const int mrc = mix_plan_create(H, W, u, c->p.method, c->p.in_dtype, c->p.eps, kMixTauInt,
                                        sn ? mix_tau0_sn(H) : kMixTau0, sn ? kMixTau1Sn : kMixTau1, optin, &gp.mp, &mm);
        if (mrc > 0) {
            for (void* q : gp.mem) cudaFree(q);
            return fail(c, CCST_E_CUDA, std::string("FP32 general-size plan: ") + cudaGetErrorString((cudaError_t)mrc));
        }
        if (mrc == 0) {
            gp.mem.push_back(mm);
            gp.mp.uHd = pl.uH;                         // the double-float level's phase tables
            gp.mp.uWd = pl.uW;
            const void* k = mix_kernel_ptr(H, W);
            const int cl = gp.mp.CL;
            cudaError_t ea = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, gp.mp.smem);
            int sms = 0, resident = 0;
            if (ea == cudaSuccess) ea = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device);
            if (ea == cudaSuccess && cl == 1) {
                int occ = 0;
                ea = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k, gp.mp.NT, gp.mp.smem);
                resident = occ * sms;
            } else if (ea == cudaSuccess) {
                cudaLaunchConfig_t cfg = {};
                cfg.gridDim = dim3((unsigned)(cl * sms));
                cfg.blockDim = dim3((unsigned)gp.mp.NT);
                cfg.dynamicSmemBytes = (size_t)gp.mp.smem;
                int ncl = 0;
                ea = cudaOccupancyMaxActiveClusters(&ncl, k, &cfg);
                resident = ncl * cl;
            }
            if (ea != cudaSuccess) {
                for (void* q : gp.mem) cudaFree(q);
                return fail(c, CCST_E_CUDA, std::string("FP32 general-size kernel: ") + cudaGetErrorString(ea));
            }
            if (resident >= cl) {
                gp.mix = true;
                gp.mix_grid = resident;
            }
        }
    }
    c->gplans.push_back(gp);
    *gcls = (int)c->gplans.size() - 1;
    c->rois_dirty = true;
    c->gen_dirty = true;
    return CCST_OK;
}

// The half spectrum F[b] of a reference into Fb (H x (W/2 + 1) double-floats), from an FP32
// image (host or device, `frame_kind` 0) or from a frame on the device in the context's
// input type with row pitch `pitch` (`frame_kind` 1). Synchronous on the context's stream.
static int gen_ref_spectrum(ccst_ctx* c, int H, int W, const void* src, int frame_kind, long long pitch, dfc* Fb) {
    const size_t HW = (size_t)H * W, HWh = (size_t)H * (W / 2 + 1);
    const size_t ntmp = HWh * sizeof(double2) + HW * sizeof(float);
    if (c->addref_tmp_bytes < ntmp) {
        if (c->d_addref_tmp) cudaFree(c->d_addref_tmp);
        c->d_addref_tmp = nullptr;
        c->addref_tmp_bytes = 0;
        CK(c, cudaMalloc(&c->d_addref_tmp, ntmp));
        c->addref_tmp_bytes = ntmp;
    }
    double2* R = (double2*)c->d_addref_tmp;
    float* ref32 = (float*)((char*)c->d_addref_tmp + HWh * sizeof(double2));
    int method = c->p.method, in_dtype = c->p.in_dtype;
    float eps = c->p.eps;
    cudaError_t e;
    if (frame_kind == 0) {
        e = cudaMemcpyAsync(ref32, src, HW * sizeof(float), cudaMemcpyDefault, c->stream);
    } else {
        void* af[] = {&H, &W, &in_dtype, (void*)&src, &pitch, &ref32};
        e = cudaLaunchKernel(gen_frame_to_f32_ptr(), dim3(64), dim3(256), af, 0, c->stream);
    }
    if (e == cudaSuccess) {
        void* ar[] = {&H, &W, &method, &eps, &ref32, &R};
        e = cudaLaunchKernel(gen_ref_rows_ptr(), dim3(64), dim3(256), ar, 0, c->stream);
    }
    if (e == cudaSuccess) {
        void* ac[] = {&H, &W, &R, &Fb};
        e = cudaLaunchKernel(gen_ref_cols_ptr(), dim3(64), dim3(256), ac, 0, c->stream);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return fail(c, CCST_E_CUDA, std::string("general-size reference: ") + cudaGetErrorString(e));
    return CCST_OK;
}

static int add_generic_reference(ccst_ctx* c, const float* ref, int H, int W, int* ref_id) {
    int gcls = 0, rc;
    if ((rc = gen_plan(c, H, W, &gcls))) return rc;
    ccst_ctx::RefEntry re;
    re.gcls = gcls;
    dfc* Fb = nullptr;
    CK(c, cudaMalloc(&Fb, (size_t)H * (W / 2 + 1) * sizeof(dfc)));
    if ((rc = gen_ref_spectrum(c, H, W, ref, 0, W, Fb))) {
        cudaFree(Fb);
        return rc;
    }
    re.mem.push_back(Fb);
    re.gFb = Fb;
    c->refs.push_back(re);
    c->rois_dirty = true;
    c->gen_dirty = true;
    *ref_id = (int)c->refs.size() - 1;
    return CCST_OK;
}

// The kernel's grid (CTAs per SM x SMs) and the device copies of the plans and references.
static int gen_prepare(ccst_ctx* c) {
    if (!c->gen_grid) {
        int sms = 0, occ = 0;
        CK(c, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device));
        CK(c, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, track_generic_kernel_ptr(), c->gen_threads, 0));
        if (occ < 1) return fail(c, CCST_E_SHAPE, "the general-size kernel does not fit on an SM");
        c->gen_grid = sms * occ;
    }
    if (!c->gen_dirty) return CCST_OK;
    if (c->gplans_cap < c->gplans.size()) {
        if (c->d_gplans) cudaFree(c->d_gplans);
        c->d_gplans = nullptr;
        c->gplans_cap = 0;
        CK(c, cudaMalloc(&c->d_gplans, 2 * c->gplans.size() * sizeof(GenPlan)));
        c->gplans_cap = 2 * c->gplans.size();
    }
    if (c->grefs_cap < c->refs.size()) {
        if (c->d_grefs) cudaFree(c->d_grefs);
        c->d_grefs = nullptr;
        c->grefs_cap = 0;
        CK(c, cudaMalloc(&c->d_grefs, 2 * c->refs.size() * sizeof(dfc*)));
        c->grefs_cap = 2 * c->refs.size();
    }
    std::vector<GenPlan> gp;
    for (auto& g : c->gplans) gp.push_back(g.p);
    std::vector<const dfc*> gr;
    for (auto& re : c->refs) gr.push_back(re.gFb);
    CK(c, cudaMemcpy(c->d_gplans, gp.data(), gp.size() * sizeof(GenPlan), cudaMemcpyHostToDevice));
    CK(c, cudaMemcpy(c->d_grefs, gr.data(), gr.size() * sizeof(dfc*), cudaMemcpyHostToDevice));
    c->gen_dirty = false;
    return CCST_OK;
}

// The FP32 kernel's device state of a lane for batches of up to n items: its counters and
// a fallback list of n items. *grew: a buffer was (re)allocated (graphs that captured the
// old ones must go).
static int mix_reserve(ccst_ctx* c, GenLane& lane, long long n, bool* grew) {
    *grew = false;
    if (!lane.d_mixc) {
        CK(c, cudaMalloc(&lane.d_mixc, kMixCounters * sizeof(unsigned)));
        *grew = true;
    }
    if (lane.fb_cap < (size_t)n) {
        if (lane.d_fb) cudaFree(lane.d_fb);
        lane.d_fb = nullptr;
        lane.fb_cap = 0;
        CK(c, cudaMalloc(&lane.d_fb, (size_t)n * sizeof(GenItem)));
        lane.fb_cap = (size_t)n;
        *grew = true;
    }
    return CCST_OK;
}

// Plan p runs on the FP32 general-size kernel (not while ccst_autotune times the
// double-float kernel).
static bool plan_mix(ccst_ctx* c, int p) { return c->gplans[p].mix && !c->mix_off; }

static bool any_mix_plan(ccst_ctx* c) {
    for (int p = 0; p < (int)c->gplans.size(); ++p)
        if (plan_mix(c, p)) return true;
    return false;
}

// A kernel launch on `stream`; with `chained`, by programmatic dependent launch behind the
// kernel launched just before it on that stream: it may start once every CTA of that kernel
// has taken its last item (pdl_trigger), and it calls pdl_wait before it exits.
static cudaError_t launch_kernel(const void* k, int grid, int block, void** args, size_t smem, cudaStream_t stream,
                                 bool chained) {
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3((unsigned)block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = stream;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = chained ? at : nullptr;
    cfg.numAttrs = chained ? 1 : 0;
    return cudaLaunchKernelExC(&cfg, k, args);
}

// The general-size part of a batch (gb.items already on the device, ordered by gen_sort,
// with `items_host` its host copy; or null for a uniform batch): items whose plan has the
// FP32 kernel come last, equal plans together, and each such run is one FP32 launch (a
// segment); the frames it cannot certify join a fallback list. The double-float kernel then
// takes the other items (the first `ndirect`) and the fallback list.
struct MixSeg { long long first, n; int plan; };
struct GenSplit {
    MixSeg segs[kMixCounters - 2];
    int ns = 0;
    long long ndirect = 0;
};

static int gen_split_items(ccst_ctx* c, const GenBatch& gb, const GenItem* items_host, const GenLane& lane,
                           GenSplit* sp) {
    sp->ns = 0;
    sp->ndirect = gb.n;
    if (!gb.items) {
        if (plan_mix(c, gb.plan)) {
            sp->segs[sp->ns++] = MixSeg{0, gb.n, gb.plan};
            sp->ndirect = 0;
        }
    } else if (items_host) {
        long long i = 0;
        while (i < gb.n && !plan_mix(c, items_host[i].plan)) ++i;
        sp->ndirect = i;
        while (i < gb.n && sp->ns < kMixCounters - 2) {
            long long j = i;
            while (j < gb.n && items_host[j].plan == items_host[i].plan) ++j;
            sp->segs[sp->ns++] = MixSeg{i, j - i, items_host[i].plan};
            i = j;
        }
        if (i < gb.n) return fail(c, CCST_E_INVALID, "general-size batch: too many FP32 plans in one batch");
    }
    if (sp->ns > 0 && (!lane.d_mixc || lane.fb_cap < (size_t)(gb.n - sp->ndirect)))
        return fail(c, CCST_E_INVALID, "general-size batch: FP32 lane state not reserved");
    return CCST_OK;
}

// Zero the general-size part's counters: the FP32 launches' (with the fallback count) and
// the double-float kernel's.
static int gen_zero(ccst_ctx* c, const GenSplit& sp, const GenLane& lane, unsigned* counter, cudaStream_t stream) {
    if (sp.ns > 0) CK(c, cudaMemsetAsync(lane.d_mixc, 0, (size_t)(1 + sp.ns) * sizeof(unsigned), stream));
    CK(c, cudaMemsetAsync(counter, 0, sizeof(unsigned), stream));
    return CCST_OK;
}

// The FP32 launches, one per segment, each chained behind the kernel before it (*chained:
// a chained kernel was the last launch on `stream`). dbg: diagnostic outputs (uniform
// batches).
static int gen_mix_launch(ccst_ctx* c, const GenBatch& gb, const GenSplit& sp, const GenLane& lane,
                          cudaStream_t stream, bool* chained, const MixDbg* dbg = nullptr) {
    for (int k = 0; k < sp.ns; ++k) {
        const ccst_ctx::GenPlanH& gp = c->gplans[sp.segs[k].plan];
        MixArgs ma{};
        ma.items = gb.items;
        ma.first = sp.segs[k].first;
        ma.n = sp.segs[k].n;
        ma.frames = gb.frames;
        ma.frame_bytes = gb.frame_bytes;
        ma.pitch = gb.pitch;
        ma.plan = gb.plan;
        ma.ref = gb.ref;
        ma.p = gp.mp;
        ma.refs = c->d_grefs;
        ma.out = gb.out;
        ma.next = lane.d_mixc + 1 + k;
        ma.fb = lane.d_fb;
        ma.fb_count = lane.d_mixc;
        if (dbg) {
            ma.dbg_int = dbg->dbg_int;
            ma.dbg_sub = dbg->dbg_sub;
            ma.dbg_pairs = dbg->pairs;
            ma.dbg_d32 = dbg->d32;
        }
        const int cl = gp.mp.CL;
        const long long want = sp.segs[k].n * cl;
        const int grid = (int)(want < gp.mix_grid ? want : gp.mix_grid) / cl * cl;
        void* margs[] = {&ma};
        CK(c, launch_kernel(mix_kernel_ptr(gp.mp.H, gp.mp.W), grid, gp.mp.NT, margs, (size_t)gp.mp.smem, stream,
                            *chained));
        *chained = true;
    }
    return CCST_OK;
}

// The double-float kernel over the first sp.ndirect items and the fallback list, with
// per-CTA scratch of `stride` elements: a plain launch, so it starts once everything before
// it on `stream` has completed (the fallback list is whole).
static int gen_direct_launch(ccst_ctx* c, GenBatch gb, const GenSplit& sp, const GenLane& lane, long long stride,
                             unsigned* counter, cudaStream_t stream) {
    const long long ntot = gb.n;
    gb.fb_items = sp.ns > 0 ? lane.d_fb : nullptr;
    gb.fb_count = sp.ns > 0 ? lane.d_mixc : nullptr;
    const int grid = (int)(ntot < c->gen_grid ? ntot : c->gen_grid);
    gb.n = sp.ndirect;
    gb.plans = c->d_gplans;
    gb.refs = c->d_grefs;
    gb.next = counter;
    gb.scratch = lane.scratch;
    gb.scratch_stride = stride;
    void* args[] = {&gb};
    CK(c, cudaLaunchKernel(track_generic_kernel_ptr(), dim3(grid), dim3(c->gen_threads), args, 0, stream));
    return CCST_OK;
}

// The whole general-size part on `stream`: counters, the FP32 launches chained one behind
// the other, then the double-float kernel.
static int gen_kernel_launch(ccst_ctx* c, const GenBatch& gb, GenLane& lane, long long stride, cudaStream_t stream,
                             unsigned* counter, const GenItem* items_host, const MixDbg* dbg = nullptr) {
    GenSplit sp;
    int rc = gen_split_items(c, gb, items_host, lane, &sp);
    if (!rc) rc = gen_zero(c, sp, lane, counter, stream);
    bool chained = false;
    if (!rc) rc = gen_mix_launch(c, gb, sp, lane, stream, &chained, dbg);
    if (!rc) rc = gen_direct_launch(c, gb, sp, lane, stride, counter, stream);
    return rc;
}

// Per-CTA scratch stride of the general-size kernel over every plan of the context.
static long long gen_stride(ccst_ctx* c) {
    long long stride = 0;
    for (auto& g : c->gplans) stride = std::max(stride, gen_scratch_stride(g.p.H, g.p.W, g.p.M));
    return stride;
}

// A lane's device buffers for general-size batches of up to n frames: the double-float
// kernel's scratch, the work-list copy and the FP32 kernel's counters and fallback list.
// Grows them (a reallocation synchronises the device) and never shrinks them.
static int lane_reserve(ccst_ctx* c, GenLane& lane, long long n) {
    if (n <= 0) return CCST_OK;
    int rc = gen_prepare(c);
    if (rc) return rc;
    const long long stride = gen_stride(c);
    const int grid = (int)(n < c->gen_grid ? n : c->gen_grid);
    if (lane.scratch_elems < (size_t)grid * stride) {
        if (lane.scratch) cudaFree(lane.scratch);
        lane.scratch = nullptr;
        lane.scratch_elems = 0;
        CK(c, cudaMalloc(&lane.scratch, (size_t)grid * stride * sizeof(dfc)));
        lane.scratch_elems = (size_t)grid * stride;
    }
    if (lane.items_cap < (size_t)n) {
        if (lane.d_items) cudaFree(lane.d_items);
        lane.d_items = nullptr;
        lane.items_cap = 0;
        CK(c, cudaMalloc(&lane.d_items, (size_t)n * sizeof(GenItem)));
        lane.items_cap = (size_t)n;
    }
    if (any_mix_plan(c)) {
        bool grew = false;
        if ((rc = mix_reserve(c, lane, n, &grew))) return rc;
    }
    return CCST_OK;
}

// Device state of a general-size batch of gb->n frames on `lane` (lane_reserve), and the
// work list `items_host` copied to the lane on `stream` (the caller orders it; gb->items is
// set to the copy, or null for a uniform batch). *stride: the scratch stride of each CTA.
static int gen_stage(ccst_ctx* c, GenLane& lane, GenBatch* gb, const GenItem* items_host, cudaStream_t stream,
                     long long* stride) {
    int rc = lane_reserve(c, lane, gb->n);
    if (rc) return rc;
    *stride = gen_stride(c);
    gb->items = nullptr;
    if (items_host) {
        CK(c, cudaMemcpyAsync(lane.d_items, items_host, (size_t)gb->n * sizeof(GenItem), cudaMemcpyHostToDevice,
                              stream));
        gb->items = lane.d_items;
    }
    return CCST_OK;
}

// Launch the general-size kernels on `stream` over gb.n frames: the work list `items_host`
// (copied to the lane at once; the caller orders it) or, if null, the uniform batch that
// gb describes. gb.out is set by the caller; the rest is filled in here.
static int gen_launch(ccst_ctx* c, GenLane& lane, GenBatch gb, const GenItem* items_host, cudaStream_t stream,
                      unsigned* counter, const MixDbg* dbg = nullptr) {
    if (gb.n == 0) return CCST_OK;
    long long stride = 0;
    int rc = gen_stage(c, lane, &gb, items_host, stream, &stride);
    if (rc) return rc;
    return gen_kernel_launch(c, gb, lane, stride, stream, counter, items_host, dbg);
}

// Items of plans without the FP32 kernel first, then those with it; within each part the
// largest frames first (the longest work starts first; equal plans stay together).
static void gen_sort(ccst_ctx* c, GenItem* items, int64_t n) {
    std::stable_sort(items, items + n, [&](const GenItem& a, const GenItem& b) {
        const auto &ga = c->gplans[a.plan], &gb = c->gplans[b.plan];
        const bool ma = plan_mix(c, a.plan), mb = plan_mix(c, b.plan);
        if (ma != mb) return !ma;
        if (ga.p.H * ga.p.W != gb.p.H * gb.p.W) return ga.p.H * ga.p.W > gb.p.H * gb.p.W;
        return a.plan < b.plan;
    });
}

// A batch of a general-shape context: frame i at frames + i * H * pitch elements.
static int gen_track(ccst_ctx* c, const Batch& b, cudaStream_t stream, GenLane& lane, unsigned* counter,
                     const MixDbg* dbg) {
    const size_t elem = c->p.in_dtype == CCST_U16 ? 2 : 4;
    GenBatch gb{};
    gb.n = b.n;
    gb.out = b.out;
    gb.frames = b.frames;
    gb.frame_bytes = (long long)c->g.H * b.pitch * (long long)elem;
    gb.pitch = b.pitch;
    gb.plan = c->refs[0].gcls;
    gb.ref = 0;
    return gen_launch(c, lane, gb, nullptr, stream, counter, dbg);
}

// Two-level splits worth timing for an N-point DFT: the default (largest divisor not above
// sqrt(N)), its cofactor, and the next divisor below the default.
static std::vector<int> split_candidates(int N) {
    const int d0 = gen_split(N);
    std::vector<int> out = {d0};
    if (N / d0 != d0) out.push_back(N / d0);
    for (int d = d0 - 1; d > 1; --d)
        if (N % d == 0) {
            out.push_back(d);
            break;
        }
    return out;
}

extern "C" int ccst_track_rois(ccst_ctx* c, const ccst_roi* rois, int64_t n, ccst_result* out_dev);

extern "C" int ccst_autotune(ccst_ctx* c, int reps, const ccst_roi* rois, int64_t n_rois, ccst_tune_result* out,
                             int max_out, int* n_out) {
    int rc = check_ctx(c);
    if (rc) return rc;
    if (reps < 1 || max_out < 0 || (max_out > 0 && !out) || n_rois < 0 || (n_rois > 0 && !rois))
        return fail(c, CCST_E_INVALID, "ccst_autotune: bad arguments");
    if (n_out) *n_out = 0;
    const int np = (int)c->gplans.size();
    if (np == 0) return CCST_OK;
    drop_roi_graphs(c);           // schedules change below: captured launches would go stale
    c->mix_off = true;            // time the double-float kernel itself, on every plan
    std::vector<int> ref_of(np, -1);
    for (int i = 0; i < (int)c->refs.size(); ++i)
        if (c->refs[i].gcls >= 0 && ref_of[c->refs[i].gcls] < 0) ref_of[c->refs[i].gcls] = i;
    CK(c, cudaStreamSynchronize(c->stream));
    const size_t elem = c->p.in_dtype == CCST_U16 ? 2 : 4;
    std::vector<void*> frames(np, nullptr);
    Result* recs = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    GenLane lane;
    unsigned* counter = c->d_next + 32;
    std::vector<std::pair<int, int>> saved(np);
    for (int p = 0; p < np; ++p) saved[p] = {c->gplans[p].p.H1, c->gplans[p].p.W1};
    const int saved_threads = c->gen_threads;
    auto set_split = [&](int p, int h1, int w1) {
        GenPlan& pl = c->gplans[p].p;
        pl.H1 = h1; pl.H2 = pl.H / h1; pl.W1 = w1; pl.W2 = pl.W / w1;
        c->gen_dirty = true;
    };
    auto cleanup = [&]() {
        for (void* f : frames)
            if (f) cudaFree(f);
        if (recs) cudaFree(recs);
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        lane_free(lane);
    };
    auto bail = [&](int code) {
        cleanup();
        c->mix_off = false;
        for (int p = 0; p < np; ++p) set_split(p, saved[p].first, saved[p].second);
        c->gen_threads = saved_threads;
        c->gen_grid = 0;
        c->gen_dirty = true;
        return code;
    };
    // the best of `reps` timed launches (after one untimed), in ms
    auto time_launch = [&](GenBatch gb, const GenItem* items, double* ms_out) -> int {
        double best = 1e300;
        for (int r = -1; r < reps; ++r) {
            if (cudaEventRecord(e0, c->stream) != cudaSuccess) return fail(c, CCST_E_CUDA, "ccst_autotune: event");
            const int lrc = gen_launch(c, lane, gb, items, c->stream, counter);
            if (lrc) return lrc;
            if (cudaEventRecord(e1, c->stream) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess)
                return fail(c, CCST_E_CUDA, "ccst_autotune: launch");
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (r >= 0) best = std::min(best, (double)ms);
        }
        *ms_out = best;
        return CCST_OK;
    };
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
        return bail(fail(c, CCST_E_CUDA, "ccst_autotune: event"));
    // synthetic frames: two waves of the 512-thread grid per plan
    c->gen_threads = 512;
    c->gen_grid = 0;
    if ((rc = gen_prepare(c))) return bail(rc);
    const long long nf = 2LL * c->gen_grid;
    if (cudaMalloc(&recs, std::max((size_t)nf * np, (size_t)n_rois) * sizeof(Result)) != cudaSuccess)
        return bail(fail(c, CCST_E_NOMEM, "ccst_autotune: records"));
    for (int p = 0; p < np; ++p) {
        if (ref_of[p] < 0) continue;
        int H = c->gplans[p].p.H, W = c->gplans[p].p.W, dt = c->p.in_dtype;
        long long n = nf;
        if (cudaMalloc(&frames[p], (size_t)nf * H * W * elem) != cudaSuccess)
            return bail(fail(c, CCST_E_NOMEM, "ccst_autotune: frames"));
        void* af[] = {&H, &W, &dt, &n, &frames[p]};
        if (cudaLaunchKernel(gen_fill_synthetic_ptr(), dim3(256), dim3(256), af, 0, c->stream) != cudaSuccess)
            return bail(fail(c, CCST_E_CUDA, "ccst_autotune: synthetic frames"));
    }
    // 1. per plan, with 512-thread CTAs: the two-level splits, on a uniform batch of the plan
    int timed = 0;
    std::vector<double> us(np, 0.0);
    for (int p = 0; p < np; ++p) {
        if (ref_of[p] < 0) continue;
        const int H = c->gplans[p].p.H, W = c->gplans[p].p.W;
        GenBatch gb{};
        gb.n = nf;
        gb.out = recs;
        gb.frames = frames[p];
        gb.frame_bytes = (long long)H * W * (long long)elem;
        gb.pitch = W;
        gb.plan = p;
        gb.ref = ref_of[p];
        double best = 1e300;
        int bh = saved[p].first, bw = saved[p].second;
        for (int h1 : split_candidates(H))
            for (int w1 : split_candidates(W)) {
                set_split(p, h1, w1);
                double ms = 0.0;
                if ((rc = time_launch(gb, nullptr, &ms))) return bail(rc);
                ++timed;
                if (ms < best) { best = ms; bh = h1; bw = w1; }
            }
        set_split(p, bh, bw);
        us[p] = 1e3 * best / (double)nf;
    }
    // 2. the CTA size (one per launch): on the caller's ROI batch through ccst_track_rois, or
    // else on a work list of every plan's frames, largest first (as a mixed ROI batch runs)
    const int threads[2] = {512, 256};
    double tms[2] = {0.0, 0.0};
    if (n_rois > 0) {
        for (int ti = 0; ti < 2; ++ti) {
            c->gen_threads = threads[ti];
            c->gen_grid = 0;
            c->gen_dirty = true;      // a graph-captured ROI batch must be captured again
            double best = 1e300;
            for (int r = -1; r < reps; ++r) {
                if (cudaEventRecord(e0, c->stream) != cudaSuccess) return bail(fail(c, CCST_E_CUDA, "ccst_autotune: event"));
                if ((rc = ccst_track_rois(c, rois, n_rois, (ccst_result*)recs))) return bail(rc);
                if (cudaEventRecord(e1, c->stream) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess)
                    return bail(fail(c, CCST_E_CUDA, "ccst_autotune: ROI batch"));
                float ms = 0.f;
                cudaEventElapsedTime(&ms, e0, e1);
                if (r >= 0) best = std::min(best, (double)ms);
            }
            tms[ti] = best;
            ++timed;
        }
    }
    std::vector<GenItem> items;
    for (int p = 0; p < np; ++p) {
        if (ref_of[p] < 0) continue;
        const GenPlan& pl = c->gplans[p].p;
        for (long long i = 0; i < nf; ++i)
            items.push_back(GenItem{(const char*)frames[p] + (size_t)i * pl.H * pl.W * elem, (long long)pl.W,
                                    (long long)items.size(), p, ref_of[p]});
    }
    gen_sort(c, items.data(), (int64_t)items.size());
    for (int ti = 0; ti < 2 && n_rois == 0; ++ti) {
        c->gen_threads = threads[ti];
        c->gen_grid = 0;
        GenBatch gb{};
        gb.n = (long long)items.size();
        gb.out = recs;
        if ((rc = time_launch(gb, items.data(), &tms[ti]))) return bail(rc);
        ++timed;
    }
    cleanup();
    c->mix_off = false;
    c->gen_threads = tms[1] < tms[0] ? 256 : 512;
    c->gen_grid = 0;
    c->gen_dirty = true;
    if ((rc = gen_prepare(c))) return rc;
    int n = 0;
    for (int p = 0; p < np && n < max_out; ++p) {
        const GenPlan& pl = c->gplans[p].p;
        out[n++] = ccst_tune_result{pl.H, pl.W, pl.H1, pl.W1, c->gen_threads, timed, us[p]};
    }
    if (n_out) *n_out = n;
    return CCST_OK;
}

static int not_general(ccst_ctx* c, const char* who) {
    if (c && c->general)
        return fail(c, CCST_E_UNSUPPORTED, std::string(who) + ": not available on a general-shape context");
    return CCST_OK;
}

// Sort items largest first (the longest work starts first; size classes stay contiguous).
static void rois_sort(ccst_ctx* c, RoiItem* items, int64_t n) {
    std::stable_sort(items, items + n, [&](const RoiItem& a, const RoiItem& b) {
        return c->plans[a.cls].g.H > c->plans[b.cls].g.H;
    });
}

// The power-of-two ROI kernels over n items already on the device (items: their host copy),
// ordered by rois_sort: one launch per side over that side's run of items, largest side
// first, each chained behind the kernel launched before it (*chained) and with its own
// counter (counter[0 .. kRoiCounters), zeroed by the caller).
static int rois_kernel_launch(ccst_ctx* c, const RoiItem* items_dev, const RoiItem* items, int64_t n, Result* out,
                              cudaStream_t stream, unsigned* counter, bool* chained) {
    int k = 0;
    for (int64_t s = 0; s < n; ++k) {
        const int side = c->plans[items[s].cls].g.H;
        int64_t e = s + 1;
        while (e < n && c->plans[items[e].cls].g.H == side) ++e;
        RoiKernel& rk = c->rois_k[roi_side_slot(side)];
        if (!rk.fn || k >= kRoiCounters)
            return fail(c, CCST_E_SHAPE, "ccst_track_rois: no ROI kernel for a side of the work list");
        RoiBatch rb;
        rb.items = items_dev + s;
        rb.n = e - s;
        rb.refs = c->d_refs;
        rb.out = out;
        rb.next = counter + k;
        const int grid = (int)(rb.n < rk.grid ? rb.n : rk.grid);
        void* args[] = {&rb, &rk.g};
        CK(c, launch_kernel(rk.fn, grid, track_threads(side, side), args, rk.smem, stream, *chained));
        *chained = true;
        s = e;
    }
    return CCST_OK;
}

// One uneven-ROI batch on `stream`, its work lists already on the device and sorted:
//   - every counter zeroed;
//   - on side.st, forked from `stream`: the FP32 general-size launches (largest side
//     first), then the double-float kernel over the general items without an FP32 plan
//     and the fallback list, a plain launch that starts once the FP32 launches have
//     completed;
//   - on `stream`: the ROI kernel of each side present, 128 down to 16;
//   - joined.
// (Without power-of-two items, or without general ones, everything runs on `stream`.)
// On each stream a kernel is chained behind the one before it (programmatic dependent
// launch): it may start once every CTA of that one has taken its last item, so a tail
// overlaps the next kernel's start and a batch too small to fill the GPU runs side by side.
// The general-size launches are issued first: their items are the longest (about 100 us per
// CTA, against 45 us for the power-of-two kernels), and starting them first, with the 128 x
// 128 kernel taking SMs as they drain, packed the survey's uneven mix about 8% tighter in a
// captured graph than the other way round or one chain of all four kernels.
struct RoiPart {
    const RoiItem* items_dev;   // n items, largest first
    const RoiItem* items;       // their host copy
    int64_t n;
    unsigned* counter;          // kRoiCounters counters
};
struct GenPart {
    GenBatch gb;                // gb.items on the device (gen_sort order), gb.n items, gb.out
    const GenItem* items;       // their host copy
    GenLane* lane;
    long long stride;           // double-float scratch per CTA
    unsigned* counter;
};
static int rois_chain_launch(ccst_ctx* c, const RoiPart& rp, const GenPart& gp, Result* out, cudaStream_t stream,
                             SideStream& side) {
    GenSplit sp;
    int rc;
    if (gp.gb.n > 0) {
        if ((rc = gen_split_items(c, gp.gb, gp.items, *gp.lane, &sp))) return rc;
        if ((rc = gen_zero(c, sp, *gp.lane, gp.counter, stream))) return rc;
    }
    if (rp.n > 0) CK(c, cudaMemsetAsync(rp.counter, 0, kRoiCounters * sizeof(unsigned), stream));
    const bool fork = gp.gb.n > 0 && rp.n > 0;
    cudaStream_t gs = stream;
    if (fork) {
        CK(c, side_make(side));
        CK(c, cudaEventRecord(side.fork, stream));
        CK(c, cudaStreamWaitEvent(side.st, side.fork, 0));
        gs = side.st;
    }
    bool chained = false;
    if (sp.ns > 0 && (rc = gen_mix_launch(c, gp.gb, sp, *gp.lane, gs, &chained))) return rc;
    if (fork) chained = false;
    if (rp.n > 0 && (rc = rois_kernel_launch(c, rp.items_dev, rp.items, rp.n, out, stream, rp.counter, &chained)))
        return rc;
    if (gp.gb.n > 0 && (rc = gen_direct_launch(c, gp.gb, sp, *gp.lane, gp.stride, gp.counter, gs))) return rc;
    if (fork) {
        CK(c, cudaEventRecord(side.join, side.st));
        CK(c, cudaStreamWaitEvent(stream, side.join, 0));
    }
    return CCST_OK;
}

// Sort the power-of-two items, upload the plans and references, copy the items to
// items_dev (n slots) on `stream`. The host items must stay valid until the copy has run
// (pageable memory is staged at once).
static int rois_stage(ccst_ctx* c, RoiItem* items, int64_t n, cudaStream_t stream, RoiItem* items_dev) {
    rois_sort(c, items, n);
    int rc = rois_upload(c);
    if (rc) return rc;
    CK(c, cudaMemcpyAsync(items_dev, items, (size_t)n * sizeof(RoiItem), cudaMemcpyHostToDevice, stream));
    return CCST_OK;
}

constexpr size_t kMaxRoiGraphs = 64;

static uint64_t fnv1a(const void* p, size_t bytes) {
    const unsigned char* b = (const unsigned char*)p;
    uint64_t h = 1469598103934665603ull;
    for (size_t i = 0; i < bytes; ++i) h = (h ^ b[i]) * 1099511628211ull;
    return h;
}

// ccst_track_rois as a replay of a graph captured once per (stream, out, work list): the
// batch's chain of launches (rois_chain_launch). The work items (sorted as the direct path
// sorts them) are uploaded at capture.
// c->h_items[0, np) and c->h_gitems[0, ng) hold the validated items.
static int rois_graph_track(ccst_ctx* c, const ccst_roi* rois, int64_t n, ccst_result* out_dev, int64_t np,
                            int64_t ng) {
    // captured pointers and launch shapes would go stale; the general-size state matters
    // only once the context has general-size plans
    if (c->rois_dirty || (c->gen_dirty && !c->gplans.empty())) drop_roi_graphs(c);
    int rc = rois_upload(c);
    if (rc) return rc;
    if (!c->gplans.empty() && (rc = gen_prepare(c))) return rc;
    const auto key = std::make_tuple(c->stream, (void*)out_dev, n, fnv1a(rois, (size_t)n * sizeof(ccst_roi)));
    auto it = c->roi_graphs.find(key);
    if (it != c->roi_graphs.end() &&
        std::memcmp(it->second.rois.data(), rois, (size_t)n * sizeof(ccst_roi)) != 0) {   // hash collision
        free_roi_graph(it->second);
        c->roi_graphs.erase(it);
        it = c->roi_graphs.end();
    }
    if (it == c->roi_graphs.end()) {
        if (c->roi_graphs.size() >= kMaxRoiGraphs) drop_roi_graphs(c);
        GenLane* lane = nullptr;
        const long long stride = ng > 0 ? gen_stride(c) : 0;
        if (ng > 0) {
            lane = &c->roi_lanes[c->stream];
            const size_t need = (size_t)c->gen_grid * (size_t)stride;
            if (lane->scratch_elems < need) {
                drop_roi_graphs(c);                               // graphs on this stream use the lane
                if (lane->scratch) cudaFree(lane->scratch);
                lane->scratch = nullptr;
                lane->scratch_elems = 0;
                CK(c, cudaMalloc(&lane->scratch, need * sizeof(dfc)));
                lane->scratch_elems = need;
            }
            if (any_mix_plan(c) && (!lane->d_mixc || lane->fb_cap < (size_t)ng)) {
                drop_roi_graphs(c);
                bool grew = false;
                if ((rc = mix_reserve(c, *lane, ng, &grew))) return rc;
            }
        }
        ccst_ctx::RoiGraph e;
        e.rois.assign(rois, rois + n);
        auto bail = [&](int code) { free_roi_graph(e); return code; };
        cudaError_t err;
        if ((err = cudaEventCreateWithFlags(&e.done, cudaEventDisableTiming)) != cudaSuccess ||
            (err = cudaMalloc(&e.counters, (kRoiCounters + 1) * sizeof(unsigned))) != cudaSuccess)
            return bail(fail(c, CCST_E_CUDA, std::string("ccst_track_rois: ") + cudaGetErrorString(err)));
        if (np > 0) {
            rois_sort(c, c->h_items.data(), np);
            if ((err = cudaMalloc(&e.d_items, (size_t)np * sizeof(RoiItem))) != cudaSuccess ||
                (err = cudaMemcpy(e.d_items, c->h_items.data(), (size_t)np * sizeof(RoiItem), cudaMemcpyHostToDevice)) !=
                    cudaSuccess)
                return bail(fail(c, err == cudaErrorMemoryAllocation ? CCST_E_NOMEM : CCST_E_CUDA,
                                 std::string("ccst_track_rois: ") + cudaGetErrorString(err)));
        }
        if (ng > 0) {
            gen_sort(c, c->h_gitems.data(), ng);
            if ((err = cudaMalloc(&e.d_gitems, (size_t)ng * sizeof(GenItem))) != cudaSuccess ||
                (err = cudaMemcpy(e.d_gitems, c->h_gitems.data(), (size_t)ng * sizeof(GenItem),
                                  cudaMemcpyHostToDevice)) != cudaSuccess)
                return bail(fail(c, err == cudaErrorMemoryAllocation ? CCST_E_NOMEM : CCST_E_CUDA,
                                 std::string("ccst_track_rois: ") + cudaGetErrorString(err)));
        }
        if ((err = side_make(c->rside)) != cudaSuccess)               // not made during capture
            return bail(fail(c, CCST_E_CUDA, std::string("ccst_track_rois: ") + cudaGetErrorString(err)));
        cudaGraph_t graph = nullptr;
        if ((err = cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal)) != cudaSuccess)
            return bail(fail(c, CCST_E_CUDA, std::string("ccst_track_rois: capture: ") + cudaGetErrorString(err)));
        GenPart gpart{};
        gpart.gb.n = ng;
        gpart.gb.out = (Result*)out_dev;
        gpart.gb.items = e.d_gitems;
        gpart.items = c->h_gitems.data();
        gpart.lane = lane;
        gpart.stride = stride;
        gpart.counter = e.counters + kRoiCounters;
        const int lrc = rois_chain_launch(c, RoiPart{e.d_items, c->h_items.data(), np, e.counters}, gpart,
                                          (Result*)out_dev, c->stream, c->rside);
        err = cudaStreamEndCapture(c->stream, &graph);
        if (lrc) {
            if (graph) cudaGraphDestroy(graph);
            c->dead = true;                                       // a broken capture leaves the stream unusable
            return bail(lrc);
        }
        if (err != cudaSuccess) return bail(fail(c, CCST_E_CUDA, std::string("ccst_track_rois: capture: ") +
                                                                     cudaGetErrorString(err)));
        err = cudaGraphInstantiate(&e.exec, graph, 0);
        cudaGraphDestroy(graph);
        if (err != cudaSuccess)
            return bail(fail(c, CCST_E_CUDA, std::string("ccst_track_rois: instantiate: ") + cudaGetErrorString(err)));
        ++c->roi_graph_instantiations;
        it = c->roi_graphs.emplace(key, std::move(e)).first;
    }
    CK(c, cudaGraphLaunch(it->second.exec, c->stream));
    CK(c, cudaEventRecord(it->second.done, c->stream));
    ++c->roi_graph_replays;
    return CCST_OK;
}

extern "C" int ccst_track_rois(ccst_ctx* c, const ccst_roi* rois, int64_t n, ccst_result* out_dev) {
    int rc = check_ctx(c);
    if (rc) return rc;
    if (n < 0) return fail(c, CCST_E_INVALID, "ccst_track_rois: n < 0");
    if (n == 0) return CCST_OK;
    if (!rois || !out_dev) return fail(c, CCST_E_INVALID, "ccst_track_rois: null rois or out");
    rois_init(c);
    const size_t elem = c->p.in_dtype == CCST_U16 ? 2 : 4;
    c->h_items.resize((size_t)n);
    c->h_gitems.resize((size_t)n);
    int64_t np = 0, ng = 0;
    for (int64_t i = 0; i < n; ++i) {
        const ccst_roi& q = rois[i];
        if (q.ref_id < 0 || q.ref_id >= (int)c->refs.size() || (c->refs[q.ref_id].cls < 0 && c->refs[q.ref_id].gcls < 0))
            return fail(c, CCST_E_INVALID, "ccst_track_rois: unknown or unusable ref_id");
        const auto& re = c->refs[q.ref_id];
        const int rh = re.cls >= 0 ? c->plans[re.cls].g.H : c->gplans[re.gcls].p.H;
        const int rw = re.cls >= 0 ? c->plans[re.cls].g.W : c->gplans[re.gcls].p.W;
        if (q.H != rh || q.W != rw) return fail(c, CCST_E_SHAPE, "ccst_track_rois: ROI size differs from its reference");
        const int64_t pitch = q.pitch_elems == 0 ? q.W : q.pitch_elems;
        if (!q.frame || pitch < q.W) return fail(c, CCST_E_INVALID, "ccst_track_rois: null frame or pitch < W");
        if (re.gcls >= 0) {
            c->h_gitems[(size_t)ng++] = GenItem{q.frame, (long long)pitch, i, re.gcls, q.ref_id};
            continue;
        }
        RoiItem& it = c->h_items[(size_t)np++];
        it.frame = q.frame;
        it.pitch = pitch;
        it.out_index = i;
        it.cls = re.cls;
        it.ref = q.ref_id;
        it.vec_ok = ((uintptr_t)q.frame % 16 == 0) && ((size_t)pitch * elem % 16 == 0) ? 1 : 0;
        it.pad = 0;
    }
    if ((c->p.flags & CCST_FLAG_GRAPHS) && c->stream != nullptr) return rois_graph_track(c, rois, n, out_dev, np, ng);
    CK(c, shared_acquire(c, c->stream));
    GenPart gpart{};
    if (ng > 0) {
        gen_sort(c, c->h_gitems.data(), ng);
        gpart.gb.n = ng;
        gpart.gb.out = (Result*)out_dev;
        if ((rc = gen_stage(c, c->glane[0], &gpart.gb, c->h_gitems.data(), c->stream, &gpart.stride))) return rc;
        gpart.items = c->h_gitems.data();
        gpart.lane = &c->glane[0];
        gpart.counter = c->d_next + 24;
    }
    if (np > 0) {
        if (c->items_cap < (size_t)np) {
            if (c->d_items) cudaFree(c->d_items);
            c->d_items = nullptr;
            c->items_cap = 0;
            CK(c, cudaMalloc(&c->d_items, (size_t)np * sizeof(RoiItem)));
            c->items_cap = (size_t)np;
        }
        if ((rc = rois_stage(c, c->h_items.data(), np, c->stream, c->d_items))) return rc;
    }
    if ((rc = rois_chain_launch(c, RoiPart{c->d_items, c->h_items.data(), np, c->d_next + 16}, gpart,
                                (Result*)out_dev, c->stream, c->rside)))
        return rc;
    CK(c, shared_release(c, c->stream));
    return CCST_OK;
}

// ---------------------------------------------------------------------- serving
// Continuous batching over the uneven-ROI kernel: clients submit single frames of any of
// the context's references (cameras); a worker thread takes everything pending as one
// batch and launches one ROI kernel per batch, up to kRing batches in flight on their own
// streams. Frame slots are pinned host memory mapped into the device's address space,
// reserved at creation: the submit copies a frame into its slot and the kernel reads it in
// place, so the worker issues no per-frame copy. A submit without a free slot is refused
// (admission control).
struct ccst_server {
    static constexpr int kRing = 4;
    static constexpr size_t kAlign = 256;
    struct Req {
        int ref = 0;
        uint64_t vstart = 0;           // the frame's bytes in the arena: virtual offset (see reserve)
        uint64_t ticket = 0;
        bool keep = false;
        std::chrono::steady_clock::time_point t0;
    };
    // one reservation of the arena, in reservation order
    struct Span {
        uint64_t vstart = 0, vend = 0;
        bool released = false;
    };
    struct InFlight {
        cudaStream_t st = nullptr;
        cudaEvent_t ev = nullptr;
        SideStream side;               // the batch's general-size part, beside st
        Result* d_out = nullptr;
        Result* h_out = nullptr;
        RoiItem* d_items = nullptr;
        RoiItem* h_items = nullptr;    // pinned, so the item upload is asynchronous
        GenItem* h_gitems = nullptr;   // pinned: the batch's general-size frames
        GenLane lane;                  // the general-size kernel's scratch for this entry
        std::vector<Req> reqs;
        bool busy = false;
    };
    ccst_ctx* c = nullptr;
    int max_batch = 0, depth = kRing;
    size_t elem = 0;
    // Admission arena: `cap` bytes of pinned host memory mapped into the device's address
    // space (the kernels read each frame in place). A frame takes its own size rounded to
    // 256 bytes, reserved at the head of a ring in virtual offsets (physical = virtual mod
    // cap; a frame never straddles the end: the rest of the ring is skipped). Reservations
    // free in completion order, but the tail only moves past the oldest live one.
    uint64_t cap = 0, head = 0, tail = 0, max_used = 0;
    std::deque<Span> spans;
    char* h_frames = nullptr;
    char* d_frames = nullptr;          // the same memory as the device addresses it
    unsigned* d_counters = nullptr;    // kRoiCounters + 1 item counters per ring entry (power-of-two sides; general)
    InFlight ring[kRing];
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Req> pending;
    std::atomic<int> npending{0};
    std::unordered_map<uint64_t, std::pair<bool, Result>> results;
    uint64_t next_ticket = 1, submitted = 0, completed = 0, rejected = 0, batches = 0, batched = 0;
    std::vector<float> lat_us;
    int error = 0;
    bool stop = false;
    std::thread worker;

    // Reserve `bytes` (a multiple of kAlign) at the head; false when the budget is full.
    // Call with mu held.
    bool reserve(uint64_t bytes, uint64_t* vstart) {
        uint64_t v = head;
        const uint64_t off = v % cap;
        if (off + bytes > cap) v += cap - off;            // skip the end of the ring
        if (v + bytes - tail > cap) return false;
        spans.push_back(Span{v, v + bytes, false});
        head = v + bytes;
        max_used = std::max(max_used, head - tail);
        *vstart = v;
        return true;
    }
    // Release the reservation starting at vstart (mu held).
    void release(uint64_t vstart) {
        for (auto& sp : spans)
            if (sp.vstart == vstart) {
                sp.released = true;
                break;
            }
        while (!spans.empty() && spans.front().released) {
            tail = spans.front().vend;
            spans.pop_front();
        }
        if (spans.empty()) tail = head;
    }
};

// The frame shape of reference `ref`, for either kernel.
static void ref_shape(const ccst_ctx* c, int ref, int* H, int* W) {
    const auto& re = c->refs[ref];
    if (re.cls >= 0) {
        *H = c->plans[re.cls].g.H;
        *W = c->plans[re.cls].g.W;
    } else {
        *H = c->gplans[re.gcls].p.H;
        *W = c->gplans[re.gcls].p.W;
    }
}

static bool ref_usable(const ccst_ctx* c, int ref) {
    return ref >= 0 && ref < (int)c->refs.size() && (c->refs[ref].cls >= 0 || c->refs[ref].gcls >= 0);
}

static void server_fail(ccst_server* s, int code) {
    std::lock_guard<std::mutex> lk(s->mu);
    if (!s->error) s->error = code;
    s->cv_done.notify_all();
}

// Retire the ring entry if its batch has finished (or `block`: wait for it).
static bool server_retire(ccst_server* s, ccst_server::InFlight& b, bool block) {
    if (!b.busy) return false;
    const cudaError_t q = block ? cudaEventSynchronize(b.ev) : cudaEventQuery(b.ev);
    if (q == cudaErrorNotReady) return false;
    if (q != cudaSuccess) {
        server_fail(s, CCST_E_CUDA);
        return false;
    }
    const auto t1 = std::chrono::steady_clock::now();
    {
        std::lock_guard<std::mutex> lk(s->mu);
        for (size_t i = 0; i < b.reqs.size(); ++i) {
            const auto& r = b.reqs[i];
            s->lat_us.push_back(std::chrono::duration<float, std::micro>(t1 - r.t0).count());
            if (r.keep) s->results[r.ticket] = {true, b.h_out[i]};
            s->release(r.vstart);
            ++s->completed;
        }
    }
    b.reqs.clear();
    b.busy = false;
    s->cv_done.notify_all();
    return true;
}

static void server_loop(ccst_server* s) {
    ccst_ctx* c = s->c;
    int next = 0;
    for (;;) {
        bool any_busy = false;
        for (auto& b : s->ring) {
            server_retire(s, b, false);
            any_busy |= b.busy;
        }
        ccst_server::InFlight& b = s->ring[next];
        std::vector<ccst_server::Req> take;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            if (s->stop && s->pending.empty() && !any_busy) return;
            if (s->error) {
                if (s->stop) return;
                s->cv_work.wait_for(lk, std::chrono::milliseconds(10));
                continue;
            }
            if (!b.busy && !s->pending.empty()) {
                const size_t m = std::min(s->pending.size(), (size_t)s->max_batch);
                take.assign(s->pending.begin(), s->pending.begin() + m);
                s->pending.erase(s->pending.begin(), s->pending.begin() + m);
                s->npending -= (int)m;
            } else if (!any_busy && s->pending.empty()) {
                // idle: poll for a new frame for up to 200 us (a thread wake-up costs tens of
                // microseconds of latency), then sleep until one is submitted
                lk.unlock();
                const auto spin_end = std::chrono::steady_clock::now() + std::chrono::microseconds(200);
                while (s->npending.load() == 0 && std::chrono::steady_clock::now() < spin_end) std::this_thread::yield();
                lk.lock();
                if (s->pending.empty() && !s->stop) s->cv_work.wait_for(lk, std::chrono::milliseconds(10));
                continue;
            }
        }
        if (take.empty()) {
            if (b.busy) server_retire(s, b, true);      // the ring is full: wait for its oldest
            else std::this_thread::yield();
            continue;
        }
        const int m = (int)take.size();
        int np = 0, ng = 0;
        for (int i = 0; i < m; ++i) {
            const auto& r = take[i];
            const auto& re = c->refs[r.ref];
            int H = 0, W = 0;
            ref_shape(c, r.ref, &H, &W);
            const char* frame = s->d_frames + (size_t)(r.vstart % s->cap);
            if (re.cls >= 0) b.h_items[np++] = RoiItem{frame, (long long)W, i, re.cls, r.ref, 1, 0};
            else b.h_gitems[ng++] = GenItem{frame, (long long)W, i, re.gcls, r.ref};
        }
        // each kernel writes record i of the batch to d_out[i]; out_index survives the sorts
        bool ok = true;
        GenPart gpart{};
        if (ng > 0) {
            gen_sort(c, b.h_gitems, ng);
            gpart.gb.n = ng;
            gpart.gb.out = b.d_out;
            ok = gen_stage(c, b.lane, &gpart.gb, b.h_gitems, b.st, &gpart.stride) == CCST_OK;
            gpart.items = b.h_gitems;
            gpart.lane = &b.lane;
            gpart.counter = s->d_counters + (kRoiCounters + 1) * next + kRoiCounters;
        }
        if (ok && np > 0) ok = rois_stage(c, b.h_items, np, b.st, b.d_items) == CCST_OK;
        ok = ok && rois_chain_launch(c, RoiPart{b.d_items, b.h_items, np, s->d_counters + (kRoiCounters + 1) * next}, gpart, b.d_out,
                                     b.st, b.side) == CCST_OK;
        ok = ok && cudaMemcpyAsync(b.h_out, b.d_out, (size_t)m * sizeof(Result), cudaMemcpyDeviceToHost, b.st) ==
                       cudaSuccess;
        ok = ok && cudaEventRecord(b.ev, b.st) == cudaSuccess;
        if (!ok) {
            server_fail(s, CCST_E_CUDA);
            continue;
        }
        b.reqs = std::move(take);
        b.busy = true;
        {
            std::lock_guard<std::mutex> lk(s->mu);
            ++s->batches;
            s->batched += (uint64_t)m;
        }
        next = (next + 1) % s->depth;
    }
}

static void server_free(ccst_server* s) {
    for (auto& b : s->ring) {
        if (b.st) cudaStreamSynchronize(b.st);
        side_free(b.side);
        if (b.ev) cudaEventDestroy(b.ev);
        if (b.st) cudaStreamDestroy(b.st);
        if (b.d_out) cudaFree(b.d_out);
        if (b.h_out) cudaFreeHost(b.h_out);
        if (b.d_items) cudaFree(b.d_items);
        if (b.h_items) cudaFreeHost(b.h_items);
        if (b.h_gitems) cudaFreeHost(b.h_gitems);
        lane_free(b.lane);
    }
    if (s->h_frames) cudaFreeHost(s->h_frames);
    if (s->d_counters) cudaFree(s->d_counters);
}

// Bytes a frame of reference `ref` takes in the admission arena.
static uint64_t frame_bytes(const ccst_server* s, int ref) {
    int H = 0, W = 0;
    ref_shape(s->c, ref, &H, &W);
    const uint64_t b = (uint64_t)H * W * s->elem;
    return (b + ccst_server::kAlign - 1) / ccst_server::kAlign * ccst_server::kAlign;
}

extern "C" int ccst_server_create_ex(ccst_ctx* c, const ccst_server_config* cfg, ccst_server** out) {
    int rc = check_ctx(c);
    if (rc) return rc;
    if (!out || !cfg || cfg->max_batch < 1 || cfg->max_in_flight < 1 || cfg->max_in_flight > ccst_server::kRing ||
        cfg->budget_bytes < (int64_t)ccst_server::kAlign)
        return fail(c, CCST_E_INVALID, "ccst_server_create_ex: bad configuration");
    *out = nullptr;
    rois_init(c);
    if ((rc = rois_upload(c))) return rc;
    if (!c->gplans.empty() && (rc = gen_prepare(c))) return rc;
    ccst_server* s = new (std::nothrow) ccst_server();
    if (!s) return fail(c, CCST_E_NOMEM, "ccst_server_create: host allocation failed");
    s->c = c;
    s->max_batch = cfg->max_batch;
    s->depth = cfg->max_in_flight;
    s->elem = c->p.in_dtype == CCST_U16 ? 2 : 4;
    s->cap = ((uint64_t)cfg->budget_bytes + ccst_server::kAlign - 1) / ccst_server::kAlign * ccst_server::kAlign;
    bool any = false;
    for (int i = 0; i < (int)c->refs.size(); ++i) any |= ref_usable(c, i);
    if (!any) {
        delete s;
        return fail(c, CCST_E_INVALID, "ccst_server_create: no reference usable by ROI batches");
    }
    auto bad = [&](cudaError_t e) {
        server_free(s);
        delete s;
        return fail(c, e == cudaErrorMemoryAllocation ? CCST_E_NOMEM : CCST_E_CUDA,
                    std::string("ccst_server_create: ") + cudaGetErrorString(e));
    };
    cudaError_t e;
    if ((e = cudaHostAlloc(&s->h_frames, (size_t)s->cap, cudaHostAllocMapped)) != cudaSuccess) return bad(e);
    if ((e = cudaHostGetDevicePointer((void**)&s->d_frames, s->h_frames, 0)) != cudaSuccess) return bad(e);
    if ((e = cudaMalloc(&s->d_counters, (kRoiCounters + 1) * ccst_server::kRing * sizeof(unsigned))) != cudaSuccess) return bad(e);
    for (int k = 0; k < s->depth; ++k) {
        auto& b = s->ring[k];
        if ((e = cudaStreamCreateWithFlags(&b.st, cudaStreamNonBlocking)) != cudaSuccess) return bad(e);
        if ((e = cudaEventCreateWithFlags(&b.ev, cudaEventDisableTiming)) != cudaSuccess) return bad(e);
        if ((e = side_make(b.side)) != cudaSuccess) return bad(e);     // not made while serving
        if ((e = cudaMalloc(&b.d_out, (size_t)s->max_batch * sizeof(Result))) != cudaSuccess) return bad(e);
        if ((e = cudaHostAlloc(&b.h_out, (size_t)s->max_batch * sizeof(Result), cudaHostAllocDefault)) != cudaSuccess)
            return bad(e);
        if ((e = cudaMalloc(&b.d_items, (size_t)s->max_batch * sizeof(RoiItem))) != cudaSuccess) return bad(e);
        if ((e = cudaHostAlloc(&b.h_items, (size_t)s->max_batch * sizeof(RoiItem), cudaHostAllocDefault)) != cudaSuccess)
            return bad(e);
        if ((e = cudaHostAlloc(&b.h_gitems, (size_t)s->max_batch * sizeof(GenItem), cudaHostAllocDefault)) != cudaSuccess)
            return bad(e);
        // the general-size lane for a whole batch: growing it while serving would
        // reallocate, and so synchronise the device under every batch in flight
        if (!c->gplans.empty() && (rc = lane_reserve(c, b.lane, s->max_batch)) != CCST_OK) {
            server_free(s);
            delete s;
            return rc;
        }
    }
    s->worker = std::thread(server_loop, s);
    *out = s;
    return CCST_OK;
}

extern "C" int ccst_server_create(ccst_ctx* c, int slots, int max_batch, ccst_server** out) {
    int rc = check_ctx(c);
    if (rc) return rc;
    if (!out || slots < 1 || max_batch < 1) return fail(c, CCST_E_INVALID, "ccst_server_create: bad arguments");
    rois_init(c);
    // the budget of `slots` frames of the largest reference present now
    uint64_t largest = 0;
    const size_t elem = c->p.in_dtype == CCST_U16 ? 2 : 4;
    for (int i = 0; i < (int)c->refs.size(); ++i)
        if (ref_usable(c, i)) {
            int H = 0, W = 0;
            ref_shape(c, i, &H, &W);
            largest = std::max(largest, ((uint64_t)H * W * elem + 255) / 256 * 256);
        }
    if (largest == 0) return fail(c, CCST_E_INVALID, "ccst_server_create: no reference usable by ROI batches");
    ccst_server_config cfg{};
    cfg.max_batch = std::min(max_batch, slots);
    cfg.max_in_flight = ccst_server::kRing;
    cfg.budget_bytes = (int64_t)(largest * (uint64_t)slots);
    return ccst_server_create_ex(c, &cfg, out);
}

extern "C" int ccst_server_submit(ccst_server* s, int ref_id, const void* frame_host, int64_t pitch_elems,
                                  uint64_t* ticket) {
    if (!s || !frame_host) return CCST_E_INVALID;
    ccst_ctx* c = s->c;
    if (!ref_usable(c, ref_id)) return CCST_E_INVALID;
    int H = 0, W = 0;
    ref_shape(c, ref_id, &H, &W);
    const uint64_t bytes = frame_bytes(s, ref_id);
    if (bytes > s->cap) return CCST_E_INVALID;                 // can never be admitted
    if (pitch_elems == 0) pitch_elems = W;
    if (pitch_elems < W) return CCST_E_INVALID;
    ccst_server::Req r;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->error) return s->error;
        if (!s->reserve(bytes, &r.vstart)) {
            ++s->rejected;
            return CCST_E_BUSY;
        }
    }
    char* dst = s->h_frames + (size_t)(r.vstart % s->cap);
    const size_t row = (size_t)W * s->elem;
    for (int y = 0; y < H; ++y) std::memcpy(dst + y * row, (const char*)frame_host + (size_t)y * pitch_elems * s->elem, row);
    r.ref = ref_id;
    r.keep = ticket != nullptr;
    r.t0 = std::chrono::steady_clock::now();
    {
        std::lock_guard<std::mutex> lk(s->mu);
        r.ticket = s->next_ticket++;
        if (r.keep) {
            s->results[r.ticket] = {false, Result{}};
            *ticket = r.ticket;
        }
        s->pending.push_back(r);
        ++s->npending;
        ++s->submitted;
    }
    s->cv_work.notify_one();
    return CCST_OK;
}

extern "C" int ccst_server_poll(ccst_server* s, uint64_t ticket, int timeout_us, ccst_result* out, int* done) {
    if (!s || !done) return CCST_E_INVALID;
    *done = 0;
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->results.find(ticket);
    if (it == s->results.end()) return CCST_E_INVALID;
    const auto until = std::chrono::steady_clock::now() + std::chrono::microseconds(timeout_us > 0 ? timeout_us : 0);
    while (!it->second.first && !s->error) {
        if (s->cv_done.wait_until(lk, until) == std::cv_status::timeout) break;
        it = s->results.find(ticket);
    }
    if (!it->second.first) return s->error ? s->error : CCST_E_TIMEOUT;
    if (out) std::memcpy(out, &it->second.second, sizeof(Result));
    s->results.erase(it);
    *done = 1;
    return CCST_OK;
}

extern "C" int ccst_server_read_stats(ccst_server* s, int reset, ccst_server_stats* out) {
    if (!s || !out) return CCST_E_INVALID;
    std::lock_guard<std::mutex> lk(s->mu);
    out->submitted = s->submitted;
    out->completed = s->completed;
    out->rejected = s->rejected;
    out->batches = s->batches;
    out->mean_batch = s->batches ? (double)s->batched / (double)s->batches : 0.0;
    std::vector<float> v = s->lat_us;
    std::sort(v.begin(), v.end());
    auto pct = [&](double q) { return v.empty() ? 0.0 : (double)v[std::min(v.size() - 1, (size_t)(q * v.size()))]; };
    out->p50_us = pct(0.50);
    out->p99_us = pct(0.99);
    out->max_us = v.empty() ? 0.0 : (double)v.back();
    out->in_flight = (int64_t)(s->submitted - s->completed);
    out->bytes_in_flight = (int64_t)(s->head - s->tail);
    out->max_bytes_in_flight = (int64_t)s->max_used;
    out->budget_bytes = (int64_t)s->cap;
    if (reset) {
        s->lat_us.clear();
        s->submitted = s->completed = s->rejected = s->batches = s->batched = 0;
        s->max_used = s->head - s->tail;
    }
    return s->error;
}

extern "C" void ccst_server_destroy(ccst_server* s) {
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv_work.notify_all();
    if (s->worker.joinable()) s->worker.join();
    server_free(s);
    delete s;
}

// Offered-load generator for measuring the server: one host thread per camera submits frames
// of its pool (cycled) at exponential inter-arrival times of mean 1/rate for `seconds`,
// without tickets (results are counted, not kept); refused submits are counted and dropped.
// Then it waits for all admitted frames and reports the server's statistics.
extern "C" int ccst_server_loadgen(ccst_server* s, int ncams, const int* ref_ids, const double* rates_hz,
                                   const void* const* pools, const int* pool_len, double seconds, uint64_t seed,
                                   ccst_server_stats* out) {
    if (!s || ncams < 1 || !ref_ids || !rates_hz || !pools || !pool_len || !(seconds > 0) || !out)
        return CCST_E_INVALID;
    for (int k = 0; k < ncams; ++k)
        if (!ref_usable(s->c, ref_ids[k]) || !(rates_hz[k] > 0) || !pools[k] || pool_len[k] < 1) return CCST_E_INVALID;
    ccst_server_stats dummy;
    ccst_server_read_stats(s, 1, &dummy);
    std::atomic<int> err{0};
    std::vector<std::thread> th;
    const auto t_start = std::chrono::steady_clock::now() + std::chrono::milliseconds(5);
    for (int k = 0; k < ncams; ++k) {
        th.emplace_back([&, k]() {
            std::mt19937_64 rng(seed + 7919u * (uint64_t)k);
            std::exponential_distribution<double> gap(rates_hz[k]);
            int H = 0, W = 0;
            ref_shape(s->c, ref_ids[k], &H, &W);
            const size_t fb = (size_t)H * W * s->elem;
            double t = 0.0;
            for (int64_t i = 0;; ++i) {
                t += gap(rng);
                if (t >= seconds) break;
                const auto at = t_start + std::chrono::duration_cast<std::chrono::steady_clock::duration>(
                                              std::chrono::duration<double>(t));
                while (std::chrono::steady_clock::now() < at) {
                }
                const char* f = (const char*)pools[k] + (size_t)(i % pool_len[k]) * fb;
                const int rc = ccst_server_submit(s, ref_ids[k], f, 0, nullptr);
                if (rc && rc != CCST_E_BUSY) {
                    err = rc;
                    return;
                }
            }
        });
    }
    for (auto& t : th) t.join();
    for (int it = 0; it < 200000; ++it) {                   // drain: admitted frames finish
        ccst_server_stats st;
        const int rc = ccst_server_read_stats(s, 0, &st);
        if (rc) return rc;
        if (st.in_flight == 0) break;
        std::this_thread::sleep_for(std::chrono::microseconds(50));
    }
    const int rc = ccst_server_read_stats(s, 0, out);
    return err ? (int)err : rc;
}

// Grid size M of the refinement square for this context (tests and bindings).
extern "C" int ccst_grid_size(ccst_ctx* c) { return c ? c->g.M : CCST_E_INVALID; }

// ------------------------------------------------------------------------------------
// Allocation-free tracking (ccst_track_static).
//
// For callers that are not allowed to allocate device memory at run time: for
// instance a camera/feedback loop that reserves all GPU memory when it starts and
// must never stall on cudaMalloc (which can synchronise the device), or a plug-in
// inside a host program that owns the device memory pool. Everything ccst_create
// would allocate (reference spectra, upsampling tables, FFT twiddles and the FP64
// FFT workspace used to build the reference spectrum) lives instead in one
// file-scope device array of fixed size, shared by every call in the process.
namespace {

constexpr size_t kStaticScratchBytes = (size_t)2 << 20;   // 2 MiB per device
static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

struct StaticDevice {
    bool ready = false;
    unsigned char* scratch = nullptr;   // device address of g_static_scratch on this device
    size_t smem_limit = 0;
    int sms = 0;
};
constexpr int kStaticMaxDevices = 64;
std::mutex g_static_mu;
StaticDevice g_static_dev[kStaticMaxDevices];
char g_static_err[256] = "no error";

int static_fail(int code, const char* msg, const char* detail = "") {
    std::lock_guard<std::mutex> lk(g_static_mu);
    snprintf(g_static_err, sizeof(g_static_err), "%s%s", msg, detail);
    return code;
}

// Once per device, with that device current: resolve the array's device address
// (the host-side symbol is only a stand-in) and raise the kernels' shared-memory limit.
int static_setup(int dev, StaticDevice* out) {
    if (dev < 0 || dev >= kStaticMaxDevices) return static_fail(CCST_E_UNSUPPORTED, "ccst_track_static: device ordinal >= 64");
    std::lock_guard<std::mutex> lk(g_static_mu);
    StaticDevice& d = g_static_dev[dev];
    if (!d.ready) {
        cudaError_t e = cudaGetSymbolAddress((void**)&d.scratch, g_static_scratch);
        if (e != cudaSuccess) {
            snprintf(g_static_err, sizeof(g_static_err), "cudaGetSymbolAddress: %s", cudaGetErrorString(e));
            return CCST_E_CUDA;
        }
        cudaDeviceProp prop;
        if ((e = cudaGetDeviceProperties(&prop, dev)) != cudaSuccess) {
            snprintf(g_static_err, sizeof(g_static_err), "cudaGetDeviceProperties: %s", cudaGetErrorString(e));
            return CCST_E_CUDA;
        }
        d.smem_limit = prop.sharedMemPerBlockOptin;
        d.sms = prop.multiProcessorCount;
        for (int h = 8; h <= 128; h *= 2)
            for (int w = 8; w <= 128; w *= 2) {
                if ((e = cudaFuncSetAttribute(track_kernel_for(h, w), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              (int)d.smem_limit - ((h == 128 && w == 128) ? kTcStaticSmem : 0))) !=
                    cudaSuccess) {
                    snprintf(g_static_err, sizeof(g_static_err), "cudaFuncSetAttribute: %s", cudaGetErrorString(e));
                    return CCST_E_CUDA;
                }
            }
        d.ready = true;
    }
    *out = d;
    return CCST_OK;
}

}  // namespace

extern "C" int ccst_track_static(const float* ref_dev, int H, int W, const ccst_params* pin,
                                 const void* frames_dev, int64_t n, int64_t pitch_elems,
                                 ccst_result* out_dev) {
    ccst_params p;
    if (pin) p = *pin; else ccst_default_params(&p);
    if (!ref_dev) return static_fail(CCST_E_INVALID, "ccst_track_static: null reference");
    if (n < 0) return static_fail(CCST_E_INVALID, "ccst_track_static: n < 0");
    if (n > 0 && (!frames_dev || !out_dev)) return static_fail(CCST_E_INVALID, "ccst_track_static: null frames or out");
    if (!is_pow2(H) || !is_pow2(W) || H < 8 || W < 8 || H > 128 || W > 128)
        return static_fail(CCST_E_SHAPE, "ccst_track_static: H and W must be powers of two in [8, 128]");
    if (p.upsample < 1 || p.upsample > 16384)
        return static_fail(CCST_E_INVALID, "ccst_track_static: upsample must be in [1, 16384]");
    if (p.method != CCST_CC_U && p.method != CCST_CC_SN)
        return static_fail(CCST_E_INVALID, "ccst_track_static: unknown method");
    if (p.method == CCST_CC_SN && !(p.eps == p.eps))
        return static_fail(CCST_E_INVALID, "ccst_track_static: eps is NaN");
    if (p.in_dtype != CCST_U16 && p.in_dtype != CCST_F32)
        return static_fail(CCST_E_INVALID, "ccst_track_static: unknown in_dtype");
    if (pitch_elems == 0) pitch_elems = W;
    if (pitch_elems < W) return static_fail(CCST_E_INVALID, "ccst_track_static: pitch_elems < W");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return static_fail(CCST_E_CUDA, "cudaGetDevice: ", cudaGetErrorString(e));
    StaticDevice sd;
    int rc = static_setup(dev, &sd);
    if (rc) return rc;
    cudaStream_t stream = (cudaStream_t)p.stream;

    // geometry: the same choices ccst_create makes
    Geom g{};
    if (!plan_geometry(H, W, p, sd.smem_limit, &g))
        return static_fail(CCST_E_SHAPE, "ccst_track_static: frame too large for shared memory");
    const size_t smem = smem_plan(g).total;
    const long long Dy = (long long)g.u * H, Dx = (long long)g.u * W;
    g.By = 1; while ((long long)g.By * g.By < Dy) ++g.By;
    g.Bx = 1; while ((long long)g.Bx * g.Bx < Dx) ++g.Bx;
    const int ncy = (int)((Dy + g.By - 1) / g.By), ncx = (int)((Dx + g.Bx - 1) / g.Bx);

    // carve the static array (256-byte aligned regions)
    const size_t HW = (size_t)H * W, HWc = (size_t)H * g.Wc;
    const size_t tabA = (size_t)g.Hh * g.T1p, tabB = (size_t)g.Wc * g.T1p;
    const size_t ndf = (size_t)(g.Ntw / 2) + HWc + ncy + g.By + ncx + g.Bx;
    const size_t work = (size_t)(H / 2) * W + (size_t)H * g.Wcp;
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t o = off; off = align_up(off + bytes, 256); return sd.scratch + o; };
    double* b64 = (double*)take(HW * sizeof(double));
    double2* FE64 = (double2*)take(HWc * sizeof(double2));
    float2* FE32 = (float2*)take(HWc * sizeof(float2));
    double2* tw64 = (double2*)take((size_t)(g.Ntw / 2) * sizeof(double2));
    float2* tw32 = (float2*)take((size_t)(g.Ntw / 2) * sizeof(float2));
    float* tab = (float*)take((2 * tabA + 3 * tabB) * sizeof(float) + table_bytes(g));
    dfc* dfb = (dfc*)take(ndf * sizeof(dfc));
    double2* wk = (double2*)take(work * sizeof(double2));
    if (off > kStaticScratchBytes)
        return static_fail(CCST_E_SHAPE, "ccst_track_static: this H, W and upsample need more scratch than "
                                         "the 2 MiB static array holds (lower upsample)");
    g.FE32 = FE32; g.FE64 = FE64; g.b64 = b64; g.tw32 = tw32; g.tw64 = tw64;
    g.tA_cm1 = tab; g.tA_s = tab + tabA; g.tB_wc = tab + 2 * tabA; g.tB_ws = g.tB_wc + tabB; g.tB_gc = g.tB_ws + tabB;
    g.tAh = (const uint2*)(g.tB_gc + tabB);
    g.tBh = (const uint2*)((const char*)g.tAh + ta_bytes(g));
    dfc* twdf = dfb;
    dfc* FEdf = twdf + g.Ntw / 2;
    dfc* eyc = FEdf + HWc;
    dfc* eyf = eyc + ncy;
    dfc* exc = eyf + g.By;
    dfc* exf = exc + ncx;
    g.twdf = twdf; g.FEdf = FEdf; g.eyc = eyc; g.eyf = eyf; g.exc = exc; g.exf = exf;

    // every region is rewritten in full below before anything reads it
    init_twiddles<<<1, 256, 0, stream>>>(g.Ntw, tw64, tw32);
    init_tables<<<64, 256, 0, stream>>>(g, tab, tab + tabA, tab + 2 * tabA, tab + 2 * tabA + tabB,
                                        tab + 2 * tabA + 2 * tabB, (uint2*)g.tAh, (uint2*)g.tBh);
    init_ref_operand<<<32, 256, 0, stream>>>(g, ref_dev, b64);
    init_ref_spectrum<<<1, 256, 0, stream>>>(g, wk, FE64, FE32);
    init_dfloat<<<32, 256, 0, stream>>>(g, tw64, FE64, twdf, FEdf, eyc, eyf, exc, exf, ncy, ncx);
    if (n > 0) {
        Batch b{};
        b.frames = frames_dev;
        b.n = n;
        b.pitch = pitch_elems;
        b.out = (Result*)out_dev;
        const size_t el = p.in_dtype == CCST_U16 ? 2 : 4;
        b.vec_ok = ((uintptr_t)frames_dev % 16 == 0) && ((size_t)pitch_elems * el % 16 == 0) ? 1 : 0;
        const void* kern = track_kernel_for(H, W);
        int occ = 1;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, track_threads(H, W), smem);
        const long long cap = (long long)sd.sms * (occ > 0 ? occ : 1);
        const int grid = (int)(n < cap ? n : cap);
        void* args[] = {&g, &b};
        if ((e = cudaLaunchKernel(kern, dim3(grid), dim3(track_threads(H, W)), args, smem, stream)) != cudaSuccess)
            return static_fail(CCST_E_CUDA, "ccst_track_static launch: ", cudaGetErrorString(e));
    }
    if ((e = cudaGetLastError()) != cudaSuccess)
        return static_fail(CCST_E_CUDA, "ccst_track_static launch: ", cudaGetErrorString(e));
    return CCST_OK;
}

extern "C" const char* ccst_static_last_error(void) {
    std::lock_guard<std::mutex> lk(g_static_mu);
    return g_static_err;
}
