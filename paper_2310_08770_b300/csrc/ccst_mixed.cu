// ccst_mixed.cu -- the tracking path of Secs. II-III in FP32 for square frames of 48, 96,
// 192 and 256 pixels a side, whose FFT lengths factor into 2s and 3s.
//
// Per frame, one cluster of CL CTAs (CL = 1, 2 or 4; ccst_mixed.cuh):
//   a1  each CTA loads its H/CL rows (16-byte vector loads where aligned) and forms the
//       operand a = I (CC-U, Eq. 4) or (I + eps)^2 (CC-SN, Eq. 7);
//   a2  real rows -> half spectra through a W/2-point complex FFT per row (even samples
//       real, odd samples imaginary, then the even/odd split); each CTA writes column kx
//       of every row straight into the shared memory of the CTA that owns kx;
//   a3  column FFTs over the CTA's band and the product X = F[a] conj F[b];
//   a4  inverse column FFTs, then the inverse rows (reading the owners' bands), scanned
//       for the integer extremum (lowest flat index on ties); a near-tie within the
//       integer threshold sends the frame to the fallback;
//   a6  the upsampled DFT on the M x M grid around the peak (Sec. III) in the peak-relative
//       folded form, as two FP32 contractions over the CTA's band whose partial sums the
//       CTAs add through distributed shared memory:
//         X'(k) = X(k) e^{2 pi i k.p/N};  P(m) = X'(m) + X'(-m), Q(m) = X'(m) - X'(-m);
//         U'(t) = sum_m (cos th_mt - 1) P(m),  V(t) = sum_m sin th_mt Q(m),  th_mt = 2 pi m t/(uH);
//         T'(+-t) = U'(t) +- i V(t);
//         D(ty, tx) = Re sum_kx g(kx) T'(ty, kx) e^{2 pi i kx' tx/(uW)} + gsum(tx),
//         gsum(tx) = Re sum_kx g(kx) R(kx) (e^{2 pi i kx' tx/(uW)} - 1),  R(kx) = sum_ky X'(ky, kx);
//       D is cu(t) - cu(0) in units of HW (g = 1 at kx = 0 and kx = W/2, 2 elsewhere: the
//       Hermitian fold; kx' the signed frequency, -W/2 at the Nyquist column). In the
//       columns 0 < kx < W/2 the y-Nyquist row enters through cos only (Q(H/2) = 0); in
//       the x-Nyquist column it keeps its full phase (Q(H/2) = -P(H/2)).
//   a7  the sub-pixel extremum: unique within tau0 sum g|X| -> the record; a few points
//       within tau0 -> exact pair differences v(j) - v(j1), from factors
//       E(a) - E(b) = 2i sin(.) e^{i .} (level 1); still within tau1 -> fallback.
// A frame sent to the fallback is appended to a list that the double-float general-size
// kernel (ccst_generic.cu) tracks in a second launch, so the records of this path are
// FP32 decisions certified by the guard thresholds, or the double-float path's own.
#include "ccst_mixed.cuh"
#include "ccst_mixfft.cuh"

#include <cooperative_groups.h>
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

namespace cg = cooperative_groups;

namespace ccst {
namespace mix {

// Threads per CTA and CTAs per SM. A small frame is latency-bound (each phase is a few
// hundred tasks between barriers), so 48 and 96 run 4 and 2 smaller CTAs per SM; 192 takes
// a whole SM per CTA, and 256 takes 384 threads, whose 16-point register DFTs want more
// than the 128 registers a 512-thread CTA leaves each thread.
__host__ __device__ constexpr int mix_threads(int H, int W) {
    return H * W <= 48 * 48 ? 128 : H * W <= 96 * 96 ? 256 : (H >= 256 || W >= 256) ? 384 : 512;
}
__host__ __device__ constexpr int mix_min_ctas(int H, int W) { return H * W <= 48 * 48 ? 4 : H * W <= 96 * 96 ? 2 : 1; }
constexpr int kTM = 8;            // t rows per contraction task

template <int CL>
struct Clu {
    __device__ __forceinline__ static int rank() {
        if constexpr (CL == 1) return 0;
        else return (int)cg::this_cluster().block_rank();
    }
    // every thread of every CTA of the cluster; orders shared-memory accesses across them
    __device__ __forceinline__ static void sync() {
        if constexpr (CL == 1) __syncthreads();
        else cg::this_cluster().sync();
    }
    template <class T>
    __device__ __forceinline__ static T* at(T* p, int r) {
        if constexpr (CL == 1) return p;
        else return cg::this_cluster().map_shared_rank(p, r);
    }
};

// Shared-memory layout (byte offsets in MixPlan; mix_carve is used by the host to size it).
struct MixSh {
    float2* X;       // [H][KB]: the band of the spectrum; rows are FFT slots (X(ky) at mix_pos(ky))
    float2* Y;       // [H][KB]: inverse column transforms, natural rows
    float2* SG;      // [G][RSG]: staged rows
    float4* CE;      // [TCp][KB]: stage-A output (C0, E0, C1, E1)
    float4* PS;      // [TC][TX]: stage-B partial sums (CL > 1)
    float2* TBs;     // [Wc][TXp]: the stage-B table (p.tbs; CL = 1), at PS's place
    float2* gy;      // level 1: [Hh] E(m, ry)
    float2* fy;      // level 1: [kMaxCand][Hh] E(m, ty) - E(m, ry)
    float2* acol;    // level 1: [kMaxCand][KB]
    float2* bcol;    // level 1: [KB]
    float2 *t4h, *t4r, *rtw, *phH, *phW, *R;
    float *gP, *gM, *gpart;
    int *pslot, *qslot;
    float *rv, *rs, *xf, *cv, *cd;
    int *rj, *xi, *misc, *cj, *gj;
};

__host__ __device__ inline size_t mal(size_t x) { return (x + 15) / 16 * 16; }

// sizes of the small arrays, in carve order
__host__ __device__ inline size_t mix_small_bytes(const MixPlan& p) {
    size_t s = 0;
    s += mal(sizeof(float2) * p.H) + mal(sizeof(float2) * p.L) + mal(sizeof(float2) * (p.L / 2 + 1)) +
         mal(sizeof(float2) * p.H) + mal(sizeof(float2) * p.W) + mal(sizeof(float2) * p.KB);
    s += 4 * mal(sizeof(float) * p.TX);
    s += 2 * mal(sizeof(int) * p.Hh);
    s += 3 * mal(sizeof(float) * 32) + 2 * mal(sizeof(float) * kMaxCand);
    s += mal(sizeof(int) * 32) + mal(sizeof(int) * 32) + mal(sizeof(int) * 16) + 2 * mal(sizeof(int) * kMaxCand);
    return s;
}

__host__ __device__ inline MixSh mix_carve(const MixPlan& p, unsigned char* base) {
    MixSh s;
    s.X = (float2*)base;
    unsigned char* w = base + p.off_w;
    s.Y = (float2*)w;
    s.SG = (float2*)(w + mal(sizeof(float2) * (size_t)p.H * p.KB));
    s.CE = (float4*)w;
    const int TCp = (p.TC + kTM - 1) / kTM * kTM;
    s.PS = (float4*)(w + mal(sizeof(float4) * (size_t)TCp * p.KB));
    s.TBs = (float2*)s.PS;
    s.gy = (float2*)w;
    s.fy = s.gy + mal(sizeof(float2) * p.Hh) / sizeof(float2);
    s.acol = s.fy + (size_t)kMaxCand * p.Hh;
    s.bcol = s.acol + (size_t)kMaxCand * p.KB;
    unsigned char* m = base + p.off_small;
    auto take = [&](size_t bytes) { unsigned char* r = m; m += mal(bytes); return r; };
    s.t4h = (float2*)take(sizeof(float2) * p.H);
    s.t4r = (float2*)take(sizeof(float2) * p.L);
    s.rtw = (float2*)take(sizeof(float2) * (p.L / 2 + 1));
    s.phH = (float2*)take(sizeof(float2) * p.H);
    s.phW = (float2*)take(sizeof(float2) * p.W);
    s.R = (float2*)take(sizeof(float2) * p.KB);
    s.gP = (float*)take(sizeof(float) * p.TX);
    s.gM = (float*)take(sizeof(float) * p.TX);
    s.gpart = (float*)take(sizeof(float) * 2 * p.TX);
    s.pslot = (int*)take(sizeof(int) * p.Hh);
    s.qslot = (int*)take(sizeof(int) * p.Hh);
    s.rv = (float*)take(sizeof(float) * 32);
    s.rs = (float*)take(sizeof(float) * 32);
    s.xf = (float*)take(sizeof(float) * 32);
    s.cv = (float*)take(sizeof(float) * kMaxCand);
    s.cd = (float*)take(sizeof(float) * kMaxCand);
    s.rj = (int*)take(sizeof(int) * 32);
    s.xi = (int*)take(sizeof(int) * 32);
    s.misc = (int*)take(sizeof(int) * 16);
    s.cj = (int*)take(sizeof(int) * kMaxCand);
    s.gj = (int*)take(sizeof(int) * kMaxCand);
    return s;
}

__device__ __forceinline__ float2 ldg2(const float2* p) { return __ldg(p); }
__device__ __forceinline__ float4 ldg4(const float2* p) { return __ldg(reinterpret_cast<const float4*>(p)); }

// e^{i pi x}
__device__ __forceinline__ float2 expipi(float x) {
    float s, c;
    sincospif(x, &s, &c);
    return make_float2(c, s);
}
// E(a) - E(b) for E(n) = e^{2 pi i n / D}: 2i sin(pi (a - b)/D) e^{i pi (a + b)/D}
__device__ __forceinline__ float2 ediff(long long a, long long b, long long D) {
    long long dm = (a - b) % (2 * D), sm = (a + b) % (2 * D);
    const float s = sinpif((float)dm / (float)D);
    const float2 e = expipi((float)sm / (float)D);
    return make_float2(-2.f * s * e.y, 2.f * s * e.x);
}
__device__ __forceinline__ float2 eat(long long a, long long D) { return expipi((float)((2 * a) % (2 * D)) / (float)D); }

template <int H, int W, int CL>
struct Geo {
    static constexpr int L = W / 2, Wc = L + 1, Hh = H / 2, RH = H / CL;
    static constexpr int KB = (Wc + CL - 1) / CL;
    static constexpr int N1h = MSplit<H>::N1, N2h = MSplit<H>::N2, N1r = MSplit<L>::N1, N2r = MSplit<L>::N2;
    static constexpr int RSG = mix_padded_len<L>();
    static_assert(N2h > 1 && N2r > 1, "two-pass lengths only");
};

    // Level 2: the candidates S.gj[0, nc) re-evaluated from a double-float product
    // spectrum (about 48 significant bits) computed here: the forward transforms of the
    // rows and the band's columns in double-float into [0, off_small) (the FP32 band and
    // the work area are no longer needed), then per candidate the double-float kernel's
    // own sums, cu(j) = sum_kx g Re[e^{2 pi i kx' qx/(uW)} sum_ky X(ky, kx) e^{2 pi i ky' qy/(uH)}],
    // qy = py u + ty, qx = px u + tx (the y-Nyquist row through its real part in the
    // folded columns). Returns the winner's slot in S.gj and its raw value, or -1 when the
    // two best are within 2^-36 sum g|X| (a tie in all but name: the fallback decides it
    // exactly as the double-float kernel does everywhere). With `integer` the candidates are
    // integer shifts (flat indices y W + x) and the values those of the integer surface.
template <int H, int W, int CL>
__device__ __forceinline__ int mix_level2(const MixArgs& a, const MixSh& S, unsigned char* mix_smem, const GenItem& it,
                                          const dfc* Fb, int nc, int py, int px, float scale, double* vbest,
                                          bool integer) {
    using Gm = Geo<H, W, CL>;
    constexpr int L = Gm::L, Wc = Gm::Wc, RH = Gm::RH, KB = Gm::KB;
    constexpr int N1h = Gm::N1h, N2h = Gm::N2h, N1r = Gm::N1r, N2r = Gm::N2r, RSG = Gm::RSG;
    constexpr int NP = L / 2 + 1;
    constexpr int kNT = mix_threads(H, W);
    const MixPlan& P = a.p;
    const int rank = Clu<CL>::rank(), tid = threadIdx.x;
    const int b0 = rank * KB, nb = min(KB, Wc - b0), row0 = rank * RH;
    const int M = P.M, h0 = P.h0;
    const float sense = P.sense;
    const int elem = P.in_dtype == 0 ? 2 : 4;
    const char* frame = (const char*)it.frame;
        dfc* Xd = reinterpret_cast<dfc*>(mix_smem);
        dfc* Sd = reinterpret_cast<dfc*>(mix_smem + P.off_l2s);
        df* cs = reinterpret_cast<df*>(mix_smem + P.off_l2c);
        const int G2 = P.G2;
        Clu<CL>::sync();
        for (int g0 = 0; g0 < RH; g0 += G2) {
            const char* rbase = frame + (size_t)(row0 + g0) * it.pitch * elem;
            for (int i = tid; i < G2 * L; i += kNT) {
                const int s2 = i / L, n = i - s2 * L;
                const long long o = (long long)s2 * it.pitch + 2 * n;
                float i0, i1;
                if (elem == 2) {
                    i0 = (float)__ldg((const unsigned short*)rbase + o);
                    i1 = (float)__ldg((const unsigned short*)rbase + o + 1);
                } else {
                    i0 = __ldg((const float*)rbase + o);
                    i1 = __ldg((const float*)rbase + o + 1);
                }
                df d0 = df_make(i0), d1 = df_make(i1);
                if (P.method != 0) {                      // (I + eps)^2, exactly formed
                    float sh, sl;
                    two_sum(i0, P.eps, sh, sl);
                    d0 = df_mul(df{sh, sl}, df{sh, sl});
                    two_sum(i1, P.eps, sh, sl);
                    d1 = df_mul(df{sh, sl}, df{sh, sl});
                }
                Sd[s2 * RSG + mix_phys<L>(n)] = dfc{d0, d1};
            }
            __syncthreads();
            fwd_pass_s<N1r, N2r, false, kNT>(
                G2, P.t4r_d, [&](int s2, int n2, int n1) { return Sd[s2 * RSG + mix_phys<L>(N2r * n1 + n2)]; },
                [&](int s2, int n2, int k1, dfc v) { Sd[s2 * RSG + mix_phys<L>(N2r * k1 + n2)] = v; });
            __syncthreads();
            fwd_pass_c<N1r, N2r, false, kNT>(
                G2, [&](int s2, int k1, int n2) { return Sd[s2 * RSG + mix_phys<L>(N2r * k1 + n2)]; },
                [&](int s2, int k1, int k2, dfc v) { Sd[s2 * RSG + mix_phys<L>(N2r * k1 + k2)] = v; });
            __syncthreads();
            for (int task = tid; task < G2 * NP; task += kNT) {
                const int s2 = task / NP, k = task - s2 * NP, y = row0 + g0 + s2;
                const dfc* zr = Sd + s2 * RSG;
                const dfc zk = zr[mix_phys<L>(mix_pos<L>(k))];
                auto put = [&](int kx, dfc v) {
                    const int r = kx / KB;
                    Clu<CL>::at(Xd, r)[y * KB + (kx - r * KB)] = v;
                };
                const df zero{0.f, 0.f};
                if (k == 0) {
                    put(0, dfc{df_add_abs(zk.re, zk.im), zero});
                    put(L, dfc{df_add_abs(zk.re, df_neg(zk.im)), zero});
                } else {
                    const dfc zm = zr[mix_phys<L>(mix_pos<L>(L - k))];
                    const dfc fe = {df_scale(df_add_abs(zk.re, zm.re), 0.5f), df_scale(df_add_abs(zk.im, df_neg(zm.im)), 0.5f)};
                    const dfc fo = {df_scale(df_add_abs(zk.im, zm.im), 0.5f), df_scale(df_add_abs(zm.re, df_neg(zk.re)), 0.5f)};
                    const dfc rt = *reinterpret_cast<const dfc*>(P.rtw_d + k);
                    const dfc t = cmul(rt, fo);
                    put(k, cadd(fe, t));
                    if (2 * k != L) put(L - k, cconj(csub(fe, t)));
                }
            }
            __syncthreads();
        }
        Clu<CL>::sync();
        fwd_pass_s<N1h, N2h, true, kNT>(
            nb, P.t4h_d, [&](int c, int n2, int n1) { return Xd[(N2h * n1 + n2) * KB + c]; },
            [&](int c, int n2, int k1, dfc v) { Xd[(N2h * k1 + n2) * KB + c] = v; });
        __syncthreads();
        fwd_pass_c<N1h, N2h, true, kNT>(
            nb, [&](int c, int k1, int n2) { return Xd[(N2h * k1 + n2) * KB + c]; },
            [&](int c, int k1, int k2, dfc v) {
                const int ky = k1 + N1h * k2, kx = b0 + c;
                const float4 f = __ldg(reinterpret_cast<const float4*>(Fb + (size_t)ky * Wc + kx));
                Xd[(N2h * k1 + k2) * KB + c] = cmul(v, dfc{df{f.x, f.y}, df{-f.z, -f.w}});
            });
        __syncthreads();
        // per (candidate, column): the double-float kernel's column sum and x-phase
        const long long DH = (long long)P.u * H, DW = (long long)P.u * W;
        for (int e = tid; e < nc * nb; e += kNT) {
            const int k = e / nb, c = e - k * nb, kx = b0 + c, j = S.gj[k];
            const bool folded = kx != 0 && kx != L;
            long long qy, qx;
            if (integer) {                        // j = y W + x: the shift (y, x), wrapped, t = 0
                const int y = j / W, x = j - (j / W) * W;
                qy = (long long)(y > H / 2 ? y - H : y) * P.u;
                qx = (long long)(x > W / 2 ? x - W : x) * P.u;
            } else {
                qy = (long long)py * P.u + j / M - h0;
                qx = (long long)px * P.u + j % M - h0;
            }
            dfc acc = {df{0.f, 0.f}, df{0.f, 0.f}};
            for (int ky = 0; ky < H; ++ky) {
                const long long ks = 2 * ky >= H ? ky - H : ky;
                long long m = (ks * qy) % DH;
                if (m < 0) m += DH;
                const float4 ev = __ldg(reinterpret_cast<const float4*>(P.uHd + m));
                dfc ey = {df{ev.x, ev.y}, df{ev.z, ev.w}};
                if (2 * ky == H && folded) ey.im = df{0.f, 0.f};
                acc = cadd(acc, cmul(Xd[mix_pos<H>(ky) * KB + c], ey));
            }
            long long mx = ((long long)(kx == L ? -L : kx) * qx) % DW;
            if (mx < 0) mx += DW;
            const float4 xv = __ldg(reinterpret_cast<const float4*>(P.uWd + mx));
            df re = df_add_abs(df_mul(acc.re, df{xv.x, xv.y}), df_neg(df_mul(acc.im, df{xv.z, xv.w})));
            if (folded) re = df_scale(re, 2.f);
            cs[e] = re;
        }
        __syncthreads();
        {
            const int lane = tid & 31, wid = tid >> 5;
            for (int k = wid; k < nc; k += kNT / 32) {
                if (lane == 0) {
                    df sum{0.f, 0.f};
                    for (int c = 0; c < nb; ++c) sum = df_add_abs(sum, cs[k * nb + c]);
                    S.cv[k] = sum.hi;
                    S.cd[k] = sum.lo;
                }
            }
        }
        Clu<CL>::sync();
        int kb = -1;
        double bv = -INFINITY, second = -INFINITY;
        for (int k = 0; k < nc; ++k) {
            df tot{0.f, 0.f};
            for (int r = 0; r < CL; ++r)
                tot = df_add_abs(tot, df{Clu<CL>::at(S.cv, r)[k], Clu<CL>::at(S.cd, r)[k]});
            const double v = (double)sense * df_to_double(tot);
            if (kb < 0 || v > bv || (v == bv && S.gj[k] < S.gj[kb])) {
                second = bv;
                bv = v;
                kb = k;
            } else if (v > second) {
                second = v;
            }
        }
        Clu<CL>::sync();                                   // the partial sums are read
        *vbest = (double)sense * bv;
        return (bv - second > 0x1p-36 * (double)scale) ? kb : -1;
    }

// The 256-pixel kernel calls it out of line: its 16-point double-float DFTs do not fit
// beside the main loop's registers. The smaller sides inline it, which spills nothing.
template <int H, int W, int CL>
__device__ __noinline__ int mix_level2_call(const MixArgs& a, const MixSh& S, unsigned char* mix_smem,
                                            const GenItem& it, const dfc* Fb, int nc, int py, int px, float scale,
                                            double* vbest, bool integer) {
    return mix_level2<H, W, CL>(a, S, mix_smem, it, Fb, nc, py, px, scale, vbest, integer);
}

template <int H, int W, int CL>
__global__ void __launch_bounds__(mix_threads(H, W), mix_min_ctas(H, W)) __cluster_dims__(CL, 1, 1)
    mix_track_kernel(const MixArgs a) {
    constexpr int kNT = mix_threads(H, W);
    using Gm = Geo<H, W, CL>;
    constexpr int L = Gm::L, Wc = Gm::Wc, Hh = Gm::Hh, RH = Gm::RH, KB = Gm::KB;
    constexpr int N1h = Gm::N1h, N2h = Gm::N2h, N1r = Gm::N1r, N2r = Gm::N2r, RSG = Gm::RSG;
    constexpr int NP = L / 2 + 1;
    extern __shared__ __align__(16) unsigned char mix_smem[];
    const MixPlan& P = a.p;
    const MixSh S = mix_carve(P, mix_smem);
    const int rank = Clu<CL>::rank();
    const int b0 = rank * KB, nb = min(KB, Wc - b0);
    const int row0 = rank * RH;
    const int G = P.G;
    const int tid = threadIdx.x;

    // frame-independent tables -> shared memory
    for (int i = tid; i < H; i += kNT) { S.t4h[i] = ldg2(P.t4h + i); S.phH[i] = ldg2(P.phH + i); }
    for (int i = tid; i < L; i += kNT) S.t4r[i] = ldg2(P.t4r + i);
    for (int i = tid; i < NP; i += kNT) S.rtw[i] = ldg2(P.rtw + i);
    for (int i = tid; i < W; i += kNT) S.phW[i] = ldg2(P.phW + i);
    for (int i = tid; i < Hh; i += kNT) {
        S.pslot[i] = mix_pos<H>(i + 1);
        S.qslot[i] = mix_pos<H>((H - i - 1) % H);
    }
    const float sense = P.sense;

    for (;;) {
        // next item: rank 0 takes it and hands it to every CTA of the cluster
        Clu<CL>::sync();
        if (rank == 0 && tid == 0) {
            const int v = (int)atomicAdd(a.next, 1u);
            for (int r = 0; r < CL; ++r) Clu<CL>::at(S.misc, r)[0] = v;
        }
        Clu<CL>::sync();
        const long long idx = S.misc[0];
        if (idx >= a.n - (long long)(gridDim.x / CL)) pdl_trigger();      // the last wave
        if (idx >= a.n) break;
        GenItem it;
        if (a.items) {
            it = a.items[a.first + idx];
        } else {
            it.frame = (const char*)a.frames + idx * a.frame_bytes;
            it.pitch = a.pitch;
            it.out_index = idx;
            it.plan = a.plan;
            it.ref = a.ref;
        }
        const dfc* Fb = a.refs[it.ref];
        // a per-ROI reference is cold in L2 and the product step reads it after the row
        // FFTs: each CTA of the cluster prefetches its share of the rows
        if (tid == 0) prefetch_l2(Fb + (size_t)row0 * Wc, (size_t)RH * Wc * sizeof(dfc));
        const int elem = P.in_dtype == 0 ? 2 : 4;
        const char* frame = (const char*)it.frame;
        const bool vec = ((uintptr_t)frame % 16 == 0) && ((it.pitch * elem) % 16 == 0) && ((W * elem) % 16 == 0);
        float* dbg_int = a.dbg_int ? a.dbg_int + (size_t)idx * H * W : nullptr;
        float* dbg_sub = a.dbg_sub ? a.dbg_sub + (size_t)idx * P.M * P.M : nullptr;
        auto opnd = [&](float I) {
            if (P.method == 0) return I;
            const float ip = I + P.eps;
            return ip * ip;
        };
        auto to_owner = [&](int y, int kx, float2 v) {
            const int r = kx / KB;
            Clu<CL>::at(S.X, r)[y * KB + (kx - r * KB)] = v;
        };

        // ---- a1-a3: the product spectrum X in the bands (sabs: this thread's part of sum g|X|)
        float sabs = 0.f;
        auto forward = [&]() {
        // a1-a2: rows -> half spectra in the owners' bands
        for (int g0 = 0; g0 < RH; g0 += G) {
            const char* rbase = frame + (size_t)(row0 + g0) * it.pitch * elem;
            if (vec && elem == 2) {
                constexpr int NV = L / 4;                       // uint4 = 8 pixels = 4 complex samples
                for (int i = tid; i < G * NV; i += kNT) {
                    const int s = i / NV, q = i - s * NV;
                    const uint4 v = __ldg((const uint4*)(rbase + (size_t)s * it.pitch * 2) + q);
                    const unsigned w4[4] = {v.x, v.y, v.z, v.w};
                    float2* zr = S.SG + s * RSG;
#pragma unroll
                    for (int k = 0; k < 4; ++k)
                        zr[mix_phys<L>(4 * q + k)] = make_float2(opnd((float)(w4[k] & 0xffffu)), opnd((float)(w4[k] >> 16)));
                }
            } else if (vec) {
                constexpr int NV = L / 2;                       // float4 = 4 pixels = 2 complex samples
                for (int i = tid; i < G * NV; i += kNT) {
                    const int s = i / NV, q = i - s * NV;
                    const float4 v = __ldg((const float4*)(rbase + (size_t)s * it.pitch * 4) + q);
                    float2* zr = S.SG + s * RSG;
                    zr[mix_phys<L>(2 * q)] = make_float2(opnd(v.x), opnd(v.y));
                    zr[mix_phys<L>(2 * q + 1)] = make_float2(opnd(v.z), opnd(v.w));
                }
            } else {
                for (int i = tid; i < G * L; i += kNT) {
                    const int s = i / L, n = i - s * L;
                    const long long o = (long long)s * it.pitch + 2 * n;
                    float a0, a1;
                    if (elem == 2) {
                        a0 = (float)__ldg((const unsigned short*)rbase + o);
                        a1 = (float)__ldg((const unsigned short*)rbase + o + 1);
                    } else {
                        a0 = __ldg((const float*)rbase + o);
                        a1 = __ldg((const float*)rbase + o + 1);
                    }
                    S.SG[s * RSG + mix_phys<L>(n)] = make_float2(opnd(a0), opnd(a1));
                }
            }
            __syncthreads();
            fwd_pass_s<N1r, N2r, false, kNT>(
                G, S.t4r, [&](int s, int n2, int n1) { return S.SG[s * RSG + mix_phys<L>(N2r * n1 + n2)]; },
                [&](int s, int n2, int k1, float2 v) { S.SG[s * RSG + mix_phys<L>(N2r * k1 + n2)] = v; });
            __syncthreads();
            fwd_pass_c<N1r, N2r, false, kNT>(
                G, [&](int s, int k1, int n2) { return S.SG[s * RSG + mix_phys<L>(N2r * k1 + n2)]; },
                [&](int s, int k1, int k2, float2 v) { S.SG[s * RSG + mix_phys<L>(N2r * k1 + k2)] = v; });
            __syncthreads();
            // even/odd split: A(k) = Fe + w^k Fo, A(L - k) = conj(Fe - w^k Fo), A(0), A(L) real
            for (int task = tid; task < G * NP; task += kNT) {
                const int s = task / NP, k = task - s * NP, y = row0 + g0 + s;
                const float2* zr = S.SG + s * RSG;
                const float2 zk = zr[mix_phys<L>(mix_pos<L>(k))];
                if (k == 0) {
                    to_owner(y, 0, make_float2(zk.x + zk.y, 0.f));
                    to_owner(y, L, make_float2(zk.x - zk.y, 0.f));
                } else {
                    const float2 zm = zr[mix_phys<L>(mix_pos<L>(L - k))];
                    const float2 fe = make_float2(0.5f * (zk.x + zm.x), 0.5f * (zk.y - zm.y));
                    const float2 fo = make_float2(0.5f * (zk.y + zm.y), -0.5f * (zk.x - zm.x));
                    const float2 t = cmul(S.rtw[k], fo);
                    to_owner(y, k, cadd(fe, t));
                    if (2 * k != L) to_owner(y, L - k, cconj(csub(fe, t)));
                }
            }
            __syncthreads();
        }
        Clu<CL>::sync();

        // a3: column FFTs over the band, product with conj F[b]
        fwd_pass_s<N1h, N2h, true, kNT>(
            nb, S.t4h, [&](int c, int n2, int n1) { return S.X[(N2h * n1 + n2) * KB + c]; },
            [&](int c, int n2, int k1, float2 v) { S.X[(N2h * k1 + n2) * KB + c] = v; });
        __syncthreads();
        sabs = 0.f;
        fwd_pass_c<N1h, N2h, true, kNT>(
            nb, [&](int c, int k1, int n2) { return S.X[(N2h * k1 + n2) * KB + c]; },
            [&](int c, int k1, int k2, float2 v) {
                const int ky = k1 + N1h * k2, kx = b0 + c;
                const float4 f = __ldg(reinterpret_cast<const float4*>(Fb + (size_t)ky * Wc + kx));
                const float2 x = cmul(v, make_float2(f.x, -f.z));
                S.X[(N2h * k1 + k2) * KB + c] = x;
                sabs += (kx == 0 || kx == L ? 1.f : 2.f) * (fabsf(x.x) + fabsf(x.y));
            });
        __syncthreads();
        };
        forward();

        // ---- a4: inverse columns (X -> Y), then inverse rows scanned for the extremum
        inv_pass_c<N1h, N2h, true, kNT>(
            nb, S.t4h, [&](int c, int k1, int k2) { return S.X[(N2h * k1 + k2) * KB + c]; },
            [&](int c, int k1, int n2, float2 v) { S.Y[(N2h * k1 + n2) * KB + c] = v; });
        __syncthreads();
        inv_pass_s<N1h, N2h, true, kNT>(
            nb, [&](int c, int n2, int k1) { return S.Y[(N2h * k1 + n2) * KB + c]; },
            [&](int c, int n2, int n1, float2 v) { S.Y[(N2h * n1 + n2) * KB + c] = v; });
        Clu<CL>::sync();
        // the CTA's rows of HW c(y, x), each value handed to visit(value, flat index)
        auto inverse_rows = [&](auto&& visit) {
        for (int g0 = 0; g0 < RH; g0 += G) {
            for (int task = tid; task < G * NP; task += kNT) {
                const int s = task / NP, k = task - s * NP, y = row0 + g0 + s;
                auto yat = [&](int kx) {
                    const int r = kx / KB;
                    return Clu<CL>::at(S.Y, r)[y * KB + (kx - r * KB)];
                };
                float2* zr = S.SG + s * RSG;
                if (k == 0) {
                    const float a0 = yat(0).x, aL = yat(L).x;
                    zr[mix_phys<L>(mix_pos<L>(0))] = make_float2(a0 + aL, a0 - aL);
                } else {
                    // Z(k) = [A(k) + conj A(L-k)] + i e^{2 pi i k/W} [A(k) - conj A(L-k)]
                    const float2 ak = yat(k), am = yat(L - k), wk = S.rtw[k];
                    const float2 s1 = cadd(ak, cconj(am)), d1 = csub(ak, cconj(am));
                    const float2 t1 = cmul(cconj(wk), d1);
                    zr[mix_phys<L>(mix_pos<L>(k))] = make_float2(s1.x - t1.y, s1.y + t1.x);
                    if (2 * k != L) {
                        const float2 s2 = cadd(am, cconj(ak)), d2 = csub(am, cconj(ak));
                        const float2 t2v = cmul(make_float2(-wk.x, -wk.y), d2);
                        zr[mix_phys<L>(mix_pos<L>(L - k))] = make_float2(s2.x - t2v.y, s2.y + t2v.x);
                    }
                }
            }
            __syncthreads();
            inv_pass_c<N1r, N2r, false, kNT>(
                G, S.t4r, [&](int s, int k1, int k2) { return S.SG[s * RSG + mix_phys<L>(N2r * k1 + k2)]; },
                [&](int s, int k1, int n2, float2 v) { S.SG[s * RSG + mix_phys<L>(N2r * k1 + n2)] = v; });
            __syncthreads();
            inv_pass_s<N1r, N2r, false, kNT>(
                G, [&](int s, int n2, int k1) { return S.SG[s * RSG + mix_phys<L>(N2r * k1 + n2)]; },
                [&](int s, int n2, int n1, float2 v) {
                    const int y = row0 + g0 + s, x = 2 * (n2 + N2r * n1), fe = y * W + x;
                    visit(v.x, fe);
                    visit(v.y, fe + 1);
                });
            __syncthreads();
        }
        };
        Best2 t2;
        t2.init();
        inverse_rows([&](float v, int fe) {
            if (dbg_int) dbg_int[fe] = v;
            t2.push(sense * v, fe);
        });
        // a5: the integer extremum and the spectral scale over the cluster
        float v1 = t2.v1;
        int best = t2.j1;
        float scale = block_argmax_sum(v1, best, sabs, S.rv, S.rj, S.rs);
        if constexpr (CL > 1) {
            if (tid == 0) { S.xf[0] = v1; S.xf[1] = scale; S.xi[0] = best; }
            Clu<CL>::sync();
            float bv = -INFINITY, sc = 0.f;
            int bj = INT_MAX;
            for (int r = 0; r < CL; ++r) {
                const float* xf = Clu<CL>::at(S.xf, r);
                const int j = Clu<CL>::at(S.xi, r)[0];
                if (better(xf[0], j, bv, bj)) { bv = xf[0]; bj = j; }
                sc += xf[1];
            }
            v1 = bv;
            best = bj;
            scale = sc;
        }
        const float tau_i = P.tau_int * scale;
        int near = __syncthreads_count((t2.v1 >= v1 - tau_i && t2.j1 != best) || t2.v2 >= v1 - tau_i);
        if constexpr (CL > 1) {
            if (tid == 0) S.xi[1] = near;
            Clu<CL>::sync();
            near = 0;
            for (int r = 0; r < CL; ++r) near += Clu<CL>::at(S.xi, r)[1];
        }
        auto to_fallback = [&]() {
            if (rank == 0 && tid == 0) {
                const unsigned s = atomicAdd(a.fb_count, 1u);
                a.fb[s] = it;
            }
        };
        if (!(v1 > -INFINITY) || !(scale < INFINITY)) {
            to_fallback();
            continue;
        }
        float c0 = sense * v1;                               // HW c(p)
        unsigned iflags = 0;
        if (near > 0 && !dbg_sub) {
            // integer near-ties: every shift within tau_int of the best, evaluated from the
            // double-float spectrum (the interpolant at a whole-pixel offset is the integer
            // surface), then the FP32 spectrum again for the sub-pixel stage
            if (tid == 0) S.misc[2] = 0;
            __syncthreads();
            const float thr_i = v1 - tau_i;
            inverse_rows([&](float v, int fe) {
                if (sense * v >= thr_i) {
                    const int slot = atomicAdd(&S.misc[2], 1);
                    if (slot < kMaxCand) S.cj[slot] = fe;
                }
            });
            int ni = S.misc[2];
            if constexpr (CL > 1) {
                Clu<CL>::sync();
                ni = 0;
                for (int r = 0; r < CL; ++r) ni += Clu<CL>::at(S.misc, r)[2];
                if (tid == 0 && ni <= kMaxCand) {
                    int n = 0;
                    for (int r = 0; r < CL; ++r) {
                        const int cnt = Clu<CL>::at(S.misc, r)[2];
                        const int* cj = Clu<CL>::at(S.cj, r);
                        for (int k = 0; k < cnt; ++k) S.gj[n++] = cj[k];
                    }
                }
            } else {
                for (int k = tid; k < ni && ni <= kMaxCand; k += kNT) S.gj[k] = S.cj[k];
            }
            __syncthreads();
            if (ni > kMaxCand || ni < 1) {
                to_fallback();
                continue;
            }
            double vi = 0.0;
            int ki;
            if constexpr (H >= 256) ki = mix_level2_call<H, W, CL>(a, S, mix_smem, it, Fb, ni, 0, 0, scale, &vi, true);
            else ki = mix_level2<H, W, CL>(a, S, mix_smem, it, Fb, ni, 0, 0, scale, &vi, true);
            if (ki < 0) {
                to_fallback();
                continue;
            }
            best = S.gj[ki];
            c0 = (float)vi;
            iflags = 0x01u;
            forward();
        }
        const int iy = best / W, ix = best - (best / W) * W;
        const int py = iy > H / 2 ? iy - H : iy, px = ix > W / 2 ? ix - W : ix;
        const int pyy = iy, pxx = ix;

        // ---- a6 prologue: X' and P/Q in place, R(kx), gsum(+-tx)
        for (int task = tid; task < (Hh + 1) * nb; task += kNT) {
            const int m = task / nb, c = task - m * nb, kx = b0 + c;
            const float2 ex = S.phW[(kx * pxx) % W];
            if (m == 0) {
                float2* p0 = S.X + mix_pos<H>(0) * KB + c;
                *p0 = cmul(*p0, ex);
            } else if (m == Hh) {
                float2* ph = S.X + mix_pos<H>(Hh) * KB + c;
                *ph = cmul(*ph, cmul(S.phH[(Hh * pyy) % H], ex));
            } else {
                float2* pp = S.X + mix_pos<H>(m) * KB + c;
                float2* pm = S.X + mix_pos<H>(H - m) * KB + c;
                const float2 xp = cmul(*pp, cmul(S.phH[(m * pyy) % H], ex));
                const float2 xm = cmul(*pm, cmul(S.phH[((H - m) * pyy) % H], ex));
                *pp = cadd(xp, xm);
                *pm = csub(xp, xm);
            }
        }
        __syncthreads();
        for (int c = tid; c < nb; c += kNT) {
            float2 r = S.X[mix_pos<H>(0) * KB + c];
            for (int i = 0; i < Hh; ++i) r = cadd(r, S.X[S.pslot[i] * KB + c]);
            S.R[c] = r;
        }
        __syncthreads();
        const int TX = P.TX;
        for (int tx = tid; tx < TX; tx += kNT) {
            float gp = 0.f, gm = 0.f;
            for (int c = 0; c < nb; ++c) {
                const int kx = b0 + c;
                const float gc = __ldg(P.tG + (size_t)kx * P.TXp + tx), ws = ldg2(P.tB + (size_t)kx * P.TXp + tx).y;
                const float2 r = S.R[c];
                const float u1 = gc * r.x, u2 = ws * r.y;
                gp += u1 - u2;
                gm += u1 + u2;
            }
            S.gpart[tx] = gp;
            S.gpart[TX + tx] = gm;
        }
        Clu<CL>::sync();
        for (int tx = tid; tx < TX; tx += kNT) {
            float gp = 0.f, gm = 0.f;
            for (int r = 0; r < CL; ++r) {
                const float* gq = Clu<CL>::at(S.gpart, r);
                gp += gq[tx];
                gm += gq[TX + tx];
            }
            S.gP[tx] = gp;
            S.gM[tx] = gm;
        }
        __syncthreads();

        const int M = P.M, h0 = P.h0, pmax = P.pmax;
        // Level 1: d_k = v(j_k) - v(j1) for the candidates S.gj[0, nc) against j1 = jw, into
        // S.cv[k] (cluster totals): per column the sums over m against the factors
        // E(m, ty_k) - E(m, ry) and E(m, ry), then the sum over the band's kx against
        // E(kx, tx_k) and E(kx, tx_k) - E(kx, rx), g-weighted (the y-Nyquist rule as in stage A).
        auto pair_diffs = [&](int nc, int jw) {
            const long long DH = (long long)P.u * H, DW = (long long)P.u * W;
            const int ry = jw / M - h0, rx = jw % M - h0;
            // factors: gy(m) = E(m, ry), fy_k(m) = E(m, ty_k) - E(m, ry), m = i + 1
            for (int i = tid; i < Hh; i += kNT) S.gy[i] = eat((long long)(i + 1) * ry, DH);
            for (int e = tid; e < nc * Hh; e += kNT) {
                const int k = e / Hh, i = e - k * Hh, ty = S.gj[k] / M - h0;
                S.fy[e] = ediff((long long)(i + 1) * ty, (long long)(i + 1) * ry, DH);
            }
            __syncthreads();
            // column sums over m: acol_k = sum P Re fy + i Q Im fy, bcol = X'(0) + sum P Re gy + i Q Im gy
            for (int e = tid; e < (nc + 1) * nb; e += kNT) {
                const int k = e / nb, c = e - k * nb, kx = b0 + c;
                const float2* f = k < nc ? S.fy + (size_t)k * Hh : S.gy;
                float2 acc = k < nc ? make_float2(0.f, 0.f) : S.X[mix_pos<H>(0) * KB + c];
                for (int i = 0; i < Hh; ++i) {
                    const float2 p = S.X[S.pslot[i] * KB + c];
                    float2 q;
                    if (i < Hh - 1) q = S.X[S.qslot[i] * KB + c];
                    else q = kx == L ? make_float2(-p.x, -p.y) : make_float2(0.f, 0.f);
                    const float2 fv = f[i];
                    acc.x = fmaf(p.x, fv.x, fmaf(-q.y, fv.y, acc.x));
                    acc.y = fmaf(p.y, fv.x, fmaf(q.x, fv.y, acc.y));
                }
                if (k < nc) S.acol[(size_t)k * KB + c] = acc;
                else S.bcol[c] = acc;
            }
            __syncthreads();
            // d_k = sum_kx g Re[acol_k E(kx, tx_k) + bcol (E(kx, tx_k) - E(kx, rx))], one warp per candidate
            {
                const int lane = tid & 31, wid = tid >> 5;
                for (int k = wid; k < nc; k += kNT / 32) {
                    const int tx = S.gj[k] % M - h0;
                    float d = 0.f;
                    for (int c = lane; c < nb; c += 32) {
                        const int kx = b0 + c, ks = kx == L ? -L : kx;
                        const float2 ex = eat((long long)ks * tx, DW);
                        const float2 fx = ediff((long long)ks * tx, (long long)ks * rx, DW);
                        const float2 ac = S.acol[(size_t)k * KB + c], bc = S.bcol[c];
                        const float re = ac.x * ex.x - ac.y * ex.y + bc.x * fx.x - bc.y * fx.y;
                        d = fmaf(kx == 0 || kx == L ? 1.f : 2.f, re, d);
                    }
                    d = warp_sum(d);
                    if (lane == 0) S.cd[k] = d;
                }
            }
            if constexpr (CL > 1) {
                Clu<CL>::sync();
                for (int k = tid; k < nc; k += kNT) {
                    float d = 0.f;
                    for (int r = 0; r < CL; ++r) d += Clu<CL>::at(S.cd, r)[k];
                    S.cv[k] = d;
                }
            } else {
                __syncthreads();
                for (int k = tid; k < nc; k += kNT) S.cv[k] = S.cd[k];
            }
            __syncthreads();
        };
        // ---- a6: the contraction, chunk by chunk of t (skipped by the pair diagnostic)
        TopK<kTopK> top;
        top.init();
        // D(0, 0) = 0 is a candidate, so no point below -tau0 sum w|X| can matter. Each thread
        // raises that bound as it keeps points: no point below its best so far minus the
        // band can be within the band of the maximum. Twice the band keeps the raised bound,
        // rounding included, below the level-0 threshold applied later.
        const float lb = -P.tau0 * scale;
        float lb_run = lb;
        auto emit = [&](float D, int ty, int tx) {
            const int j = (ty + h0) * M + (tx + h0);
            if (dbg_sub) dbg_sub[j] = D;
            const float v = sense * D;
            if (v >= lb_run) {
                top.push(v, j);
                if (!dbg_sub) lb_run = fmaxf(lb_run, v + 2.f * lb);
            }
        };
        auto epilogue = [&](int t, int tx, float4 s) {
            if (t <= pmax) {
                if (tx <= pmax) emit(s.x - s.y + S.gP[tx], t, tx);
                if (tx >= 1) emit(s.x + s.y + S.gM[tx], t, -tx);
            }
            if (tx <= pmax) emit(s.z - s.w + S.gP[tx], -t, tx);
            if (tx >= 1) emit(s.z + s.w + S.gM[tx], -t, -tx);
        };
        if (rank == 0) {
            for (int tx = tid; tx < TX; tx += kNT) {
                if (tx <= pmax) emit(S.gP[tx], 0, tx);
                if (tx >= 1) emit(S.gM[tx], 0, -tx);
            }
        }
        const int TC = P.TC, TAp = P.TAp, TXp = P.TXp;
        const int ntx = (TX + 1) / 2;
        if (P.tbs) {
            // the stage-B table into shared memory (one CTA: the band is every column); the
            // barrier after stage A orders these stores before stage B reads them
            const float4* src = reinterpret_cast<const float4*>(P.tB);
            float4* dst = reinterpret_cast<float4*>(S.TBs);
            const int n4 = Wc * TXp / 2;
            for (int i = tid; i < n4; i += kNT) dst[i] = __ldg(src + i);
        }
        for (int t0 = 1; t0 <= (a.dbg_pairs ? 0 : h0); t0 += TC) {
            const int tcn = min(TC, h0 - t0 + 1), ntg = (tcn + kTM - 1) / kTM;
            // stage A: (C0, E0, C1, E1)(t, kx) for the band
            for (int task = tid; task < ntg * nb; task += kNT) {
                const int tg = task / nb, c = task - tg * nb, kx = b0 + c;
                float ur[kTM], ui[kTM], vr[kTM], vi[kTM];
#pragma unroll
                for (int r = 0; r < kTM; ++r) ur[r] = ui[r] = vr[r] = vi[r] = 0.f;
                const float2* ta = P.tA + (t0 - 1) + tg * kTM;
                for (int i = 0; i < Hh; ++i) {
                    const float2 p = S.X[S.pslot[i] * KB + c];
                    float2 q;
                    if (i < Hh - 1) q = S.X[S.qslot[i] * KB + c];
                    else q = kx == L ? make_float2(-p.x, -p.y) : make_float2(0.f, 0.f);
                    const float2* tr = ta + (size_t)i * TAp;
#pragma unroll
                    for (int r2 = 0; r2 < kTM / 2; ++r2) {
                        const float4 aa = ldg4(tr + 2 * r2);
                        ur[2 * r2] = fmaf(aa.x, p.x, ur[2 * r2]);
                        ui[2 * r2] = fmaf(aa.x, p.y, ui[2 * r2]);
                        vr[2 * r2] = fmaf(aa.y, q.x, vr[2 * r2]);
                        vi[2 * r2] = fmaf(aa.y, q.y, vi[2 * r2]);
                        ur[2 * r2 + 1] = fmaf(aa.z, p.x, ur[2 * r2 + 1]);
                        ui[2 * r2 + 1] = fmaf(aa.z, p.y, ui[2 * r2 + 1]);
                        vr[2 * r2 + 1] = fmaf(aa.w, q.x, vr[2 * r2 + 1]);
                        vi[2 * r2 + 1] = fmaf(aa.w, q.y, vi[2 * r2 + 1]);
                    }
                }
#pragma unroll
                for (int r = 0; r < kTM; ++r)
                    S.CE[(tg * kTM + r) * KB + c] = make_float4(ur[r] - vi[r], ui[r] + vr[r], ur[r] + vi[r], ui[r] - vr[r]);
            }
            __syncthreads();
            // stage B: per (t, tx) the four sums over the band, the table entries from
            // `ldtb` (shared memory with p.tbs, else global memory)
            auto stage_b = [&](auto ldtb) {
            for (int task = tid; task < ntg * ntx; task += kNT) {
                const int tg = task / ntx, q = task - tg * ntx;
                const int txa = q, txb = q + ntx;
                float acc[kTM][2][4];
#pragma unroll
                for (int r = 0; r < kTM; ++r)
#pragma unroll
                    for (int h = 0; h < 2; ++h)
#pragma unroll
                        for (int e = 0; e < 4; ++e) acc[r][h][e] = 0.f;
                for (int c = 0; c < nb; ++c) {
                    const float2 ba = ldtb((size_t)c * TXp + txa), bb = ldtb((size_t)c * TXp + txb);
#pragma unroll
                    for (int r = 0; r < kTM; ++r) {
                        const float4 ce = S.CE[(tg * kTM + r) * KB + c];
                        acc[r][0][0] = fmaf(ce.x, ba.x, acc[r][0][0]);
                        acc[r][0][1] = fmaf(ce.y, ba.y, acc[r][0][1]);
                        acc[r][0][2] = fmaf(ce.z, ba.x, acc[r][0][2]);
                        acc[r][0][3] = fmaf(ce.w, ba.y, acc[r][0][3]);
                        acc[r][1][0] = fmaf(ce.x, bb.x, acc[r][1][0]);
                        acc[r][1][1] = fmaf(ce.y, bb.y, acc[r][1][1]);
                        acc[r][1][2] = fmaf(ce.z, bb.x, acc[r][1][2]);
                        acc[r][1][3] = fmaf(ce.w, bb.y, acc[r][1][3]);
                    }
                }
#pragma unroll
                for (int r = 0; r < kTM; ++r) {
                    const int lt = tg * kTM + r;
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const int tx = h ? txb : txa;
                        if (lt < tcn && tx < TX) {
                            const float4 s4 = make_float4(acc[r][h][0], acc[r][h][1], acc[r][h][2], acc[r][h][3]);
                            if constexpr (CL == 1) epilogue(t0 + lt, tx, s4);
                            else S.PS[lt * TX + tx] = s4;
                        }
                    }
                }
            }
            };
            if (P.tbs) {
                const float2* tbs = S.TBs;
                stage_b([&](size_t i) { return tbs[i]; });
            } else {
                const float2* tb = P.tB + (size_t)b0 * TXp;
                stage_b([&](size_t i) { return ldg2(tb + i); });
            }
            if constexpr (CL > 1) {
                Clu<CL>::sync();
                const int ne = tcn * TX, share = (ne + CL - 1) / CL;
                const int lo = rank * share, hi = min(ne, lo + share);
                for (int e = lo + tid; e < hi; e += kNT) {
                    float4 s4 = make_float4(0.f, 0.f, 0.f, 0.f);
                    for (int r = 0; r < CL; ++r) {
                        const float4 v = Clu<CL>::at(S.PS, r)[e];
                        s4.x += v.x; s4.y += v.y; s4.z += v.z; s4.w += v.w;
                    }
                    const int lt = e / TX;
                    epilogue(t0 + lt, e - lt * TX, s4);
                }
                Clu<CL>::sync();
            } else {
                __syncthreads();
            }
        }

        // ---- a7: level 0 -- the best point and its near-ties within tau0 (the pair
        // diagnostic instead takes its pair as the candidates, ja first, and stops after level 1)
        float vw = top.v[0];
        int jw = top.j[0];
        if (a.dbg_pairs) {
            vw = 0.f;
            jw = a.dbg_pairs[2 * idx];
        }
        block_argmax(vw, jw, S.rv, S.rj);
        if constexpr (CL > 1) {
            if (tid == 0) { S.xf[2] = vw; S.xi[2] = jw; }
            Clu<CL>::sync();
            float bv = -INFINITY;
            int bj = INT_MAX;
            for (int r = 0; r < CL; ++r) {
                const float v = Clu<CL>::at(S.xf, r)[2];
                const int j = Clu<CL>::at(S.xi, r)[2];
                if (better(v, j, bv, bj)) { bv = v; bj = j; }
            }
            vw = bv;
            jw = bj;
        }
        if (!(vw > -INFINITY)) {
            to_fallback();
            continue;
        }
        const float thr = vw - P.tau0 * scale;
        int nc = 0;
#pragma unroll
        for (int k = 0; k < kTopK; ++k) nc += __syncthreads_count(top.v[k] >= thr);
        int full = __syncthreads_or(top.v[kTopK - 1] >= thr);
        if (a.dbg_pairs) {
            nc = 2;
            full = 0;
        }
        if constexpr (CL > 1) {
            if (tid == 0) { S.xi[3] = nc; S.xi[4] = full; }
            Clu<CL>::sync();
            nc = 0;
            full = 0;
            for (int r = 0; r < CL; ++r) {
                nc += Clu<CL>::at(S.xi, r)[3];
                full |= Clu<CL>::at(S.xi, r)[4];
            }
        }
        unsigned flags = kRMixed | iflags;
        float dwin = 0.f;
        double raw_peak = NAN;                               // HW cu(winner) from level 2, if it ran
        if (nc > 1) {
            if (full || nc > kMaxCand) {
                to_fallback();
                continue;
            }
            // ---- level 1: exact pair differences d(j) = v(j) - v(j1) over the candidates
            flags |= 0x02u;
            if (tid == 0) S.misc[1] = 0;
            __syncthreads();
            if (a.dbg_pairs) {
                if (tid == 0 && rank == 0) {
                    S.cj[0] = a.dbg_pairs[2 * idx];
                    S.cj[1] = a.dbg_pairs[2 * idx + 1];
                    S.misc[1] = 2;
                }
            } else {
#pragma unroll
                for (int k = 0; k < kTopK; ++k)
                    if (top.v[k] >= thr) {
                        const int slot = atomicAdd(&S.misc[1], 1);
                        S.cj[slot] = top.j[k];
                    }
            }
            if constexpr (CL > 1) {
                Clu<CL>::sync();
                if (tid == 0) {
                    int n = 0;
                    for (int r = 0; r < CL; ++r) {
                        const int cnt = Clu<CL>::at(S.misc, r)[1];
                        const int* cj = Clu<CL>::at(S.cj, r);
                        for (int k = 0; k < cnt; ++k) S.gj[n++] = cj[k];
                    }
                }
            } else {
                __syncthreads();
                for (int k = tid; k < nc; k += kNT) S.gj[k] = S.cj[k];
            }
            __syncthreads();
            pair_diffs(nc, jw);
            if (a.dbg_pairs) {
                if (rank == 0 && tid == 0) a.dbg_d32[idx] = S.cv[1];
                continue;
            }
            // the winner must beat every other candidate by more than 2 tau1 sum g|X|
            int kb = -1;
            for (int k = 0; k < nc; ++k) {
                const float v = sense * S.cv[k];
                if (kb < 0 || better(v, S.gj[k], sense * S.cv[kb], S.gj[kb])) kb = k;
            }
            bool ok = true;
            const float need = 2.f * P.tau1 * scale;
            for (int k = 0; k < nc; ++k)
                if (k != kb && !(sense * (S.cv[kb] - S.cv[k]) > need)) ok = false;
            if (ok) {
                // d of j1 itself is exactly zero (its factors vanish), so S.cv[kb] is v(winner) - v(j1)
                jw = S.gj[kb];
                dwin = S.cv[kb];
            } else {
                double v2 = 0.0;
                int k2;
                if constexpr (H >= 256) k2 = mix_level2_call<H, W, CL>(a, S, mix_smem, it, Fb, nc, py, px, scale, &v2, false);
                else k2 = mix_level2<H, W, CL>(a, S, mix_smem, it, Fb, nc, py, px, scale, &v2, false);
                if (k2 < 0) {
                    to_fallback();
                    continue;
                }
                jw = S.gj[k2];
                flags |= 0x04u;
                raw_peak = v2;
            }
        }
        if (rank == 0 && tid == 0) {
            const int jy = jw / M, jx = jw % M;
            Result r;
            r.dy = (float)(((double)py * P.u + (jy - h0)) / P.u);
            r.dx = (float)(((double)px * P.u + (jx - h0)) / P.u);
            r.peak = raw_peak == raw_peak ? (float)(raw_peak / ((double)H * W)) : (c0 + sense * vw + dwin) / (float)(H * W);
            r.ipy = py;
            r.ipx = px;
            r.flags = flags;
            a.out[it.out_index] = r;
        }
    }
    pdl_wait();
}

template <int H, int W>
const void* kernel_for() {
    return (const void*)mix_track_kernel<H, W, mix_cluster(H, W)>;
}

}  // namespace mix

const void* mix_kernel_ptr(int H, int W) {
    if (H == 48 && W == 48) return mix::kernel_for<48, 48>();
    if (H == 96 && W == 96) return mix::kernel_for<96, 96>();
    if (H == 192 && W == 192) return mix::kernel_for<192, 192>();
    if (H == 256 && W == 256) return mix::kernel_for<256, 256>();
    if (H == 256 && W == 128) return mix::kernel_for<256, 128>();
    if (H == 128 && W == 256) return mix::kernel_for<128, 256>();
    return nullptr;
}

// ------------------------------------------------------------------ host: the plan
namespace {
constexpr double kPi = 3.14159265358979323846;
// e^{i 2 pi n / D} with n reduced exactly
void cexp2pi(long long n, long long D, double* c, double* s) {
    n %= D;
    if (n < 0) n += D;
    const double th = 2.0 * kPi * (double)n / (double)D;
    *c = std::cos(th);
    *s = std::sin(th);
}
// cos(2 pi n / D) - 1 = -2 sin^2(pi n / D), without cancellation
double cosm1_2pi(long long n, long long D) {
    n %= D;
    if (n < 0) n += D;
    const double h = std::sin(kPi * (double)n / (double)D);
    return -2.0 * h * h;
}
// the kernel's four-step split of length N (mix::MSplit), false if it has none
bool msplit(int N, int* n1, int* n2) {
    switch (N) {
#define CCST_SPLIT(n) case n: *n1 = mix::MSplit<n>::N1; *n2 = mix::MSplit<n>::N2; return true;
        CCST_SPLIT(24) CCST_SPLIT(48) CCST_SPLIT(64) CCST_SPLIT(96) CCST_SPLIT(128) CCST_SPLIT(192) CCST_SPLIT(256)
#undef CCST_SPLIT
        default: return false;
    }
}
// W_N^{n2 k1} laid out [k1][n2] for the split of N, through `put(c, s)`
template <class PUT>
bool pass_twiddles_n(int N, PUT put) {
    int n1 = 0, n2 = 0;
    if (!msplit(N, &n1, &n2)) return false;
    for (int k1 = 0; k1 < n1; ++k1)
        for (int j = 0; j < n2; ++j) {
            double c, s;
            cexp2pi(-(long long)j * k1, N, &c, &s);
            put(c, s);
        }
    return true;
}
// staged rows per group: the largest divisor of the CTA's row count up to 64 whose staging
// buffer stays within 36 KB
int staged_rows(int RH, int rsg) {
    int g = 0;
    for (int d = 1; d <= RH && d <= 64; ++d)
        if (RH % d == 0 && (size_t)d * rsg * sizeof(float2) <= 36 * 1024) g = d;
    return g;
}
}  // namespace

int mix_plan_create(int H, int W, int u, int method, int in_dtype, float eps, float tau_int, float tau0, float tau1,
                    int smem_optin, MixPlan* out, void** mem) {
    *mem = nullptr;
    if (!mix_shape_ok(H, W) || u < 1 || u > 256) return -1;
    MixPlan p{};
    p.H = H;
    p.W = W;
    p.L = W / 2;
    p.Wc = p.L + 1;
    p.Hh = H / 2;
    p.CL = mix_cluster(H, W);
    p.NT = mix::mix_threads(H, W);
    p.KB = (p.Wc + p.CL - 1) / p.CL;
    p.u = u;
    p.M = (3 * u + 1) / 2;
    p.h0 = p.M / 2;
    p.pmax = p.M - 1 - p.h0;
    p.TX = p.h0 + 1;
    p.method = method;
    p.in_dtype = in_dtype;
    p.eps = eps;
    p.sense = method == 1 ? -1.f : 1.f;
    p.tau_int = tau_int;
    p.tau0 = tau0;
    p.tau1 = tau1;
    p.RSX = p.KB;
    int n1r = 0, n2r = 0;
    if (!msplit(p.L, &n1r, &n2r) || !msplit(H, &n1r, &n2r)) return -1;
    msplit(p.L, &n1r, &n2r);
    p.RSG = n2r > 1 ? p.L + n1r : p.L;          // mix_padded_len of the half-row length
    p.G = staged_rows(H / p.CL, p.RSG);
    if (p.G < 1) return -1;
    p.G2 = 1;                                   // double-float staging: up to 8 rows per group
    for (int d = 1; d <= 8; ++d)
        if ((H / p.CL) % d == 0) p.G2 = d;
    // stage A reads 8 t entries per task from t' = t0 - 1 + 8 tg: one spare group of padding
    p.TAp = (p.h0 + mix::kTM - 1) / mix::kTM * mix::kTM + mix::kTM;
    p.TXp = 2 * ((p.TX + 1) / 2);
    // shared memory: band, work area (Y + staging | contraction chunk | level 1), small arrays
    const size_t band = mix::mal(sizeof(float2) * (size_t)H * p.KB);
    const size_t ysg = band + mix::mal(sizeof(float2) * (size_t)p.G * p.RSG);
    const size_t lvl1 = mix::mal(sizeof(float2) * p.Hh) + sizeof(float2) * ((size_t)kMaxCand * p.Hh + (size_t)kMaxCand * p.KB + p.KB);
    // the double-float level from offset 0: band, staging, per-(candidate, column) sums
    const size_t l2s = mix::mal(sizeof(dfc) * (size_t)H * p.KB);
    const size_t l2c = l2s + mix::mal(sizeof(dfc) * (size_t)p.G2 * p.RSG);
    const size_t lvl2 = l2c + sizeof(df) * (size_t)kMaxCand * p.KB;
    p.off_l2s = (int)l2s;
    p.off_l2c = (int)l2c;
    const size_t lvl2w = lvl2 > band ? lvl2 - band : 0;
    p.off_w = (int)band;
    p.TC = 1;
    p.off_small = 0;
    const size_t small = mix::mix_small_bytes(p);
    const size_t limit = (size_t)smem_optin > 2048 ? (size_t)smem_optin - 1024 : 0;
    auto contraction = [&](int tc) {
        const size_t tcp = (size_t)(tc + mix::kTM - 1) / mix::kTM * mix::kTM;
        return mix::mal(sizeof(float4) * tcp * p.KB) + (p.CL > 1 ? sizeof(float4) * (size_t)tc * p.TX : 0);
    };
    // one chunk of all h0 rows if it fits, else a multiple of 8 rows (the stage-A loads of
    // 8 t entries then stay 16-byte aligned)
    int tc = p.h0;
    while (tc > 8) {
        const size_t work = std::max(std::max(std::max(ysg, lvl1), lvl2w), contraction(tc));
        if (band + work + small <= limit) break;
        tc = (tc - 1) / 8 * 8;
    }
    const size_t work = std::max(std::max(std::max(ysg, lvl1), lvl2w), contraction(tc));
    if (band + work + small > limit) return -1;
    p.TC = tc;
    // one-CTA sides from 96 px: a smaller chunk (a multiple of 8 rows, at least 32) beside a
    // copy of the stage-B table, if both fit in the same work area (the same shared memory,
    // so the same CTAs per SM); stage B then reads the table from shared memory instead of
    // through L1. At 48 px the second chunk cost more than the copy saved (6.89 -> 6.54 M
    // ROIs/s); at 96 px it gained (2.94 -> 2.97 M)
    p.tbs = 0;
    if (p.CL == 1 && H >= 96) {
        const size_t tb = mix::mal(sizeof(float2) * (size_t)p.Wc * p.TXp);
        for (int tc2 = tc / 8 * 8; tc2 >= 32; tc2 -= 8)
            if (contraction(tc2) + tb <= work) {
                p.TC = tc2;
                p.tbs = 1;
                break;
            }
    }
    p.off_small = (int)(band + mix::mal(work));
    p.smem = (int)(p.off_small + small);

    // tables, in one device block
    std::vector<float2> t4h, t4r, rtw, phH, phW, tA((size_t)p.Hh * p.TAp), tB((size_t)p.Wc * p.TXp);
    std::vector<float> tG((size_t)p.Wc * p.TXp);
    // inter-pass twiddles in FP32 and as double-floats (hi = the FP32 rounding, lo = the rest)
    auto to_df = [](double x) { const float h = (float)x; return df{h, (float)(x - (double)h)}; };
    std::vector<dfc> t4h_d, t4r_d, rtw_d;
    pass_twiddles_n(H, [&](double c, double sn) {
        t4h.push_back(make_float2((float)c, (float)sn));
        t4h_d.push_back(dfc{to_df(c), to_df(sn)});
    });
    pass_twiddles_n(p.L, [&](double c, double sn) {
        t4r.push_back(make_float2((float)c, (float)sn));
        t4r_d.push_back(dfc{to_df(c), to_df(sn)});
    });
    if ((int)t4h.size() != H || (int)t4r.size() != p.L) return -1;
    for (int k = 0; k <= p.L / 2; ++k) {
        double c, sn;
        cexp2pi(-k, W, &c, &sn);
        rtw_d.push_back(dfc{to_df(c), to_df(sn)});
    }
    for (int k = 0; k <= p.L / 2; ++k) {
        double c, s;
        cexp2pi(-k, W, &c, &s);
        rtw.push_back(make_float2((float)c, (float)s));
    }
    for (int m = 0; m < H; ++m) {
        double c, s;
        cexp2pi(m, H, &c, &s);
        phH.push_back(make_float2((float)c, (float)s));
    }
    for (int m = 0; m < W; ++m) {
        double c, s;
        cexp2pi(m, W, &c, &s);
        phW.push_back(make_float2((float)c, (float)s));
    }
    const long long DH = (long long)u * H, DW = (long long)u * W;
    for (int i = 0; i < p.Hh; ++i)
        for (int tt = 0; tt < p.TAp; ++tt) {
            const int t = tt + 1;
            if (t > p.h0) { tA[(size_t)i * p.TAp + tt] = make_float2(0.f, 0.f); continue; }
            const long long n = (long long)(i + 1) * t;
            double c, s;
            cexp2pi(n, DH, &c, &s);
            tA[(size_t)i * p.TAp + tt] = make_float2((float)cosm1_2pi(n, DH), (float)s);
        }
    for (int kx = 0; kx < p.Wc; ++kx) {
        const int ks = kx == p.L ? -p.L : kx;
        const double g = (kx == 0 || kx == p.L) ? 1.0 : 2.0;
        for (int tx = 0; tx < p.TXp; ++tx) {
            const size_t o = (size_t)kx * p.TXp + tx;
            if (tx >= p.TX) { tB[o] = make_float2(0.f, 0.f); tG[o] = 0.f; continue; }
            const long long n = (long long)ks * tx;
            double c, s;
            cexp2pi(n, DW, &c, &s);
            tB[o] = make_float2((float)(g * c), (float)(g * s));
            tG[o] = (float)(g * cosm1_2pi(n, DW));
        }
    }
    const size_t n2 = t4h.size() + t4r.size() + rtw.size() + phH.size() + phW.size() + tA.size() + tB.size();
    const size_t bytes = n2 * sizeof(float2) + tG.size() * sizeof(float) +
                         (t4h_d.size() + t4r_d.size() + rtw_d.size()) * sizeof(dfc) + 512;
    char* d = nullptr;
    cudaError_t e = cudaMalloc(&d, bytes);
    if (e != cudaSuccess) return (int)e;
    std::vector<char> h(bytes, 0);
    size_t off = 0;
    auto put = [&](const void* src, size_t nbytes) {
        off = (off + 15) / 16 * 16;
        std::memcpy(h.data() + off, src, nbytes);
        const size_t at = off;
        off += nbytes;
        return d + at;
    };
    p.t4h = (const float2*)put(t4h.data(), t4h.size() * sizeof(float2));
    p.t4r = (const float2*)put(t4r.data(), t4r.size() * sizeof(float2));
    p.rtw = (const float2*)put(rtw.data(), rtw.size() * sizeof(float2));
    p.phH = (const float2*)put(phH.data(), phH.size() * sizeof(float2));
    p.phW = (const float2*)put(phW.data(), phW.size() * sizeof(float2));
    p.tA = (const float2*)put(tA.data(), tA.size() * sizeof(float2));
    p.tB = (const float2*)put(tB.data(), tB.size() * sizeof(float2));
    p.tG = (const float*)put(tG.data(), tG.size() * sizeof(float));
    p.t4h_d = (const dfc*)put(t4h_d.data(), t4h_d.size() * sizeof(dfc));
    p.t4r_d = (const dfc*)put(t4r_d.data(), t4r_d.size() * sizeof(dfc));
    p.rtw_d = (const dfc*)put(rtw_d.data(), rtw_d.size() * sizeof(dfc));
    e = cudaMemcpy(d, h.data(), bytes, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(d);
        return (int)e;
    }
    *mem = d;
    *out = p;
    return 0;
}

}  // namespace ccst
