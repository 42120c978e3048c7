// ccst_kernels.cuh -- the tracking kernel for sm_103a.
//
// One CTA tracks one frame at a time (grid-stride over the batch). Every step
// stays in shared memory:
//   a1  ingest the frame (uint16 or float32, 16-byte vector loads) and form the
//       surface operand: the frame itself for CC-U, (I + eps)^2 for CC-SN
//       (Sec. II, Eqs. (4), (7));
//   a2  2-D R2C FFT: two real rows per complex row, four-step passes with the
//       small DFTs in registers; the real/complex split is fused into the column
//       pass loads, and the DC and Nyquist columns travel as one complex column;
//   a3  product with the resident reference spectrum, X = F[a] conj(F[b]), fused
//       into the last column pass;
//   a4  inverse 2-D FFT -> integer surface c(s) (right-hand side of Eq. (4)/(7));
//   a5  integer extremum, lowest row-major index on ties, wrapped shift;
//       near-ties re-decided by FP64 direct sums sum_r a(r+s) b(r);
//   a6  upsampled DFT on the M x M grid around it (Sec. III), as two dense
//       contractions with frame-independent tables staged in shared memory;
//   a7  sub-pixel extremum and the output record.
//
// a6 is evaluated relative to the integer peak (the "delta" form): with
// X'(k) = X(k) exp(2 pi i k'.p/N) and E(k,t) = exp(2 pi i k' t/(uN)),
//   cu(ty,tx) - cu(0,0) = S(ty,tx) + g(tx),
//   S(ty,tx) = Re sum_kx w(kx) T'(ty,kx) E(kx,tx),  T'(ty,kx) = sum_ky X'(ky,kx) (E(ky,ty) - 1),
//   g(tx)    = Re sum_kx w(kx) R(kx) (E(kx,tx) - 1),  R(kx) = sum_ky X'(ky,kx),
// with w = 1 at kx = 0 and kx = W/2 and 2 elsewhere (Hermitian folding of the
// real-input spectrum). The pairs +-ky and +-t are folded too:
//   T'(+-t) = U'(t) +- i V(t),  U'(t) = sum_m (cos th_mt - 1) P(m),  V(t) = sum_m sin th_mt Q(m),
//   P(m) = X'(m) + X'(-m),  Q(m) = X'(m) - X'(-m),  th_mt = 2 pi m t / (uH).
// The interpolant is the real part of the full signed-frequency sum (Nyquist bin
// at -N/2). For the y-Nyquist row (ky = H/2) in the columns 0 < kx < W/2 that
// real part pairs each term with its Hermitian partner so that the row's y-phase
// enters only through its real part cos(pi s_y); the folded sums reproduce this by
// keeping only the cosine part of that row (Q(H/2, kx) = 0 for kx < W/2).
// The same algebra is exact in real arithmetic; in FP32 it keeps the rounding
// error proportional to the surface's variation over the grid rather than to
// its value, which is what decides the sub-pixel argmax.
//
// Near-ties of the FP32 sub-pixel surface are re-decided from exact pair
// differences v(j) - v(j1) = Re sum_k w X'(k) [E(ty)E(tx) - E(ry)E(rx)], split
// into terms with small factors (E(tx) - E(rx) = 2i sin(.) exp(i .)), and, if
// still tied, by re-evaluating the tied candidates from a double-float product
// spectrum (about 48 significant bits) computed in the same CTA.
#pragma once

#include "ccst_device.cuh"
#include "ccst_fft.cuh"
#include "ccst_tc.cuh"
#include <cuda_fp16.h>

namespace ccst {

// g(+-tx) row sums: partial sums per tx, each of at most kGTerms table terms
// (kGParts * kGTerms >= W/2 + 1 for W <= 128)
constexpr int kGParts = 6, kGTerms = 11;

struct Geom {
    int H, W, logH, logW, Hh, Wc, Wcp;  // Wc = W/2+1 (half spectrum), Wcp = Wc rounded up to even
    int SA;                             // column slots of the spectrum buffer: W/2 (slot 0 = DC, + Nyquist array)
    int SZ;                             // padded row stride (float2) of the packed-row buffer
    int u, M, h0, pmax;                 // grid: M points, offsets t = j - h0 in [-h0, pmax]
    int T1p;                            // table row length for tx in [0, h0] (padded to 4)
    int T1p8;                           // tx extent of the tensor-core stage-B tables (padded to 8)
    int TAB;                            // t rows 1..TAB of the stage tables (h0 rounded up to 15)
    int TC, nchunk;                     // t rows per stage chunk (multiple of 15) and number of chunks
    int tables_smem;                    // stage tables staged in shared memory (else read from global)
    int Ntw, logNtw;                    // twiddle table length = max(H, W)
    int lN1h, lN2h, lN1w, lN2w;         // log2 of the four-step splits of H and W
    int method, in_dtype;
    float eps, sense;                   // sense = +1 (CC-U maximum) or -1 (CC-SN minimum)
    float tau_int, tau0, tau1;          // guard thresholds, relative to sum w|X|
    int guard;                          // tie guard on/off
    int tc;                             // the contraction runs on tcgen05 (H = W = 128, one chunk, tables in smem)
    int RA, NB;                         // tc: rows of a stage-A table matrix (TAB rounded to 8), stage-B N (TC to 16)
    // resident device data (owned by the context)
    const float2* FE32;                 // H x Wc   F[b]
    const double2* FE64;                // H x Wc   F[b] in FP64
    const double* b64;                  // H x W    reference operand b (E or 1/(E+eps))
    const float2* tw32;                 // Ntw/2    exp(-2 pi i k/Ntw)
    const double2* tw64;
    const float* tA_cm1;                // [Hh][T1p]  cos(2 pi m t/(uH)) - 1, m = 1..Hh
    const float* tA_s;                  // [Hh][T1p]  sin(2 pi m t/(uH))
    const uint2* tAh;                   // stage-A tensor-core tables (layout of Smem::TA)
    const uint2* tBh;                   // stage-B tensor-core tables (layout of Smem::TB)
    const float* tB_wc;                 // [Wc][T1p]  w cos(2 pi kx' t/(uW))
    const float* tB_ws;                 // [Wc][T1p]  w sin(2 pi kx' t/(uW))
    const float* tB_gc;                 // [Wc][T1p]  w (cos(2 pi kx' t/(uW)) - 1)
    // double-float data for the last guard level
    const dfc* FEdf;                    // H x Wc   F[b]
    const dfc* twdf;                    // Ntw/2    exp(-2 pi i k/Ntw)
    const dfc* eyc; const dfc* eyf;     // exp(2 pi i n/(uH)) = eyc[n / By] * eyf[n % By]
    const dfc* exc; const dfc* exf;     // exp(2 pi i n/(uW)) = exc[n / Bx] * exf[n % Bx]
    int By, Bx;
};

// Uneven-ROI batches (ccst_track_rois): resident spectra of one reference, one work item per
// ROI, and the launch's arguments.
struct RefSpectra {
    const float2* FE32;
    const double2* FE64;
    const double* b64;
    const dfc* FEdf;
};

struct Result;

struct RoiItem {
    const void* frame;      // the ROI's pixels (in_dtype), rows `pitch` elements apart
    long long pitch;
    long long out_index;    // record slot
    int cls;                // size class: the plan of the ROI's side
    int ref;                // reference: index into RoiBatch::refs
    int vec_ok;             // 16-byte vector loads allowed
    int pad;
};

struct RoiBatch {
    const RoiItem* items;   // items of one side
    long long n;
    const RefSpectra* refs;
    Result* out;
    unsigned* next;         // item counter, zeroed before the launch
};

// General square sizes (ccst_generic.cu): one plan per side N, items, launch arguments.
struct Result {  // mirrors ccst_result
    float dx, dy, peak;
    int ipy, ipx;
    unsigned flags;
};

struct Batch {
    const void* frames;
    long long n;
    long long pitch;     // row pitch in elements
    int vec_ok;          // frames and pitch allow 16-byte vector loads
    Result* out;
    float* dbg_int;      // optional: n x H x W integer surfaces (unnormalised), or null
    float* dbg_sub;      // optional: n x M x M delta surfaces (unnormalised), or null
    const int* dbg_pairs;  // optional: n x 2 grid indices (ja, jb); then only the pair difference runs
    float* dbg_d32;        // n: v(jb) - v(ja) by the FP32 pair-difference guard
    double* dbg_d64;       // n: the same difference accumulated in FP64 from the FP32 spectrum
    int dbg_no_copy;       // tests of the bounded wait: withhold the table copies (the wait runs out)
    unsigned* next;        // optional: frame counter (zero at launch); CTAs take frames from it in
                           // order, so that a slow frame delays no other. Null: CTA i takes frames
                           // i, i + gridDim.x, ...
};

// --------------------------------------------------------------------- helpers
__device__ __forceinline__ int signed_k(int k, int N) { return k < (N >> 1) ? k : k - N; }
__device__ __forceinline__ int wrap_shift(int p, int N) { return p > (N >> 1) ? p - N : p; }

// exp(+2 pi i r / N) from the FP32 table exp(-2 pi i k / Ntw), 0 <= r < N, N | Ntw.
__device__ __forceinline__ float2 twiddle_pos(const float2* tw, int r, int logN, int logNtw) {
    const int halfN = 1 << (logN - 1);
    const int sh = logNtw - logN;
    if (r < halfN) {
        const float2 t = tw[r << sh];
        return make_float2(t.x, -t.y);
    }
    const float2 t = tw[(r - halfN) << sh];
    return make_float2(-t.x, t.y);
}

template <typename T>
__device__ __forceinline__ double load_pixel(const T* f, long long idx);
template <>
__device__ __forceinline__ double load_pixel<unsigned short>(const unsigned short* f, long long idx) {
    return (double)__ldg(f + idx);
}
template <>
__device__ __forceinline__ double load_pixel<float>(const float* f, long long idx) {
    return (double)__ldg(f + idx);
}

__device__ __forceinline__ float pixel_f32(const void* frames, int in_dtype, long long idx) {
    if (in_dtype == 0) return (float)__ldg((const unsigned short*)frames + idx);
    return __ldg((const float*)frames + idx);
}

// Surface operand of one pixel: the pixel (CC-U) or (I + eps)^2 (CC-SN).
__device__ __forceinline__ float operand_f32(float I, const Geom& g) {
    if (g.method == 0) return I;
    const float ip = I + g.eps;
    return ip * ip;
}
__device__ __forceinline__ double operand_f64(double I, const Geom& g) {
    if (g.method == 0) return I;
    const double ip = I + (double)g.eps;
    return ip * ip;
}

// ------------------------------------------------- fp16 hi/lo operand pairs
// The contractions run on the tensor cores as m16n8k16 FP16 MMAs with FP32 accumulation.
// Each FP32 operand x (scaled by a power of two into [2^-14, 2^14]) is stored as
// x = hi + lo + r, hi = fp16(x), lo = fp16(x - hi), |r| <= 2^-22 |x| (plus the fp16
// subnormal floor, far below the contraction's error budget after scaling), and a product
// is accumulated as lo*hi + hi*lo + hi*hi (the dropped lo*lo is below 2^-22 of it). Two
// consecutive K elements share one 32-bit register as the MMA fragments want them; an
// operand row is stored as uint2 {hi pair, lo pair} per K pair.
// two floats -> one register of two fp16 (a in the low half), round to nearest; and back
__device__ __forceinline__ unsigned pack_f16x2(float a, float b) {
    unsigned r;
    asm("cvt.rn.f16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(b), "f"(a));
    return r;
}
__device__ __forceinline__ float2 unpack_f16x2(unsigned v) {
    float a, b;
    asm("{\n.reg .f16 lo, hi;\nmov.b32 {lo, hi}, %2;\ncvt.f32.f16 %0, lo;\ncvt.f32.f16 %1, hi;\n}"
        : "=f"(a), "=f"(b) : "r"(v));
    return make_float2(a, b);
}
__device__ __forceinline__ uint2 split_pair(float a, float b) {
    const unsigned h = pack_f16x2(a, b);
    const float2 hf = unpack_f16x2(h);
    return make_uint2(h, pack_f16x2(a - hf.x, b - hf.y));
}
__device__ __forceinline__ float2 unsplit_pair(uint2 v) {
    const float2 h = unpack_f16x2(v.x), l = unpack_f16x2(v.y);
    return make_float2(h.x + l.x, h.y + l.y);
}
// Pair-index swizzle of an operand row with kp pairs: pair p of row r sits at p ^ pswz(r).
// The 16 lanes of a half-warp (4 rows x 4 pairs) of every fragment load then hit distinct
// 8-byte bank pairs.
__host__ __device__ __forceinline__ int pswz(int r, int kp) { return ((r & 3) << 2) & (kp - 1); }
// (not volatile: the compiler may interleave independent accumulations)
__device__ __forceinline__ void mma_f16(float (&d)[4], const unsigned (&a)[4], unsigned b0, unsigned b1) {
    asm("mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
                 "{%0,%1,%2,%3};\n"
                 : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
                 : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}
// Fragment addressing of a swizzled [row][KP] operand: the thread reads K pairs
// 8 s + tq and 8 s + tq + 4 of k16 step s. Writing 8 s = 16 a + 8 b, the swizzle only
// touches bits 2-3, so pair 16 a + ((8 b + 4 h + tq) ^ pswz(r)): the four row offsets
// o[b][h] are computed once per task and every load is one of them plus 16 a.
// The operand lives in the kernel's dynamic shared memory; the offsets are 32-bit byte
// offsets into it, so that each load is one shared load with an immediate displacement.
extern __shared__ __align__(16) unsigned char ccst_smem[];
struct RowOffsets {
    unsigned o[2][2];
    __device__ __forceinline__ RowOffsets(const uint2* P, int KP, int r, int tq) {
        const int c = pswz(r, KP);
        const unsigned base = (unsigned)((const unsigned char*)(P + r * KP) - ccst_smem);
#pragma unroll
        for (int b = 0; b < 2; ++b)
#pragma unroll
            for (int h = 0; h < 2; ++h) o[b][h] = base + 8u * (unsigned)(((8 * b + 4 * h + tq) ^ c) & (KP - 1));
    }
    __device__ __forceinline__ uint2 at(int s, int h) const {
        return *reinterpret_cast<const uint2*>(ccst_smem + o[s & 1][h] + 128 * (s >> 1));
    }
    // the same pair of row r + dr (same swizzle when dr is a multiple of 4) of an operand
    // starting `delta` bytes further
    __device__ __forceinline__ uint2 at(int s, int h, unsigned delta) const {
        return *reinterpret_cast<const uint2*>(ccst_smem + o[s & 1][h] + delta + 128 * (s >> 1));
    }
};
// A fragment of k16 step s: rows r (offsets ro, plus `delta` bytes) and r + 8 (8 rows of
// KP pairs further, `r8` bytes)
__device__ __forceinline__ void load_afrag(const RowOffsets& ro, unsigned delta, unsigned r8, int s, unsigned (&h)[4],
                                           unsigned (&l)[4]) {
    const uint2 v0 = ro.at(s, 0, delta), v1 = ro.at(s, 0, delta + r8), v2 = ro.at(s, 1, delta),
                v3 = ro.at(s, 1, delta + r8);
    h[0] = v0.x; h[1] = v1.x; h[2] = v2.x; h[3] = v3.x;
    l[0] = v0.y; l[1] = v1.y; l[2] = v2.y; l[3] = v3.y;
}

// Power-of-two exponent for the per-frame operands: with sum|X| <= scale, every P/Q value
// is <= 2 scale and every stage-A combination <= 4 scale; 2^kexp brings them to <= 2^14.
__device__ __forceinline__ int operand_exponent(float scale) {
    int e = 0;
    if (scale > 0.f && isfinite(scale)) (void)frexpf(scale, &e);   // scale <= 2^e
    return max(-120, min(120, 12 - e));
}

// ------------------------------------------------------------- shared layout
// R1: A (H x SA float2: the spectrum, later X' with P/Q rows) and XN (H float2: the
//     x-Nyquist column kx = W/2 of the same).
// R2, FFT phase: B (H x SA float2, inverse-FFT workspace) and ZC (H/2 x SZ float2,
//     packed rows: the frame, then the integer surface).
// R2, contraction phase: TA (stage-A table), TB (stage-B tables), UV (TC x SA float4),
//     UVN (TC float4, x-Nyquist column). After the contraction R2 holds the guard
//     scratch. The last guard level uses R1 + R2 as one block.
struct Smem {
    float2* A;
    float2* XN;
    float2* B;
    float2* ZC;
    uint2* PQ;             // = A after the P/Q build: [4][SA][Hh/2] planes Pr, Pi, Qr, Qi (fp16 pairs)
    uint2* TA;             // stage-A tables [2][TAB][Hh/2]: 2^13 (cos - 1), 2^13 sin (fp16 pairs)
    uint2* TB;             // stage-B tables [2][T1p][SA/2]: 2^13 w cos, 2^13 w sin (fp16 pairs),
                           //   then float [2][T1p8]: w cos, w sin at kx = W/2
    float4* UV;            // the contraction area, also scratch before and after it
    float4* UVN;
    uint2* CB;             // = UV: stage-A output [4][TC][SA/2] (C0, C1, E0, E1 as fp16 pairs)
    float* CBN;            // = UVN: [4][TC] the same at kx = W/2 (FP32)
    unsigned char* r1;     // start of R1
    size_t r12_bytes;      // bytes of R1 + R2
    float2* tw;            // Ntw/2
    float2* t4h;           // H: four-step inter-pass twiddles of length H, [k1][n2]
    float2* t4w;           // W: the same for length W
    float2* X0;            // SA: X'(0, kx)
    float* gP;             // T1p: g(+tx)
    float* gM;             // T1p: g(-tx)
    float* rv;             // reduction scratch (floats)
    int* rj;               // reduction scratch (ints)
    double* rd;            // reduction scratch (doubles)
    unsigned long long* bar;  // mbarrier of the bulk table copies
    float2* ex;            // Wc: e^{2 pi i kx px / W} per column slot (slot W/2 = x-Nyquist column)
    float2* ey;            // Hh + 1: e^{2 pi i m py / H}, m = 0 .. Hh
    int* cj;               // candidate list
    float* cv;             // candidate values
    int* misc;             // small broadcast ints
    // the frame's reference spectra, when they are not the geometry's own (an uneven-ROI
    // item's, in shared memory), else null
    const RefSpectra* ref;
};

__host__ __device__ inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Stride (float2) of the packed rows: >= W + W/PG (the padded row) and = 8 (mod 16), which
// keeps the row passes' lane groups on distinct banks.
__host__ __device__ constexpr int packed_row_stride(int W) {
    const int pg = split_n2(W) > 1 ? split_n2(W) : W;
    const int len = W + W / pg;
    const int sz = ((len + 7) / 16) * 16 + 8;
    return sz < len ? sz + 16 : sz;
}

struct SmemPlan {
    size_t a, xn, r1, b, zc, ta, tb, uv, uvn, r2, misc, total;
};

// sizes (bytes) of the two tensor-core table blocks. With g.tc: stage A's four matrices
// (2^13 (cos - 1) and 2^13 sin, fp16 hi and lo each; rows t - 1, K = m - 1) and stage B's four
// (2^13 w cos and 2^13 w sin, hi and lo; rows tx, K = kx), 128-byte-swizzled K-major, then
// the kx = W/2 column in FP32.
__host__ __device__ inline size_t ta_bytes(const Geom& g) {
    if (g.tc) return (size_t)4 * g.RA * 128;
    return sizeof(uint2) * 2 * (size_t)g.TAB * (g.Hh / 2);
}
__host__ __device__ inline size_t tb_bytes(const Geom& g) {
    if (g.tc) return (size_t)4 * g.T1p8 * 128 + sizeof(float) * 2 * (size_t)g.T1p8;
    return sizeof(uint2) * 2 * (size_t)g.T1p * (g.SA / 2) + sizeof(float) * 2 * (size_t)g.T1p8;
}
__host__ __device__ inline size_t table_bytes(const Geom& g) { return ta_bytes(g) + tb_bytes(g); }

// The tcgen05 plan (g.tc). R1 starts on a 1024-byte boundary (the dynamic base is padded at
// run time; the total counts 1024 for it). R1 holds the spectrum, then the P/Q planes as eight
// matrices [Pr, Pi, Qr, Qi] x [hi, lo] of SA rows (kx) by 64 K values (m - 1). R2 in the
// contraction phase: TB (the stage-B tables, read as 128-row A operands: rows past T1p8 fall
// in what follows), then one block that holds TA (stage A's A operands, also read as 128
// rows) and, once stage A has finished, CB: stage B's B operands, eight matrices
// [C0, C1, E0, E1] x [hi, lo] of NB rows (t) by 64 K values (kx). Then the scratch area UV
// (R, partial sums, guard scratch) and UVN (the x-Nyquist combinations in FP32).
__host__ __device__ inline SmemPlan smem_plan_tc(const Geom& g) {
    SmemPlan p;
    const size_t pq = (size_t)8 * g.SA * 128, spec = sizeof(float2) * (size_t)g.H * g.SA;
    p.a = align_up(pq > spec ? pq : spec, 16);
    p.xn = align_up(sizeof(float2) * (size_t)g.H, 16);
    p.r1 = align_up(p.a + p.xn, 1024);
    p.b = align_up(sizeof(float2) * (size_t)g.H * g.SA, 16);
    p.zc = align_up(sizeof(float2) * (size_t)(g.H / 2) * g.SZ, 16);
    const size_t fft = p.b + p.zc;
    p.tb = align_up(tb_bytes(g), 1024);
    const size_t ta_read = (size_t)4 * g.RA * 128 + (size_t)(128 - g.RA) * 128;   // last matrix read as 128 rows
    const size_t cb = (size_t)8 * g.NB * 128;
    p.ta = align_up(ta_read > cb ? ta_read : cb, 1024);
    // the epilogue stages float2 [2][TC][T1p8] over TB and this block
    const size_t stg = sizeof(float2) * 2 * (size_t)g.TC * g.T1p8;
    if (p.tb + p.ta < stg) p.ta = align_up(stg - p.tb, 1024);
    size_t rscr = sizeof(float2) * ((size_t)g.Wcp + 8 * (size_t)(g.SA + 1)) + sizeof(float) * 2 * kGParts * (size_t)g.T1p;
    const size_t gscr = sizeof(float2) * (size_t)(4 * g.Wc + 23 * g.H + 17);
    const size_t dscr = sizeof(double2) * (size_t)(2 * g.H + 2 * g.Wc);
    if (rscr < gscr) rscr = gscr;
    if (rscr < dscr) rscr = dscr;
    p.uv = align_up(rscr, 16);
    p.uvn = align_up(sizeof(float4) * (size_t)g.TC, 16);
    const size_t k6 = p.tb + p.ta + p.uv + p.uvn;
    p.r2 = fft > k6 ? fft : k6;
    const size_t chunk = (size_t)g.W > (size_t)(g.H + g.Wc) ? (size_t)g.W : (size_t)(g.H + g.Wc);
    const size_t dfl = sizeof(dfc) * ((size_t)g.H * g.Wcp + (size_t)(g.Ntw / 2) + g.W + g.H + chunk);
    if (p.r1 + p.r2 < dfl) p.r2 = align_up(dfl - p.r1, 16);
    p.misc = sizeof(double) * 32 + 16 + sizeof(float2) * (size_t)(g.Wc + g.Hh + 1) +
             sizeof(float2) * (size_t)(g.Ntw / 2 + g.H + g.W) + sizeof(float2) * (size_t)g.SA +
             sizeof(float) * 2 * (size_t)g.T1p + sizeof(float) * 64 + sizeof(int) * 64 +
             (sizeof(int) + sizeof(float)) * kMaxCand + sizeof(int) * 16 + 64;
    p.total = align_up(1024 + p.r1 + p.r2 + p.misc, 16);
    return p;
}

__host__ __device__ inline SmemPlan smem_plan(const Geom& g) {
    if (g.tc) return smem_plan_tc(g);
    SmemPlan p;
    p.a = align_up(sizeof(float2) * (size_t)g.H * g.SA, 16);
    p.xn = align_up(sizeof(float2) * (size_t)g.H, 16);
    p.r1 = p.a + p.xn;
    p.b = align_up(sizeof(float2) * (size_t)g.H * g.SA, 16);
    p.zc = align_up(sizeof(float2) * (size_t)(g.H / 2) * g.SZ, 16);
    const size_t fft = p.b + p.zc;
    p.ta = g.tables_smem ? align_up(ta_bytes(g), 16) : 0;
    p.tb = g.tables_smem ? align_up(tb_bytes(g), 16) : 0;
    p.uv = align_up(sizeof(uint2) * 4 * (size_t)g.TC * (g.SA / 2), 16);
    // the P/Q build keeps R(kx), its 8 partial sums and the g partial sums here first
    size_t rscr = sizeof(float2) * ((size_t)g.Wcp + 8 * (size_t)(g.SA + 1)) + sizeof(float) * 2 * kGParts * (size_t)g.T1p;
    // ... and afterwards the guard scratch (FP32 pair differences, or the FP64 diagnostic)
    const size_t gscr = sizeof(float2) * (size_t)(4 * g.Wc + 23 * g.H + 17);   // pair-difference guard
    const size_t dscr = sizeof(double2) * (size_t)(2 * g.H + 2 * g.Wc);
    if (rscr < gscr) rscr = gscr;
    if (rscr < dscr) rscr = dscr;
    if (p.uv < rscr) p.uv = align_up(rscr, 16);
    p.uvn = align_up(sizeof(float4) * (size_t)g.TC, 16);
    const size_t k6 = p.ta + p.tb + p.uv + p.uvn;
    p.r2 = fft > k6 ? fft : k6;
    // the double-float level needs H x Wcp dfc, the FFT twiddles (Ntw/2 + W + H) and one
    // packed-row chunk (at least one row of W dfc), which later holds the H + Wc candidate
    // twiddles
    const size_t chunk = (size_t)g.W > (size_t)(g.H + g.Wc) ? (size_t)g.W : (size_t)(g.H + g.Wc);
    const size_t dfl = sizeof(dfc) * ((size_t)g.H * g.Wcp + (size_t)(g.Ntw / 2) + g.W + g.H + chunk);
    if (p.r1 + p.r2 < dfl) p.r2 = align_up(dfl - p.r1, 16);
    p.misc = sizeof(double) * 32 + 16 + sizeof(float2) * (size_t)(g.Wc + g.Hh + 1) +
             sizeof(float2) * (size_t)(g.Ntw / 2 + g.H + g.W) + sizeof(float2) * (size_t)g.SA +
             sizeof(float) * 2 * (size_t)g.T1p + sizeof(float) * 64 + sizeof(int) * 64 +
             (sizeof(int) + sizeof(float)) * kMaxCand + sizeof(int) * 16 + 64;
    // the tensor-core stages read up to 15 rows past the last stage-A output plane (rows of
    // the last 16-row tile that feed only discarded outputs): keep them inside the allocation
    const size_t over = 15 * sizeof(uint2) * (size_t)(g.SA / 2);
    const size_t tail = p.uvn + p.misc;
    p.total = align_up(p.r1 + p.r2 + p.misc + (over > tail ? over - tail : 0), 16);
    return p;
}

static __device__ inline Smem carve(const Geom& g, unsigned char* base) {
    const SmemPlan p = smem_plan(g);
    Smem s;
    if (g.tc) base += (1024u - (smem_addr(base) & 1023u)) & 1023u;     // R1 on a 1024-byte boundary
    s.r1 = base;
    s.A = (float2*)base;
    s.XN = (float2*)(base + p.a);
    unsigned char* r2 = base + p.r1;
    s.B = (float2*)r2;
    s.ZC = (float2*)(r2 + p.b);
    s.PQ = (uint2*)base;
    if (g.tc) {
        s.TB = (uint2*)r2;
        s.TA = (uint2*)(r2 + p.tb);
        s.UV = (float4*)(r2 + p.tb + p.ta);
        s.UVN = (float4*)(r2 + p.tb + p.ta + p.uv);
    } else {
        s.TA = (uint2*)r2;
        s.TB = (uint2*)(r2 + p.ta);
        s.UV = (float4*)(r2 + p.ta + p.tb);
        s.UVN = (float4*)(r2 + p.ta + p.tb + p.uv);
    }
    s.CB = g.tc ? s.TA : (uint2*)s.UV;      // tc: stage B's operands replace the stage-A tables
    s.CBN = (float*)s.UVN;
    s.r12_bytes = p.r1 + p.r2;
    unsigned char* m = r2 + p.r2;
    s.rd = (double*)m; m += sizeof(double) * 32;
    s.bar = (unsigned long long*)m; m += 16;
    s.ex = (float2*)m; m += sizeof(float2) * g.Wc;
    s.ey = (float2*)m; m += sizeof(float2) * (g.Hh + 1);
    s.tw = (float2*)m; m += sizeof(float2) * (g.Ntw / 2);
    s.t4h = (float2*)m; m += sizeof(float2) * g.H;
    s.t4w = (float2*)m; m += sizeof(float2) * g.W;
    s.X0 = (float2*)m; m += sizeof(float2) * g.SA;
    s.gP = (float*)m; m += sizeof(float) * g.T1p;
    s.gM = (float*)m; m += sizeof(float) * g.T1p;
    s.rv = (float*)m; m += sizeof(float) * 64;
    s.rj = (int*)m; m += sizeof(int) * 64;
    s.cj = (int*)m; m += sizeof(int) * kMaxCand;
    s.cv = (float*)m; m += sizeof(float) * kMaxCand;
    s.misc = (int*)m;
    s.ref = nullptr;
    return s;
}

// Positions: spectrum rows after the column passes, packed-row elements after the row passes
// (all sizes are powers of two: shifts and masks).
__device__ __forceinline__ int posH(const Geom& g, int ky) {
    return ((ky & ((1 << g.lN1h) - 1)) << g.lN2h) | (ky >> g.lN1h);
}
__device__ __forceinline__ int posW(const Geom& g, int kx) {
    return ((kx & ((1 << g.lN1w) - 1)) << g.lN2w) | (kx >> g.lN1w);
}
__device__ __forceinline__ int unposW(const Geom& g, int q) {
    return ((q & ((1 << g.lN2w) - 1)) << g.lN1w) | (q >> g.lN2w);
}
__device__ __forceinline__ int physZ(const Geom& g, int q) {
    const int lpg = g.lN2w > 0 ? g.lN2w : g.logW;      // padding group: N2, or W for one-pass rows
    return q + (q >> lpg);
}

// ------------------------------------------------------- a1-a4: FFT correlation
// Also scans the integer surface as the last inverse pass stores it: t2 receives each
// thread's best (sense * HW c(y, x), y * W + x) and runner-up value; dbg, if set, the
// whole surface. *scale_out gets this thread's part of the spectral sum sum |X|.
template <int H, int W>
static __device__ void fft_correlate_t(const Geom& g, const Smem& S, const void* frame, long long pitch, int vec_ok,
                                float* scale_out, Best2& t2, float* dbg) {
    constexpr int N1w = Split<W>::N1, N2w = Split<W>::N2, N1h = Split<H>::N1, N2h = Split<H>::N2;
    constexpr int Hh = H / 2, SA = W / 2;
    constexpr int PG = N2w > 1 ? N2w : W;          // padding group of the packed rows
    constexpr int SZ = packed_row_stride(W);
    float2* Z = S.ZC;
    float2* A = S.A;
    float2* B = S.B;
    float2* XN = S.XN;
    auto zphys = [&](int q) { return q + q / PG; };

    // a1: ingest: packed rows Z[r][x] = (a(2r, x), a(2r+1, x)), natural x order
    if (vec_ok && g.in_dtype == 0) {
        for (int idx = threadIdx.x; idx < H * W / 8; idx += blockDim.x) {
            const int y = idx / (W / 8), x0 = (idx - y * (W / 8)) * 8;
            const uint4 v = __ldg((const uint4*)((const unsigned short*)frame + (long long)y * pitch + x0));
            const unsigned int w[4] = {v.x, v.y, v.z, v.w};
            float* zr = (float*)&Z[(y >> 1) * SZ] + (y & 1);
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                zr[2 * zphys(x0 + 2 * k)] = operand_f32((float)(w[k] & 0xffffu), g);
                zr[2 * zphys(x0 + 2 * k + 1)] = operand_f32((float)(w[k] >> 16), g);
            }
        }
    } else if (vec_ok) {
        for (int idx = threadIdx.x; idx < H * W / 4; idx += blockDim.x) {
            const int y = idx / (W / 4), x0 = (idx - y * (W / 4)) * 4;
            const float4 v = __ldg((const float4*)((const float*)frame + (long long)y * pitch + x0));
            float* zr = (float*)&Z[(y >> 1) * SZ] + (y & 1);
            zr[2 * zphys(x0)] = operand_f32(v.x, g);
            zr[2 * zphys(x0 + 1)] = operand_f32(v.y, g);
            zr[2 * zphys(x0 + 2)] = operand_f32(v.z, g);
            zr[2 * zphys(x0 + 3)] = operand_f32(v.w, g);
        }
    } else {
        for (int idx = threadIdx.x; idx < H * W; idx += blockDim.x) {
            const int y = idx / W, x = idx - y * W;
            float* zr = (float*)&Z[(y >> 1) * SZ] + (y & 1);
            zr[2 * zphys(x)] = operand_f32(pixel_f32(frame, g.in_dtype, (long long)y * pitch + x), g);
        }
    }
    __syncthreads();
    // element n of a packed row sits at Z[r][n + n / PG]; for n = N2w a + b (b < N2w) that
    // is (N2w + 1) a + b, linear in the unrolled index a
    constexpr int RP = N2w > 1 ? N2w + 1 : 1;        // padded stride of a row-pass group
    // a2: row FFTs (forward), in place
    fft_pass1<N1w, N2w, false, false>(
        Hh, S.t4w, [&](int s, int n2, int n1) { return Z[s * SZ + RP * n1 + n2]; },
        [&](int s, int n2, int k1, float2 v) { Z[s * SZ + RP * k1 + n2] = v; });
    __syncthreads();
    if (N2w > 1) {
        fft_pass2<N1w, N2w, false, false>(
            Hh, [&](int s, int k1, int n2) { return Z[s * SZ + RP * k1 + n2]; },
            [&](int s, int k1, int k2, float2 v) { Z[s * SZ + RP * k1 + k2] = v; });
        __syncthreads();
    }
    // Z_r(k) now sits at Z[r][zphys(fft_pos(k))]. Column pass 1 (forward) with the
    // real/complex split fused into the loads; slot 0 carries the DC and Nyquist columns
    // as one complex column (both are real sequences along y for real rows).
    fft_pass1<N1h, N2h, false, true>(
        SA, S.t4h,
        [&](int s, int n2, int n1) {
            const int y = N2h * n1 + n2;
            const float2* zr = Z + (y >> 1) * SZ;
            if (s == 0) {
                const float2 z0 = zr[0], zn = zr[zphys(fft_pos(W / 2, N1w, N2w))];
                return (y & 1) ? make_float2(z0.y, zn.y) : make_float2(z0.x, zn.x);
            }
            const float2 z = zr[zphys(fft_pos(s, N1w, N2w))], zc = zr[zphys(fft_pos(W - s, N1w, N2w))];
            if (y & 1) return make_float2(0.5f * (z.y + zc.y), -0.5f * (z.x - zc.x));   // (z - conj zc)/(2i)
            return make_float2(0.5f * (z.x + zc.x), 0.5f * (z.y - zc.y));               // (z + conj zc)/2
        },
        [&](int s, int n2, int k1, float2 v) { A[(N2h * k1 + n2) * SA + s] = v; });
    __syncthreads();
    // column pass 2 + a3: product with conj(F[b]) (slot 0 is unpacked afterwards)
    const float2* FE32 = S.ref ? S.ref->FE32 : g.FE32;
    float sabs = 0.f;
    fft_pass2<N1h, N2h, false, true>(
        SA, [&](int s, int k1, int n2) { return A[(N2h * k1 + n2) * SA + s]; },
        [&](int s, int k1, int k2, float2 v) {
            if (s != 0) {
                const int ky = k1 + N1h * k2;
                const float2 x = cmul(v, cconj(__ldg(&FE32[ky * (W / 2 + 1) + s])));
                sabs += 2.f * (fabsf(x.x) + fabsf(x.y));
                v = x;
            }
            A[(N2h * k1 + k2) * SA + s] = v;
        });
    __syncthreads();
    // unpack slot 0 into X(ky, 0) (kept in slot 0) and X(ky, W/2) (in XN)
    for (int ky = threadIdx.x; ky < H; ky += blockDim.x) {
        const int q = fft_pos(ky, N1h, N2h), qm = fft_pos((H - ky) & (H - 1), N1h, N2h);
        const float2 zp = A[q * SA], zm = cconj(A[qm * SA]);
        const float2 f0 = make_float2(0.5f * (zp.x + zm.x), 0.5f * (zp.y + zm.y));
        const float2 d = csub(zp, zm);
        const float2 fn = make_float2(0.5f * d.y, -0.5f * d.x);
        const float2 x0 = cmul(f0, cconj(__ldg(&FE32[ky * (W / 2 + 1)])));
        const float2 xn = cmul(fn, cconj(__ldg(&FE32[ky * (W / 2 + 1) + W / 2])));
        sabs += fabsf(x0.x) + fabsf(x0.y) + fabsf(xn.x) + fabsf(xn.y);
        XN[q] = xn;
        B[q] = x0;                       // staged: other threads still read slot 0
    }
    __syncthreads();
    for (int q = threadIdx.x; q < H; q += blockDim.x) A[q * SA] = B[q];
    __syncthreads();
    *scale_out = sabs;                    // this thread's part; reduced with the integer argmax
    // a4: inverse column pass 1 (slot 0 packs X(.,0) + i X(.,W/2), whose transforms are real).
    // X(ky) sits at row fft_pos(ky); ky = N2h n1 + n2.
    fft_pass1<N1h, N2h, true, true>(
        SA, S.t4h,
        [&](int s, int n2, int n1) {
            const int q = fft_pos(N2h * n1 + n2, N1h, N2h);
            if (s == 0) {
                const float2 a = A[q * SA], n = XN[q];
                return make_float2(a.x - n.y, a.y + n.x);
            }
            return A[q * SA + s];
        },
        [&](int s, int n2, int k1, float2 v) { B[(N2h * k1 + n2) * SA + s] = v; });
    __syncthreads();
    fft_pass2<N1h, N2h, true, true>(
        SA, [&](int s, int k1, int n2) { return B[(N2h * k1 + n2) * SA + s]; },
        [&](int s, int k1, int k2, float2 v) { B[(N2h * k1 + k2) * SA + s] = v; });
    __syncthreads();
    // packed row r holds HW c(2r, x) + i HW c(2r+1, x) once the row passes are done
    t2.init();
    auto scan = [&](int r, int x, float2 v) {
        const int fe = (2 * r) * W + x;
        if (dbg) { dbg[fe] = v.x; dbg[fe + W] = v.y; }
        t2.push(g.sense * v.x, fe);
        t2.push(g.sense * v.y, fe + W);
    };
    // C2R rows: packed row r = Y(2r,.) + i Y(2r+1,.), Hermitian extension for kx > W/2.
    // kx = N2w n1 + n2 lies below W/2 exactly when n1 < N1w/2.
    fft_pass1<N1w, N2w, true, false>(
        Hh, S.t4w,
        [&](int r, int n2, int n1) {
            const float2* be = B + fft_pos(2 * r, N1h, N2h) * SA;
            const float2* bo = B + fft_pos(2 * r + 1, N1h, N2h) * SA;
            const int kx = N2w * n1 + n2;
            float2 ye, yo;
            if (2 * n1 < N1w) {
                if (kx == 0) { ye = make_float2(be[0].x, 0.f); yo = make_float2(bo[0].x, 0.f); }
                else { ye = be[kx]; yo = bo[kx]; }
            } else {
                if (2 * kx == W) { ye = make_float2(be[0].y, 0.f); yo = make_float2(bo[0].y, 0.f); }
                else { ye = cconj(be[W - kx]); yo = cconj(bo[W - kx]); }
            }
            return make_float2(ye.x - yo.y, ye.y + yo.x);
        },
        [&](int r, int n2, int k1, float2 v) {
            Z[r * SZ + RP * k1 + n2] = v;
            if (N2w == 1) scan(r, k1, v);
        });
    __syncthreads();
    if (N2w > 1) {
        fft_pass2<N1w, N2w, true, false>(
            Hh, [&](int s, int k1, int n2) { return Z[s * SZ + RP * k1 + n2]; },
            [&](int s, int k1, int k2, float2 v) {
                Z[s * SZ + RP * k1 + k2] = v;
                scan(s, k1 + N1w * k2, v);
            });
        __syncthreads();
    }
}

// Integer surface HW*c(y, x) from the packed-row buffer.
__device__ __forceinline__ float int_surface(const Geom& g, const Smem& S, int flat) {
    const int y = flat >> g.logW, x = flat & (g.W - 1);
    const float2 z = S.ZC[(y >> 1) * g.SZ + physZ(g, posW(g, x))];
    return (y & 1) ? z.y : z.x;
}

// FP64 direct sum c(s) = sum_r a((r + s) mod N) b(r) (left-hand side of Eq. (4)/(7)).
static __device__ double direct_sum_f64(const Geom& g, const Smem& S, const void* frame, long long pitch,
                                 int sy, int sx) {
    const double* b64 = S.ref ? S.ref->b64 : g.b64;
    double acc = 0.0;
    for (int idx = threadIdx.x; idx < g.H * g.W; idx += blockDim.x) {
        const int y = idx >> g.logW, x = idx & (g.W - 1);
        const int yy = (y + sy) & (g.H - 1), xx = (x + sx) & (g.W - 1);
        double I;
        if (g.in_dtype == 0) I = load_pixel((const unsigned short*)frame, (long long)yy * pitch + xx);
        else I = load_pixel((const float*)frame, (long long)yy * pitch + xx);
        acc = fma(operand_f64(I, g), __ldg(&b64[idx]), acc);
    }
    return block_sum(acc, S.rd);
}

// ------------------------------------------------------ a5: integer extremum
// Rare path of the integer search: collect every integer shift whose FP32 value is >= thr
// and re-decide among them by FP64 direct sums.
static __device__ int integer_collect(const Geom& g, const Smem& S, const void* frame, long long pitch,
                                                   float thr, int best, unsigned* flags) {
    if (threadIdx.x == 0) S.misc[0] = 0;
    __syncthreads();
    for (int idx = threadIdx.x; idx < g.H * g.W; idx += blockDim.x) {
        if (g.sense * int_surface(g, S, idx) >= thr) {
            const int k = atomicAdd(&S.misc[0], 1);
            if (k < kMaxIntCand) S.cj[k] = idx;
        }
    }
    __syncthreads();
    const int nc = S.misc[0];
    __syncthreads();
    *flags |= 0x01u;
    if (nc > kMaxIntCand) { *flags |= 0x08u; return best; }
    double bestv = -INFINITY;
    int bestj = INT_MAX;
    for (int k = 0; k < nc; ++k) {
        const int j = S.cj[k];
        const double v = (double)g.sense * direct_sum_f64(g, S, frame, pitch, j >> g.logW, j & (g.W - 1));
        if (v > bestv || (v == bestv && j < bestj)) { bestv = v; bestj = j; }
    }
    return bestj;
}


// t2: each thread's best point of the integer surface (value, natural flat index) and its
// runner-up value, collected while the inverse FFT stored them.
// *scale: in, this thread's part of the spectral sum; out, the block total.
__device__ __forceinline__ int integer_peak(const Geom& g, const Smem& S, const void* frame, long long pitch,
                                            float* scale_io, unsigned* flags, const Best2& t2) {
    float v1 = t2.v1;
    int best = t2.j1;
    const float scale = block_argmax_sum(v1, best, *scale_io, S.rv, S.rj, S.rv + 32);
    *scale_io = scale;
    if (!(v1 > -INFINITY)) { *flags |= 0x10u; return 0; }
    const float tau = g.tau_int * scale;
    if (!g.guard) return best;
    // unique unless some other shift lies within tau of the best
    const int near = __syncthreads_count((t2.v1 >= v1 - tau && t2.j1 != best) || t2.v2 >= v1 - tau);
    if (near == 0) return best;
    return integer_collect(g, S, frame, pitch, v1 - tau, best, flags);
}

// Stage tables -> shared memory by two bulk copies on the TMA engine (contiguous tables,
// 16-byte aligned, sizes multiples of 16 bytes), completing on the mbarrier S.bar.
__device__ __forceinline__ void tables_bar_init(const Smem& S) {
    if (threadIdx.x == 0) {
        const unsigned b = (unsigned)__cvta_generic_to_shared(S.bar);
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(b) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
}
// Issued by lane 0 of the last warp (idle in the step that follows, so the proxy fence's
// latency hides) after a __syncthreads that ends every generic access to the destination.
__device__ __forceinline__ void stage_tables_async(const Geom& g, const Smem& S) {
    if (!g.tables_smem || threadIdx.x != blockDim.x - 32) return;     // the last warp idles next
    const unsigned na = (unsigned)ta_bytes(g), nb = (unsigned)tb_bytes(g);
    const unsigned b = (unsigned)__cvta_generic_to_shared(S.bar);
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(b), "r"(na + nb) : "memory");
    const void* src[2] = {g.tAh, g.tBh};
    const void* dst[2] = {S.TA, S.TB};
    const unsigned n[2] = {na, nb};
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const unsigned d = (unsigned)__cvta_generic_to_shared(dst[i]);
        asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n"
                     ::"r"(d), "l"(src[i]), "r"(n[i]), "r"(b) : "memory");
    }
}
// Waits for the copies of phase `parity`. Bounded: returns false if they have not landed
// after `limit` polls (2^22 normally, far beyond any real copy time), true otherwise.
__device__ __forceinline__ bool stage_tables_wait(const Geom& g, const Smem& S, unsigned parity,
                                                  int limit = 1 << 22) {
    if (!g.tables_smem) return true;
    const unsigned b = (unsigned)__cvta_generic_to_shared(S.bar);
    for (int it = 0; it < limit; ++it) {
        unsigned done;
        asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
                     : "=r"(done) : "r"(b), "r"(parity) : "memory");
        if (done) return true;
    }
    return false;
}

// --------------------------------------------- a6 prologue: X' and P/Q, R, g
// Builds the stage-A operand planes S.PQ from the spectrum in S.A (and XN in place),
// X'(0, kx) in S.X0, R(kx) and g(+-tx).
static __device__ void build_pq_and_g(const Geom& g, const Smem& S, int py, int px, float scale) {
    const int H = g.H, W = g.W, SA = g.SA, Hh = g.Hh;
    const int pyy = py & (H - 1), pxx = px & (W - 1);
    const int ncol = SA + 1;          // slots 0..SA-1 and the Nyquist column
    // g(+-tx) sums the gc and ws tables (global, L2-resident) against R: a thread's first
    // task (part, tx) loads its kGTerms table entries now, so that their latency hides
    // behind the P/Q build. Task (part, tx) covers kx = part + kGParts j.
    const int ngt = kGParts * g.T1p;
    float pgc[kGTerms], pws[kGTerms];
    {
        const int task = threadIdx.x, part = task / g.T1p, tx = task - part * g.T1p;
#pragma unroll
        for (int j = 0; j < kGTerms; ++j) {
            const int kx = part + kGParts * j;
            const bool ok = task < ngt && kx < g.Wc;
            pgc[j] = ok ? __ldg(&g.tB_gc[kx * g.T1p + tx]) : 0.f;
            pws[j] = ok ? __ldg(&g.tB_ws[kx * g.T1p + tx]) : 0.f;
        }
    }
    // per-frame phase factors: ex(c) for the column slots, ey(m) for m = 0 .. Hh
    // (ey(-m) = conj ey(m); the Nyquist row's factor (-1)^py is real)
    for (int i = threadIdx.x; i < ncol + Hh + 1; i += blockDim.x) {
        if (i < ncol) {
            const int kx = (i == SA) ? W / 2 : i;
            S.ex[i] = twiddle_pos(S.tw, (signed_k(kx, W) * pxx) & (W - 1), g.logW, g.logNtw);
        } else {
            const int m = i - ncol;
            S.ey[m] = twiddle_pos(S.tw, (signed_k(m, H) * pyy) & (H - 1), g.logH, g.logNtw);
        }
    }
    __syncthreads();
    // X' = X e^{2 pi i k'.p/N} folded into P(m) = X'(m) + X'(-m), Q(m) = X'(m) - X'(-m),
    // m = 1 .. Hh (P(Hh) = X'(Hh); Q(Hh) = 0 outside the x-Nyquist column), and 8 partial
    // column sums of R(kx) = X'(0) + sum_{m<Hh} P(m) + X'(Hh). Regular column c, task
    // (part, c): the row pairs (2p+1, 2p+2), p = part (mod 8), and row 0 for part 0. The
    // planes reuse the spectrum's memory, so every task reads into registers first and
    // writes after a barrier (8 SA <= blockDim: one task per thread). The x-Nyquist column
    // stays FP32, folded in place in XN.
    const int Hq = Hh / 2, kexp = operand_exponent(scale);
    const float sc = ldexpf(1.f, kexp);
    if (threadIdx.x == 0) S.misc[3] = kexp;
    float2* R = (float2*)S.UV;
    float2* Rp = R + g.Wcp;                         // [8][ncol] partials
    constexpr int kMaxPairs = 4;                    // Hq / 8 (H <= 128)
    float2 pq[kMaxPairs][4];                        // P(m1), Q(m1), P(m2), Q(m2), scaled
    const int task = threadIdx.x;
    const int part = task / SA, c = task - part * SA;
    const bool mine = task < 8 * SA;
    if (mine) {
        const float2 ex = S.ex[c];
        float2 r = make_float2(0.f, 0.f);
        if (part == 0) {
            const float2 x0 = cmul(S.A[posH(g, 0) * SA + c], cmul(S.ey[0], ex));
            S.X0[c] = x0;
            r = x0;
        }
#pragma unroll
        for (int j = 0; j < kMaxPairs; ++j) {
            const int p = part + 8 * j;
            if (p >= Hq) break;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int m = 2 * p + 1 + h;
                const float2 ey = S.ey[m];
                float2 P, Q;
                if (m == Hh) {
                    P = cmul(S.A[posH(g, m) * SA + c], cmul(ey, ex));
                    Q = make_float2(0.f, 0.f);
                } else {
                    const float2 xp = cmul(S.A[posH(g, m) * SA + c], cmul(ey, ex));
                    const float2 xm = cmul(S.A[posH(g, H - m) * SA + c], cmul(cconj(ey), ex));
                    P = cadd(xp, xm);
                    Q = csub(xp, xm);
                }
                r = cadd(r, P);
                pq[j][2 * h] = make_float2(P.x * sc, P.y * sc);
                pq[j][2 * h + 1] = make_float2(Q.x * sc, Q.y * sc);
            }
        }
        Rp[part * ncol + c] = r;
    }
    // x-Nyquist column, folded in place in XN (FP32) by the last two warps, one row m (and
    // its mirror H - m) per thread; their P sums are reduced per warp into parts 0 and 1
    {
        const int l = (int)threadIdx.x - ((int)blockDim.x - 64);
        if (l >= 0) {
            const float2 ex = S.ex[SA];
            float2 r = make_float2(0.f, 0.f);
            for (int m = l; m <= Hh; m += 64) {
                const float2 ey = S.ey[m];
                if (m == 0 || m == Hh) {
                    float2* p = S.XN + posH(g, m);
                    const float2 x = cmul(*p, cmul(ey, ex));
                    *p = x;
                    r = cadd(r, x);
                } else {
                    float2* rp = S.XN + posH(g, m);
                    float2* rm = S.XN + posH(g, H - m);
                    const float2 xp = cmul(*rp, cmul(ey, ex));
                    const float2 xm = cmul(*rm, cmul(cconj(ey), ex));
                    const float2 pm = cadd(xp, xm);
                    *rp = pm;
                    *rm = csub(xp, xm);
                    r = cadd(r, pm);
                }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                r.x += __shfl_xor_sync(0xffffffffu, r.x, o);
                r.y += __shfl_xor_sync(0xffffffffu, r.y, o);
            }
            if ((l & 31) == 0) Rp[(l >> 5) * ncol + SA] = r;
            if (l < 6) Rp[(2 + l) * ncol + SA] = make_float2(0.f, 0.f);
        }
    }
    __syncthreads();
    if (mine && g.tc) {
        // eight matrices [Pr hi, Pi hi, Pr lo, Pi lo, Qr hi, Qi hi, Qr lo, Qi lo] (so that Pr and
        // Pi, and Qr and Qi, form one 2 SA-row operand): row c, K = m - 1; the pair (m1, m2) is
        // two adjacent K values, one 32-bit store per matrix
        unsigned char* pqb = (unsigned char*)S.PQ;
        const size_t ms = (size_t)SA * 128;
#pragma unroll
        for (int j = 0; j < kMaxPairs; ++j) {
            const int p = part + 8 * j;
            if (p >= Hq) break;
            const uint32_t off = sw128_off(c, 2 * p);
            const uint2 v[4] = {split_pair(pq[j][0].x, pq[j][2].x), split_pair(pq[j][0].y, pq[j][2].y),
                                split_pair(pq[j][1].x, pq[j][3].x), split_pair(pq[j][1].y, pq[j][3].y)};
#pragma unroll
            for (int pl = 0; pl < 4; ++pl) {
                const int mi = (pl >> 1) * 4 + (pl & 1);
                *(unsigned*)(pqb + mi * ms + off) = v[pl].x;
                *(unsigned*)(pqb + (mi + 2) * ms + off) = v[pl].y;
            }
        }
    } else if (mine) {
        const int sw = pswz(c, Hq);
#pragma unroll
        for (int j = 0; j < kMaxPairs; ++j) {
            const int p = part + 8 * j;
            if (p >= Hq) break;
            const int q = p ^ sw;
            S.PQ[(0 * SA + c) * Hq + q] = split_pair(pq[j][0].x, pq[j][2].x);     // Pr
            S.PQ[(1 * SA + c) * Hq + q] = split_pair(pq[j][0].y, pq[j][2].y);     // Pi
            S.PQ[(2 * SA + c) * Hq + q] = split_pair(pq[j][1].x, pq[j][3].x);     // Qr
            S.PQ[(3 * SA + c) * Hq + q] = split_pair(pq[j][1].y, pq[j][3].y);     // Qi
        }
    }
    __syncthreads();
    for (int c = threadIdx.x; c < ncol; c += blockDim.x) {
        float2 r = make_float2(0.f, 0.f);
        for (int part = 7; part >= 0; --part) r = cadd(r, Rp[part * ncol + c]);
        R[c == SA ? W / 2 : c] = r;
    }
    __syncthreads();
    // g(+-tx) = sum_kx gc Rr -+ ws Ri: kGParts partial sums per tx, then totals
    float* gpart = (float*)(Rp + 8 * ncol);          // [kGParts][T1p][2]
    for (int task = threadIdx.x; task < ngt; task += blockDim.x) {
        const int part = task / g.T1p, tx = task - part * g.T1p;
        float a = 0.f, b = 0.f;
        int kx = part + kGParts * (kGTerms - 1);
        if (task == (int)threadIdx.x) {
#pragma unroll
            for (int j = kGTerms - 1; j >= 0; --j, kx -= kGParts) {
                if (kx < g.Wc) {
                    const float2 r = R[kx];
                    a = fmaf(pgc[j], r.x, a);
                    b = fmaf(pws[j], r.y, b);
                }
            }
        } else {
            for (; kx >= 0; kx -= kGParts) {
                if (kx < g.Wc) {
                    const float2 r = R[kx];
                    a = fmaf(__ldg(&g.tB_gc[kx * g.T1p + tx]), r.x, a);
                    b = fmaf(__ldg(&g.tB_ws[kx * g.T1p + tx]), r.y, b);
                }
            }
        }
        gpart[2 * task] = a;
        gpart[2 * task + 1] = b;
    }
    __syncthreads();
    for (int tx = threadIdx.x; tx < g.T1p; tx += blockDim.x) {
        float a = 0.f, b = 0.f;
        for (int part = kGParts - 1; part >= 0; --part) {
            a += gpart[2 * (part * g.T1p + tx)];
            b += gpart[2 * (part * g.T1p + tx) + 1];
        }
        S.gP[tx] = a - b;
        S.gM[tx] = a + b;
    }
    __syncthreads();
}

// --------------------------------------------------- a6: stage A (one chunk)
// For t = t0 + lt, lt in [0, TC) and every regular column kx < SA:
//   U'r, U'i = sum_m (cos - 1)(2 pi m t/(uH)) (Pr, Pi)(m, kx),  Vr, Vi = sum_m sin(..) (Qr, Qi)(m, kx),
// stored as the combinations stage B contracts, C0 = U'r - Vi, C1 = U'r + Vi,
// E0 = U'i + Vr, E1 = U'i - Vr (scaled by 2^kexp, fp16 pairs, CB); CBN gets them in FP32
// for the x-Nyquist column, whose Nyquist row keeps the full phase (Q(Hh) = -P(Hh)).

// the four combinations from (U'r, U'i, Vr, Vi)
__device__ __forceinline__ float4 combos(float ur, float ui, float vr, float vi) {
    return make_float4(ur - vi, ur + vi, ui + vr, ui - vr);
}

__device__ __forceinline__ void stage_a_nyquist(const Geom& g, const Smem& S, int t0, const uint2* TA) {
    const int H = g.H, Hh = g.Hh, Hq = Hh / 2, TC = g.TC;
    const uint2* Tc = TA;
    const uint2* Ts = TA + (size_t)g.TAB * Hq;
    const float un = ldexpf(1.f, -13);
    // item (lt, part): the m pairs p = part (mod 4); the four parts of one row are adjacent
    // lanes and are summed by shuffles
    for (int base = 0; base < 4 * TC; base += blockDim.x) {
        const int item = base + threadIdx.x, lt = item >> 2, part = item & 3;
        float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
        if (lt < TC) {
            const int ta = t0 - 1 + lt, sw = pswz(ta, Hq);
            for (int p = Hq - 1 - part; p >= 0; p -= 4) {
                const int m1 = 2 * p + 1, m2 = 2 * p + 2;
                float2 cm, sn;
                if (g.tc) {
                    // matrices [cos - 1, sin] x [hi, lo] of RA rows; row ta, K = m - 1
                    const size_t ms = (size_t)g.RA * 128;
                    const unsigned char* b = (const unsigned char*)TA + sw128_off(ta, 2 * p);
                    const __half2 ch = *(const __half2*)b, cl = *(const __half2*)(b + ms);
                    const __half2 shv = *(const __half2*)(b + 2 * ms), slv = *(const __half2*)(b + 3 * ms);
                    cm = make_float2(__low2float(ch) + __low2float(cl), __high2float(ch) + __high2float(cl));
                    sn = make_float2(__low2float(shv) + __low2float(slv), __high2float(shv) + __high2float(slv));
                } else {
                    cm = unsplit_pair(Tc[ta * Hq + (p ^ sw)]);
                    sn = unsplit_pair(Ts[ta * Hq + (p ^ sw)]);
                }
                const float2 p1 = S.XN[posH(g, m1)], p2 = S.XN[posH(g, m2)], q1 = S.XN[posH(g, H - m1)];
                const float2 q2 = (m2 == Hh) ? make_float2(-p2.x, -p2.y) : S.XN[posH(g, H - m2)];
                acc.x = fmaf(cm.x * un, p1.x, fmaf(cm.y * un, p2.x, acc.x));
                acc.y = fmaf(cm.x * un, p1.y, fmaf(cm.y * un, p2.y, acc.y));
                acc.z = fmaf(sn.x * un, q1.x, fmaf(sn.y * un, q2.x, acc.z));
                acc.w = fmaf(sn.x * un, q1.y, fmaf(sn.y * un, q2.y, acc.w));
            }
        }
#pragma unroll
        for (int o = 1; o < 4; o <<= 1) {
            acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
            acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
            acc.z += __shfl_xor_sync(0xffffffffu, acc.z, o);
            acc.w += __shfl_xor_sync(0xffffffffu, acc.w, o);
        }
        if (lt < TC && part == 0) {
            const float4 cb = combos(acc.x, acc.y, acc.z, acc.w);
            S.CBN[lt] = cb.x;
            S.CBN[TC + lt] = cb.y;
            S.CBN[2 * TC + lt] = cb.z;
            S.CBN[3 * TC + lt] = cb.w;
        }
    }
}

// write the combinations of (row lt, K pair kp) of the four accumulators (already in the
// 2^kexp scale) as fp16 pairs
__device__ __forceinline__ void store_combo_pairs(const Geom& g, const Smem& S, int lt, int kp, float2 ur, float2 ui,
                                                  float2 vr, float2 vi) {
    const int SAq = g.SA / 2, TC = g.TC;
    const int q = kp ^ pswz(lt, SAq);
    const float4 a = combos(ur.x, ui.x, vr.x, vi.x), b = combos(ur.y, ui.y, vr.y, vi.y);
    S.CB[(0 * TC + lt) * SAq + q] = split_pair(a.x, b.x);
    S.CB[(1 * TC + lt) * SAq + q] = split_pair(a.y, b.y);
    S.CB[(2 * TC + lt) * SAq + q] = split_pair(a.z, b.z);
    S.CB[(3 * TC + lt) * SAq + q] = split_pair(a.w, b.w);
}

// Tensor-core form (Hh a multiple of 16): M = t, N = kx, K = m. A warp task is one t tile
// of 16 by one kx tile of 8, with the four products (Cm1 Pr, Cm1 Pi, S Qr, S Qi) sharing
// the A fragments. Rows past the chunk read its last row and are not stored.
template <int H, int W>
__device__ __forceinline__ void stage_a_mma(const Geom& g, const Smem& S, int t0, const uint2* TA) {
    constexpr int Hq = H / 4, NKS = Hq / 8, SA = W / 2;
    constexpr unsigned R8 = 8u * Hq * 8u;                        // 8 table rows, bytes
    constexpr unsigned PL = (unsigned)SA * Hq * 8u;              // one P/Q plane, bytes
    const int TC = g.TC;
    const uint2* Tc = TA;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    const int gq = lane >> 2, tq = lane & 3;
    const int ntt = (TC + 15) >> 4, nnt = SA >> 3;
    const float un = ldexpf(1.f, -13);
    for (int task = warp; task < ntt * nnt; task += nwarp) {
        const int tt = task / nnt, nt = task - tt * nnt;
        if (t0 + 16 * tt > g.h0) continue;                       // warp-uniform: all rows past h0
        // table rows t0 - 1 + lt for lt = 16 tt + gq (+ 8); rows past the chunk read the
        // following table rows (in bounds: TAB >= t0 - 1 + 16 ceil(TC / 16) or the next
        // table / region) and are not stored
        const RowOffsets tr(Tc, Hq, t0 - 1 + 16 * tt + gq, tq);
        const unsigned dts = (unsigned)((size_t)g.TAB * Hq * 8u);   // Ts - Tc, bytes
        const RowOffsets pq(S.PQ, Hq, 8 * nt + gq, tq);
        float d[4][4];
#pragma unroll
        for (int pl = 0; pl < 4; ++pl)
#pragma unroll
            for (int e = 0; e < 4; ++e) d[pl][e] = 0.f;
#pragma unroll
        for (int s = 0; s < NKS; ++s) {
            unsigned ch[4], cl[4], sh[4], sl[4];
            load_afrag(tr, 0u, R8, s, ch, cl);
            load_afrag(tr, dts, R8, s, sh, sl);
            const uint2 b0[4] = {pq.at(s, 0), pq.at(s, 0, PL), pq.at(s, 0, 2 * PL), pq.at(s, 0, 3 * PL)};
            const uint2 b1[4] = {pq.at(s, 1), pq.at(s, 1, PL), pq.at(s, 1, 2 * PL), pq.at(s, 1, 3 * PL)};
            // the three split products, each issued across the four independent accumulators
#pragma unroll
            for (int pl = 0; pl < 4; ++pl) mma_f16(d[pl], pl < 2 ? cl : sl, b0[pl].x, b1[pl].x);
#pragma unroll
            for (int pl = 0; pl < 4; ++pl) mma_f16(d[pl], pl < 2 ? ch : sh, b0[pl].y, b1[pl].y);
#pragma unroll
            for (int pl = 0; pl < 4; ++pl) mma_f16(d[pl], pl < 2 ? ch : sh, b0[pl].x, b1[pl].x);
        }
        // element e: row gq + 8 (e >> 1), kx 8 nt + 2 tq + (e & 1)
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int lt = 16 * tt + gq + 8 * h;
            if (lt >= TC) continue;
            store_combo_pairs(g, S, lt, 4 * nt + tq, make_float2(d[0][2 * h] * un, d[0][2 * h + 1] * un),
                              make_float2(d[1][2 * h] * un, d[1][2 * h + 1] * un),
                              make_float2(d[2][2 * h] * un, d[2][2 * h + 1] * un),
                              make_float2(d[3][2 * h] * un, d[3][2 * h + 1] * un));
        }
    }
}

// Plain form for Hh < 16: one thread per (t, kx pair), operands reconstructed in FP32.
__device__ __forceinline__ void stage_a_simt(const Geom& g, const Smem& S, int t0, const uint2* TA) {
    const int Hq = g.Hh / 2, SA = g.SA, SAq = SA / 2, TC = g.TC;
    const uint2* Tc = TA;
    const uint2* Ts = TA + (size_t)g.TAB * Hq;
    const float un = ldexpf(1.f, -13);
    for (int task = threadIdx.x; task < TC * SAq; task += blockDim.x) {
        const int lt = task / SAq, kp = task - lt * SAq, ta = t0 - 1 + lt;
        float2 acc[4] = {};
        for (int x = 0; x < 2; ++x) {
            const int kx = 2 * kp + x, sb = pswz(kx, Hq);
            for (int p = Hq - 1; p >= 0; --p) {
                const float2 cm = unsplit_pair(Tc[ta * Hq + (p ^ pswz(ta, Hq))]);
                const float2 sn = unsplit_pair(Ts[ta * Hq + (p ^ pswz(ta, Hq))]);
                float v[4];
#pragma unroll
                for (int pl = 0; pl < 4; ++pl) {
                    const float2 w = unsplit_pair(S.PQ[(size_t)(pl * SA + kx) * Hq + (p ^ sb)]);
                    const float2 t = pl < 2 ? cm : sn;
                    v[pl] = t.x * w.x + t.y * w.y;
                }
                if (x == 0) { acc[0].x += v[0]; acc[1].x += v[1]; acc[2].x += v[2]; acc[3].x += v[3]; }
                else { acc[0].y += v[0]; acc[1].y += v[1]; acc[2].y += v[2]; acc[3].y += v[3]; }
            }
        }
        store_combo_pairs(g, S, lt, kp, make_float2(acc[0].x * un, acc[0].y * un), make_float2(acc[1].x * un, acc[1].y * un),
                          make_float2(acc[2].x * un, acc[2].y * un), make_float2(acc[3].x * un, acc[3].y * un));
    }
}

template <int H, int W>
__device__ __forceinline__ void stage_a(const Geom& g, const Smem& S, int t0, const uint2* TA) {
    // the warp-MMA form takes kx tiles of 8 columns: W >= 16 (W = 8 has W/2 = 4 columns)
    if constexpr (H % 32 == 0 && W >= 16) {
        if (g.tables_smem) stage_a_mma<H, W>(g, S, t0, TA);
        else stage_a_simt(g, S, t0, TA);
    } else {
        stage_a_simt(g, S, t0, TA);
    }
    stage_a_nyquist(g, S, t0, TA);
    __syncthreads();
}

__device__ __forceinline__ int grid_index(const Geom& g, int ty, int tx) {
    return (ty + g.h0) * g.M + (tx + g.h0);
}

// --------------------------------------------------- a6: stage B (one chunk)
// Stage B evaluates v = sense * (S + g) at every grid point whose |ty| lies in the chunk
// (t = t0 .. t0 + TC - 1, t >= 1) and feeds the top-K (with kCollect: appends every point
// with v >= thr to the candidate list instead). With the stage-A combinations,
//   A0 = sum_kx wc C0, B0 = sum_kx ws E0 give S(+t, +-tx) = A0 -+ B0 (+ g(+-tx)),
//   A1 = sum_kx wc C1, B1 = sum_kx ws E1 give S(-t, +-tx) = A1 -+ B1 (+ g(+-tx)),
// where wc = w cos(2 pi kx tx/(uW)), ws = w sin(..), w = 1 at kx = 0 and W/2, else 2.
template <bool kCollect>
struct Emitter {
    const Geom& g;
    const Smem& S;
    TopK<kTopK>& top;
    // thr: candidate-list threshold (kCollect), else a lower bound below which no point can
    // be the maximum or within the near-tie band of it (the (0, 0) point's value minus that
    // band): most points stop at this one comparison. In top-K mode each thread raises it
    // as it keeps points: no point below the thread's best so far minus the band can be
    // within the band of the maximum. The raise uses twice the band, so that its rounding
    // (an ulp of values of a few percent of sum w|X|, against a band of eps32 sum w|X|)
    // keeps it below the threshold the guard applies later.
    mutable float thr;
    float* dbg;
    float band;
    __device__ __forceinline__ Emitter(const Geom& g_, const Smem& S_, TopK<kTopK>& top_, float thr_, float* dbg_)
        : g(g_), S(S_), top(top_), thr(thr_), dbg(dbg_), band(2.f * (g_.sense * S_.gP[0] - thr_)) {}
    __device__ __forceinline__ void raise(float v) const {
        if (!kCollect && !dbg) thr = fmaxf(thr, v - band);
    }
    __device__ __forceinline__ void operator()(float raw, int ty, int tx) const {
        const float v = g.sense * raw;
        if (!kCollect && dbg) dbg[grid_index(g, ty, tx)] = raw;
        if (!(v >= thr)) return;
        const int j = grid_index(g, ty, tx);
        if (kCollect) {
            const int k = atomicAdd(&S.misc[1], 1);
            if (k < kMaxCand) { S.cj[k] = j; S.cv[k] = v; }
        } else {
            top.push(v, j);
            raise(v);
        }
    }
    // the two points (+-tx) of row t of the sign `sg` (0: +t, 1: -t) from (A, B)
    __device__ __forceinline__ void quad(int sg, int t, int x, float A, float B) const {
        const float rp = A - B + S.gP[x], rm = A + B + S.gM[x];
        if (!kCollect && dbg) {
            const int ts = sg ? -t : t;
            if ((sg || t <= g.pmax) && x <= g.pmax) dbg[grid_index(g, ts, x)] = rp;
            if ((sg || t <= g.pmax) && x >= 1) dbg[grid_index(g, ts, -x)] = rm;
        }
        if (!(g.sense * rp >= thr) && !(g.sense * rm >= thr)) return;      // the common case
        const int ts = sg ? -t : t;
        if ((sg || t <= g.pmax) && x <= g.pmax) keep(g.sense * rp, ts, x);
        if ((sg || t <= g.pmax) && x >= 1) keep(g.sense * rm, ts, -x);
    }
    __device__ __forceinline__ void keep(float v, int ty, int tx) const {
        if (!(v >= thr)) return;
        const int j = grid_index(g, ty, tx);
        if (kCollect) {
            const int k = atomicAdd(&S.misc[1], 1);
            if (k < kMaxCand) { S.cj[k] = j; S.cv[k] = v; }
        } else {
            top.push(v, j);
            raise(v);
        }
    }
};

// Tensor-core form (SA a multiple of 16): M = t, N = tx, K = kx < SA; the x-Nyquist column
// is a rank-one FP32 term. A warp task is (t tile of 16, sign, two tx tiles of 8). Rows
// past the chunk (or the tables) read the last row and are discarded. dsc = 2^-(13+kexp)
// undoes the operand scales.
template <int W, bool kCollect>
__device__ __forceinline__ void stage_b_mma(const Geom& g, const Smem& S, int t0, const uint2* TB, float dsc,
                                            const Emitter<kCollect>& emit) {
    constexpr int SAq = W / 4, NKS = SAq / 8;
    constexpr unsigned R8 = 8u * SAq * 8u;                       // 8 operand rows, bytes
    const int T1 = g.T1p, T8 = g.T1p8, TC = g.TC;
    const uint2* WC = TB;
    const float* WCN = (const float*)(TB + 2 * (size_t)T1 * SAq);
    const float* WSN = WCN + T8;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    const int gq = lane >> 2, tq = lane & 3;
    const int ntt = (TC + 15) >> 4, nnt = T8 >> 3, nng = (nnt + 1) >> 1;
    const int ntask = ntt * 2 * nng;
    for (int task = warp; task < ntask; task += nwarp) {
        const int tt = task / (2 * nng);
        const int rem = task - tt * 2 * nng;
        const int sg = rem / nng;
        const int nt0 = 2 * (rem - sg * nng);
        if (t0 + 16 * tt > g.h0) continue;                       // warp-uniform
        const bool two = nt0 + 1 < nnt;                          // warp-uniform
        const uint2* Ca = S.CB + (size_t)sg * TC * SAq;          // C0 / C1 (E0 / E1 at deb bytes on)
        // rows 16 tt + gq (+ 8) of the combinations and tx rows 8 nt0 + gq (+ 8) of the tables;
        // rows past the chunk / the tables read the following rows of the shared area (in
        // bounds) and only feed discarded outputs
        const RowOffsets ra(Ca, SAq, 16 * tt + gq, tq), rx(WC, SAq, 8 * nt0 + gq, tq);
        const unsigned deb = (unsigned)((size_t)2 * TC * SAq * 8u);       // Eb - Ca, bytes
        const unsigned dws = (unsigned)((size_t)T1 * SAq * 8u);           // WS - WC, bytes
        const unsigned x8 = two ? R8 : 0u;                                // second tx tile
        float dA[2][4], dB[2][4];
#pragma unroll
        for (int j = 0; j < 2; ++j)
#pragma unroll
            for (int e = 0; e < 4; ++e) { dA[j][e] = 0.f; dB[j][e] = 0.f; }
#pragma unroll
        for (int s = 0; s < NKS; ++s) {
            unsigned ah[4], al[4], eh[4], el[4];
            load_afrag(ra, 0u, R8, s, ah, al);
            load_afrag(ra, deb, R8, s, eh, el);
            const uint2 c0[2] = {rx.at(s, 0), rx.at(s, 0, x8)}, c1[2] = {rx.at(s, 1), rx.at(s, 1, x8)};
            const uint2 s0[2] = {rx.at(s, 0, dws), rx.at(s, 0, dws + x8)}, s1[2] = {rx.at(s, 1, dws), rx.at(s, 1, dws + x8)};
            // the three split products, each issued across the four independent accumulators
            // (for a single tx tile, x1 = x0 repeats a valid row and its results are unused)
#pragma unroll
            for (int j = 0; j < 2; ++j) { mma_f16(dA[j], al, c0[j].x, c1[j].x); mma_f16(dB[j], el, s0[j].x, s1[j].x); }
#pragma unroll
            for (int j = 0; j < 2; ++j) { mma_f16(dA[j], ah, c0[j].y, c1[j].y); mma_f16(dB[j], eh, s0[j].y, s1[j].y); }
#pragma unroll
            for (int j = 0; j < 2; ++j) { mma_f16(dA[j], ah, c0[j].x, c1[j].x); mma_f16(dB[j], eh, s0[j].x, s1[j].x); }
        }
        // epilogue: fragment element e sits at row gq + 8 (e >> 1), column 2 tq + (e & 1).
        // Per row h: the x-Nyquist terms; per column: the tables' kx = W/2 entries and g(+-x).
        const float* CaN = S.CBN + (size_t)sg * TC;
        const float* EbN = S.CBN + (size_t)(2 + sg) * TC;
        const int lt0 = 16 * tt + gq;
        const int ltc[2] = {min(lt0, TC - 1), min(lt0 + 8, TC - 1)};
        const float can[2] = {CaN[ltc[0]], CaN[ltc[1]]}, ebn[2] = {EbN[ltc[0]], EbN[ltc[1]]};
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            if (j == 1 && !two) break;
#pragma unroll
            for (int xo = 0; xo < 2; ++xo) {
                const int x = 8 * (nt0 + j) + 2 * tq + xo;
                if (x > g.h0) continue;
                const float wcn = WCN[x], wsn = WSN[x];
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int lt = lt0 + 8 * h, t = t0 + lt;
                    if (lt >= TC || t > g.h0) continue;
                    const int e = 2 * h + xo;
                    emit.quad(sg, t, x, fmaf(wcn, can[h], dA[j][e] * dsc), fmaf(wsn, ebn[h], dB[j][e] * dsc));
                }
            }
        }
    }
}

// Plain form for SA < 16: one thread per (t, tx), operands reconstructed in FP32.
template <bool kCollect>
__device__ __forceinline__ void stage_b_simt(const Geom& g, const Smem& S, int t0, const uint2* TB, float dsc,
                                             const Emitter<kCollect>& emit) {
    const int SAq = g.SA / 2, T1 = g.T1p, T8 = g.T1p8, TC = g.TC;
    const uint2* WC = TB;
    const uint2* WS = TB + (size_t)T1 * SAq;
    const float* WCN = (const float*)(TB + 2 * (size_t)T1 * SAq);
    const float* WSN = WCN + T8;
    for (int task = threadIdx.x; task < TC * T1; task += blockDim.x) {
        const int lt = task / T1, x = task - lt * T1, t = t0 + lt;
        if (t > g.h0 || x > g.h0) continue;
        const int sl = pswz(lt, SAq), sx = pswz(x, SAq);
        for (int sg = 0; sg < 2; ++sg) {
            const uint2* Ca = S.CB + ((size_t)sg * TC + lt) * SAq;
            const uint2* Eb = S.CB + ((size_t)(2 + sg) * TC + lt) * SAq;
            float A = 0.f, B = 0.f;
            for (int kp = SAq - 1; kp >= 0; --kp) {
                const float2 wc = unsplit_pair(WC[x * SAq + (kp ^ sx)]), ws = unsplit_pair(WS[x * SAq + (kp ^ sx)]);
                const float2 ca = unsplit_pair(Ca[kp ^ sl]), eb = unsplit_pair(Eb[kp ^ sl]);
                A += wc.x * ca.x + wc.y * ca.y;
                B += ws.x * eb.x + ws.y * eb.y;
            }
            A = fmaf(WCN[x], S.CBN[sg * TC + lt], A * dsc);
            B = fmaf(WSN[x], S.CBN[(2 + sg) * TC + lt], B * dsc);
            emit.quad(sg, t, x, A, B);
        }
    }
}

// The upsampled surface on the 5th-generation tensor cores (g.tc: H = W = 128, one chunk,
// tables in shared memory). One thread issues every MMA; the accumulators live in Tensor
// Memory, and the other threads never hold them in registers.
//   Stage A: D_a[t][kx] = sum_m T[t][m] P_a[kx][m] for a = (Cm1 Pr, Cm1 Pi, S Qr, S Qi), four
//   M = 128 (t rows; rows past TC are discarded), N = 64 (kx), K = 64 (m) accumulators in
//   columns 64 a, each as lo*hi + hi*lo + hi*hi of the fp16 pairs.
//   Its rows are read back one t row per lane, combined (C0, C1, E0, E1) and written as
//   stage B's fp16 pair operands over the stage-A tables.
//   Stage B: D_b[tx][t] = sum_kx Wtab[tx][kx] CE_b[t][kx] for b = (wc C0, ws E0, wc C1, ws E1),
//   four M = 128 (tx lanes), N = NB (t) accumulators in columns NB b; the epilogue feeds
//   the same Emitter as the warp-level form. The x-Nyquist column and the t = 0 row are FP32,
//   as in the other forms.
// A batch of MMAs that does not complete within the bounded wait marks the CTA failed
// (TcShared::failed): no further MMA is issued and the caller stops the CTA.
template <bool kCollect>
__device__ void upsampled_pass_tc(const Geom& g, const Smem& S, TopK<kTopK>& top, float thr, float* dbg) {
    TcShared* ts = tc_shared();
    const uint32_t tmem = ts->tmem, bar = smem_addr(&ts->bar);
    const float dsc = ldexpf(1.f, -13 - S.misc[3]);
    const float un = ldexpf(1.f, -13);
    const Emitter<kCollect> emit{g, S, top, thr, dbg};
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, sp = warp & 3, grp = warp >> 2;
    const int SA = g.SA, TC = g.TC, NB = g.NB, RA = g.RA, T8 = g.T1p8;
    const uint32_t pq = smem_addr(S.PQ), ta = smem_addr(S.TA), tb = smem_addr(S.TB);
    unsigned char* cb = (unsigned char*)S.CB;
    const uint32_t lanes = (uint32_t)(32 * sp) << 16;          // this warp's Tensor Memory lanes
    constexpr int kWait = 1 << 22;
    // the P/Q planes were written by ordinary stores: make them visible to the tensor cores
    tc_fence_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const bool live = ts->failed == 0;
    // the MMAs are issued by the last thread, idle in the x-Nyquist step (4 TC items) and in
    // the t = 0 row (h0 + 1 items) that run beside them; issue takes about as long as the MMAs
    const bool issuer = threadIdx.x == blockDim.x - 1;
    if (issuer && live) {
        // two N = 2 SA MMAs: U = Cm1 [Pr; Pi] (columns 0 .. 127), V = S [Qr; Qi] (128 .. 255)
        const uint32_t id = tc_idesc(128, 2 * SA);
        for (int a = 0; a < 2; ++a) {
            const uint32_t am = ta + (uint32_t)(2 * a * RA * 128), al = am + (uint32_t)(RA * 128);
            const uint32_t bm = pq + (uint32_t)(4 * a * SA * 128), bl = bm + (uint32_t)(2 * SA * 128);
            const uint32_t d = tmem + (uint32_t)(2 * SA * a);
            for (int st = 0; st < 4; ++st) {
                const uint32_t ko = 32u * st;
                tc_mma(d, tc_desc(al + ko), tc_desc(bm + ko), id, st > 0 ? 1u : 0u);
                tc_mma(d, tc_desc(am + ko), tc_desc(bl + ko), id, 1u);
                tc_mma(d, tc_desc(am + ko), tc_desc(bm + ko), id, 1u);
            }
        }
        tc_commit(bar);
    }
    stage_a_nyquist(g, S, 1, S.TA);                            // FP32, beside the MMAs
    bool ok = live && tc_bar_wait(bar, ts->batches & 1u, kWait);
    tc_fence_after();
    if (__syncthreads_or(live && !ok)) {
        if (threadIdx.x == 0) ts->failed = 1;
    }
    const bool liveA = live && __syncthreads_and(ok);          // (also: the table reads are done)
    if (threadIdx.x == 0 && live) ts->batches++;
    // stage A read back: lane = t row lt, this warp's 16 kx of each accumulator
    {
        const int lt = 32 * sp + lane;
        float ur[16], ui[16], vr[16], vi[16];
        tc_ld16(tmem + lanes + 0 * 64 + 16 * grp, ur);
        tc_ld16(tmem + lanes + 1 * 64 + 16 * grp, ui);
        tc_ld16(tmem + lanes + 2 * 64 + 16 * grp, vr);
        tc_ld16(tmem + lanes + 3 * 64 + 16 * grp, vi);
        tc_ld_wait();
        if (lt < NB && liveA) {
            const size_t ms = (size_t)NB * 128;
            const bool row = lt < TC;
#pragma unroll
            for (int j = 0; j < 16; j += 2) {
                const uint32_t off = sw128_off(lt, 16 * grp + j);
                float4 a = make_float4(0.f, 0.f, 0.f, 0.f), b = a;
                if (row) {
                    a = combos(ur[j] * un, ui[j] * un, vr[j] * un, vi[j] * un);
                    b = combos(ur[j + 1] * un, ui[j + 1] * un, vr[j + 1] * un, vi[j + 1] * un);
                }
                const uint2 v[4] = {split_pair(a.x, b.x), split_pair(a.y, b.y), split_pair(a.z, b.z), split_pair(a.w, b.w)};
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    // [C0 hi, C1 hi, C0 lo, C1 lo, E0 hi, E1 hi, E0 lo, E1 lo]
                    const int mi = (c >> 1) * 4 + (c & 1);
                    *(unsigned*)(cb + mi * ms + off) = v[c].x;
                    *(unsigned*)(cb + (mi + 2) * ms + off) = v[c].y;
                }
            }
        }
    }
    tc_fence_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (issuer && liveA) {
        // two N = 2 NB MMAs: wc [C0; C1] (columns 0 .. 2 NB - 1: A0, A1) and ws [E0; E1]
        // (2 NB .. 4 NB - 1: B0, B1)
        const uint32_t id = tc_idesc(128, 2 * NB);
        const uint32_t cbs = smem_addr(cb);
        for (int b = 0; b < 2; ++b) {
            const uint32_t am = tb + (uint32_t)(2 * b * T8 * 128), al = am + (uint32_t)(T8 * 128);
            const uint32_t bm = cbs + (uint32_t)(4 * b * NB * 128), bl = bm + (uint32_t)(2 * NB * 128);
            const uint32_t d = tmem + (uint32_t)(2 * NB * b);
            for (int st = 0; st < 4; ++st) {
                const uint32_t ko = 32u * st;
                tc_mma(d, tc_desc(al + ko), tc_desc(bm + ko), id, st > 0 ? 1u : 0u);
                tc_mma(d, tc_desc(am + ko), tc_desc(bl + ko), id, 1u);
                tc_mma(d, tc_desc(am + ko), tc_desc(bm + ko), id, 1u);
            }
        }
        tc_commit(bar);
    }
    // the t = 0 row: S = 0, the surface is g(tx)
    float vmax = -INFINITY;                                     // this thread's largest surface value
    for (int x = threadIdx.x; x <= g.h0; x += blockDim.x) {
        if (x <= g.pmax) { emit(S.gP[x], 0, x); vmax = fmaxf(vmax, g.sense * S.gP[x]); }
        if (x >= 1) { emit(S.gM[x], 0, -x); vmax = fmaxf(vmax, g.sense * S.gM[x]); }
    }
    ok = liveA && tc_bar_wait(bar, ts->batches & 1u, kWait);
    tc_fence_after();
    if (__syncthreads_or(liveA && !ok)) {
        if (threadIdx.x == 0) ts->failed = 1;
    }
    const bool liveB = liveA && __syncthreads_and(ok);
    if (threadIdx.x == 0 && liveA) ts->batches++;
    // epilogue, in two steps. The warps that own the accumulator lanes (tx rows; only the
    // tx <= h0 of them matter, so one SMSP's warps would idle) move the final stage-B values
    // (A, B) of each (sign, t, tx), with the x-Nyquist terms, into the dead table area as
    // float2 [sg][lt][tx]; then every warp feeds the Emitter from there.
    float2* stg = (float2*)S.TB;                                // TB + TA/CB are dead now
    {
        const int x = 32 * sp + lane;
        const bool xok = liveB && x <= g.h0;
        const float* WCN = (const float*)((const unsigned char*)S.TB + (size_t)4 * T8 * 128);
        const float* WSN = WCN + T8;
        const float wcn = xok ? WCN[x] : 0.f, wsn = xok ? WSN[x] : 0.f;
        __syncthreads();                                        // the weights are read before stg overwrites them
        const int q = NB >> 2;
        for (int c = grp * q; c < grp * q + q; c += 4) {
            float a0[4], a1[4], b0[4], b1[4];
            tc_ld4(tmem + lanes + c, a0);
            tc_ld4(tmem + lanes + NB + c, a1);
            tc_ld4(tmem + lanes + 2 * NB + c, b0);
            tc_ld4(tmem + lanes + 3 * NB + c, b1);
            tc_ld_wait();
            if (!xok) continue;
            const float gpx = S.gP[x], gmx = S.gM[x];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int lt = c + i, t = 1 + lt;
                if (lt >= TC) continue;
                const float2 v0 = make_float2(fmaf(wcn, S.CBN[lt], a0[i] * dsc), fmaf(wsn, S.CBN[2 * TC + lt], b0[i] * dsc));
                const float2 v1 = make_float2(fmaf(wcn, S.CBN[TC + lt], a1[i] * dsc), fmaf(wsn, S.CBN[3 * TC + lt], b1[i] * dsc));
                stg[(size_t)lt * T8 + x] = v0;
                stg[(size_t)(TC + lt) * T8 + x] = v1;
                if (t <= g.h0) {                                // the grid points of rows +-t
                    if (t <= g.pmax && x <= g.pmax) vmax = fmaxf(vmax, g.sense * (v0.x - v0.y + gpx));
                    if (t <= g.pmax && x >= 1) vmax = fmaxf(vmax, g.sense * (v0.x + v0.y + gmx));
                    if (x <= g.pmax) vmax = fmaxf(vmax, g.sense * (v1.x - v1.y + gpx));
                    if (x >= 1) vmax = fmaxf(vmax, g.sense * (v1.x + v1.y + gmx));
                }
            }
        }
    }
    // the surface's maximum: only points within the near-tie band of it can matter, so the
    // top-K pass pushes no point below it minus the band (thr = the (0, 0) value minus the
    // band; taking twice the band keeps the raised threshold, rounding included, below the
    // one the guard applies later)
    for (int o = 16; o; o >>= 1) vmax = fmaxf(vmax, __shfl_xor_sync(0xffffffffu, vmax, o));
    if (lane == 0) S.rv[warp] = vmax;
    __syncthreads();
    if (!kCollect && !dbg) {
        float m = -INFINITY;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = fmaxf(m, S.rv[w]);
        const float band = g.sense * S.gP[0] - thr;
        const float raised = m - 2.f * band;
        if (raised > thr) thr = raised;
    }
    __syncthreads();
    if (liveB) {
        // one staged row (sign, t) per warp at a time, tx = lane + 32 k: the row's loads are
        // issued together before its points are emitted
        const int nt = TC < g.h0 ? TC : g.h0, nwarp = blockDim.x >> 5;
        // this lane's columns: g(+-tx) and whether +tx / -tx are grid points, hoisted out
        // of the row loop; the surface values are sense * (A -+ B + g(+-tx))
        float gp[4], gm[4];
        bool okp[4], okm[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int x = lane + 32 * k;
            const bool in = x <= g.h0;
            gp[k] = in ? S.gP[x] : 0.f;
            gm[k] = in ? S.gM[x] : 0.f;
            okp[k] = in && x <= g.pmax;
            okm[k] = in && x >= 1;
        }
        const float sense = g.sense;
        if (dbg) {                                              // debug surfaces: the generic path
            for (int r = warp; r < 2 * nt; r += nwarp) {
                const int sg = r >= nt ? 1 : 0, lt = r - sg * nt, t = 1 + lt;
                const float2* row = stg + (size_t)(sg * TC + lt) * T8;
                for (int k = 0; k < 4; ++k)
                    if (lane + 32 * k <= g.h0) emit.quad(sg, t, lane + 32 * k, row[lane + 32 * k].x, row[lane + 32 * k].y);
            }
        } else {
            // the hot loop only loads a row and compares its points with the threshold; the
            // rare points at or above it (about one a frame) are kept in one block after it
            for (int r = warp; r < 2 * nt; r += nwarp) {
                const int sg = r >= nt ? 1 : 0, lt = r - sg * nt;
                const bool rowok = sg || 1 + lt <= g.pmax;
                const float2* row = stg + (size_t)(sg * TC + lt) * T8;
                float vp[4], vm[4];
                bool hit = false;
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const float2 v = lane + 32 * k <= g.h0 ? row[lane + 32 * k] : make_float2(0.f, 0.f);
                    vp[k] = sense * (v.x - v.y + gp[k]);
                    vm[k] = sense * (v.x + v.y + gm[k]);
                    hit |= (rowok && okp[k] && vp[k] >= thr) || (rowok && okm[k] && vm[k] >= thr);
                }
                if (__builtin_expect(hit, 0)) {
                    const int ts = sg ? -(1 + lt) : 1 + lt;
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        if (rowok && okp[k] && vp[k] >= thr) emit.keep(vp[k], ts, lane + 32 * k);
                        if (rowok && okm[k] && vm[k] >= thr) emit.keep(vm[k], ts, -(lane + 32 * k));
                    }
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
}

// Full upsampled surface pass (all chunks): top-K, or candidate collection.
// kTcOnly: the 128 x 128 instantiation for plans that use tcgen05 (g.tc), compiled without
// the warp-MMA stages (a smaller kernel: its first stall was instruction fetch).
template <int H, int W, bool kCollect, bool kTcOnly = false>
__device__ __forceinline__ void upsampled_pass(const Geom& g, const Smem& S, TopK<kTopK>& top, float thr,
                                               float* dbg) {
    if constexpr (kTcOnly) {
        upsampled_pass_tc<kCollect>(g, S, top, thr, dbg);
    } else {
        if constexpr (H == 128 && W == 128 && !kTcOnly) {
            if (g.tc) {
                upsampled_pass_tc<kCollect>(g, S, top, thr, dbg);
                return;
            }
        }
        const uint2* TA = g.tables_smem ? S.TA : g.tAh;
        const uint2* TB = g.tables_smem ? S.TB : g.tBh;
        const float dsc = ldexpf(1.f, -13 - S.misc[3]);
        const Emitter<kCollect> emit{g, S, top, thr, dbg};
        for (int c = 0; c < g.nchunk; ++c) {
            const int t0 = 1 + c * g.TC;
            stage_a<H, W>(g, S, t0, TA);
            if constexpr (W % 32 == 0) {
                if (g.tables_smem) stage_b_mma<W, kCollect>(g, S, t0, TB, dsc, emit);
                else stage_b_simt<kCollect>(g, S, t0, TB, dsc, emit);
            } else {
                stage_b_simt<kCollect>(g, S, t0, TB, dsc, emit);
            }
            // the t = 0 row: S = 0, the surface is g(tx)
            if (t0 == 1) {
                for (int x = threadIdx.x; x <= g.h0; x += blockDim.x) {
                    if (x <= g.pmax) emit(S.gP[x], 0, x);
                    if (x >= 1) emit(S.gM[x], 0, -x);
                }
            }
            __syncthreads();
        }
    }
}

// Second surface pass that lists every point with v >= thr (S.cj/S.cv, count returned).
template <int H, int W, bool kTcOnly = false>
static __device__ int collect_near(const Geom& g, const Smem& S, float thr) {
    TopK<kTopK> unused;
    unused.init();
    if (threadIdx.x == 0) S.misc[1] = 0;
    __syncthreads();
    upsampled_pass<H, W, true, kTcOnly>(g, S, unused, thr, nullptr);
    const int nc = S.misc[1];
    __syncthreads();
    return nc;
}

// ---------------------------------- a7 guard: exact FP32 pair differences
// X'(ky, kx) for any row and column, from the P/Q layout.
// P(m, kx) and Q(m, kx), m = 1 .. Hh, of a regular column from the fp16 planes (unscaled
// by inv = 2^-kexp)
// (tc layout) plane pl (Pr, Pi, Qr, Qi) at row kx, K index k: hi + lo
__device__ __forceinline__ float pq_tc(const Geom& g, const Smem& S, int pl, int kx, int k) {
    const size_t ms = (size_t)g.SA * 128;
    const unsigned char* b = (const unsigned char*)S.PQ + (size_t)((pl >> 1) * 4 + (pl & 1)) * ms + sw128_off(kx, k);
    return __half2float(*(const __half*)b) + __half2float(*(const __half*)(b + 2 * ms));
}

__device__ __forceinline__ void pq_at(const Geom& g, const Smem& S, int m, int kx, float inv, float2* P, float2* Q) {
    if (g.tc) {
        const int k = m - 1;
        *P = make_float2(pq_tc(g, S, 0, kx, k) * inv, pq_tc(g, S, 1, kx, k) * inv);
        *Q = make_float2(pq_tc(g, S, 2, kx, k) * inv, pq_tc(g, S, 3, kx, k) * inv);
        return;
    }
    const int SA = g.SA, Hq = g.Hh / 2, k = m - 1, q = (k >> 1) ^ pswz(kx, Hq);
    const float2 pr = unsplit_pair(S.PQ[(0 * SA + kx) * Hq + q]), pi = unsplit_pair(S.PQ[(1 * SA + kx) * Hq + q]);
    const float2 qr = unsplit_pair(S.PQ[(2 * SA + kx) * Hq + q]), qi = unsplit_pair(S.PQ[(3 * SA + kx) * Hq + q]);
    *P = (k & 1) ? make_float2(pr.y * inv, pi.y * inv) : make_float2(pr.x * inv, pi.x * inv);
    *Q = (k & 1) ? make_float2(qr.y * inv, qi.y * inv) : make_float2(qr.x * inv, qi.x * inv);
}

// X'(ky, kx) for any row and column: X'(0) from S.X0, X'(Hh) = P(Hh), X'(+-m) = (P -+... ) / 2
// from the planes, and the x-Nyquist column from the FP32 P/Q rows in XN.
__device__ __forceinline__ float2 xprime(const Geom& g, const Smem& S, int ky, int kx) {
    const int Hh = g.Hh;
    if (2 * kx == g.W) {
        const float2* colbase = S.XN;
        if (ky == 0 || ky == Hh) return colbase[posH(g, ky)];
        if (ky < Hh) {
            const float2 p = colbase[posH(g, ky)], q = colbase[posH(g, g.H - ky)];
            return make_float2(0.5f * (p.x + q.x), 0.5f * (p.y + q.y));
        }
        const int m = g.H - ky;
        const float2 p = colbase[posH(g, m)], q = colbase[posH(g, ky)];
        return make_float2(0.5f * (p.x - q.x), 0.5f * (p.y - q.y));
    }
    if (ky == 0) return S.X0[kx];
    const float inv = ldexpf(1.f, -S.misc[3]);
    float2 p, q;
    pq_at(g, S, ky <= Hh ? ky : g.H - ky, kx, inv, &p, &q);
    if (ky == Hh) return p;
    if (ky < Hh) return make_float2(0.5f * (p.x + q.x), 0.5f * (p.y + q.y));
    return make_float2(0.5f * (p.x - q.x), 0.5f * (p.y - q.y));
}

// exp(i pi n / D) for an integer n (reduced mod 2D first).
__device__ __forceinline__ float2 expi_pi_frac(long long n, long long D) {
    long long r = n % (2 * D);
    if (r < 0) r += 2 * D;
    float s, c;
    sincospif((float)r / (float)D, &s, &c);
    return make_float2(c, s);
}
__device__ __forceinline__ float sin_pi_frac(long long n, long long D) {
    return sinpif((float)n / (float)D);
}
// the same in 32-bit integers (u <= 16384, H, W <= 128: |n| and 2D stay below 2^31)
__device__ __forceinline__ float2 expi_pi_frac32(int n, int D) {
    int r = n % (2 * D);
    if (r < 0) r += 2 * D;
    float s, c;
    sincospif((float)r / (float)D, &s, &c);
    return make_float2(c, s);
}

// X'(ky, kx) along one row over the regular columns kx < W/2, with the row's case and its
// plane pair resolved once: X'(0) from S.X0, X'(Hh) = P(Hh), X'(+-m) = (P +- Q)/2.
struct XRow {
    int mode;          // 0: row 0; 1: the Nyquist row (P only); 2: (P + Q)/2; 3: (P - Q)/2
    int p, h;          // pair index of m = |row| and its half
    float sa, sb;      // weights of P and Q, including the 2^-kexp unscale
    __device__ __forceinline__ XRow(const Geom& g, const Smem& S, int ky) {
        const int Hh = g.Hh, m = ky <= Hh ? ky : g.H - ky;
        const float inv = ldexpf(1.f, -S.misc[3]);
        mode = ky == 0 ? 0 : (ky == Hh ? 1 : (ky < Hh ? 2 : 3));
        p = (m - 1) >> 1;
        h = (m - 1) & 1;
        sa = mode == 1 ? inv : 0.5f * inv;
        sb = mode == 2 ? 0.5f * inv : (mode == 3 ? -0.5f * inv : 0.f);
    }
    __device__ __forceinline__ float2 at(const Geom& g, const Smem& S, int kx) const {
        if (mode == 0) return S.X0[kx];
        if (g.tc) {
            const int k = 2 * p + h;
            const float pr = pq_tc(g, S, 0, kx, k), pi = pq_tc(g, S, 1, kx, k);
            if (mode == 1) return make_float2(sa * pr, sa * pi);
            const float qr = pq_tc(g, S, 2, kx, k), qi = pq_tc(g, S, 3, kx, k);
            return make_float2(fmaf(sa, pr, sb * qr), fmaf(sa, pi, sb * qi));
        }
        const int SA = g.SA, Hq = g.Hh / 2, q = p ^ pswz(kx, Hq);
        auto half = [&](uint2 v) {
            const float2 hh = unpack_f16x2(v.x), ll = unpack_f16x2(v.y);
            return h ? hh.y + ll.y : hh.x + ll.x;
        };
        const float pr = half(S.PQ[(0 * SA + kx) * Hq + q]), pi = half(S.PQ[(1 * SA + kx) * Hq + q]);
        if (mode == 1) return make_float2(sa * pr, sa * pi);
        const float qr = half(S.PQ[(2 * SA + kx) * Hq + q]), qi = half(S.PQ[(3 * SA + kx) * Hq + q]);
        return make_float2(fmaf(sa, pr, sb * qr), fmaf(sa, pi, sb * qi));
    }
};

// Full twiddle exp(2 pi i k' t / (uH)) of the stage tables (FP64-rounded values).
__device__ __forceinline__ float2 table_twiddle_y(const Geom& g, int ks, int t) {
    const int m = ks < 0 ? -ks : ks, at = t < 0 ? -t : t;
    if (m == 0 || at == 0) return make_float2(1.f, 0.f);
    const float c = 1.f + __ldg(&g.tA_cm1[(m - 1) * g.T1p + at]);
    const float s = __ldg(&g.tA_s[(m - 1) * g.T1p + at]);
    return make_float2(c, ((ks < 0) != (t < 0)) ? -s : s);
}

// Decide among the candidates S.cj[0..nc) (S.cj[0] is the FP32 best j1) with exact
// pair differences D(j) = v(j) - v(j1). Returns the winner; sets *nl2 when the two
// best remain within tau1, leaving the tied candidates in S.cj[0..*nl2).
//   v(j) - v(j1) = Re sum_ky [ Ey(ky, ty) F_j(ky) + (Ey(ky, ty) - Ey(ky, ry)) G(ky) ],
//   G(ky) = sum_kx X'(ky, kx) w Ex(kx, rx),  F_j(ky) = sum_kx X'(ky, kx) w (Ex(kx, tx) - Ex(kx, rx)),
// with both differences in the small-factor form 2i sin(a) e^{ib}. The row sums of up to
// kPdGroup factor vectors share one sweep over X' (G rides along with the first group);
// each row sum is split kPdParts ways over the CTA. Scratch: the UV area (dead after
// stage B).
constexpr int kPdGroup = 3, kPdParts = 4;

static __device__ int pair_difference_guard(const Geom& g, const Smem& S, int nc, float scale, int* nl2,
                                            float* dwin) {
    const int H = g.H, Wc = g.Wc, u = g.u, Hh = g.Hh, T1p = g.T1p;
    const float* TBc = g.tB_wc;
    const float* TBs = g.tB_ws;
    constexpr int NF = kPdGroup + 1;
    float2* fx = (float2*)S.UV;             // [NF][Wc]   factor vectors over kx (slot 0: G's)
    float2* Eyc = fx + NF * Wc;             // [kPdGroup][H]  Ey(ky, ty)
    float2* dEy = Eyc + kPdGroup * H;       // [kPdGroup][H]  Ey(ky, ty) - Ey(ky, ry)
    float2* G = dEy + kPdGroup * H;         // [H]
    float2* GN = G + H;                     // [1]  the Nyquist row's x-Nyquist term of G
    float2* part = GN + 1;                  // [kPdParts][NF][H]
    float2* partN = part + kPdParts * NF * H;   // [kPdParts][NF]
    const int j1 = S.cj[0];
    const int ry = j1 / g.M - g.h0, rx = j1 % g.M - g.h0;
    const int kn = g.W >> 1;
    const int arx = rx < 0 ? -rx : rx;
    if (threadIdx.x == 0) S.cv[0] = 0.f;
    for (int c0 = 1; c0 < nc; c0 += kPdGroup) {
        const int ng = min(kPdGroup, nc - c0);
        const bool first = (c0 == 1);
        // factor vectors and y twiddles of this group (slot 0 = G's factor, first group only)
        for (int k = threadIdx.x; k < ng * (H + Wc) + (first ? Wc : 0); k += blockDim.x) {
            if (k >= ng * (H + Wc)) {
                const int kx = k - ng * (H + Wc);
                const float c = TBc[kx * T1p + arx], s = TBs[kx * T1p + arx];
                fx[kx] = make_float2(c, rx < 0 ? -s : s);
                continue;
            }
            const int ci = k / (H + Wc), kk = k - ci * (H + Wc);
            const int jc = S.cj[c0 + ci];
            const int ty = jc / g.M - g.h0, tx = jc % g.M - g.h0;
            if (kk < H) {
                const int ks = signed_k(kk, H);
                Eyc[ci * H + kk] = table_twiddle_y(g, ks, ty);
                // E(ty) - E(ry) = 2i sin(pi k'(ty - ry)/(uH)) exp(i pi k'(ty + ry)/(uH))
                const float s1 = sinpif((float)(ks * (ty - ry)) / (float)(u * H));
                const float2 e2 = expi_pi_frac32(ks * (ty + ry), u * H);
                dEy[ci * H + kk] = make_float2(-2.f * s1 * e2.y, 2.f * s1 * e2.x);
            } else {
                const int kx = kk - H;
                const int ks = signed_k(kx, g.W);
                const float w = (kx == 0 || 2 * kx == g.W) ? 1.f : 2.f;
                const float s1 = sinpif((float)(ks * (tx - rx)) / (float)(u * g.W));
                const float2 e2 = expi_pi_frac32(ks * (tx + rx), u * g.W);
                fx[(1 + ci) * Wc + kx] = make_float2(-2.f * w * s1 * e2.y, 2.f * w * s1 * e2.x);
            }
        }
        __syncthreads();
        // one sweep over X': row sums of the factor vectors f0 (first group) and f1..f_ng
        const int fbeg = first ? 0 : 1, fend = 1 + ng;
        for (int task = threadIdx.x; task < kPdParts * H; task += blockDim.x) {
            const int q = task / H, ky = task - q * H;
            float2 acc[NF], accn[NF];
#pragma unroll
            for (int f = 0; f < NF; ++f) { acc[f] = make_float2(0.f, 0.f); accn[f] = acc[f]; }
            const XRow xr(g, S, ky);
            for (int kx = Wc - 1 - q; kx >= 0; kx -= kPdParts) {
                const float2 xp = kx == kn ? xprime(g, S, ky, kx) : xr.at(g, S, kx);
                const bool nn = (ky == Hh && kx == kn);
#pragma unroll
                for (int f = 0; f < NF; ++f) {
                    if (f < fbeg || f >= fend) continue;
                    const float2 t = cmul(xp, fx[f * Wc + kx]);
                    if (nn) accn[f] = t; else acc[f] = cadd(acc[f], t);
                }
            }
#pragma unroll
            for (int f = 0; f < NF; ++f) {
                if (f < fbeg || f >= fend) continue;
                part[(q * NF + f) * H + ky] = acc[f];
                if (ky == Hh) partN[q * NF + f] = accn[f];
            }
        }
        __syncthreads();
        if (first) {
            for (int ky = threadIdx.x; ky < H; ky += blockDim.x) {
                float2 s = make_float2(0.f, 0.f);
                for (int q = 0; q < kPdParts; ++q) s = cadd(s, part[q * NF * H + ky]);
                G[ky] = s;
                if (ky == Hh) {
                    float2 sn = make_float2(0.f, 0.f);
                    for (int q = 0; q < kPdParts; ++q) sn = cadd(sn, partN[q * NF]);
                    *GN = sn;
                }
            }
            __syncthreads();
        }
        // D for each candidate of the group: per-thread partial sums, then a block reduction
        float acc[kPdGroup];
#pragma unroll
        for (int ci = 0; ci < kPdGroup; ++ci) acc[ci] = 0.f;
        for (int ky = threadIdx.x; ky < H; ky += blockDim.x) {
#pragma unroll
            for (int ci = 0; ci < kPdGroup; ++ci) {
                if (ci >= ng) continue;
                const int f = 1 + ci;
                float2 F = make_float2(0.f, 0.f);
                for (int q = 0; q < kPdParts; ++q) F = cadd(F, part[(q * NF + f) * H + ky]);
                const float2 ey = Eyc[ci * H + ky], dy = dEy[ci * H + ky];
                if (ky == Hh) {
                    float2 FN = make_float2(0.f, 0.f);
                    for (int q = 0; q < kPdParts; ++q) FN = cadd(FN, partN[q * NF + f]);
                    // real part of the row's y-phase, except in the x-Nyquist column
                    acc[ci] += ey.x * F.x + dy.x * G[ky].x;
                    acc[ci] += cmul(ey, FN).x + cmul(dy, GN[0]).x;
                } else {
                    acc[ci] += cmul(ey, F).x + cmul(dy, G[ky]).x;
                }
            }
        }
        // block sums of the group's values (S.rv holds kWarps x kPdGroup partials)
        const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
        for (int ci = 0; ci < kPdGroup; ++ci) {
            const float v = warp_sum(acc[ci]);
            if (lane == 0) S.rv[wid * kPdGroup + ci] = v;
        }
        __syncthreads();
        if (threadIdx.x < ng) {
            float D = 0.f;
            for (int w = 0; w < nw; ++w) D += S.rv[w * kPdGroup + threadIdx.x];
            S.cv[c0 + threadIdx.x] = g.sense * D;
        }
        __syncthreads();
    }
    // winner and runner-up by (D, lowest index)
    float bv = S.cv[0], sv = -INFINITY;
    int bj = S.cj[0], sj = INT_MAX;
    for (int c = 1; c < nc; ++c) {
        const float v = S.cv[c];
        const int j = S.cj[c];
        if (better(v, j, bv, bj)) { sv = bv; sj = bj; bv = v; bj = j; }
        else if (better(v, j, sv, sj)) { sv = v; sj = j; }
    }
    *nl2 = 0;
    *dwin = bv;
    const float tau1 = g.tau1 * scale;
    if (nc > 1 && bv - sv <= tau1) {
        // keep every candidate within tau1 of the winner for the last level
        __syncthreads();
        if (threadIdx.x == 0) {
            int k = 0;
            int keep[kMaxCandL2];
            for (int c = 0; c < nc && k < kMaxCandL2; ++c)
                if (bv - S.cv[c] <= tau1) keep[k++] = S.cj[c];
            for (int c = 0; c < k; ++c) S.cj[c] = keep[c];
            S.misc[2] = k;
        }
        __syncthreads();
        *nl2 = S.misc[2];
        __syncthreads();
    }
    return bj;
}

// v(jb) - v(ja) from the FP32 X' in shared memory, with FP64 twiddles and FP64
// accumulation (the Nyquist-row rule included). Scratch: the UV area.
static __device__ double pair_difference_f64(const Geom& g, const Smem& S, int ja, int jb, double* red) {
    const int H = g.H, Wc = g.Wc;
    double2* eyA = (double2*)(S.UV);
    double2* eyB = eyA + H;
    double2* exA = eyB + H;
    double2* exB = exA + Wc;
    const int tya = ja / g.M - g.h0, txa = ja % g.M - g.h0;
    const int tyb = jb / g.M - g.h0, txb = jb % g.M - g.h0;
    const long long Dy = (long long)g.u * H, Dx = (long long)g.u * g.W;
    for (int k = threadIdx.x; k < H + Wc; k += blockDim.x) {
        const bool isy = k < H;
        const int kk = isy ? k : k - H;
        const long long ks = isy ? signed_k(kk, H) : signed_k(kk, g.W);
        const long long D = isy ? Dy : Dx;
        long long na = (ks * (isy ? tya : txa)) % D, nb = (ks * (isy ? tyb : txb)) % D;
        if (na < 0) na += D;
        if (nb < 0) nb += D;
        double sa, ca, sb, cb;
        sincospi(2.0 * (double)na / (double)D, &sa, &ca);
        sincospi(2.0 * (double)nb / (double)D, &sb, &cb);
        if (isy) { eyA[kk] = make_double2(ca, sa); eyB[kk] = make_double2(cb, sb); }
        else {
            const double w = (kk == 0 || 2 * kk == g.W) ? 1.0 : 2.0;
            exA[kk] = make_double2(w * ca, w * sa); exB[kk] = make_double2(w * cb, w * sb);
        }
    }
    __syncthreads();
    double acc = 0.0;
    for (int idx = threadIdx.x; idx < H * Wc; idx += blockDim.x) {
        const int ky = idx / Wc, kx = idx - ky * Wc;
        const float2 xf = xprime(g, S, ky, kx);
        const double2 x = make_double2(xf.x, xf.y);
        double2 ea = eyA[ky], eb = eyB[ky];
        if (ky == g.Hh && 2 * kx != g.W) { ea.y = 0.0; eb.y = 0.0; }
        const double2 pa = cmul(ea, exA[kx]), pb = cmul(eb, exB[kx]);
        acc += x.x * (pb.x - pa.x) - x.y * (pb.y - pa.y);
    }
    return block_sum(acc, red);
}

// ------------------------------------------- last guard level: double-float
__device__ __forceinline__ dfc df_twiddle(const dfc* coarse, const dfc* fine, int B, long long n) {
    return cmul(coarse[n / B], fine[n % B]);
}

static __device__ df block_sum_df(df v, double* red) {
    // double-float sum across the block; the warp partials are combined in FP64 (few ops)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        df w = {__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o)};
        v = df_add(v, w);
    }
    const double d = df_to_double(v);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[wid] = d;
    __syncthreads();
    double r = 0.0;
    const int nw = (blockDim.x + 31) >> 5;
    for (int k = 0; k < nw; ++k) r += red[k];
    __syncthreads();
    return df_from_double(r);
}

// Re-evaluate the candidates S.cj[0..nc) from a double-float product spectrum
// X = F[a] conj(F[b]): R2C FFT of the operand in double-float (the first H x Wcp
// dfc of R1 + R2 hold the half spectrum, the rest the packed row chunks), then
//   cu(j) = Re sum_{ky,kx} w X(ky,kx) E_y(ky, py u + ty) E_x(kx, px u + tx)
// with exactly reduced angles. Returns the winner (sense-adjusted maximum,
// lowest index on ties) and its unnormalised value in *val.
template <int H, int W>
static __device__ int df_reevaluate(const Geom& g, const Smem& S, const void* frame, long long pitch,
                                    int py, int px, int nc, double* val) {
    constexpr int N1w = Split<W>::N1, N2w = Split<W>::N2, N1h = Split<H>::N1, N2h = Split<H>::N2;
    constexpr int Hh = H / 2, Wc = W / 2 + 1;
    const int Wcp = g.Wcp;
    dfc* Xd = (dfc*)S.r1;                      // [H][Wcp]; after the column passes row fft_pos(ky) holds X(ky, .)
    dfc* twd = Xd + (size_t)H * Wcp;           // Ntw/2 FFT twiddles, staged from global
    dfc* t4w = twd + g.Ntw / 2;                // W: inter-pass twiddles of length W
    dfc* t4h = t4w + W;                        // H: the same for length H
    dfc* Zc = t4h + H;                         // packed-row chunk, later the candidate phases
    const long long cbytes =
        (long long)S.r12_bytes - (long long)sizeof(dfc) * ((long long)H * Wcp + g.Ntw / 2 + W + H);
    for (int k2 = threadIdx.x; k2 < g.Ntw / 2; k2 += blockDim.x) twd[k2] = g.twdf[k2];
    __syncthreads();
    build_pass_twiddles_df<W>(t4w, twd, g.logNtw);
    build_pass_twiddles_df<H>(t4h, twd, g.logNtw);
    int R = 1;                                 // packed rows per chunk
    while (2 * R <= Hh && 2LL * R * W * (long long)sizeof(dfc) <= cbytes) R *= 2;
    __syncthreads();
    // rows: packed pair (2r, 2r+1) as one complex row, four-step passes, then the split into
    // the two real rows' half spectra, stored in natural row order
    for (int r0 = 0; r0 < Hh; r0 += R) {
        for (int idx = threadIdx.x; idx < R * W; idx += blockDim.x) {
            const int rl = idx / W, x = idx - rl * W;
            const int y = 2 * (r0 + rl);
            df a[2];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const float I = pixel_f32(frame, g.in_dtype, (long long)(y + h) * pitch + x);
                a[h] = df_make(I);
                if (g.method != 0) {
                    float s, e;
                    two_sum(I, g.eps, s, e);
                    const df ip = {s, e};
                    a[h] = df_mul(ip, ip);
                }
            }
            Zc[rl * W + x] = dfc{a[0], a[1]};
        }
        __syncthreads();
        fft_pass1_df<N1w, N2w, false>(
            R, t4w, [&](int s, int n2, int n1) { return Zc[s * W + N2w * n1 + n2]; },
            [&](int s, int n2, int k1, dfc v) { Zc[s * W + N2w * k1 + n2] = v; });
        __syncthreads();
        if (N2w > 1) {
            fft_pass2_df<N1w, N2w, false>(
                R, [&](int s, int k1, int n2) { return Zc[s * W + N2w * k1 + n2]; },
                [&](int s, int k1, int k2, dfc v) { Zc[s * W + N2w * k1 + k2] = v; });
            __syncthreads();
        }
        for (int idx = threadIdx.x; idx < R * Wc; idx += blockDim.x) {
            const int rl = idx / Wc, kx = idx - rl * Wc;
            const dfc z = Zc[rl * W + fft_pos(kx & (W - 1), N1w, N2w)];
            const dfc zc = cconj(Zc[rl * W + fft_pos((W - kx) & (W - 1), N1w, N2w)]);
            const dfc sp = cadd(z, zc), dm = csub(z, zc);
            const int r = r0 + rl;
            Xd[(2 * r) * Wcp + kx] = {df_scale(sp.re, 0.5f), df_scale(sp.im, 0.5f)};
            Xd[(2 * r + 1) * Wcp + kx] = {df_scale(dm.im, 0.5f), df_scale(df_neg(dm.re), 0.5f)};   // (z - zc)/(2i)
        }
        __syncthreads();
    }
    // columns, with the product X = F[a] conj F[b] fused into the last pass
    const dfc* FEdf = S.ref ? S.ref->FEdf : g.FEdf;
    auto product = [&](int ky, int kx, dfc v) { return cmul(v, cconj(FEdf[ky * Wc + kx])); };
    fft_pass1_df<N1h, N2h, true>(
        Wc, t4h, [&](int s, int n2, int n1) { return Xd[(N2h * n1 + n2) * Wcp + s]; },
        [&](int s, int n2, int k1, dfc v) {
            if (N2h == 1) v = product(k1, s, v);
            Xd[(N2h * k1 + n2) * Wcp + s] = v;
        });
    __syncthreads();
    if (N2h > 1) {
        fft_pass2_df<N1h, N2h, true>(
            Wc, [&](int s, int k1, int n2) { return Xd[(N2h * k1 + n2) * Wcp + s]; },
            [&](int s, int k1, int k2, dfc v) { Xd[(N2h * k1 + k2) * Wcp + s] = product(k1 + N1h * k2, s, v); });
        __syncthreads();
    }
    // candidates: v(j) = Re sum_ky Ey(ky) sum_kx X(ky, kx) Ex(kx), the Nyquist row taking only
    // the real part of its phase outside the x-Nyquist column; row sums split kParts ways
    constexpr int kParts = (H * 4 <= 512) ? 4 : 2;
    dfc* Ey = Zc;            // H
    dfc* Ex = Zc + H;        // Wc
    const long long Dy = (long long)g.u * H, Dx = (long long)g.u * W;
    double bestv = -INFINITY, bestraw = 0.0;
    int bestj = INT_MAX;
    for (int c = 0; c < nc; ++c) {
        const int j = S.cj[c];
        const int ty = j / g.M - g.h0, tx = j % g.M - g.h0;
        for (int k = threadIdx.x; k < H + Wc; k += blockDim.x) {
            if (k < H) {
                long long n = ((long long)signed_k(k, H) * ((long long)py * g.u + ty)) % Dy;
                if (n < 0) n += Dy;
                Ey[k] = df_twiddle(g.eyc, g.eyf, g.By, n);
            } else {
                const int kx = k - H;
                long long n = ((long long)signed_k(kx, W) * ((long long)px * g.u + tx)) % Dx;
                if (n < 0) n += Dx;
                dfc e = df_twiddle(g.exc, g.exf, g.Bx, n);
                if (kx != 0 && 2 * kx != W) e = {df_scale(e.re, 2.f), df_scale(e.im, 2.f)};
                Ex[kx] = e;
            }
        }
        __syncthreads();
        df acc = {0.f, 0.f};
        for (int task = threadIdx.x; task < H * kParts; task += blockDim.x) {
            const int ky = task / kParts, part = task - ky * kParts;
            const dfc* xr = Xd + (size_t)fft_pos(ky, N1h, N2h) * Wcp;
            dfc F = {{0.f, 0.f}, {0.f, 0.f}}, FN = F;
            for (int kx = part; kx < Wc; kx += kParts) {
                const dfc t = cmul(xr[kx], Ex[kx]);
                if (2 * kx == W) FN = t; else F = cadd(F, t);
            }
            const dfc ey = Ey[ky];
            df v;
            if (ky == Hh) {
                v = df_add_abs(df_mul(ey.re, F.re), cmul(ey, FN).re);     // real part of the phase only
            } else {
                const dfc t = cmul(ey, cadd(F, FN));
                v = t.re;
            }
            acc = df_add_abs(acc, v);
        }
        const double vv = df_to_double(block_sum_df(acc, S.rd));
        const double sv = (double)g.sense * vv;
        if (sv > bestv || (sv == bestv && j < bestj)) { bestv = sv; bestj = j; bestraw = vv; }
        __syncthreads();
    }
    *val = bestraw;
    return bestj;
}

// ---------------------------------------------------------- the FP32 kernel
// One instantiation per frame size (H, W); the host picks it through track_kernel_for().
// Per-CTA set-up for frames of size H x W: FFT twiddles and the four-step pass twiddles.
template <int H, int W>
__device__ __forceinline__ void track_setup(const Geom& g, const Smem& S) {
    for (int k = threadIdx.x; k < g.Ntw / 2; k += blockDim.x) S.tw[k] = g.tw32[k];
    __syncthreads();
    build_pass_twiddles<H>(S.t4h, S.tw, g.logNtw);
    build_pass_twiddles<W>(S.t4w, S.tw, g.logNtw);
}

// A tensor-core batch of this CTA never completed (upsampled_pass_tc): the frame's record
// says so (CCST_R_TIMEOUT) and the CTA must stop. CTA-uniform (read after a barrier).
template <int H, int W>
__device__ __forceinline__ bool tc_failed(const Geom& g, const Batch& b, long long f, unsigned flags) {
    if constexpr (H == 128 && W == 128) {
        if (g.tc && tc_shared()->failed) {
            if (threadIdx.x == 0) {
                Result r{};
                r.flags = flags | 0x20u;
                b.out[f] = r;
            }
            __syncthreads();
            return true;
        }
    }
    return false;
}

// a1-a7 for one frame (rows b.pitch elements apart) against the reference of g; the record
// goes to b.out[f], and f indexes the optional debug outputs of b. Returns false when the
// stage tables never arrived (the record says so; the CTA must stop).
template <int H, int W, bool kTcOnly = false>
__device__ __forceinline__ bool track_frame(const Geom& g, const Batch& b, const Smem& S, long long f,
                                            const char* frame, unsigned& bar_parity) {
    unsigned flags = 0;
    float scale = 0.f;
    Best2 t2;
    fft_correlate_t<H, W>(g, S, frame, b.pitch, b.vec_ok, &scale, t2,
                          b.dbg_int ? b.dbg_int + (size_t)f * g.H * g.W : nullptr);
    const int ip = integer_peak(g, S, frame, b.pitch, &scale, &flags, t2);
    const float c0 = int_surface(g, S, ip);           // HW * c(p)
    const int py = wrap_shift(ip >> g.logW, g.H), px = wrap_shift(ip & (g.W - 1), g.W);
    __syncthreads();
    if (!b.dbg_no_copy) stage_tables_async(g, S);      // overlaps the P/Q build
    build_pq_and_g(g, S, py, px, scale);
    const int wait_limit = b.dbg_no_copy ? (1 << 10) : (1 << 22);
    const bool staged = stage_tables_wait(g, S, bar_parity, wait_limit);
    if (__syncthreads_or(!staged)) {
        // the copies never completed: report it for this frame and stop this CTA, after
        // one more bounded wait so that no copy is left writing into this CTA's memory
        if (threadIdx.x == 0) {
            (void)stage_tables_wait(g, S, bar_parity, wait_limit);
            Result r{};
            r.flags = flags | 0x20u;
            b.out[f] = r;
        }
        return false;
    }
    bar_parity ^= 1u;
    if (b.dbg_pairs) {
        const int ja = b.dbg_pairs[2 * f], jb = b.dbg_pairs[2 * f + 1];
        const double d64 = pair_difference_f64(g, S, ja, jb, S.rd);
        if (threadIdx.x == 0) { S.cj[0] = ja; S.cj[1] = jb; }
        __syncthreads();
        int nl2dummy = 0;
        float dw = 0.f;
        pair_difference_guard(g, S, 2, 0.f, &nl2dummy, &dw);
        if (threadIdx.x == 0) {
            b.dbg_d32[f] = g.sense * S.cv[1];
            b.dbg_d64[f] = d64;
        }
        __syncthreads();
        return true;
    }
    TopK<kTopK> top;
    top.init();
    float* dbg = b.dbg_sub ? b.dbg_sub + (size_t)f * g.M * g.M : nullptr;
    // no point below the (0, 0) point's value minus the near-tie band can matter
    const float lb = g.sense * S.gP[0] - g.tau0 * scale;
    upsampled_pass<H, W, false, kTcOnly>(g, S, top, lb, dbg);
    if (tc_failed<H, W>(g, b, f, flags)) return false;
    float vw = top.v[0];
    int jw = top.j[0];
    block_argmax(vw, jw, S.rv, S.rj);
    float dwin = 0.f;
    int nl2 = 0;
    if (!(vw > -INFINITY)) {
        flags |= 0x10u;
        jw = 0;
    } else if (g.guard) {
        const float thr = vw - g.tau0 * scale;
        // each thread kept its best kTopK points; count those within tau0 of the maximum,
        // and whether some thread kept kTopK of them (it may have dropped more): one warp
        // reduction each, then one barrier (S.rj[32 ..], apart from block_argmax's entries)
        unsigned mine = 0;
#pragma unroll
        for (int k = 0; k < kTopK; ++k) mine |= (top.v[k] >= thr ? 1u : 0u) << k;
        {
            const int cw = (int)__reduce_add_sync(0xffffffffu, (unsigned)__popc(mine));
            const bool fw = __any_sync(0xffffffffu, top.v[kTopK - 1] >= thr);
            if ((threadIdx.x & 31) == 0) S.rj[32 + (threadIdx.x >> 5)] = cw | (fw ? 1 << 16 : 0);
        }
        __syncthreads();
        int nc = 0;
        bool full = false;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            const int e = S.rj[32 + w];
            nc += e & 0xffff;
            full |= (e >> 16) != 0;
        }
        if (nc > 1) {
            flags |= 0x02u;
            if (!full && nc <= kMaxCand) {
                // every point within tau0 is among the kept ones: gather them, j1 first
                if (threadIdx.x == 0) { S.misc[1] = 1; S.cj[0] = jw; S.cv[0] = vw; }
                __syncthreads();
#pragma unroll
                for (int k = 0; k < kTopK; ++k)
                    if (((mine >> k) & 1u) && top.j[k] != jw) {
                        const int slot = atomicAdd(&S.misc[1], 1);
                        S.cj[slot] = top.j[k];
                        S.cv[slot] = top.v[k];
                    }
                __syncthreads();
            } else {
                // a thread holds more near-ties than it kept: collect them all with a second pass
                nc = collect_near<H, W, kTcOnly>(g, S, thr);
                if (tc_failed<H, W>(g, b, f, flags)) return false;
                if (nc > kMaxCand) {
                    flags |= 0x08u;
                    nc = 1;
                } else if (threadIdx.x == 0) {
                    // put the FP32 best first
                    for (int k = 0; k < nc; ++k)
                        if (S.cj[k] == jw) { S.cj[k] = S.cj[0]; S.cj[0] = jw; }
                }
                __syncthreads();
            }
            if (nc > 1) jw = pair_difference_guard(g, S, nc, scale, &nl2, &dwin);
        }
    }
    __syncthreads();
    // raw value at the winner: c(p) + sense * (v(j1) + D(winner))
    float peak = (c0 + ((flags & 0x10u) ? 0.f : g.sense * (vw + dwin))) / (float)(g.H * g.W);
    if (nl2 > 0) {
        double raw = 0.0;
        jw = df_reevaluate<H, W>(g, S, frame, b.pitch, py, px, nl2, &raw);
        peak = (float)(raw / ((double)g.H * g.W));
        flags |= 0x04u;
    }
    if (threadIdx.x == 0) {
        const int jy = jw / g.M, jx = jw % g.M;
        const int ty = jy - g.h0, tx = jx - g.h0;
        Result r;
        r.dy = (float)(((double)py * g.u + ty) / g.u);
        r.dx = (float)(((double)px * g.u + tx) / g.u);
        r.peak = peak;
        r.ipy = py;
        r.ipx = px;
        r.flags = flags;
        b.out[f] = r;
    }
    __syncthreads();
    return true;
}

// CTA size and CTAs per SM of track_kernel<H, W>: frames up to 64 x 64 are latency-bound
// with one 512-thread CTA per SM (a few hundred tasks per phase between barriers), so they
// run two 256-thread CTAs per SM. The P/Q build takes one task per thread for 4 W tasks,
// which 256 threads cover up to W = 64.
__host__ __device__ constexpr int track_threads(int H, int W) { return (H <= 64 && W <= 64) ? 256 : kThreads; }
__host__ __device__ constexpr int track_min_ctas(int H, int W) { return (H <= 64 && W <= 64) ? 2 : 1; }

template <int H, int W, bool kTcOnly = false>
__global__ void __launch_bounds__(track_threads(H, W), track_min_ctas(H, W)) track_kernel(Geom g, Batch b) {
    const Smem S = carve(g, ccst_smem);
    track_setup<H, W>(g, S);
    tables_bar_init(S);
    unsigned bar_parity = 0;
    if constexpr (H == 128 && W == 128) {
        if (g.tc) tc_setup();                       // Tensor Memory for the contraction
    }
    __syncthreads();
    const size_t elem = g.in_dtype == 0 ? 2 : 4;
    // next frame: from the shared counter (every thread has read the current index at the
    // barrier before thread 0 fetches the next), else grid-stride
    auto fetch = [&](long long cur) -> long long {
        if (!b.next) return cur < 0 ? (long long)blockIdx.x : cur + gridDim.x;
        __syncthreads();
        if (threadIdx.x == 0) S.misc[4] = (int)atomicAdd(b.next, 1u);
        __syncthreads();
        return S.misc[4];
    };
    for (long long f = fetch(-1); f < b.n; f = fetch(f)) {
        const char* frame = (const char*)b.frames + (size_t)f * g.H * b.pitch * elem;
        if (!track_frame<H, W, kTcOnly>(g, b, S, f, frame, bar_parity)) break;
    }
    if constexpr (H == 128 && W == 128) {
        if (g.tc) tc_teardown();                    // every exit path releases the columns
    }
}

// Address of the uneven-ROI kernel for one side (ccst_rois.cu: 16, 32, 64 or 128; null for
// another), with track_threads(side, side) threads; at 128, tc_only picks the instantiation
// for a tcgen05 plan (compiled without the warp-MMA stages).
const void* track_rois_kernel_ptr(int side, bool tc_only);

// Address of track_kernel<H, W> (defined in the per-height translation units).
const void* track_kernel_h8(int W);
const void* track_kernel_h16(int W);
const void* track_kernel_h32(int W);
const void* track_kernel_h64(int W);
const void* track_kernel_h128(int W);
const void* track_kernel_128_tc();      // track_kernel<128, 128, true>
inline const void* track_kernel_for(int H, int W) {
    switch (H) {
        case 8: return track_kernel_h8(W);
        case 16: return track_kernel_h16(W);
        case 32: return track_kernel_h32(W);
        case 64: return track_kernel_h64(W);
        case 128: return track_kernel_h128(W);
        default: return nullptr;
    }
}

// ------------------------------------------------------ FP64 re-evaluation
// For frames whose FP32 pair differences stayed within tau1, recompute the product
// spectrum in FP64 (R2C FFT of the operand, product with the FP64 reference
// spectrum) and evaluate the upsampled surface at the candidates directly:
//   cu(j) = Re sum_{ky,kx} w X(ky,kx) exp(2 pi i [ky'(py u + ty)/(uH) + kx'(px u + tx)/(uW)]).
// Workspace: per CTA, H/2*W + H*Wcp double2 in global memory.
static __device__ void fft_r2c_f64_global(const Geom& g, const double* a_or_null, const void* frame,
                                   long long pitch, double2* Z, double2* Xh, double* red) {
    const int H = g.H, W = g.W, Hh = g.Hh, Wc = g.Wc, Wcp = g.Wcp;
    for (int idx = threadIdx.x; idx < H * W; idx += blockDim.x) {
        const int y = idx >> g.logW, x = idx & (W - 1);
        double a;
        if (a_or_null) a = a_or_null[idx];
        else {
            double I;
            if (g.in_dtype == 0) I = load_pixel((const unsigned short*)frame, (long long)y * pitch + x);
            else I = load_pixel((const float*)frame, (long long)y * pitch + x);
            a = operand_f64(I, g);
        }
        double* dst = (double*)&Z[(y >> 1) * W + brev(x, g.logW)];
        dst[y & 1] = a;
    }
    __syncthreads();
    fft_r2_passes(Z, g.logW, Hh, W, 1, g.tw64, g.logNtw, false);
    for (int idx = threadIdx.x; idx < Hh * Wcp; idx += blockDim.x) {
        const int r = idx / Wcp, kx = idx - r * Wcp;
        double2 fe = make_double2(0.0, 0.0), fo = make_double2(0.0, 0.0);
        if (kx < Wc) {
            const double2 z = Z[r * W + kx];
            const double2 zc = cconj(Z[r * W + ((W - kx) & (W - 1))]);
            fe = make_double2(0.5 * (z.x + zc.x), 0.5 * (z.y + zc.y));
            const double2 d = csub(z, zc);
            fo = make_double2(0.5 * d.y, -0.5 * d.x);
        }
        Xh[brev(2 * r, g.logH) * Wcp + kx] = fe;
        Xh[brev(2 * r + 1, g.logH) * Wcp + kx] = fo;
    }
    __syncthreads();
    fft_r2_passes(Xh, g.logH, Wc, 1, Wcp, g.tw64, g.logNtw, false);
    (void)red;
}

}  // namespace ccst
