// ccst_kernels.cuh -- the tracking kernels for sm_103a.
//
// One CTA tracks one frame at a time (grid-stride over the batch). Every step
// stays in shared memory:
//   a1  ingest the frame (uint16 or float32) and form the surface operand: the
//       frame itself for CC-U, (I + eps)^2 for CC-SN (Sec. II, Eqs. (4), (7));
//   a2  2-D R2C FFT (two real rows packed per complex row, radix-2);
//   a3  product with the resident reference spectrum, X = F[a] conj(F[b]);
//   a4  inverse 2-D FFT -> integer surface c(s) (right-hand side of Eq. (4)/(7));
//   a5  integer extremum, lowest row-major index on ties, wrapped shift;
//       near-ties re-decided by FP64 direct sums sum_r a(r+s) b(r);
//   a6  upsampled DFT on the M x M grid around it (Sec. III), as two dense
//       contractions with frame-independent tables;
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

namespace ccst {

struct Geom {
    int H, W, logH, logW, Hh, Wc, Wcp;  // Wc = W/2+1 (half spectrum), Wcp = Wc rounded up to even
    int u, M, h0, pmax;                 // grid: M points, offsets t = j - h0 in [-h0, pmax]
    int T1p;                            // table row length for t, tx in [0, h0] (padded to 4)
    int TC, nchunk;                     // stage-A chunk rows (multiple of 4) and number of chunks
    int Ntw, logNtw;                    // twiddle table length = max(H, W)
    int method, in_dtype;
    float eps, sense;                   // sense = +1 (CC-U maximum) or -1 (CC-SN minimum)
    float tau_int, tau0, tau1;          // guard thresholds, relative to sum w|X|
    int guard;                          // tie guard on/off
    // resident device data (owned by the context)
    const float2* FE32;                 // H x Wc   F[b]
    const double2* FE64;                // H x Wc   F[b] in FP64
    const double* b64;                  // H x W    reference operand b (E or 1/(E+eps))
    const float2* tw32;                 // Ntw/2    exp(-2 pi i k/Ntw)
    const double2* tw64;
    const float* tA_cm1;                // [Hh][T1p]  cos(2 pi m t/(uH)) - 1, m = 1..Hh
    const float* tA_s;                  // [Hh][T1p]  sin(2 pi m t/(uH))
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

struct Result {  // mirrors ccst_result
    float dx, dy, peak;
    int ipy, ipx;
    unsigned flags;
};

struct Batch {
    const void* frames;
    long long n;
    long long pitch;     // row pitch in elements
    Result* out;
    float* dbg_int;      // optional: n x H x W integer surfaces (unnormalised), or null
    float* dbg_sub;      // optional: n x M x M delta surfaces (unnormalised), or null
    const int* dbg_pairs;  // optional: n x 2 grid indices (ja, jb); then only the pair difference runs
    float* dbg_d32;        // n: v(jb) - v(ja) by the FP32 pair-difference guard
    double* dbg_d64;       // n: the same difference accumulated in FP64 from the FP32 spectrum
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

// ------------------------------------------------------------- shared layout
struct Smem {
    float2* A;     // H x Wcp   X, then X' with P/Q rows
    float2* B;     // H x Wcp   inverse-FFT workspace
    float4* C;     // TC x Wcp  U'/V chunk; also packed rows (H/2 x W complex) and L1 arrays
    float2* tw;    // Ntw/2
    float* gP;     // T1p: g(+tx)
    float* gM;     // T1p: g(-tx)
    float* rv;     // reduction scratch (floats)
    int* rj;       // reduction scratch (ints)
    double* rd;    // reduction scratch (doubles)
    int* cj;       // candidate list
    float* cv;     // candidate values
    int* misc;     // small broadcast ints
    float* miscf;  // small broadcast floats
};

__host__ __device__ inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

__host__ __device__ inline size_t smem_bytes(const Geom& g) {
    size_t off = 0;
    off += sizeof(float2) * (size_t)g.H * g.Wcp;            // A
    off += sizeof(float2) * (size_t)g.H * g.Wcp;            // B
    size_t cbytes = sizeof(float4) * (size_t)g.TC * g.Wcp;
    const size_t packed = sizeof(float2) * (size_t)(g.H / 2) * g.W;
    const size_t l1 = sizeof(float2) * (size_t)(3 * g.H + 2 * g.Wcp + 2);
    if (cbytes < packed) cbytes = packed;
    if (cbytes < l1) cbytes = l1;
    off += align_up(cbytes, 16);                            // C
    off += sizeof(float2) * (size_t)(g.Ntw / 2);            // tw
    off += sizeof(float) * 2 * (size_t)g.T1p;               // gP, gM
    off += sizeof(float) * 128 + sizeof(int) * 128;         // rv, rj
    off = align_up(off, 8);
    off += sizeof(double) * 32;                             // rd
    off += (sizeof(int) + sizeof(float)) * kMaxCand;        // cj, cv
    off += sizeof(int) * 16 + sizeof(float) * 16;           // misc
    return align_up(off, 16);
}

__device__ inline Smem carve(const Geom& g, unsigned char* base) {
    Smem s;
    size_t off = 0;
    s.A = (float2*)(base + off); off += sizeof(float2) * (size_t)g.H * g.Wcp;
    s.B = (float2*)(base + off); off += sizeof(float2) * (size_t)g.H * g.Wcp;
    size_t cbytes = sizeof(float4) * (size_t)g.TC * g.Wcp;
    const size_t packed = sizeof(float2) * (size_t)(g.H / 2) * g.W;
    const size_t l1 = sizeof(float2) * (size_t)(3 * g.H + 2 * g.Wcp + 2);
    if (cbytes < packed) cbytes = packed;
    if (cbytes < l1) cbytes = l1;
    s.C = (float4*)(base + off); off += align_up(cbytes, 16);
    s.tw = (float2*)(base + off); off += sizeof(float2) * (size_t)(g.Ntw / 2);
    s.gP = (float*)(base + off); off += sizeof(float) * g.T1p;
    s.gM = (float*)(base + off); off += sizeof(float) * g.T1p;
    s.rv = (float*)(base + off); off += sizeof(float) * 128;
    s.rj = (int*)(base + off); off += sizeof(int) * 128;
    off = align_up(off, 8);
    s.rd = (double*)(base + off); off += sizeof(double) * 32;
    s.cj = (int*)(base + off); off += sizeof(int) * kMaxCand;
    s.cv = (float*)(base + off); off += sizeof(float) * kMaxCand;
    s.misc = (int*)(base + off); off += sizeof(int) * 16;
    s.miscf = (float*)(base + off);
    return s;
}

// ------------------------------------------------------- a1-a4: FFT correlation
// Leaves X = F[a] conj(F[b]) (H x Wc, natural order) in S.A and the unnormalised
// integer surface HW*c(s) packed in S.C as (row 2r, row 2r+1) pairs. Returns
// sum w|X| (for the guard thresholds), identical in every thread.
__device__ float fft_correlate(const Geom& g, const Smem& S, const void* frame, long long pitch) {
    const int H = g.H, W = g.W, Wc = g.Wc, Wcp = g.Wcp, Hh = g.Hh;
    float2* Z = (float2*)S.C;  // packed rows: H/2 x W

    // a1: ingest, operand, pack rows (2r, 2r+1) -> one complex row, x bit-reversed
    for (int idx = threadIdx.x; idx < H * W; idx += blockDim.x) {
        const int y = idx >> g.logW, x = idx & (W - 1);
        const float a = operand_f32(pixel_f32(frame, g.in_dtype, (long long)y * pitch + x), g);
        float* dst = (float*)&Z[(y >> 1) * W + brev(x, g.logW)];
        dst[y & 1] = a;
    }
    __syncthreads();
    // a2: row FFTs
    fft_r2_passes(Z, g.logW, Hh, W, 1, S.tw, g.logNtw, false);
    // split the packed spectra into rows 2r, 2r+1 of the half spectrum (rows bit-reversed)
    for (int idx = threadIdx.x; idx < Hh * Wcp; idx += blockDim.x) {
        const int r = idx / Wcp, kx = idx - r * Wcp;
        float2 fe = make_float2(0.f, 0.f), fo = make_float2(0.f, 0.f);
        if (kx < Wc) {
            const float2 z = Z[r * W + kx];
            const float2 zc = cconj(Z[r * W + ((W - kx) & (W - 1))]);
            fe = make_float2(0.5f * (z.x + zc.x), 0.5f * (z.y + zc.y));
            const float2 d = csub(z, zc);
            fo = make_float2(0.5f * d.y, -0.5f * d.x);   // (z - zc) / (2i)
        }
        S.A[brev(2 * r, g.logH) * Wcp + kx] = fe;
        S.A[brev(2 * r + 1, g.logH) * Wcp + kx] = fo;
    }
    __syncthreads();
    // column FFTs
    fft_r2_passes(S.A, g.logH, Wc, 1, Wcp, S.tw, g.logNtw, false);
    // a3: product with conj(F[b]); bit-reversed copy for the inverse column pass
    float sabs = 0.f;
    for (int idx = threadIdx.x; idx < H * Wc; idx += blockDim.x) {
        const int ky = idx / Wc, kx = idx - ky * Wc;
        const float2 fe = __ldg(&g.FE32[idx]);
        const float2 x = cmul(S.A[ky * Wcp + kx], cconj(fe));
        S.A[ky * Wcp + kx] = x;
        S.B[brev(ky, g.logH) * Wcp + kx] = x;
        const float w = (kx == 0 || 2 * kx == W) ? 1.f : 2.f;
        sabs += w * (fabsf(x.x) + fabsf(x.y));
    }
    __syncthreads();
    const float scale = block_sum(sabs, S.rv);
    // a4: inverse column FFTs, then C2R rows packed two per complex row
    fft_r2_passes(S.B, g.logH, Wc, 1, Wcp, S.tw, g.logNtw, true);
    for (int idx = threadIdx.x; idx < Hh * W; idx += blockDim.x) {
        const int r = idx >> g.logW, kx = idx & (W - 1);
        float2 ye, yo;
        if (kx < Wc) {
            ye = S.B[(2 * r) * Wcp + kx];
            yo = S.B[(2 * r + 1) * Wcp + kx];
        } else {
            ye = cconj(S.B[(2 * r) * Wcp + (W - kx)]);
            yo = cconj(S.B[(2 * r + 1) * Wcp + (W - kx)]);
        }
        Z[r * W + brev(kx, g.logW)] = make_float2(ye.x - yo.y, ye.y + yo.x);  // ye + i yo
    }
    __syncthreads();
    fft_r2_passes(Z, g.logW, Hh, W, 1, S.tw, g.logNtw, true);
    return scale;
}

__device__ __forceinline__ float int_surface(const Geom& g, const Smem& S, int flat) {
    const int y = flat >> g.logW, x = flat & (g.W - 1);
    const float2 z = ((const float2*)S.C)[(y >> 1) * g.W + x];
    return (y & 1) ? z.y : z.x;
}

// FP64 direct sum c(s) = sum_r a((r + s) mod N) b(r) (left-hand side of Eq. (4)/(7)).
__device__ double direct_sum_f64(const Geom& g, const Smem& S, const void* frame, long long pitch,
                                 int sy, int sx) {
    double acc = 0.0;
    for (int idx = threadIdx.x; idx < g.H * g.W; idx += blockDim.x) {
        const int y = idx >> g.logW, x = idx & (g.W - 1);
        const int yy = (y + sy) & (g.H - 1), xx = (x + sx) & (g.W - 1);
        double I;
        if (g.in_dtype == 0) I = load_pixel((const unsigned short*)frame, (long long)yy * pitch + xx);
        else I = load_pixel((const float*)frame, (long long)yy * pitch + xx);
        acc = fma(operand_f64(I, g), __ldg(&g.b64[idx]), acc);
    }
    return block_sum(acc, S.rd);
}

// ------------------------------------------------------ a5: integer extremum
// Returns the flat index of the integer peak (0..HW-1) and sets *flags.
__device__ int integer_peak(const Geom& g, const Smem& S, const void* frame, long long pitch,
                            float scale, unsigned* flags, float* dbg) {
    TopK<2> t2;
    t2.init();
    for (int idx = threadIdx.x; idx < g.H * g.W; idx += blockDim.x) {
        const float c = int_surface(g, S, idx);
        if (dbg) dbg[idx] = c;
        t2.push(g.sense * c, idx);
    }
    block_topk(t2, S.rv, S.rj);
    int best = t2.j[0];
    if (!(t2.v[0] > -INFINITY)) { *flags |= 0x10u; return 0; }
    const float tau = g.tau_int * scale;
    if (!g.guard || !(t2.v[0] - t2.v[1] <= tau)) return best;
    // collect every integer shift within tau of the best
    if (threadIdx.x == 0) S.misc[0] = 0;
    __syncthreads();
    const float thr = t2.v[0] - tau;
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

// --------------------------------------------- a6 prologue: X' and P/Q, R, g
// In place in S.A: row 0 = X'(0), row Hh = X'(Hh), row m = P(m), row H-m = Q(m).
// Writes g(+tx), g(-tx) to S.gP / S.gM.
__device__ void build_pq_and_g(const Geom& g, const Smem& S, int py, int px) {
    const int H = g.H, W = g.W, Wc = g.Wc, Wcp = g.Wcp, Hh = g.Hh;
    const int pyy = py & (H - 1), pxx = px & (W - 1);
    for (int idx = threadIdx.x; idx < (Hh + 1) * Wc; idx += blockDim.x) {
        const int m = idx / Wc, kx = idx - m * Wc;
        const int kxs = signed_k(kx, W);
        const float2 ex = twiddle_pos(S.tw, (kxs * pxx) & (W - 1), g.logW, g.logNtw);
        if (m == 0 || m == Hh) {
            const int kys = signed_k(m, H);
            const float2 ey = twiddle_pos(S.tw, (kys * pyy) & (H - 1), g.logH, g.logNtw);
            S.A[m * Wcp + kx] = cmul(S.A[m * Wcp + kx], cmul(ey, ex));
        } else {
            const float2 eyp = twiddle_pos(S.tw, (m * pyy) & (H - 1), g.logH, g.logNtw);
            const float2 eym = twiddle_pos(S.tw, (-m * pyy) & (H - 1), g.logH, g.logNtw);
            const float2 xp = cmul(S.A[m * Wcp + kx], cmul(eyp, ex));
            const float2 xm = cmul(S.A[(H - m) * Wcp + kx], cmul(eym, ex));
            S.A[m * Wcp + kx] = cadd(xp, xm);
            S.A[(H - m) * Wcp + kx] = csub(xp, xm);
        }
    }
    __syncthreads();
    // R(kx) = X'(0) + sum_{m=1}^{Hh-1} P(m) + X'(Hh), kept in S.B row 0
    for (int kx = threadIdx.x; kx < Wc; kx += blockDim.x) {
        float2 r = S.A[Hh * Wcp + kx];
        for (int m = Hh - 1; m >= 1; --m) r = cadd(r, S.A[m * Wcp + kx]);
        r = cadd(r, S.A[kx]);
        S.B[kx] = r;
    }
    __syncthreads();
    // g(+-tx) = sum_kx gc Rr -+ ws Ri
    for (int tx = threadIdx.x; tx < g.T1p; tx += blockDim.x) {
        float a = 0.f, b = 0.f;
        for (int kx = Wc - 1; kx >= 0; --kx) {
            const float2 r = S.B[kx];
            a = fmaf(__ldg(&g.tB_gc[kx * g.T1p + tx]), r.x, a);
            b = fmaf(__ldg(&g.tB_ws[kx * g.T1p + tx]), r.y, b);
        }
        S.gP[tx] = a - b;
        S.gM[tx] = a + b;
    }
    __syncthreads();
}

// --------------------------------------------------- a6: stage A (one chunk)
// UV[t - t0][kx] = (U'r, U'i, Vr, Vi)(t, kx) for t in [t0, t0 + TC).
__device__ void stage_a(const Geom& g, const Smem& S, int t0) {
    const int Wcp = g.Wcp, Hh = g.Hh, H = g.H;
    const int ntile_t = g.TC / 4, ntile_k = Wcp / 2;
    for (int tile = threadIdx.x; tile < ntile_t * ntile_k; tile += blockDim.x) {
        const int tt = tile / ntile_k, kk = tile - tt * ntile_k;
        const int tb = t0 + 4 * tt, kb = 2 * kk;
        float4 acc[4][2];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int k = 0; k < 2; ++k) acc[i][k] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (tb < g.T1p) {
            // Nyquist row first (signed -H/2): P = X'(Hh); Q = -X'(Hh) in the x-Nyquist
            // column only (elsewhere the row contributes through cos(pi t/u) alone)
            for (int m = Hh; m >= 1; --m) {
                const float4 cm = __ldg((const float4*)&g.tA_cm1[(m - 1) * g.T1p + tb]);
                const float4 sn = __ldg((const float4*)&g.tA_s[(m - 1) * g.T1p + tb]);
                const float4 p = *(const float4*)&S.A[m * Wcp + kb];
                float4 q;
                if (m == Hh) {
                    const int kn = g.W >> 1;
                    q = make_float4(kb == kn ? -p.x : 0.f, kb == kn ? -p.y : 0.f,
                                    kb + 1 == kn ? -p.z : 0.f, kb + 1 == kn ? -p.w : 0.f);
                } else {
                    q = *(const float4*)&S.A[(H - m) * Wcp + kb];
                }
                const float cmv[4] = {cm.x, cm.y, cm.z, cm.w};
                const float snv[4] = {sn.x, sn.y, sn.z, sn.w};
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    acc[i][0].x = fmaf(cmv[i], p.x, acc[i][0].x);
                    acc[i][0].y = fmaf(cmv[i], p.y, acc[i][0].y);
                    acc[i][0].z = fmaf(snv[i], q.x, acc[i][0].z);
                    acc[i][0].w = fmaf(snv[i], q.y, acc[i][0].w);
                    acc[i][1].x = fmaf(cmv[i], p.z, acc[i][1].x);
                    acc[i][1].y = fmaf(cmv[i], p.w, acc[i][1].y);
                    acc[i][1].z = fmaf(snv[i], q.z, acc[i][1].z);
                    acc[i][1].w = fmaf(snv[i], q.w, acc[i][1].w);
                }
            }
        }
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int k = 0; k < 2; ++k) S.C[(4 * tt + i) * Wcp + kb + k] = acc[i][k];
    }
    __syncthreads();
}

__device__ __forceinline__ int grid_index(const Geom& g, int ty, int tx) {
    return (ty + g.h0) * g.M + (tx + g.h0);
}

// --------------------------------------------------- a6: stage B (one chunk)
// Evaluates v = sense * (S + g) at every grid point whose |ty| lies in the chunk,
// feeding the top-K. With collect=true, also appends every point with v >= thr
// to the candidate list instead.
template <bool kCollect>
__device__ void stage_b(const Geom& g, const Smem& S, int t0, TopK<kTopK>& top, float thr, float* dbg) {
    const int Wcp = g.Wcp, Wc = g.Wc;
    const int ntile_t = g.TC / 4, ntile_x = g.T1p / 4;
    for (int tile = threadIdx.x; tile < ntile_t * ntile_x; tile += blockDim.x) {
        const int tt = tile / ntile_x, xx = tile - tt * ntile_x;
        const int tb = t0 + 4 * tt, xb = 4 * xx;
        if (tb > g.h0) continue;
        float aU[4][4], aV[4][4], bU[4][4], bV[4][4];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int l = 0; l < 4; ++l) { aU[i][l] = 0.f; aV[i][l] = 0.f; bU[i][l] = 0.f; bV[i][l] = 0.f; }
        for (int kx = Wc - 1; kx >= 0; --kx) {
            const float4 wc = __ldg((const float4*)&g.tB_wc[kx * g.T1p + xb]);
            const float4 ws = __ldg((const float4*)&g.tB_ws[kx * g.T1p + xb]);
            const float wcv[4] = {wc.x, wc.y, wc.z, wc.w};
            const float wsv[4] = {ws.x, ws.y, ws.z, ws.w};
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const float4 uv = S.C[(4 * tt + i) * Wcp + kx];
#pragma unroll
                for (int l = 0; l < 4; ++l) {
                    aU[i][l] = fmaf(wcv[l], uv.x, aU[i][l]);
                    aV[i][l] = fmaf(wcv[l], uv.w, aV[i][l]);
                    bU[i][l] = fmaf(wsv[l], uv.y, bU[i][l]);
                    bV[i][l] = fmaf(wsv[l], uv.z, bV[i][l]);
                }
            }
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int t = tb + i;
            if (t > g.h0) continue;
#pragma unroll
            for (int l = 0; l < 4; ++l) {
                const int x = xb + l;
                if (x > g.h0) continue;
                const float gp = S.gP[x], gm = S.gM[x];
                const float A0 = aU[i][l] - aV[i][l], A1 = aU[i][l] + aV[i][l];
                float vals[4];
                int js[4];
                int nv = 0;
                // (+t, +x)
                if (t <= g.pmax && x <= g.pmax) {
                    vals[nv] = A0 - bU[i][l] - bV[i][l] + gp; js[nv++] = grid_index(g, t, x);
                }
                // (+t, -x)
                if (t <= g.pmax && x >= 1) {
                    vals[nv] = A0 + bU[i][l] + bV[i][l] + gm; js[nv++] = grid_index(g, t, -x);
                }
                // (-t, +x)
                if (t >= 1 && x <= g.pmax) {
                    vals[nv] = A1 - bU[i][l] + bV[i][l] + gp; js[nv++] = grid_index(g, -t, x);
                }
                // (-t, -x)
                if (t >= 1 && x >= 1) {
                    vals[nv] = A1 + bU[i][l] - bV[i][l] + gm; js[nv++] = grid_index(g, -t, -x);
                }
                for (int q = 0; q < nv; ++q) {
                    const float v = g.sense * vals[q];
                    if (kCollect) {
                        if (v >= thr) {
                            const int k = atomicAdd(&S.misc[1], 1);
                            if (k < kMaxCand) { S.cj[k] = js[q]; S.cv[k] = v; }
                        }
                    } else {
                        if (dbg) dbg[js[q]] = vals[q];
                        top.push(v, js[q]);
                    }
                }
            }
        }
    }
}

// Full upsampled surface pass (all chunks): top-K, or candidate collection.
template <bool kCollect>
__device__ void upsampled_pass(const Geom& g, const Smem& S, TopK<kTopK>& top, float thr, float* dbg) {
    for (int c = 0; c < g.nchunk; ++c) {
        const int t0 = c * g.TC;
        stage_a(g, S, t0);
        stage_b<kCollect>(g, S, t0, top, thr, dbg);
        __syncthreads();
    }
}

// ---------------------------------- a7 guard: exact FP32 pair differences
// X'(ky, kx) for any row, from the P/Q layout of S.A.
__device__ __forceinline__ float2 xprime(const Geom& g, const Smem& S, int ky, int kx) {
    const int Hh = g.Hh, Wcp = g.Wcp;
    if (ky == 0 || ky == Hh) return S.A[ky * Wcp + kx];
    if (ky < Hh) {
        const float2 p = S.A[ky * Wcp + kx], q = S.A[(g.H - ky) * Wcp + kx];
        return make_float2(0.5f * (p.x + q.x), 0.5f * (p.y + q.y));
    }
    const int m = g.H - ky;
    const float2 p = S.A[m * Wcp + kx], q = S.A[ky * Wcp + kx];
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

// Full twiddle exp(2 pi i k' t / (uN)) of the stage tables (FP64-rounded values).
__device__ __forceinline__ float2 table_twiddle_y(const Geom& g, int ks, int t) {
    const int m = ks < 0 ? -ks : ks, at = t < 0 ? -t : t;
    if (m == 0 || at == 0) return make_float2(1.f, 0.f);
    const float c = 1.f + __ldg(&g.tA_cm1[(m - 1) * g.T1p + at]);
    const float s = __ldg(&g.tA_s[(m - 1) * g.T1p + at]);
    return make_float2(c, ((ks < 0) != (t < 0)) ? -s : s);
}

// Decide among the candidates S.cj[0..nc) (S.cj[0] is the FP32 best j1) with exact
// pair differences D(j) = v(j) - v(j1). Returns the winner; sets *l2 when the two
// best remain within tau1, leaving the tied candidates in S.cj[0..*nl2).
__device__ int pair_difference_guard(const Geom& g, const Smem& S, int nc, float scale, int* nl2,
                                     float* dwin) {
    const int H = g.H, Wc = g.Wc, Wcp = g.Wcp, u = g.u;
    float2* G = (float2*)S.C;          // H      G(ky) = sum_kx w X'(ky,kx) E(kx, rx)
    float2* Eyc = G + H;               // H      E(ky, ty_c)
    float2* dEy = Eyc + H;             // H      E(ky, ty_c) - E(ky, ry)
    float2* dEx = dEy + H;             // Wcp    w (E(kx, tx_c) - E(kx, rx))
    const int j1 = S.cj[0];
    const int ry = j1 / g.M - g.h0, rx = j1 % g.M - g.h0;
    // G(ky), using the table twiddles w E(kx, rx) = wc -+ i ws. For the Nyquist row the
    // x-Nyquist column is kept apart in slot H + 3H + Wcp (it takes the full y-phase).
    float2* GN = dEx + Wcp;
    const int kn = g.W >> 1;
    for (int ky = threadIdx.x; ky < H; ky += blockDim.x) {
        float2 acc = make_float2(0.f, 0.f), accn = make_float2(0.f, 0.f);
        const int arx = rx < 0 ? -rx : rx;
        for (int kx = Wc - 1; kx >= 0; --kx) {
            const float c = __ldg(&g.tB_wc[kx * g.T1p + arx]);
            float s = __ldg(&g.tB_ws[kx * g.T1p + arx]);
            if (rx < 0) s = -s;
            const float2 t = cmul(xprime(g, S, ky, kx), make_float2(c, s));
            if (ky == g.Hh && kx == kn) accn = t; else acc = cadd(acc, t);
        }
        G[ky] = acc;
        if (ky == g.Hh) GN[0] = accn;
    }
    __syncthreads();
    if (threadIdx.x == 0) S.cv[0] = 0.f;
    for (int c = 1; c < nc; ++c) {
        const int jc = S.cj[c];
        const int ty = jc / g.M - g.h0, tx = jc % g.M - g.h0;
        for (int ky = threadIdx.x; ky < H; ky += blockDim.x) {
            const int ks = signed_k(ky, H);
            Eyc[ky] = table_twiddle_y(g, ks, ty);
            // E(ty) - E(ry) = 2i sin(pi k'(ty - ry)/(uH)) exp(i pi k'(ty + ry)/(uH))
            const float s1 = sin_pi_frac((long long)ks * (ty - ry), (long long)u * H);
            const float2 e2 = expi_pi_frac((long long)ks * (ty + ry), (long long)u * H);
            dEy[ky] = make_float2(-2.f * s1 * e2.y, 2.f * s1 * e2.x);
        }
        for (int kx = threadIdx.x; kx < Wc; kx += blockDim.x) {
            const int ks = signed_k(kx, g.W);
            const float w = (kx == 0 || 2 * kx == g.W) ? 1.f : 2.f;
            const float s1 = sin_pi_frac((long long)ks * (tx - rx), (long long)u * g.W);
            const float2 e2 = expi_pi_frac((long long)ks * (tx + rx), (long long)u * g.W);
            dEx[kx] = make_float2(-2.f * w * s1 * e2.y, 2.f * w * s1 * e2.x);
        }
        __syncthreads();
        float part = 0.f;
        for (int ky = threadIdx.x; ky < H; ky += blockDim.x) {
            float2 F = make_float2(0.f, 0.f), FN = make_float2(0.f, 0.f);
            for (int kx = Wc - 1; kx >= 0; --kx) {
                const float2 t = cmul(xprime(g, S, ky, kx), dEx[kx]);
                if (ky == g.Hh && kx == kn) FN = t; else F = cadd(F, t);
            }
            if (ky == g.Hh) {
                // real part of the row's y-phase, except in the x-Nyquist column
                part += Eyc[ky].x * F.x + dEy[ky].x * G[ky].x;
                part += cmul(Eyc[ky], FN).x + cmul(dEy[ky], GN[0]).x;
            } else {
                part += cmul(Eyc[ky], F).x + cmul(dEy[ky], G[ky]).x;
            }
        }
        const float D = block_sum(part, S.rv);
        if (threadIdx.x == 0) S.cv[c] = g.sense * D;
        __syncthreads();
    }
    __syncthreads();
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
        // keep every candidate within tau1 of the winner for the FP64 pass
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
// accumulation (the Nyquist-row rule included). Scratch: S.C.
__device__ double pair_difference_f64(const Geom& g, const Smem& S, int ja, int jb, double* red) {
    const int H = g.H, Wc = g.Wc;
    double2* eyA = (double2*)S.C;
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

__device__ df block_sum_df(df v, double* red) {
    // double-float sum across the block; the 16 warp partials are combined in FP64 (few ops)
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
// X = F[a] conj(F[b]): R2C FFT of the operand in double-float (S.A..S.B hold the
// H x Wcp half spectrum, S.C the packed row chunks), then
//   cu(j) = Re sum_{ky,kx} w X(ky,kx) E_y(ky, py u + ty) E_x(kx, px u + tx)
// with exactly reduced angles. Returns the winner (sense-adjusted maximum,
// lowest index on ties) and its unnormalised value in *val.
__device__ int df_reevaluate(const Geom& g, const Smem& S, const void* frame, long long pitch,
                             int py, int px, int nc, double* val) {
    const int H = g.H, W = g.W, Wc = g.Wc, Wcp = g.Wcp, Hh = g.Hh;
    dfc* Xd = (dfc*)S.A;                        // spans S.A and S.B
    dfc* Zc = (dfc*)S.C;
    const int cbytes = (int)((char*)S.tw - (char*)S.C);
    int R = 1;
    while (2 * R <= Hh && 2 * R * W * (int)sizeof(dfc) <= cbytes) R *= 2;
    for (int r0 = 0; r0 < Hh; r0 += R) {
        for (int idx = threadIdx.x; idx < 2 * R * W; idx += blockDim.x) {
            const int yl = idx / W, x = idx - yl * W;
            const int y = 2 * r0 + yl;
            const float I = pixel_f32(frame, g.in_dtype, (long long)y * pitch + x);
            df a = df_make(I);
            if (g.method != 0) {
                float s, e;
                two_sum(I, g.eps, s, e);
                const df ip = {s, e};
                a = df_mul(ip, ip);
            }
            dfc* z = &Zc[(yl >> 1) * W + brev(x, g.logW)];
            if (y & 1) z->im = a; else z->re = a;
        }
        __syncthreads();
        fft_r2_passes(Zc, g.logW, R, W, 1, g.twdf, g.logNtw, false);
        for (int idx = threadIdx.x; idx < R * Wcp; idx += blockDim.x) {
            const int rl = idx / Wcp, kx = idx - rl * Wcp;
            dfc fe = {{0.f, 0.f}, {0.f, 0.f}}, fo = fe;
            if (kx < Wc) {
                const dfc z = Zc[rl * W + kx];
                const dfc zc = cconj(Zc[rl * W + ((W - kx) & (W - 1))]);
                const dfc sp = cadd(z, zc), dm = csub(z, zc);
                fe = {df_scale(sp.re, 0.5f), df_scale(sp.im, 0.5f)};
                fo = {df_scale(dm.im, 0.5f), df_scale(df_neg(dm.re), 0.5f)};   // (z - zc) / (2i)
            }
            const int r = r0 + rl;
            Xd[brev(2 * r, g.logH) * Wcp + kx] = fe;
            Xd[brev(2 * r + 1, g.logH) * Wcp + kx] = fo;
        }
        __syncthreads();
    }
    fft_r2_passes(Xd, g.logH, Wc, 1, Wcp, g.twdf, g.logNtw, false);
    for (int idx = threadIdx.x; idx < H * Wc; idx += blockDim.x) {
        const int ky = idx / Wc, kx = idx - ky * Wc;
        Xd[ky * Wcp + kx] = cmul(Xd[ky * Wcp + kx], cconj(g.FEdf[idx]));
    }
    __syncthreads();
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
        for (int idx = threadIdx.x; idx < H * Wc; idx += blockDim.x) {
            const int ky = idx / Wc, kx = idx - ky * Wc;
            dfc ey = Ey[ky];
            if (ky == Hh && 2 * kx != W) ey.im = {0.f, 0.f};   // real part of the Nyquist row's phase
            const dfc e = cmul(ey, Ex[kx]);
            const dfc x = Xd[ky * Wcp + kx];
            acc = df_add(acc, df_sub(df_mul(x.re, e.re), df_mul(x.im, e.im)));
        }
        const double v = df_to_double(block_sum_df(acc, S.rd));
        const double sv = (double)g.sense * v;
        if (sv > bestv || (sv == bestv && j < bestj)) { bestv = sv; bestj = j; bestraw = v; }
        __syncthreads();
    }
    *val = bestraw;
    return bestj;
}

// ---------------------------------------------------------- the FP32 kernel
__global__ void __launch_bounds__(kThreads, 1) track_kernel(Geom g, Batch b) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const Smem S = carve(g, smem_raw);
    for (int k = threadIdx.x; k < g.Ntw / 2; k += blockDim.x) S.tw[k] = g.tw32[k];
    __syncthreads();
    const size_t elem = g.in_dtype == 0 ? 2 : 4;
    for (long long f = blockIdx.x; f < b.n; f += gridDim.x) {
        const char* frame = (const char*)b.frames + (size_t)f * g.H * b.pitch * elem;
        unsigned flags = 0;
        const float scale = fft_correlate(g, S, frame, b.pitch);
        const int ip = integer_peak(g, S, frame, b.pitch, scale, &flags,
                                    b.dbg_int ? b.dbg_int + (size_t)f * g.H * g.W : nullptr);
        const float c0 = int_surface(g, S, ip);           // HW * c(p)
        const int py = wrap_shift(ip >> g.logW, g.H), px = wrap_shift(ip & (g.W - 1), g.W);
        __syncthreads();
        build_pq_and_g(g, S, py, px);
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
            continue;
        }
        TopK<kTopK> top;
        top.init();
        float* dbg = b.dbg_sub ? b.dbg_sub + (size_t)f * g.M * g.M : nullptr;
        upsampled_pass<false>(g, S, top, 0.f, dbg);
        block_topk(top, S.rv, S.rj);
        int jw = top.j[0];
        const float vw = top.v[0];
        float dwin = 0.f;
        int nl2 = 0;
        if (!(vw > -INFINITY)) {
            flags |= 0x10u;
            jw = 0;
        } else if (g.guard) {
            const float tau0 = g.tau0 * scale;
            const float thr = top.v[0] - tau0;
            int nc = 0;
#pragma unroll
            for (int k = 0; k < kTopK; ++k) nc += (top.v[k] >= thr) ? 1 : 0;
            if (nc > 1) {
                flags |= 0x02u;
                if (nc < kTopK) {
                    if (threadIdx.x == 0)
                        for (int k = 0; k < nc; ++k) S.cj[k] = top.j[k];
                    __syncthreads();
                } else {
                    // more than K-1 near ties: collect them all with a second pass
                    if (threadIdx.x == 0) S.misc[1] = 0;
                    __syncthreads();
                    upsampled_pass<true>(g, S, top, thr, nullptr);
                    nc = S.misc[1];
                    __syncthreads();
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
            jw = df_reevaluate(g, S, frame, b.pitch, py, px, nl2, &raw);
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
    }
}

// ------------------------------------------------------ FP64 re-evaluation
// For frames whose FP32 pair differences stayed within tau1, recompute the product
// spectrum in FP64 (R2C FFT of the operand, product with the FP64 reference
// spectrum) and evaluate the upsampled surface at the candidates directly:
//   cu(j) = Re sum_{ky,kx} w X(ky,kx) exp(2 pi i [ky'(py u + ty)/(uH) + kx'(px u + tx)/(uW)]).
// Workspace: per CTA, H/2*W + H*Wcp double2 in global memory.
__device__ void fft_r2c_f64_global(const Geom& g, const double* a_or_null, const void* frame,
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
