// ccst_device.cuh -- device building blocks of the tracking kernels (sm_103a).
//
// Complex arithmetic, radix-2 FFT passes over shared or global memory, block
// reductions, and the (value, index) top-K search with the lowest-row-major-index
// tie rule of the method's argmax (Sec. III).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <math.h>
#include <limits.h>

#include "ccst_dfloat.cuh"

namespace ccst {

constexpr int kThreads = 512;            // threads per CTA of the tracking kernels
constexpr int kWarps = kThreads / 32;
constexpr int kTopK = 4;                 // candidates kept by the sub-pixel search
constexpr int kMaxCand = 32;             // near-tie candidates a frame may carry to exact re-evaluation
constexpr int kMaxCandL2 = 16;           // candidates handed to the FP64 re-evaluation
constexpr int kMaxIntCand = 16;          // integer near-tie candidates

// ------------------------------------------------------------------ complex helpers
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
    return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ double2 cconj(double2 a) { return make_double2(a.x, -a.y); }

template <typename C> struct CplxTraits;
template <> struct CplxTraits<float2> { typedef float R; };
template <> struct CplxTraits<double2> { typedef double R; };

template <typename C> __device__ __forceinline__ C cmake(typename CplxTraits<C>::R x, typename CplxTraits<C>::R y);
template <> __device__ __forceinline__ float2 cmake<float2>(float x, float y) { return make_float2(x, y); }
template <> __device__ __forceinline__ double2 cmake<double2>(double x, double y) { return make_double2(x, y); }

__device__ __forceinline__ int brev(int x, int logN) { return (int)(__brev((unsigned)x) >> (32 - logN)); }

// Hint that [p, p + bytes) is read soon: bulk prefetches into L2 (cp.async.bulk.prefetch,
// sm_90 and later) over the 16-byte-aligned part of the range, in pieces of at most 32 KB.
// One thread issues them; nothing waits on them, and no byte outside the range is touched.
__device__ __forceinline__ void prefetch_l2(const void* p, size_t bytes) {
    const uintptr_t a = ((uintptr_t)p + 15) & ~(uintptr_t)15, e = ((uintptr_t)p + bytes) & ~(uintptr_t)15;
    for (uintptr_t q = a; q < e; q += 32768) {
        const unsigned n = (unsigned)(e - q < 32768 ? e - q : 32768);
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;\n" ::"l"(q), "r"(n) : "memory");
    }
}

// Programmatic dependent launch (sm_90 and later), for persistent kernels chained on one
// stream. pdl_trigger: the next kernel on the stream, if it was launched with programmatic
// stream serialization, may start once every CTA of this grid has called it or exited (a
// no-op without such a kernel). pdl_wait: returns once the grid this one was let in early
// behind has completed and its writes are visible (at once if there is none). A chained
// kernel calls pdl_wait before it exits, so that its completion implies that of every
// kernel before it in the chain.
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory"); }
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;\n" ::: "memory"); }

// ------------------------------------------------------------------ radix-2 FFT
// In-place radix-2 decimation-in-time passes over `nseq` independent sequences of
// length N = 2^logN. Element i of sequence s sits at buf[s*seq_stride + i*elem_stride].
// The input must be in bit-reversed order; the output is in natural order.
// tw[k] = exp(-2 pi i k / Ntw), k < Ntw/2, Ntw = 2^logNtw >= N. inverse=true uses
// exp(+2 pi i ...) and does not scale. Ends with __syncthreads().
template <typename C>
static __device__ void fft_r2_passes(C* buf, int logN, int nseq, int seq_stride, int elem_stride,
                              const C* tw, int logNtw, bool inverse) {
    const int halfN = 1 << (logN - 1);
    const int total = halfN * nseq;
    for (int s = 0; s < logN; ++s) {
        const int half = 1 << s;
        const int twshift = logNtw - (s + 1);
        for (int b = threadIdx.x; b < total; b += blockDim.x) {
            const int seq = b >> (logN - 1);
            const int k = b & (halfN - 1);
            const int pos = k & (half - 1);
            const int i0 = ((k >> s) << (s + 1)) + pos;
            const int i1 = i0 + half;
            C w = tw[pos << twshift];
            if (inverse) w = cconj(w);
            C* base = buf + (size_t)seq * seq_stride;
            const C a = base[(size_t)i0 * elem_stride];
            const C c = base[(size_t)i1 * elem_stride];
            const C t = cmul(w, c);
            base[(size_t)i0 * elem_stride] = cadd(a, t);
            base[(size_t)i1 * elem_stride] = csub(a, t);
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------------ reductions
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Block-wide sum; every thread gets the result. `scratch` holds >= kWarps values.
template <typename T>
__device__ T block_sum(T v, T* scratch) {
    v = warp_sum(v);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) scratch[wid] = v;
    __syncthreads();
    T r = 0;
    const int nwarps = (blockDim.x + 31) >> 5;
    if (wid == 0) {
        r = lane < nwarps ? scratch[lane] : T(0);
        r = warp_sum(r);
        if (lane == 0) scratch[0] = r;
    }
    __syncthreads();
    r = scratch[0];
    __syncthreads();
    return r;
}

// ------------------------------------------------------------------ (value, index) top-K
// "Better" = larger value; equal values: smaller flat index (the oracle's argmax rule).
__device__ __forceinline__ bool better(float va, int ja, float vb, int jb) {
    return va > vb || (va == vb && ja < jb);
}

template <int K>
struct TopK {
    float v[K];
    int j[K];
    __device__ __forceinline__ void init() {
#pragma unroll
        for (int k = 0; k < K; ++k) { v[k] = -INFINITY; j[k] = INT_MAX; }
    }
    // Sorted insertion; the K best distinct entries survive.
    __device__ __forceinline__ void push(float val, int idx) {
        if (!better(val, idx, v[K - 1], j[K - 1])) return;
#pragma unroll
        for (int k = 0; k < K; ++k) {
            if (better(val, idx, v[k], j[k])) {
                const float tv = v[k]; const int tj = j[k];
                v[k] = val; j[k] = idx;
                val = tv; idx = tj;
            }
        }
    }
    __device__ __forceinline__ void warp_merge() {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            float ov[K]; int oj[K];
#pragma unroll
            for (int k = 0; k < K; ++k) {
                ov[k] = __shfl_xor_sync(0xffffffffu, v[k], o);
                oj[k] = __shfl_xor_sync(0xffffffffu, j[k], o);
            }
#pragma unroll
            for (int k = 0; k < K; ++k) push(ov[k], oj[k]);
        }
    }
};

// The best (value, index) under better() and the runner-up's value, branch-free. The
// integer search needs the runner-up only to detect near ties.
struct Best2 {
    float v1, v2;
    int j1;
    __device__ __forceinline__ void init() { v1 = -INFINITY; v2 = -INFINITY; j1 = INT_MAX; }
    __device__ __forceinline__ void push(float v, int j) {
        const bool b = better(v, j, v1, j1);
        v2 = b ? v1 : fmaxf(v2, v);
        v1 = b ? v : v1;
        j1 = b ? j : j1;
    }
};

// Block-wide (value, index) maximum under better(); every thread gets it.
// sv/sj: >= 32 entries of scratch.
__device__ __forceinline__ void block_argmax(float& v, int& j, float* sv, int* sj) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float ov = __shfl_xor_sync(0xffffffffu, v, o);
        const int oj = __shfl_xor_sync(0xffffffffu, j, o);
        if (better(ov, oj, v, j)) { v = ov; j = oj; }
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) { sv[wid] = v; sj[wid] = j; }
    __syncthreads();
    const int nwarps = (blockDim.x + 31) >> 5;
    v = -INFINITY;
    j = INT_MAX;
    for (int w = 0; w < nwarps; ++w)
        if (better(sv[w], sj[w], v, j)) { v = sv[w]; j = sj[w]; }
    __syncthreads();
}

// block_argmax fused with a block-wide sum of s (returned); sv/sj/ss: >= 32 entries each.
__device__ __forceinline__ float block_argmax_sum(float& v, int& j, float s, float* sv, int* sj, float* ss) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float ov = __shfl_xor_sync(0xffffffffu, v, o);
        const int oj = __shfl_xor_sync(0xffffffffu, j, o);
        s += __shfl_xor_sync(0xffffffffu, s, o);
        if (better(ov, oj, v, j)) { v = ov; j = oj; }
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) { sv[wid] = v; sj[wid] = j; ss[wid] = s; }
    __syncthreads();
    const int nwarps = (blockDim.x + 31) >> 5;
    v = -INFINITY;
    j = INT_MAX;
    float tot = 0.f;
    for (int w = 0; w < nwarps; ++w) {
        if (better(sv[w], sj[w], v, j)) { v = sv[w]; j = sj[w]; }
        tot += ss[w];
    }
    __syncthreads();
    return tot;
}

// Block-wide top-K; all threads return the merged list. sv/sj: >= kWarps*K entries.
template <int K>
__device__ __forceinline__ void block_topk(TopK<K>& t, float* sv, int* sj) {
    t.warp_merge();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) {
#pragma unroll
        for (int k = 0; k < K; ++k) { sv[wid * K + k] = t.v[k]; sj[wid * K + k] = t.j[k]; }
    }
    __syncthreads();
    const int nwarps = (blockDim.x + 31) >> 5;
    if (wid == 0) {
        t.init();
        if (lane < nwarps) {
#pragma unroll
            for (int k = 0; k < K; ++k) t.push(sv[lane * K + k], sj[lane * K + k]);
        }
        t.warp_merge();
        if (lane == 0) {
#pragma unroll
            for (int k = 0; k < K; ++k) { sv[k] = t.v[k]; sj[k] = t.j[k]; }
        }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < K; ++k) { t.v[k] = sv[k]; t.j[k] = sj[k]; }
    __syncthreads();
}

}  // namespace ccst
