// ccst_tc.cuh -- 5th-generation tensor-core (tcgen05) helpers for the upsampled-DFT
// contraction: shared-memory matrix descriptors, the instruction descriptor of a
// kind::f16 MMA, MMA issue and commit, Tensor Memory allocation and loads, and the fences
// that order them against ordinary shared-memory accesses.
//
// Operand matrices are K-major with the 128-byte swizzle: a row holds 64 fp16 values
// (128 bytes), 8-row atoms are 1024 bytes, and the 16-byte chunk c of row r sits at chunk
// c ^ (r mod 8). Every matrix starts on a 1024-byte boundary; a K step of 16 values moves
// the descriptor's start address by 32 bytes inside the atom. The accumulator of an M = 128
// MMA occupies Tensor Memory lanes 0..127 (row i in lane i), one 32-bit column per N index.
#pragma once

#include <cstdint>

namespace ccst {

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// byte offset of element (row r, k) in a 64-wide K-major matrix with the 128-byte swizzle
__host__ __device__ __forceinline__ uint32_t sw128_off(int r, int k) {
    return (uint32_t)(r * 128 + ((((k >> 3) ^ r) & 7) << 4) + ((k & 7) << 1));
}

// shared-memory matrix descriptor: start address, stride between 8-row atoms 1024 bytes,
// descriptor version 1, 128-byte swizzle (the leading offset is unused for this layout)
__device__ __forceinline__ uint64_t tc_desc(uint32_t addr) {
    return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)1u << 16) | ((uint64_t)(1024u >> 4) << 32) |
           ((uint64_t)1u << 46) | ((uint64_t)2u << 61);
}

// instruction descriptor of kind::f16: F32 accumulator, F16 A and B, both K-major, M x N
__host__ __device__ constexpr uint32_t tc_idesc(int m, int n) {
    return (1u << 4) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

// D[tmem] (+)= A * B^T, issued by one thread
__device__ __forceinline__ void tc_mma(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc, uint32_t idesc,
                                       uint32_t accumulate) {
    asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                 "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
                 ::"r"(d_tmem), "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate)
                 : "memory");
}

// the MMAs issued so far by this thread arrive on the mbarrier when they complete
__device__ __forceinline__ void tc_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}

__device__ __forceinline__ void tc_bar_init(uint32_t bar) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(bar) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}

// Bounded wait for phase `parity` of an mbarrier: false after `limit` polls.
__device__ __forceinline__ bool tc_bar_wait(uint32_t bar, uint32_t parity, int limit) {
    for (int it = 0; it < limit; ++it) {
        uint32_t done;
        asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
                     : "=r"(done) : "r"(bar), "r"(parity) : "memory");
        if (done) return true;
    }
    return false;
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// ordinary shared-memory stores -> visible to the tensor cores' operand reads
__device__ __forceinline__ void tc_fence_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// Tensor Memory allocation of `cols` columns by one whole warp; the base address is
// written to the shared word `slot`.
__device__ __forceinline__ void tc_alloc(uint32_t slot, uint32_t cols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(slot), "r"(cols) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tc_dealloc(uint32_t tmem, uint32_t cols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(cols) : "memory");
}

// 16 consecutive columns of the warp's 32 lanes (lane base in bits 31..16 of the address)
__device__ __forceinline__ void tc_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                   "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
                 : "r"(taddr) : "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}
// 4 consecutive columns
__device__ __forceinline__ void tc_ld4(uint32_t taddr, float (&v)[4]) {
    uint32_t r[4];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]) : "r"(taddr) : "memory");
#pragma unroll
    for (int i = 0; i < 4; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void tc_ld_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// Per-CTA state of the tensor-core contraction, in static shared memory (the dynamic
// layout is re-carved per frame size; this must not move): the Tensor Memory base, the
// number of completed MMA batches (its parity is the mbarrier phase to wait for), and
// the mbarrier that tcgen05.commit arrives on.
struct TcShared {
    unsigned long long bar;
    uint32_t tmem;
    uint32_t batches;
    uint32_t failed;        // an MMA batch never completed: results of this CTA are void
    uint32_t pad;
};
__device__ __forceinline__ TcShared* tc_shared() {
    __shared__ __align__(16) TcShared s;
    return &s;
}

constexpr uint32_t kTcCols = 512;          // Tensor Memory columns held by a CTA of the tracking kernels

// Kernel start (all threads): allocate the columns and initialise the barrier.
__device__ __forceinline__ void tc_setup() {
    TcShared* t = tc_shared();
    if (threadIdx.x < 32) tc_alloc(smem_addr(&t->tmem), kTcCols);
    if (threadIdx.x == 0) {
        tc_bar_init(smem_addr(&t->bar));
        t->batches = 0;
        t->failed = 0;
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
}
// Kernel end (all threads, every exit path): release the columns.
__device__ __forceinline__ void tc_teardown() {
    TcShared* t = tc_shared();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (threadIdx.x < 32) tc_dealloc(t->tmem, kTcCols);
}

}  // namespace ccst
