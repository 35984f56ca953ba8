// tcgen05 / TMA helpers shared by the tensor-core kernels (inline PTX, sm_103a).
//
// Operand tiles use the canonical no-swizzle K-major layout: 8-row x 16-byte
// core matrices, K-adjacent core matrices 128 B apart (leading byte offset),
// 8-row groups KT * 32 B apart (stride byte offset) for a tile of KT FP32/TF32
// columns.  MMAs are kind::tf32 with FP32 accumulation in tensor memory, issued
// by one thread and committed to an mbarrier.  Every wait is bounded.
#pragma once

#include <cstdint>

namespace ksc {
namespace tc {

constexpr int kMaxWait = 1 << 22;  // mbarrier polls before giving up

__device__ __forceinline__ uint32_t saddr(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

// element (row, k) of a K-major tile with KT columns
template <int KT>
__host__ __device__ __forceinline__ int toff(int row, int k) {
    return (row >> 3) * (KT * 8) + (k >> 2) * 32 + (row & 7) * 4 + (k & 3);
}

template <int KT>
__device__ __forceinline__ uint64_t smem_desc(const void *p) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr(p) & 0x3FFFF) >> 4);
    d |= (uint64_t)((128u >> 4) & 0x3FFF) << 16;       // leading (K) core-matrix stride
    d |= (uint64_t)(((KT * 32u) >> 4) & 0x3FFF) << 32;  // stride (8-row group) offset
    d |= (uint64_t)1 << 46;                             // descriptor version
    return d;                                           // no swizzle, base offset 0
}

// instruction descriptor: F32 accumulator, TF32 A and B, both K-major
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N) {
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) |
           ((uint32_t)(M >> 4) << 24);
}

// x = hi + lo with hi, lo representable in TF32 (round to nearest)
__device__ __forceinline__ void split_tf32(float x, float *hi, float *lo) {
    uint32_t h;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(h) : "f"(x));
    const float hf = __uint_as_float(h);
    uint32_t l;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(l) : "f"(x - hf));
    *hi = hf;
    *lo = __uint_as_float(l);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(saddr(bar)), "r"(count));
}

// Bounded wait for the given phase parity; false if the limit ran out (after
// max_polls tries).
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity,
                                          int max_polls = kMaxWait) {
    for (int it = 0; it < max_polls; ++it) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
            " selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(saddr(bar)), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

// Bounded wait that lets the hardware suspend the thread (up to hint_ns per try)
// until the phase completes instead of spinning: for a thread with nothing else
// to do.  At most kMaxWait tries.
__device__ __forceinline__ bool mbar_wait_sleep(uint64_t *bar, uint32_t parity,
                                                uint32_t hint_ns) {
    for (int it = 0; it < kMaxWait; ++it) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n"
            " selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(saddr(bar)), "r"(parity), "r"(hint_ns)
            : "memory");
        if (done) return true;
    }
    return false;
}

__device__ __forceinline__ void mma_tf32(uint32_t tmem, uint64_t da, uint64_t db, uint32_t idesc,
                                         uint32_t acc) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
        "l"(da), "l"(db), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void mma_commit(uint64_t *bar) {
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            saddr(bar))
        : "memory");
}

// 16 consecutive 32-bit TMEM columns of this thread's lane
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t *v) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,"
        "%12,%13,%14,%15}, [%16];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
          "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]),
          "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
        : "r"(taddr));
}

__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t *v) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,"
        "%12,%13,%14,%15,%16};" ::"r"(taddr),
        "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]),
        "r"(v[8]), "r"(v[9]), "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]),
        "r"(v[15])
        : "memory");
}

__device__ __forceinline__ void tmem_wait_ld() {
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_wait_st() {
    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void fence_before_sync() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void fence_after_sync() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// generic-proxy shared-memory writes -> visible to the tensor core (async proxy)
__device__ __forceinline__ void fence_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

} // namespace tc
} // namespace ksc
