// umma.cuh -- inline-PTX helpers for the fifth-generation tensor cores
// (tcgen05.mma with accumulators in tensor memory) shared by the 3-D spread
// and gather kernels: shared-memory matrix descriptors, the TF32 MMA with A
// from shared memory or from tensor memory, bounded mbarrier waits and the
// tensor-memory load and store shapes used here.
//
// Operand layout in shared memory: K-major without swizzle, core matrices of
// 8 rows x 16 bytes (4 TF32 values); LBO = 128 bytes between the two core
// matrices of one 8-wide K step, SBO between 8-row groups.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace anova {

constexpr int kUmmaSpin = 1 << 22;          // mbarrier polls before a wait gives up

__device__ __forceinline__ uint32_t su32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint32_t tf32_rna(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}

// TF32 head (the value truncated to TF32, exactly representable) and tail
// (x - head, exact in FP32: at most 13 significant bits).  head + tail = x, and
// the tensor core's reading of the tail in TF32 loses at most 2^-21 |x|.
__device__ __forceinline__ float tf32_head(float x) { return __uint_as_float(__float_as_uint(x) & 0xFFFFE000u); }

// shared-memory matrix descriptor: K-major, no swizzle, LBO 128 bytes, SBO `sbo` bytes
__device__ __forceinline__ uint64_t umma_desc_sbo(uint32_t addr, uint32_t sbo) {
    uint64_t d = (uint64_t)((addr & 0x3FFFFu) >> 4);
    d |= (uint64_t)(128u >> 4) << 16;
    d |= (uint64_t)(sbo >> 4) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}
__device__ __forceinline__ uint64_t umma_desc(uint32_t addr) { return umma_desc_sbo(addr, 512u); }

// instruction descriptor of kind::tf32 with FP32 accumulation, both operands K-major
__host__ __device__ constexpr uint32_t umma_idesc_tf32(int M, int N) {
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// D[tmem] (+)= A[smem] B[smem]
__device__ __forceinline__ void umma_tf32(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                 "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
                 "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

// D[tmem] (+)= A[tmem] B[smem]: A's rows are tensor-memory lanes, its K values consecutive columns
__device__ __forceinline__ void umma_tf32_ts(uint32_t d_tmem, uint32_t a_tmem, uint64_t b, uint32_t idesc,
                                             uint32_t acc) {
    asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                 "tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n}\n" ::"r"(d_tmem),
                 "r"(a_tmem), "l"(b), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void umma_commit(uint32_t mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
                 : "memory");
}

__device__ __forceinline__ void mbar_init(uint32_t mbar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(mbar), "r"(count));
}

// bounded wait on the phase with the given parity; false if it did not complete within `polls` polls
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity, int polls = kUmmaSpin) {
    uint32_t done = 0;
    for (int it = 0; it < polls && !done; it++)
        asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
                     "selp.u32 %0, 1, 0, p;\n}\n"
                     : "=r"(done) : "r"(mbar), "r"(parity) : "memory");
    return done != 0;
}

__device__ __forceinline__ void tmem_alloc(uint32_t slot, uint32_t cols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(slot), "r"(cols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t cols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(cols));
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// mbarrier arrive (release, CTA scope) with a count
__device__ __forceinline__ void mbar_arrive(uint32_t mbar, uint32_t count = 1) {
    asm volatile("mbarrier.arrive.release.cta.shared::cta.b64 _, [%0], %1;" ::"r"(mbar), "r"(count) : "memory");
}

// bounded wait that also gives up once *abort is set (by another role of the block);
// the waiting thread sleeps in try_wait (suspend hint 20 us) instead of spinning; at most
// 2^14 polls (about 0.3 s)
__device__ __forceinline__ bool mbar_wait_abortable(uint32_t mbar, uint32_t parity, const volatile int* abort,
                                                    int polls = kUmmaSpin >> 8) {
    uint32_t done = 0;
    for (int it = 0; it < polls && !done; it++) {
        asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n"
                     "selp.u32 %0, 1, 0, p;\n}\n"
                     : "=r"(done) : "r"(mbar), "r"(parity), "r"(20000u) : "memory");
        if (!done && (it & 63) == 63 && *abort) return false;
    }
    return done != 0;
}

// named barrier `id` over `count` threads with an AND of the threads' predicates
__device__ __forceinline__ bool bar_and(int id, int count, bool pred) {
    uint32_t r;
    asm volatile("{\n.reg .pred p, q;\nsetp.ne.u32 p, %1, 0;\nbar.red.and.pred q, %2, %3, p;\nselp.u32 %0, 1, 0, q;\n}\n"
                 : "=r"(r) : "r"((uint32_t)pred), "r"(id), "r"(count) : "memory");
    return r != 0;
}
__device__ __forceinline__ void bar_sync(int id, int count) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}

// 4-byte asynchronous copy global -> shared; src_bytes 0 writes zero without reading
__device__ __forceinline__ void cp_async4(uint32_t dst, const void* src, uint32_t src_bytes) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(dst), "l"(src), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// 16 consecutive columns of this thread's lane (shape 32x32b: warp w reaches lanes 32 (w mod 4) ..)
#define ANOVA_TMEM_LD16(taddr, r)                                                                             \
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}," \
                 " [%16];"                                                                                    \
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),         \
                   "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),      \
                   "=r"(r[14]), "=r"(r[15])                                                                   \
                 : "r"(taddr))

// 8 consecutive columns of this thread's lane from registers
#define ANOVA_TMEM_ST8(taddr, v)                                                                     \
    asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"r"(taddr), \
                 "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]) \
                 : "memory")

// device address of the counter of abandoned waits on the current device
unsigned long long* wait_counter();

}  // namespace anova
