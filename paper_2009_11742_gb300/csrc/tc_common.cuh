// Blackwell (sm_100 family) tensor-core building blocks written as inline
// PTX: shared-memory matrix descriptors for 128-byte-swizzled K-major tiles,
// the tcgen05 instruction descriptor, TMEM allocation, MMA issue / commit,
// TMEM -> register loads, bulk global -> shared copies and mbarriers.
//
// Tile format used throughout ("SW128 K-major"): a tile of R rows whose K
// extent is exactly 128 bytes (32 tf32 or 64 bf16 values).  Rows are grouped
// in 8-row atoms of 1024 bytes; inside an atom row r sits at r * 128 bytes and
// its 16-byte chunk j is stored at chunk position j ^ r.  Tiles start on a
// 1024-byte boundary.  The bit layouts below follow the PTX ISA description
// of tcgen05 matrix and instruction descriptors.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace romk {

// Byte offset of element (row r, 16-byte chunk j) inside an SW128 K-major tile.
__host__ __device__ __forceinline__ uint32_t sw128_offset(uint32_t r, uint32_t j) {
    return (r >> 3) * 1024u + (r & 7u) * 128u + ((j ^ (r & 7u)) << 4);
}

// Shared-memory matrix descriptor (64 bit) of an SW128 K-major tile at byte
// address `saddr` (shared window): start address >> 4 in bits 0-13, leading
// byte offset (unused for swizzled K-major, encoded 1) in bits 16-29, stride
// byte offset (1024 B between 8-row atoms) >> 4 in bits 32-45, the constant
// 0b001 in bits 46-48, swizzle mode 2 (128 B) in bits 61-63.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)1u << 16;
    d |= (uint64_t)(1024u >> 4) << 32;
    d |= (uint64_t)1u << 46;
    d |= (uint64_t)2u << 61;
    return d;
}

// Instruction descriptor (32 bit) for dense kind::f16 / kind::tf32 MMA with
// FP32 accumulation, both operands K-major: D format F32 (bits 4-5 = 1),
// A / B formats in bits 7-9 / 10-12 (BF16 = 1, TF32 = 2), N >> 3 in bits
// 17-22, M >> 4 in bits 24-28.
__host__ __device__ constexpr uint32_t mma_idesc(uint32_t ab_format, uint32_t M, uint32_t N) {
    return (1u << 4) | (ab_format << 7) | (ab_format << 10) | ((N >> 3) << 17) | ((M >> 4) << 24);
}
constexpr uint32_t kFmtBF16 = 1u;
constexpr uint32_t kFmtTF32 = 2u;

__device__ __forceinline__ uint32_t cvta_shared(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

// ---- mbarrier
__device__ __forceinline__ void mbarrier_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(cvta_shared(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbarrier_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;"
                 ::"r"(cvta_shared(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbarrier_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(cvta_shared(bar)) : "memory");
}
__device__ __forceinline__ bool mbarrier_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok) : "r"(cvta_shared(bar)), "r"(parity) : "memory");
    return ok != 0;
}
// Non-blocking probe of a phase (never suspends the thread).
__device__ __forceinline__ bool mbarrier_test_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok) : "r"(cvta_shared(bar)), "r"(parity) : "memory");
    return ok != 0;
}
// Bounded spin on mbarrier_test_wait; same contract as mbarrier_wait below.
__device__ __forceinline__ bool mbarrier_spin(uint64_t* bar, uint32_t parity, long long limit,
                                              volatile int* abort) {
    if (mbarrier_test_wait(bar, parity)) return true;
    const long long t0 = clock64();
    while (!mbarrier_test_wait(bar, parity)) {
        if (*abort) return false;
        if (clock64() - t0 > limit) {
            *abort = 1;
            return false;
        }
    }
    return true;
}
// Bounded wait.  Returns false when `limit` clock cycles pass without the
// phase completing, or when *abort is raised by another thread.
__device__ __forceinline__ bool mbarrier_wait(uint64_t* bar, uint32_t parity, long long limit,
                                              volatile int* abort) {
    if (mbarrier_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    while (!mbarrier_try_wait(bar, parity)) {
        if (*abort) return false;
        if (clock64() - t0 > limit) {
            *abort = 1;
            return false;
        }
    }
    return true;
}

// ---- bulk asynchronous copy global -> shared (no tensor map); completes
// `bytes` of transaction count on `bar`.  Addresses 16-byte aligned, size a
// multiple of 16.
__device__ __forceinline__ void bulk_g2s(void* sdst, const void* gsrc, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
        ::"r"(cvta_shared(sdst)), "l"(gsrc), "r"(bytes), "r"(cvta_shared(bar))
        : "memory");
}

// Generic-proxy writes made visible to the async proxy (before bulk copies
// read global data written by threads, or MMAs read shared data written by
// threads).
__device__ __forceinline__ void fence_proxy_async_global() {
    asm volatile("fence.proxy.async.global;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async_shared() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// ---- tensor memory
__device__ __forceinline__ void tmem_alloc(uint32_t* smem_dst, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 ::"r"(cvta_shared(smem_dst)), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// D[tmem] (+)= A[smem] . B[smem]^T, one thread issues.
template <bool TF32>
__device__ __forceinline__ void mma_issue(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc,
                                          uint32_t idesc, uint32_t accumulate) {
    if (TF32) {
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "setp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}"
            ::"r"(d_tmem), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate) : "memory");
    } else {
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "setp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
            ::"r"(d_tmem), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate) : "memory");
    }
}
// Arrive once on `bar` when every MMA issued so far by this thread completed.
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                 ::"r"(cvta_shared(bar)) : "memory");
}

// 32 consecutive FP32 columns of this thread's TMEM lane (warp w reads lanes
// 32 (w % 4) .. + 31; `taddr` already carries that lane base).
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
          "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
          "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
          "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// ---- operand splitting
// x = hi + lo with hi = x rounded to the nearest TF32 value (ties to even)
// and lo = x - hi (exact in FP32) also rounded to TF32.  Both terms are
// exact TF32 numbers, so the tensor core sees them unchanged, and the
// representation error (about 2^-22 |x|) has no preferred sign.
__host__ __device__ __forceinline__ float round_tf32_rne(float x) {
#ifdef __CUDA_ARCH__
    uint32_t u = __float_as_uint(x);
    u = (u + 0x0FFFu + ((u >> 13) & 1u)) & 0xFFFFE000u;
    return __uint_as_float(u);
#else
    uint32_t u;
    __builtin_memcpy(&u, &x, 4);
    u = (u + 0x0FFFu + ((u >> 13) & 1u)) & 0xFFFFE000u;
    float y;
    __builtin_memcpy(&y, &u, 4);
    return y;
#endif
}
__host__ __device__ __forceinline__ void split_tf32_rn(float x, float& hi, float& lo) {
    hi = round_tf32_rne(x);
    lo = round_tf32_rne(x - hi);
}

}  // namespace romk
