// Building blocks of the tcgen05 kernels (tensor-core M2L of composed
// matrices, trans_tc.cu; staged RCR rotations, rcr_staged_tc.cu): operands
// in shared memory in the canonical no-swizzle K-major layout, 3xTF32 split,
// bounded mbarrier waits, MMA issue and accumulator reads.
//
// Canonical layout of a K-major operand block of KC = 16 real K values:
// 8 x 16-byte core matrices (8 rows x 4 K values), K-adjacent core matrices
// LBO = 128 bytes apart, 8-row groups SBO = 512 bytes apart; an MMA of K = 8
// reads two K-adjacent core matrices, the next one starts 2 LBO further.
#pragma once

#include <cstdint>

namespace tcx {

constexpr int KC = 16;                  // real K per pipeline stage (two MMAs of K = 8)
constexpr int SBO = (KC / 4) * 128;     // bytes between 8-row groups
constexpr int LBO = 128;                // bytes between K-adjacent core matrices
// Bound of the drain waits (copies and MMAs a CTA has issued always
// complete; the bound only keeps a broken device from hanging the kernel).
constexpr long long DRAIN_LIMIT = 1LL << 26;

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor of a canonical no-swizzle K-major block
__device__ __forceinline__ uint64_t umma_desc(uint32_t addr) {
    uint64_t d = 0;
    d |= (uint64_t)((addr & 0x3FFFF) >> 4);
    d |= (uint64_t)((LBO >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)((SBO >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;   // descriptor version of sm_100-family tcgen05
    return d;                  // base offset 0, no swizzle
}

// byte offset of element (row, k) of a canonical block (k < KC)
__host__ __device__ __forceinline__ int canon(int row, int k) {
    return (row >> 3) * SBO + (k >> 2) * LBO + (row & 7) * 16 + (k & 3) * 4;
}

// instruction descriptor of kind::tf32, FP32 accumulation, both operands K-major
__host__ __device__ __forceinline__ uint32_t idesc_tf32(int M, int N) {
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// the TF32 part of an FP32 value (low 13 mantissa bits cleared); the
// remainder v - tf32_hi(v) is exact in FP32
__device__ __forceinline__ float tf32_hi(float v) { return __uint_as_float(__float_as_uint(v) & 0xFFFFE000u); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, int count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

// Polls a phase of an mbarrier at most `limit` times; false when it did not
// complete.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, long long limit) {
    for (long long it = 0; it < limit; ++it) {
        uint32_t ok;
        asm volatile(
            "{\n\t.reg .pred P1;\n\tmbarrier.try_wait.parity.shared::cta.b64 P1, [%1], %2;\n\t"
            "selp.b32 %0, 1, 0, P1;\n\t}\n"
            : "=r"(ok)
            : "r"(bar), "r"(parity));
        if (ok) return true;
    }
    return false;
}

// D[tmem] (+)= A B^T, M x N x 8, both operands TF32 in shared memory
__device__ __forceinline__ void mma_tf32(uint32_t tmem, uint64_t da, uint64_t db, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem),
        "l"(da), "l"(db), "r"(idesc), "r"(acc));
}

// arrives on `bar` once every MMA this thread has issued so far is complete
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar)));
}

// 16 consecutive accumulator columns of this thread's lane
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&v)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
          "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;");
}

}  // namespace tcx
