// Helpers of the kernels on the 5th-generation tensor cores (tcgen05): shared-
// memory operand layout and matrix descriptors, the instruction descriptors of
// BF16 and TF32 products with FP32 accumulation, bounded mbarrier waits, the
// products and their commit, and tensor-memory loads.
//
// Operand image (K-major, 128-byte swizzle): a matrix of R rows and K
// columns is stored as K/64 blocks of R x 128 bytes; row r of a block holds
// its 64 elements as eight 16-byte chunks, chunk c at position c ^ (r mod 8);
// rows come in groups of 8 (1024 bytes).  Matrix descriptors: start address,
// stride 1024 bytes between 8-row groups, 128-byte swizzle; each K step of 16
// elements advances the start address by 32 bytes within a block.
#pragma once
#include <cstdint>

namespace klr {
namespace {

__host__ __device__ inline uint32_t swz_off(int r, int k, int rows) {
    const int kb = k >> 6, kk = k & 63;
    return (uint32_t)(kb * rows * 128 + (r >> 3) * 1024 + (r & 7) * 128 +
                      (((kk >> 3) ^ (r & 7)) << 4) + (kk & 7) * 2);
}

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr) {
    uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)1 << 16;                  // leading byte offset: unused with this layout
    d |= (uint64_t)(1024u >> 4) << 32;       // stride byte offset between 8-row groups
    d |= (uint64_t)1 << 46;                  // descriptor version
    d |= (uint64_t)2 << 61;                  // 128-byte swizzle
    return d;
}

// kind::f16 instruction descriptor: FP32 accumulator, BF16 A and B, both
// K-major, M x N
__host__ __device__ constexpr uint32_t umma_idesc_bf16(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) |
           ((uint32_t)(M >> 4) << 24);
}

// kind::tf32 instruction descriptor: FP32 accumulator, TF32 A and B, both
// K-major, M x N
__host__ __device__ constexpr uint32_t umma_idesc_tf32(int M, int N) {
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) |
           ((uint32_t)(M >> 4) << 24);
}

// byte offset of element (r, k) of a 4-byte (TF32) operand image: blocks of
// 32 elements (128 bytes) per row, the same 8-row groups and 16-byte chunk
// swizzle as the 2-byte image
__host__ __device__ inline uint32_t swz_off4(int r, int k, int rows) {
    const int kb = k >> 5, kk = k & 31;
    return (uint32_t)(kb * rows * 128 + (r >> 3) * 1024 + (r & 7) * 128 +
                      (((kk >> 2) ^ (r & 7)) << 4) + (kk & 3) * 4);
}

__device__ __forceinline__ bool mbar_wait(uint64_t* mbar, uint32_t parity) {
    // bounded: about a second of polling at most
    for (int it = 0; it < (1 << 22); ++it) {
        uint32_t ok;
        asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
                     "selp.u32 %0, 1, 0, p;\n}\n"
                     : "=r"(ok) : "r"(smem_addr(mbar)), "r"(parity) : "memory");
        if (ok) return true;
    }
    return false;
}

__device__ __forceinline__ void umma_bf16(uint32_t tmem, uint64_t ad, uint64_t bd, uint32_t idesc,
                                          uint32_t accumulate) {
    asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                 "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
                 :: "r"(tmem), "l"(ad), "l"(bd), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void umma_tf32(uint32_t tmem, uint64_t ad, uint64_t bd, uint32_t idesc,
                                          uint32_t accumulate) {
    asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                 "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n"
                 :: "r"(tmem), "l"(ad), "l"(bd), "r"(idesc), "r"(accumulate));
}

// two 16-column loads of this warp's 32 lanes (columns t0.., t1..) and one
// wait, in one statement so that no register is read early; the warp is
// reconverged first (the loads are .sync.aligned and may follow code that
// only some lanes ran)
__device__ __forceinline__ void tmem_ld16x2(uint32_t t0, uint32_t t1, float (&v)[32]) {
    uint32_t r[32];
    __syncwarp();
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%32];\n"
                 "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%33];\n"
                 "tcgen05.wait::ld.sync.aligned;\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                   "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
                   "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
                   "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
                   "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
                 : "r"(t0), "r"(t1)
                 : "memory");
#pragma unroll
    for (int j = 0; j < 32; ++j) v[j] = __uint_as_float(r[j]);
}

__device__ __forceinline__ bool mbar_try(uint64_t* mbar, uint32_t parity) {
    uint32_t ok;
    asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
                 "selp.u32 %0, 1, 0, p;\n}\n"
                 : "=r"(ok) : "r"(smem_addr(mbar)), "r"(parity) : "memory");
    return ok != 0;
}

__device__ __forceinline__ void umma_commit(uint64_t* mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                 :: "r"(smem_addr(mbar)) : "memory");
}

}  // namespace
}  // namespace klr
