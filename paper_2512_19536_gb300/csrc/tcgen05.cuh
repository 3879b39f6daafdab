// 5th-generation tensor-core helpers (tcgen05, sm_103a) shared by the kernels that run
// BF16/FP16 products with FP32 accumulation in tensor memory: operands in shared memory as
// 8-row x 16-byte core matrices without swizzle, M = 128, one issuing thread per CTA.
#pragma once

#include <cstdint>

#include "device.cuh"

namespace polydg {
namespace tc {

// Shared-memory matrix descriptor: start address, the byte distance of K-adjacent core
// matrices (lbo) and of adjacent 8-row groups (sbo), descriptor version 1, no swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);          // start address
    d |= (uint64_t)((lbo & 0x3FFFFu) >> 4) << 16;      // K-adjacent core matrices
    d |= (uint64_t)((sbo & 0x3FFFFu) >> 4) << 32;      // adjacent 8-row groups
    d |= (uint64_t)1 << 46;                             // descriptor version of tcgen05
    return d;                                           // base offset 0, no swizzle
}

// Instruction descriptor of tcgen05.mma kind::f16: D fp32, A and B of one type (BF16 when
// BF16 is true, else FP16), both K-major, M = 128, N = NB.
template <int NB, bool BF16>
__device__ __forceinline__ uint32_t instr_desc() {
    static_assert(NB % 16 == 0 && NB >= 16 && NB <= 256, "N of an M = 128 MMA");
    const uint32_t ab = BF16 ? ((1u << 7) | (1u << 10)) : 0u;
    return (1u << 4) | ab | ((uint32_t)(NB >> 3) << 17) | ((128u >> 4) << 24);
}

// D[tmem] (+)= A B^T for one K = 16 slice.
__device__ __forceinline__ void mma_f16(uint32_t tmem_d, uint64_t da, uint64_t db, uint32_t idesc,
                                        uint32_t accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
        ::"r"(tmem_d), "l"(da), "l"(db), "r"(idesc), "r"(accumulate) : "memory");
}

// One arrival on bar once every MMA this thread issued so far has completed.
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                 ::"r"(smem_addr(bar)) : "memory");
}

// NB fp32 columns of this thread's TMEM lane (32x32b shape: thread t of warp w reads lane
// 32 (w % 4) + t), starting at the column in taddr.
template <int NB>
__device__ __forceinline__ void tmem_load_row(uint32_t taddr, float* out) {
#pragma unroll
    for (int c0 = 0; c0 < NB; c0 += 16) {
        uint32_t r[16];
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
            : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
              "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
            : "r"(taddr + (uint32_t)c0) : "memory");
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
        for (int k = 0; k < 16; ++k) out[c0 + k] = __uint_as_float(r[k]);
    }
}

// Byte offset of element (row, k) of an operand stored as 8-row x 16-byte core matrices,
// K-adjacent core matrices 128 B apart and 8-row groups `sbo` bytes apart.
__device__ __forceinline__ uint32_t core_off(int row, int k, uint32_t sbo) {
    return (uint32_t)(row >> 3) * sbo + (uint32_t)(k >> 3) * 128u + (uint32_t)(row & 7) * 16u +
           (uint32_t)(k & 7) * 2u;
}

__device__ __forceinline__ void fence_after_sync() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_before_sync() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}

}  // namespace tc
}  // namespace polydg
