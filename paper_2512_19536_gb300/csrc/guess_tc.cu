// Learned PCG initial guess, inference on the 5th-generation tensor cores (tcgen05).
//
// The per-element network (features of the element and its face neighbours from the last
// three solutions, two ReLU hidden layers of kGuessHidden = 128, a linear output of n_p
// values o; x0 = U^k + s_d o) is three GEMMs over a tile of 128 elements:
//     H1 = relu(X W1^T + b1)   [128 x KF] x [KF x 128]     (KF = 9 n_p + 3 padded to 16)
//     H2 = relu(H1 W2^T + b2)  [128 x 128] x [128 x 128]
//     O  = H2 W3^T + b3        [128 x 128] x [128 x 16]    (n_p of the 16 columns used)
// with FP16 operands (the weights are stored in FP16; the features and activations are
// rounded to FP16 as they enter each product) and FP32 accumulation in tensor memory.
// One CTA of 512 threads per SM walks the tiles: the weights sit in shared memory for the
// whole launch as the B operands (8-row x 16-byte core matrices, K-major), the 16 warps
// form the tile's features into the A operand, thread 0 issues the MMAs of a layer and
// commits them to an mbarrier, and the warps read the accumulators back with tcgen05.ld
// (warp w: TMEM lanes 32 (w % 4) .., columns 32 (w / 4) ..), add the bias, apply ReLU and
// write the next layer's A operand.  Every wait is bounded: on a timeout the CTA raises
// *err, waits (bounded) once more for its MMAs, frees its tensor memory and leaves; the
// elements it did not reach keep their previous proposal, which the safeguard judges.
#include <algorithm>
#include <cstdint>

#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "device.cuh"
#include "guess_features.cuh"
#include "kernels.h"
#include "pcg_device.cuh"
#include "tcgen05.cuh"

namespace polydg {

namespace {

constexpr int kGtThreads = 512;               // 16 warps
constexpr int kGtTile = 128;                  // elements per tile: the MMA's M
constexpr int kGtH = kGuessHidden;            // 128
constexpr int kGtNO = 16;                     // output columns (n_p <= 16 used)
constexpr uint32_t kGtTmemCols = 256;         // D1 at columns 0.., D2 at 128.., O at 0..

// Shared-memory layout for n_p: byte offsets of the operands (all multiples of 128).
template <int NP>
struct GtLayout {
    static constexpr int F = guess_inputs(NP);
    static constexpr int KF = (F + 15) / 16 * 16;
    static constexpr uint32_t sbo1 = (uint32_t)(KF / 8) * 128u;     // 8-row groups of X, W1
    static constexpr uint32_t sboh = (uint32_t)(kGtH / 8) * 128u;   // of H1/H2, W2, W3
    static constexpr uint32_t w1 = 0;
    static constexpr uint32_t w2 = w1 + (uint32_t)kGtH * KF * 2;
    static constexpr uint32_t w3 = w2 + (uint32_t)kGtH * kGtH * 2;
    static constexpr uint32_t a1 = w3 + (uint32_t)kGtNO * kGtH * 2;
    static constexpr uint32_t a2 = a1 + (uint32_t)kGtTile * KF * 2;
    static constexpr uint32_t bias = a2 + (uint32_t)kGtTile * kGtH * 2;
    static constexpr uint32_t feat = bias + (uint32_t)(2 * kGtH + kGtNO) * 4;
    static constexpr uint32_t bytes = feat + (uint32_t)(kGtThreads / 32) * KF * 4;
};

// The parameter groups in the flat (canonical) layout: W1 [128][F], b1, W2 [128][128], b2,
// W3 [n_p][128], b3.
struct GtOffsets {
    int w1, b1, w2, b2, w3, b3;
};
__device__ __forceinline__ GtOffsets gt_offsets(int np) {
    const int F = guess_inputs(np);
    GtOffsets o;
    o.w1 = 0;
    o.b1 = o.w1 + kGtH * F;
    o.w2 = o.b1 + kGtH;
    o.b2 = o.w2 + kGtH * kGtH;
    o.w3 = o.b2 + kGtH;
    o.b3 = o.w3 + np * kGtH;
    return o;
}

template <int NP>
__global__ void __launch_bounds__(kGtThreads, 1)
guess_propose_tc_kernel(GuessFeat f, const __half* __restrict__ w16, const double* __restrict__ Uk,
                        const double* __restrict__ Uk1, const double* __restrict__ Uk2,
                        double* __restrict__ xg, int64_t nc, const SimScalars* ss, int* err) {
    using L = GtLayout<NP>;
    constexpr int F = L::F, KF = L::KF;
    if (ss && (ss->failed || ss->k < 2)) return;
    extern __shared__ __align__(1024) unsigned char gsm[];
    __shared__ __align__(8) uint64_t bar;
    __shared__ uint32_t tmem_slot;
    __shared__ int fail_sh;
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    unsigned char* w1 = gsm + L::w1;
    unsigned char* w2 = gsm + L::w2;
    unsigned char* w3 = gsm + L::w3;
    unsigned char* a1 = gsm + L::a1;
    unsigned char* a2 = gsm + L::a2;
    float* b1 = reinterpret_cast<float*>(gsm + L::bias);
    float* b2 = b1 + kGtH;
    float* b3 = b2 + kGtH;
    float* xw = reinterpret_cast<float*>(gsm + L::feat) + warp * KF;   // this warp's feature row

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     ::"r"(smem_addr(&tmem_slot)), "r"(kGtTmemCols) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
        tc::fence_before_sync();
    }
    if (t == 0) {
        mbar_init(&bar);
        fail_sh = 0;
    }
    // the weights as B operands (rows = output units, K-major), zero-padded
    const GtOffsets o = gt_offsets(NP);
    auto put = [](unsigned char* base, int row, int k, uint32_t sbo, float v) {
        *reinterpret_cast<__half*>(base + tc::core_off(row, k, sbo)) = __float2half_rn(v);
    };
    for (int q = t; q < kGtH * KF; q += kGtThreads) {
        const int j = q / KF, i = q - j * KF;
        put(w1, j, i, L::sbo1, i < F ? __half2float(w16[o.w1 + j * F + i]) : 0.f);
    }
    for (int q = t; q < kGtH * kGtH; q += kGtThreads) {
        const int j = q / kGtH, i = q - j * kGtH;
        put(w2, j, i, L::sboh, __half2float(w16[o.w2 + q]));
    }
    for (int q = t; q < kGtNO * kGtH; q += kGtThreads) {
        const int c = q / kGtH, i = q - c * kGtH;
        put(w3, c, i, L::sboh, c < NP ? __half2float(w16[o.w3 + c * kGtH + i]) : 0.f);
    }
    for (int q = t; q < kGtH; q += kGtThreads) {
        b1[q] = __half2float(w16[o.b1 + q]);
        b2[q] = __half2float(w16[o.b2 + q]);
    }
    if (t < kGtNO) b3[t] = t < NP ? __half2float(w16[o.b3 + t]) : 0.f;
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = tmem_slot;
    const int q4 = warp & 3, g = warp >> 2;            // TMEM lane quarter, column group
    const uint32_t lane_base = (uint32_t)(32 * q4) << 16;
    uint32_t phase = 0, commits = 0;
    bool ok = true;

    // thread 0: the MMAs of one layer, then one commit; every thread waits for it (lanes
    // 1..31 of warp 0 first wait for lane 0 at __syncwarp, not beside it on the mbarrier)
    auto layer = [&](uint32_t d_col, const unsigned char* A, const unsigned char* B, uint32_t sbo, int ksteps,
                     uint32_t idesc) {
        if (t == 0) {
            for (int kk = 0; kk < ksteps; ++kk)
                tc::mma_f16(tmem + d_col, tc::smem_desc(smem_addr(A) + kk * 256u, 128u, sbo),
                            tc::smem_desc(smem_addr(B) + kk * 256u, 128u, sbo), idesc, kk > 0 ? 1u : 0u);
            tc::mma_commit(&bar);
        }
        ++commits;
        __syncwarp();
        if (!mbar_wait(&bar, phase & 1)) fail_sh = 1;
        ++phase;
        tc::fence_after_sync();
        __syncthreads();
        ok = fail_sh == 0;
    };
    // the accumulator columns [col, col + 32) of this thread's row, bias, ReLU, FP16 into A
    auto hidden_epilogue = [&](uint32_t d_col, const float* bias, unsigned char* A) {
        float d[32];
        tc::tmem_load_row<32>(tmem + lane_base + d_col + 32u * g, d);
        const int r = 32 * q4 + lane;
#pragma unroll
        for (int c = 0; c < 32; ++c)
            put(A, r, 32 * g + c, L::sboh, fmaxf(d[c] + bias[32 * g + c], 0.f));
        tc::fence_before_sync();
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        tc::fence_after_sync();
    };

    const int64_t ntiles = (nc + kGtTile - 1) / kGtTile;
    for (int64_t tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
        const int64_t t0 = tile * kGtTile;
        const int n = (int)min((int64_t)kGtTile, nc - t0);
        // features of the tile's elements, warp by warp, into X (FP16, rows >= n zero)
        for (int sm = warp; sm < kGtTile; sm += kGtThreads / 32) {
            if (sm < n) element_features<NP>(f, Uk, Uk1, Uk2, t0 + sm, xw, [](int64_t e) { return e * NP; });
            __syncwarp();
            for (int k = lane; k < KF; k += 32) put(a1, sm, k, L::sbo1, (sm < n && k < F) ? xw[k] : 0.f);
            __syncwarp();
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        tc::fence_after_sync();
        layer(0u, a1, w1, L::sbo1, KF / 16, tc::instr_desc<kGtH, false>());
        if (!ok) break;
        hidden_epilogue(0u, b1, a2);
        layer((uint32_t)kGtH, a2, w2, L::sboh, kGtH / 16, tc::instr_desc<kGtH, false>());
        if (!ok) break;
        hidden_epilogue((uint32_t)kGtH, b2, a2);
        layer(0u, a2, w3, L::sboh, kGtH / 16, tc::instr_desc<kGtNO, false>());
        if (!ok) break;
        if (g == 0) {                             // O: rows of the four lane quarters
            float d[kGtNO];
            tc::tmem_load_row<kGtNO>(tmem + lane_base, d);
            const int r = 32 * q4 + lane;
            if (r < n) {
                const int64_t e = t0 + r;
#pragma unroll
                for (int c = 0; c < NP; ++c)
                    xg[e * NP + c] = Uk[e * NP + c] + f.s_d * (double)(d[c] + b3[c]);
            }
        }
        tc::fence_before_sync();
        __syncthreads();                          // O read before the next tile's layer 1
        tc::fence_after_sync();
    }
    if (!ok && t == 0) {
        atomicExch(err, 1);
        if (commits > 0) mbar_wait(&bar, (commits - 1) & 1);   // bounded: the last commit again
    }
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kGtTmemCols)
                     : "memory");
}

}  // namespace

size_t guess_propose_tc_smem(int np) {
    switch (np) {
        case 3: return GtLayout<3>::bytes;
        case 6: return GtLayout<6>::bytes;
        case 10: return GtLayout<10>::bytes;
        default: return 0;
    }
}

cudaError_t guess_propose_tc_prepare(int np) {
    const void* fn = nullptr;
    switch (np) {
        case 3: fn = (const void*)guess_propose_tc_kernel<3>; break;
        case 6: fn = (const void*)guess_propose_tc_kernel<6>; break;
        case 10: fn = (const void*)guess_propose_tc_kernel<10>; break;
        default: return cudaErrorInvalidValue;
    }
    return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)guess_propose_tc_smem(np));
}

cudaError_t launch_guess_propose(int np, const GuessFeat& f, const __half* w16, const double* Uk,
                                 const double* Uk1, const double* Uk2, double* xg, int64_t nc,
                                 const SimScalars* ss, int* err, int n_sm, cudaStream_t s) {
    const int64_t ntiles = (nc + kGtTile - 1) / kGtTile;
    const unsigned grid = (unsigned)std::min<int64_t>(ntiles, n_sm);
    if (grid == 0) return cudaSuccess;
    const size_t smem = guess_propose_tc_smem(np);
    switch (np) {
        case 3: guess_propose_tc_kernel<3><<<grid, kGtThreads, smem, s>>>(f, w16, Uk, Uk1, Uk2, xg, nc, ss, err); break;
        case 6: guess_propose_tc_kernel<6><<<grid, kGtThreads, smem, s>>>(f, w16, Uk, Uk1, Uk2, xg, nc, ss, err); break;
        case 10: guess_propose_tc_kernel<10><<<grid, kGtThreads, smem, s>>>(f, w16, Uk, Uk1, Uk2, xg, nc, ss, err); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace polydg
