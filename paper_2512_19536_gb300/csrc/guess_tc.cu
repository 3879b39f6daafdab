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
//
// Three kernels:
//   * guess_tc_image_kernel lays the weights out once per weight update as the B operands
//     (8-row x 16-byte core matrices, K-major, zero-padded) followed by the FP32 biases:
//     one contiguous image that a CTA copies into shared memory with one bulk copy;
//   * guess_features_tc_kernel forms every element's features (warp per element, the
//     whole GPU busy) straight into FP16 A-operand tiles in global memory;
//   * guess_propose_tc_kernel: one 512-thread CTA per SM walks the tiles, bulk-copying the
//     next tile's features while the current one runs; thread 0 issues a layer's MMAs and
//     commits them to an mbarrier, the warps read the accumulators back with tcgen05.ld
//     (warp w: TMEM lanes 32 (w % 4).., columns 32 (w / 4)..), add the bias, apply ReLU and
//     write the next layer's A operand; the output columns give x0.
// Every wait is bounded: on a timeout the CTA raises *err, waits (bounded) once more for
// its copies and MMAs, frees its tensor memory and leaves; the elements it did not reach
// keep their previous proposal, which the safeguard judges.
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
constexpr int kGfThreads = 256;               // features kernel: warp per element

// Byte layout for n_p.  The weight image (global and shared): W1 | W2 | W3 core matrices,
// then the FP32 biases b1 | b2 | b3 (b3 padded to 16).  Shared memory adds two feature
// tiles (double buffer) and the hidden-layer tile.
template <int NP>
struct GtLayout {
    static constexpr int F = guess_inputs(NP);
    static constexpr int KF = (F + 15) / 16 * 16;
    static constexpr uint32_t sbo1 = (uint32_t)(KF / 8) * 128u;     // 8-row groups of X, W1
    static constexpr uint32_t sboh = (uint32_t)(kGtH / 8) * 128u;   // of H1/H2, W2, W3
    static constexpr uint32_t w1 = 0;
    static constexpr uint32_t w2 = w1 + (uint32_t)kGtH * KF * 2;
    static constexpr uint32_t w3 = w2 + (uint32_t)kGtH * kGtH * 2;
    static constexpr uint32_t bias = w3 + (uint32_t)kGtNO * kGtH * 2;
    static constexpr uint32_t image = bias + (uint32_t)(2 * kGtH + kGtNO) * 4;   // a multiple of 16
    static constexpr uint32_t tile = (uint32_t)kGtTile * KF * 2;                 // one feature tile
    static constexpr uint32_t a1 = (image + 127u) / 128u * 128u;
    static constexpr uint32_t a2 = a1 + 2 * tile;
    static constexpr uint32_t bytes = a2 + (uint32_t)kGtTile * kGtH * 2;
};

// The parameter groups in the flat (canonical) layout: W1 [128][F], b1, W2 [128][128], b2,
// W3 [n_p][128], b3.
struct GtOffsets {
    int w1, b1, w2, b2, w3, b3;
};
__host__ __device__ inline GtOffsets gt_offsets(int np) {
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

__device__ __forceinline__ void put_half(unsigned char* base, int row, int k, uint32_t sbo, float v) {
    *reinterpret_cast<__half*>(base + tc::core_off(row, k, sbo)) = __float2half_rn(v);
}

template <int NP>
__global__ void guess_tc_image_kernel(const __half* __restrict__ w16, unsigned char* __restrict__ img) {
    using L = GtLayout<NP>;
    constexpr int F = L::F, KF = L::KF;
    const GtOffsets o = gt_offsets(NP);
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    constexpr int n1 = kGtH * KF, n2 = kGtH * kGtH, n3 = kGtNO * kGtH, nb = 2 * kGtH + kGtNO;
    if (q < n1) {
        const int j = q / KF, i = q - j * KF;
        put_half(img + L::w1, j, i, L::sbo1, i < F ? __half2float(w16[o.w1 + j * F + i]) : 0.f);
    } else if (q < n1 + n2) {
        const int r = q - n1, j = r / kGtH, i = r - j * kGtH;
        put_half(img + L::w2, j, i, L::sboh, __half2float(w16[o.w2 + r]));
    } else if (q < n1 + n2 + n3) {
        const int r = q - n1 - n2, c = r / kGtH, i = r - c * kGtH;
        put_half(img + L::w3, c, i, L::sboh, c < NP ? __half2float(w16[o.w3 + c * kGtH + i]) : 0.f);
    } else if (q < n1 + n2 + n3 + nb) {
        const int r = q - n1 - n2 - n3;
        float v = 0.f;
        if (r < kGtH) v = __half2float(w16[o.b1 + r]);
        else if (r < 2 * kGtH) v = __half2float(w16[o.b2 + r - kGtH]);
        else if (r - 2 * kGtH < NP) v = __half2float(w16[o.b3 + r - 2 * kGtH]);
        reinterpret_cast<float*>(img + L::bias)[r] = v;
    }
}

// Features of element e (rows e >= nc of the last tile zero) into tile e / 128, row e % 128.
template <int NP>
__global__ void __launch_bounds__(kGfThreads)
guess_features_tc_kernel(GuessFeat f, const double* __restrict__ Uk, const double* __restrict__ Uk1,
                         const double* __restrict__ Uk2, unsigned char* __restrict__ xt, int64_t nc,
                         int64_t nrows, const SimScalars* ss) {
    using L = GtLayout<NP>;
    constexpr int F = L::F, KF = L::KF;
    if (ss && (ss->failed || ss->k < 2)) return;
    __shared__ float xs[kGfThreads / 32][KF];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t e = ((int64_t)blockIdx.x * kGfThreads + threadIdx.x) >> 5;
    if (e >= nrows) return;
    float* x = xs[warp];
    if (e < nc) element_features<NP>(f, Uk, Uk1, Uk2, e, x, [](int64_t c) { return c * NP; });
    __syncwarp();
    unsigned char* tile = xt + (size_t)(e / kGtTile) * L::tile;
    const int r = (int)(e % kGtTile);
    for (int k = lane; k < KF; k += 32) put_half(tile, r, k, L::sbo1, (e < nc && k < F) ? x[k] : 0.f);
}

template <int NP>
__global__ void __launch_bounds__(kGtThreads, 1)
guess_propose_tc_kernel(const unsigned char* __restrict__ img, const unsigned char* __restrict__ xt,
                        const double* __restrict__ Uk, double s_d, double* __restrict__ xg, int64_t nc,
                        const SimScalars* ss, int* err) {
    using L = GtLayout<NP>;
    constexpr int KF = L::KF;
    if (ss && (ss->failed || ss->k < 2)) return;
    extern __shared__ __align__(1024) unsigned char gsm[];
    __shared__ __align__(8) uint64_t wbar, xbar[2], mbar;
    __shared__ uint32_t tmem_slot;
    __shared__ int fail_sh;
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    const float* b1 = reinterpret_cast<const float*>(gsm + L::bias);
    const float* b2 = b1 + kGtH;
    const float* b3 = b2 + kGtH;
    unsigned char* a2 = gsm + L::a2;
    const int64_t ntiles = (nc + kGtTile - 1) / kGtTile;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     ::"r"(smem_addr(&tmem_slot)), "r"(kGtTmemCols) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
        tc::fence_before_sync();
    }
    uint32_t x_issued = 0;                        // thread 0: feature tiles copied so far
    if (t == 0) {
        mbar_init(&wbar);
        mbar_init(&xbar[0]);
        mbar_init(&xbar[1]);
        mbar_init(&mbar);
        fail_sh = 0;
        const uint64_t pol = evict_first_policy();
        bulk_load(gsm, img, L::image, &wbar, pol);                    // the weights, once
        if ((int64_t)blockIdx.x < ntiles) {
            bulk_load(gsm + L::a1, xt + (size_t)blockIdx.x * L::tile, L::tile, &xbar[0], pol);
            x_issued = 1;
        }
    }
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = tmem_slot;
    const int q4 = warp & 3, g = warp >> 2;            // TMEM lane quarter, column group
    const uint32_t lane_base = (uint32_t)(32 * q4) << 16;
    uint32_t mphase = 0, x_done = 0, commits = 0;
    bool w_ok = true, ok = true;
    if (!mbar_wait(&wbar, 0)) fail_sh = 1;

    // thread 0: the MMAs of one layer, then one commit; every thread waits for it (lanes
    // 1..31 of warp 0 first wait for lane 0 at __syncwarp, not beside it on the mbarrier)
    auto layer = [&](uint32_t d_col, const unsigned char* A, const unsigned char* B, uint32_t sbo, int ksteps,
                     uint32_t idesc) {
        if (t == 0) {
            for (int kk = 0; kk < ksteps; ++kk)
                tc::mma_f16(tmem + d_col, tc::smem_desc(smem_addr(A) + kk * 256u, 128u, sbo),
                            tc::smem_desc(smem_addr(B) + kk * 256u, 128u, sbo), idesc, kk > 0 ? 1u : 0u);
            tc::mma_commit(&mbar);
        }
        ++commits;
        __syncwarp();
        if (!mbar_wait(&mbar, mphase & 1)) fail_sh = 1;
        ++mphase;
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
        for (int c = 0; c < 32; ++c) put_half(A, r, 32 * g + c, L::sboh, fmaxf(d[c] + bias[32 * g + c], 0.f));
        tc::fence_before_sync();
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        tc::fence_after_sync();
    };

    __syncthreads();
    ok = w_ok = fail_sh == 0;
    int it = 0;
    for (int64_t tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x, ++it) {
        const int b = it & 1;
        const unsigned char* a1 = gsm + L::a1 + b * L::tile;
        // the next tile's features into the other buffer (its last reader, layer 1 of the
        // previous tile, has completed)
        const int64_t next = tile + gridDim.x;
        if (t == 0 && next < ntiles) {
            bulk_load(gsm + L::a1 + (b ^ 1) * L::tile, xt + (size_t)next * L::tile, L::tile, &xbar[b ^ 1],
                      evict_first_policy());
            ++x_issued;
        }
        if (!mbar_wait(&xbar[b], (it >> 1) & 1)) fail_sh = 1;
        else ++x_done;
        __syncthreads();
        if (fail_sh != 0) { ok = false; break; }
        tc::fence_after_sync();
        const int n = (int)min((int64_t)kGtTile, nc - tile * kGtTile);
        layer(0u, a1, gsm + L::w1, L::sbo1, KF / 16, tc::instr_desc<kGtH, false>());
        if (!ok) break;
        hidden_epilogue(0u, b1, a2);
        layer((uint32_t)kGtH, a2, gsm + L::w2, L::sboh, kGtH / 16, tc::instr_desc<kGtH, false>());
        if (!ok) break;
        hidden_epilogue((uint32_t)kGtH, b2, a2);
        layer(0u, a2, gsm + L::w3, L::sboh, kGtH / 16, tc::instr_desc<kGtNO, false>());
        if (!ok) break;
        if (g == 0) {                             // O: rows of the four lane quarters
            float d[kGtNO];
            tc::tmem_load_row<kGtNO>(tmem + lane_base, d);
            const int r = 32 * q4 + lane;
            if (r < n) {
                const int64_t e = tile * kGtTile + r;
#pragma unroll
                for (int c = 0; c < NP; ++c) xg[e * NP + c] = Uk[e * NP + c] + s_d * (double)(d[c] + b3[c]);
            }
        }
        tc::fence_before_sync();
        __syncthreads();                          // O read before the next tile's layer 1
        tc::fence_after_sync();
    }
    if (!ok && t == 0) {
        atomicExch(err, 1);
        // bounded waits: the weights, the feature copies in flight, the last MMA commit
        if (!w_ok) mbar_wait(&wbar, 0);
        for (uint32_t c = x_done; c < x_issued; ++c) mbar_wait(&xbar[c & 1], (c >> 1) & 1);
        if (commits > 0) mbar_wait(&mbar, (commits - 1) & 1);
    }
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kGtTmemCols)
                     : "memory");
}

template <int NP>
const void* propose_fn() { return (const void*)guess_propose_tc_kernel<NP>; }

}  // namespace

size_t guess_tc_image_bytes(int np) {
    switch (np) {
        case 3: return GtLayout<3>::image;
        case 6: return GtLayout<6>::image;
        case 10: return GtLayout<10>::image;
        default: return 0;
    }
}

size_t guess_tc_tile_bytes(int np) {
    switch (np) {
        case 3: return GtLayout<3>::tile;
        case 6: return GtLayout<6>::tile;
        case 10: return GtLayout<10>::tile;
        default: return 0;
    }
}

cudaError_t guess_propose_tc_prepare(int np) {
    switch (np) {
        case 3: return cudaFuncSetAttribute(propose_fn<3>(), cudaFuncAttributeMaxDynamicSharedMemorySize, (int)GtLayout<3>::bytes);
        case 6: return cudaFuncSetAttribute(propose_fn<6>(), cudaFuncAttributeMaxDynamicSharedMemorySize, (int)GtLayout<6>::bytes);
        case 10: return cudaFuncSetAttribute(propose_fn<10>(), cudaFuncAttributeMaxDynamicSharedMemorySize, (int)GtLayout<10>::bytes);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_guess_tc_image(int np, const __half* w16, unsigned char* img, cudaStream_t s) {
    const int n = kGtH * 160 + kGtH * kGtH + kGtNO * kGtH + 2 * kGtH + kGtNO;   // >= every n_p's entries
    const unsigned grid = (unsigned)((n + 255) / 256);
    switch (np) {
        case 3: guess_tc_image_kernel<3><<<grid, 256, 0, s>>>(w16, img); break;
        case 6: guess_tc_image_kernel<6><<<grid, 256, 0, s>>>(w16, img); break;
        case 10: guess_tc_image_kernel<10><<<grid, 256, 0, s>>>(w16, img); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_guess_propose(int np, const GuessFeat& f, const unsigned char* img, const double* Uk,
                                 const double* Uk1, const double* Uk2, double* xg, int64_t nc,
                                 const SimScalars* ss, unsigned char* xt, int* err, int n_sm, cudaStream_t s) {
    const int64_t ntiles = (nc + kGtTile - 1) / kGtTile;
    if (ntiles == 0) return cudaSuccess;
    const int64_t nrows = ntiles * kGtTile;
    const unsigned fgrid = (unsigned)((nrows * 32 + kGfThreads - 1) / kGfThreads);
    const unsigned grid = (unsigned)std::min<int64_t>(ntiles, n_sm);
    switch (np) {
        case 3:
            guess_features_tc_kernel<3><<<fgrid, kGfThreads, 0, s>>>(f, Uk, Uk1, Uk2, xt, nc, nrows, ss);
            guess_propose_tc_kernel<3><<<grid, kGtThreads, GtLayout<3>::bytes, s>>>(img, xt, Uk, f.s_d, xg, nc, ss, err);
            break;
        case 6:
            guess_features_tc_kernel<6><<<fgrid, kGfThreads, 0, s>>>(f, Uk, Uk1, Uk2, xt, nc, nrows, ss);
            guess_propose_tc_kernel<6><<<grid, kGtThreads, GtLayout<6>::bytes, s>>>(img, xt, Uk, f.s_d, xg, nc, ss, err);
            break;
        case 10:
            guess_features_tc_kernel<10><<<fgrid, kGfThreads, 0, s>>>(f, Uk, Uk1, Uk2, xt, nc, nrows, ss);
            guess_propose_tc_kernel<10><<<grid, kGtThreads, GtLayout<10>::bytes, s>>>(img, xt, Uk, f.s_d, xg, nc, ss, err);
            break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace polydg
