// Local solves shared by up to 16 simulations of one mesh, on the 5th-generation tensor
// cores (tcgen05): the two passes over the eigenbasis of every subdomain,
//     Y = diag(1/(chi + c_s lam)) Q_i^T X,   V = Q_i Y,   X = L_i^{-1} r_s, z_s = L_i^{-T} V,
// are [n_i x n_i] x [n_i x 2R] BF16 products with FP32 accumulation (Sec. 4, Eq. prec:
// K_i(sigma)^{-1} = L_i^{-T} Q_i diag(1/(chi_cm + c lam_i)) Q_i^T L_i^{-1}, c = dt sigma/2).
//
// The right-hand sides enter as two BF16 parts each, hi = bf16(x) and lo = bf16(x - hi),
// so the inputs keep ~16 bits and the result's error is that of the BF16 eigenbasis
// alone.  One CTA of 512 threads per subdomain:
//   * thread 0 streams the 128 x 64 tiles of Q_i^T, then of Q_i (16 KB each, stored
//     pre-tiled in the core-matrix layout the MMA reads: 8-row x 16-byte core matrices,
//     K-adjacent ones 128 B apart, 8-row groups 1024 B apart) through a ring of shared-memory
//     stages with cp.async.bulk (mbarrier completion), and issues tcgen05.mma (M = 128,
//     N = 16 or 32, K = 16; four per tile) into one TMEM accumulator per 128-row tile;
//     each stage's commit frees it for the next copy;
//   * the 16 warps read the accumulators back with tcgen05.ld (warp w reads TMEM lanes
//     32 (w % 4)..32 (w % 4) + 31 of the tiles mt = w / 4, w / 4 + 4, ...), form Y (pass 1) or
//     V (pass 2) and write the next B operand;
//   * the FP64 work around the GEMMs (X = L^{-1} r, z = L^{-T} V, element by element with
//     the element's block of L^{-1} read once per right-hand side) is spread over the CTA,
//     while the first tiles are already streaming in.
// Every wait is bounded; on a timeout the CTA raises *err, waits (bounded) for its copies
// and MMAs in flight, frees its TMEM and leaves.
#include <cstdint>

#include <cuda_runtime.h>
#include <cuda_bf16.h>

#include "device.cuh"
#include "kernels.h"
#include "pcg_device.cuh"
#include "tcgen05.cuh"

namespace polydg {

namespace {

constexpr int kTcThreads = 512;                // 16 warps: warp w reads TMEM lanes 32 (w % 4)..
constexpr int kTcStages = 6;                   // ring of 16 KB A tiles
constexpr int kTcLag = 2;                      // a stage is refilled kTcLag tiles after its MMAs
constexpr uint32_t kTileBytes = 128 * 64 * 2;  // one 128 x 64 BF16 tile

using tc::smem_desc;
using tc::mma_commit;
using tc::tmem_load_row;
using tc::core_off;

// Instruction descriptor of the BF16 passes: D fp32, A and B bf16, M = 128, N = NB.
template <int NB>
__device__ __forceinline__ uint32_t instr_desc() { return tc::instr_desc<NB, true>(); }

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t da, uint64_t db, uint32_t idesc,
                                         uint32_t accumulate) {
    tc::mma_f16(tmem_d, da, db, idesc, accumulate);
}

}  // namespace

template <int NB, int NP>
__global__ void __launch_bounds__(kTcThreads, 1)
shared_tc_kernel(const TcBlock* __restrict__ blocks, const unsigned char* __restrict__ tiles,
                 const float* __restrict__ lam, const double* __restrict__ linv, double chi,
                 TcRhs p, int* err) {
    constexpr int np = NP;
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ __align__(8) uint64_t full[kTcStages], empty[kTcStages], done;
    __shared__ uint32_t tmem_slot;
    __shared__ int fail_sh;
    const TcBlock B = blocks[blockIdx.x];
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    const int R = p.nrhs, n = B.n, MT = B.mt, KT = B.kt;
    const int kpad = KT * 64, npad = MT * 128;
    const uint32_t bsbo = (uint32_t)(kpad / 8) * 128u;      // B operand: 8-row groups apart
    unsigned char* ring = smem;                              // kTcStages x 16 KB
    unsigned char* bop = smem + kTcStages * kTileBytes;      // NB x kpad bf16, core matrices
    float* vst = reinterpret_cast<float*>(smem);             // V staging (reuses the ring)
    int cols = 32;                                           // TMEM columns: a power of 2
    while (cols < MT * NB) cols *= 2;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     ::"r"(smem_addr(&tmem_slot)), "r"(cols) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    }
    if (t == 0) {
        for (int s = 0; s < kTcStages; ++s) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&full[s])) : "memory");
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&empty[s])) : "memory");
        }
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&done)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        fail_sh = 0;
    }
    __syncthreads();                                         // barriers initialised
    const int T = MT * KT;                                   // tiles per pass; tile g < 2T overall
    const unsigned char* src = tiles + B.tile_off;
    const uint32_t idesc = instr_desc<NB>();

    // thread 0: copy tile g into stage g % S (the stage's previous MMAs have completed)
    auto copy_tile = [&](int g) {
        const int s = g % kTcStages;
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;"
                     ::"r"(smem_addr(&full[s])), "r"(kTileBytes) : "memory");
        asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                     ::"r"(smem_addr(ring + (size_t)s * kTileBytes)), "l"(src + (size_t)g * kTileBytes),
                       "r"(kTileBytes), "r"(smem_addr(&full[s])) : "memory");
    };
    int issued = 0, consumed = 0, commits = 0;               // thread 0's bookkeeping
    if (t == 0)                                              // the first tiles stream during X
        while (issued < kTcStages && issued < 2 * T) copy_tile(issued++);

    // X_s = L^{-1} r_s (fp64) as hi + lo bf16 parts: B-operand rows s and R + s (rows >= 2R
    // and columns >= n are zero)
    for (int q = t; q < NB * kpad / 8; q += kTcThreads)
        reinterpret_cast<uint4*>(bop)[q] = make_uint4(0u, 0u, 0u, 0u);
    __syncthreads();
    const int ncell = n / np;
    for (int q = t; q < ncell * R; q += kTcThreads) {
        const int el = q / R, s = q - el * R;
        const double* Le = linv + (int64_t)(B.cell0 + el) * np * np;    // row-major, lower
        const double* rs = p.r[s] + B.in_off + (int64_t)el * np;
        double rv[NP];
#pragma unroll
        for (int j = 0; j < NP; ++j) rv[j] = __ldg(rs + j);
#pragma unroll
        for (int i = 0; i < NP; ++i) {
            double acc = 0.0;
#pragma unroll
            for (int j = 0; j <= i; ++j) acc = fma(__ldg(Le + i * NP + j), rv[j], acc);
            const float x = (float)acc;
            const __nv_bfloat16 hi = __float2bfloat16_rn(x);
            const int k = el * np + i;
            *reinterpret_cast<__nv_bfloat16*>(bop + core_off(s, k, bsbo)) = hi;
            *reinterpret_cast<__nv_bfloat16*>(bop + core_off(R + s, k, bsbo)) =
                __float2bfloat16_rn(x - __bfloat162float(hi));
        }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_slot;

    bool ok = true;
    // thread 0: the MMAs of pass `pass` (tiles pass*T .. pass*T + T - 1), refilling the ring
    // kTcLag tiles behind (the stage of tile g - kTcLag is free once its MMAs, committed
    // kTcLag tiles earlier, have completed: by then they usually have, so the issue loop
    // rarely waits on them), then one commit of `done` for the whole pass
    auto run_pass = [&](int pass) {
        for (int g = pass * T; g < (pass + 1) * T; ++g) {
            const int s = g % kTcStages;
            if (!mbar_wait(&full[s], (g / kTcStages) & 1)) { ok = false; break; }
            ++consumed;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const int tt = g - pass * T, mt = tt / KT, kt = tt - mt * KT;
            const uint32_t abase = smem_addr(ring + (size_t)s * kTileBytes);
            const uint32_t bbase = smem_addr(bop) + (uint32_t)kt * 8u * 128u;
#pragma unroll
            for (int kk = 0; kk < 4; ++kk)
                mma_bf16(tmem + (uint32_t)(mt * NB), smem_desc(abase + kk * 256u, 128u, 1024u),
                         smem_desc(bbase + kk * 256u, 128u, bsbo), idesc, (kt > 0 || kk > 0) ? 1u : 0u);
            mma_commit(&empty[s]);
            if (g >= kTcLag && issued < 2 * T) {
                const int gp = g - kTcLag;
                if (!mbar_wait(&empty[gp % kTcStages], (gp / kTcStages) & 1)) { ok = false; break; }
                copy_tile(issued++);
            }
        }
        mma_commit(&done);
        ++commits;
    };
    if (t == 0) {
        run_pass(0);
        if (!ok) fail_sh = 1;
    }
    // lanes 1..31 of warp 0 wait here for lane 0: spinning on `done` beside it would
    // suspend the warp in try_wait and hold lane 0's loop back
    __syncwarp();
    if (!mbar_wait(&done, 0)) fail_sh = 1;                   // pass 1 complete
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    __syncthreads();
    const bool fail1 = fail_sh != 0;
    if (!fail1) {
        // Y_s = (D hi + D lo) / (chi + c_s lam): hi/lo parts into the B operand of pass 2
        for (int mt = warp >> 2; mt < MT; mt += kTcThreads / 128) {
            float d[NB];
            tmem_load_row<NB>(tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(mt * NB), d);
            const int j = mt * 128 + 32 * (warp & 3) + lane;
            if (j < n) {                  // rows >= 2R and columns >= n keep the zeros of X
                const float lj = lam[B.lam_off + j], chif = (float)chi;
#pragma unroll
                for (int s = 0; s < NB / 2; ++s) {
                    if (s >= R) break;
                    // FP32 is ample here: y is kept to ~16 bits (hi + lo)
                    const float y = (d[s] + d[R + s]) / fmaf((float)p.c[s], lj, chif);
                    const __nv_bfloat16 hi = __float2bfloat16_rn(y);
                    *reinterpret_cast<__nv_bfloat16*>(bop + core_off(s, j, bsbo)) = hi;
                    *reinterpret_cast<__nv_bfloat16*>(bop + core_off(R + s, j, bsbo)) =
                        __float2bfloat16_rn(y - __bfloat162float(hi));
                }
            }
        }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (t == 0 && !fail1) {
        run_pass(1);
        if (!ok) fail_sh = 1;
    }
    __syncwarp();
    if (!fail1 && !mbar_wait(&done, 1)) fail_sh = 1;          // pass 2 complete
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    __syncthreads();
    const bool fail2 = fail_sh != 0;
    if (!fail2) {
        // V_s = D hi + D lo (rows k of Q_i Y), staged as fp32 in the ring
        for (int mt = warp >> 2; mt < MT; mt += kTcThreads / 128) {
            float d[NB];
            tmem_load_row<NB>(tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(mt * NB), d);
            const int k = mt * 128 + 32 * (warp & 3) + lane;
            if (k < n)
                for (int s = 0; s < R; ++s) vst[(size_t)s * npad + k] = d[s] + d[R + s];
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (!fail2) {
        // z_s = L^{-T} V_s per element: z[i] = sum_{j >= i} Linv[j][i] V[j]
        const int ncell = n / np;
        for (int q = t; q < ncell * R; q += kTcThreads) {
            const int el = q / R, s = q - el * R;
            const double* L0 = linv + (int64_t)(B.cell0 + el) * np * np;
            const float* V = vst + (size_t)s * npad + el * np;
            double* z = p.z[s] + B.in_off + (int64_t)el * np;
            double vv[NP];
#pragma unroll
            for (int j = 0; j < NP; ++j) vv[j] = (double)V[j];
#pragma unroll
            for (int i = 0; i < NP; ++i) {
                double acc = 0.0;
#pragma unroll
                for (int j = i; j < NP; ++j) acc = fma(__ldg(L0 + j * NP + i), vv[j], acc);
                z[i] = acc;
            }
        }
    }
    if (fail2 && t == 0) {
        atomicExch(err, 1);
        // bounded drain: the copies issued and not seen complete, then the last commit of
        // `done` (which covers every MMA issued)
        for (int g = consumed; g < issued; ++g)
            if (!mbar_wait(&full[g % kTcStages], (g / kTcStages) & 1)) break;
        if (commits > 0) mbar_wait(&done, (commits - 1) & 1);
    }
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(cols) : "memory");
}

size_t shared_tc_smem(int max_kpad, int nb) {
    const size_t ring = (size_t)kTcStages * kTileBytes;
    const size_t bop = (size_t)nb * max_kpad * 2;
    return ring + bop;
}

template <int NB>
static cudaError_t launch_tc_np(int np, const TcBlock* blocks, int n_blocks, const unsigned char* tiles,
                                const float* lam, const double* linv, double chi, const TcRhs& p, size_t smem,
                                int* err, cudaStream_t s) {
    const void* fn = nullptr;
    switch (np) {
        case 3: fn = (const void*)shared_tc_kernel<NB, 3>; break;
        case 6: fn = (const void*)shared_tc_kernel<NB, 6>; break;
        case 10: fn = (const void*)shared_tc_kernel<NB, 10>; break;
        case 15: fn = (const void*)shared_tc_kernel<NB, 15>; break;
        default: return cudaErrorInvalidValue;
    }
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    switch (np) {
        case 3: shared_tc_kernel<NB, 3><<<n_blocks, kTcThreads, smem, s>>>(blocks, tiles, lam, linv, chi, p, err); break;
        case 6: shared_tc_kernel<NB, 6><<<n_blocks, kTcThreads, smem, s>>>(blocks, tiles, lam, linv, chi, p, err); break;
        case 10: shared_tc_kernel<NB, 10><<<n_blocks, kTcThreads, smem, s>>>(blocks, tiles, lam, linv, chi, p, err); break;
        default: shared_tc_kernel<NB, 15><<<n_blocks, kTcThreads, smem, s>>>(blocks, tiles, lam, linv, chi, p, err); break;
    }
    return cudaGetLastError();
}

cudaError_t launch_shared_tc(const TcBlock* blocks, int n_blocks, const unsigned char* tiles,
                             const float* lam, const double* linv, int np, double chi,
                             const TcRhs& p, int max_kpad, int* err, cudaStream_t s) {
    const int nb = 2 * p.nrhs <= 16 ? 16 : 32;
    const size_t smem = shared_tc_smem(max_kpad, nb);
    return nb == 16 ? launch_tc_np<16>(np, blocks, n_blocks, tiles, lam, linv, chi, p, smem, err, s)
                    : launch_tc_np<32>(np, blocks, n_blocks, tiles, lam, linv, chi, p, smem, err, s);
}

}  // namespace polydg
