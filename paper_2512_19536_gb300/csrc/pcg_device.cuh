// Device helpers of the persistent PCG kernels (kernels_pcg.cu, kernels_group.cu):
// bounded waits, bulk copies with mbarrier completion, grid barriers and grid sums,
// and the block-row matvec from shared memory.
#pragma once

#include <type_traits>

#include <cuda_runtime.h>
#include <cuda_bf16.h>

#include "device.cuh"
#include "kernels.h"

namespace polydg {

constexpr uint32_t kSpinLimit = 1u << 22;     // bounded polls for every wait (default)

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void mbar_init(uint64_t* bar) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(bar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// L2 policy for data streamed once per iteration: evict first, so the streamed
// local inverses do not push K_h, the vectors and the coarse data out of L2.
__device__ __forceinline__ uint64_t evict_first_policy() {
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}

// L2 policy for the local inverses: a fraction `keep` of their lines evict-last (they
// stay in L2 from one iteration to the next), the rest evict-first (streamed from HBM
// without pushing K_h, the vectors and the coarse data out).  keep <= 0: all evict-first.
__device__ __forceinline__ uint64_t stream_policy(float keep) {
    if (!(keep > 0.f)) return evict_first_policy();
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_last.L2::evict_first.b64 %0, %1;"
                 : "=l"(pol)
                 : "f"(fminf(keep, 1.f)));
    return pol;
}

__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar,
                                          uint64_t pol) {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
                 "r"(bytes)
                 : "memory");
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint"
        " [%0], [%1], %2, [%3], %4;" ::"r"(smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar)), "l"(pol)
        : "memory");
}

// Bulk prefetch of [src, src + bytes) into L2 (bytes a multiple of 16, src 16-byte aligned).
__device__ __forceinline__ void prefetch_l2(const void* src, uint32_t bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
    for (uint32_t k = 0; k < kSpinLimit; ++k) {
        uint32_t ok;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
            " selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(ok)
            : "r"(smem_addr(bar)), "r"(parity)
            : "memory");
        if (ok) return true;
    }
    return false;
}

// Barrier over the G CTAs of one solve (all CTAs of a single-solve launch, or
// one simulation's CTA group of a batched launch; the launch is cooperative, so
// all of them are resident).  gs->count starts at 0 for the launch and only
// grows: barrier number k completes when it reaches (k + 1) * G, so no CTA has
// to reset or flip anything.  The arrive is a
// fire-and-forget release reduction after a fence that publishes the CTA's
// writes; waiters poll with acquire loads.  `target` lives in thread 0.
// Returns false (and raises *err) if the other CTAs did not arrive within `limit` polls.
__device__ __forceinline__ bool grid_barrier(GridSync* gs, unsigned G, unsigned& target, int* err,
                                             uint32_t limit = kSpinLimit) {
    __shared__ int ok_sh;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        target += G;
        __threadfence();
        asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(&gs->count) : "memory");
        uint32_t k = 0;
        while ((int)(ld_acquire(&gs->count) - target) < 0) {
            if (++k > limit) { ok = 0; atomicExch(err, 1); break; }
        }
        ok_sh = ok && (*((volatile int*)err) == 0);
    }
    __syncthreads();
    return ok_sh != 0;
}

// Grid barrier that also sums N <= 12 values over the G CTAs.  Each thread's values go
// to shared memory and warp 0 alone adds them (the fp64 pipe of this GPU is narrow: a
// butterfly in all 16 warps would cost 5x more fp64 instructions); the CTA's sums are
// published, and after the barrier warp 0 adds all G partials in the same order in every
// CTA, so all CTAs obtain bit-identical, deterministic sums.  fin(sums) then runs in
// thread 0 alone (scalar updates derived from the sums, written to shared memory) before
// the closing CTA barrier; every thread returns with the sums in v.
// red: shared scratch of 3 x blockDim.x doubles, outv: N shared doubles.
template <int N, typename Fin>
__device__ __forceinline__ bool barrier_sum(GridSync* gs, unsigned G, int cta, unsigned& gen, int* err,
                            double* partials, double (&v)[N], double* red, double* outv, Fin&& fin,
                            uint32_t limit = kSpinLimit) {
    static_assert(N >= 1 && N <= 12, "up to twelve sums (three at a time through red)");
    const int t = threadIdx.x, lane = t & 31;
#pragma unroll
    for (int c0 = 0; c0 < N; c0 += 3) {
        if (c0 > 0) __syncthreads();              // warp 0 is done with the previous three
#pragma unroll
        for (int k = c0; k < N && k < c0 + 3; ++k) red[(k - c0) * blockDim.x + t] = v[k];
        __syncthreads();
        if (t < 32) {
#pragma unroll
            for (int k = c0; k < N && k < c0 + 3; ++k) {
                double s0 = 0.0;
                for (int i = lane; i < (int)blockDim.x; i += 32) s0 += red[(k - c0) * blockDim.x + i];
                s0 = warp_sum(s0);
                if (lane == 0) partials[(size_t)k * G + cta] = s0;
            }
        }
    }
    const bool ok = grid_barrier(gs, G, gen, err, limit);
    if (t < 32) {
        double sum[N];
#pragma unroll
        for (int k = 0; k < N; ++k) {
            double s0 = 0.0;
            for (int i = lane; i < (int)G; i += 32) s0 += __ldcg(partials + (size_t)k * G + i);
            sum[k] = warp_sum(s0);
        }
        if (lane == 0) {
#pragma unroll
            for (int k = 0; k < N; ++k) outv[k] = sum[k];
            fin(sum);
        }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < N; ++k) v[k] = outv[k];
    return ok;
}

template <int DT>
struct StoreType {
    using T = typename std::conditional<DT == 0, double,
              typename std::conditional<DT == 1, float, __nv_bfloat16>::type>::type;
    using X = typename std::conditional<DT == 0, double, float>::type;
};

// Row dot products from shared memory (row Ar of ld entries, staged input xs),
// over the column chunks part, part + parts, ... of 32 lanes x vector width.  The
// fp32/bf16 forms return the sum in lane 0 only.
__device__ __forceinline__ double row_dot(const double* Ar, const double* xs, int ld, int lane,
                                          int part, int parts) {
    double a0 = 0.0, a1 = 0.0;
    for (int c = 2 * (lane + 32 * part); c < ld; c += 64 * parts) {
        const double2 u = *reinterpret_cast<const double2*>(Ar + c);
        const double2 v = *reinterpret_cast<const double2*>(xs + c);
        a0 = fma(u.x, v.x, a0);
        a1 = fma(u.y, v.y, a1);
    }
    return warp_sum(a0 + a1);
}

__device__ __forceinline__ double row_dot(const float* Ar, const float* xs, int ld, int lane,
                                          int part, int parts) {
    float a0 = 0.f, a1 = 0.f;
    for (int c = 4 * (lane + 32 * part); c < ld; c += 128 * parts) {
        const float4 u = *reinterpret_cast<const float4*>(Ar + c);
        const float4 v = *reinterpret_cast<const float4*>(xs + c);
        a0 = fmaf(u.x, v.x, a0); a1 = fmaf(u.y, v.y, a1);
        a0 = fmaf(u.z, v.z, a0); a1 = fmaf(u.w, v.w, a1);
    }
    const float sum = warp_sumf(a0 + a1);
    return lane == 0 ? (double)sum : 0.0;   // only lane 0's value is used: one conversion per row
}

__device__ __forceinline__ double row_dot(const __nv_bfloat16* Ar, const float* xs, int ld, int lane,
                                          int part, int parts) {
    float a0 = 0.f, a1 = 0.f;
    for (int c = 8 * (lane + 32 * part); c < ld; c += 256 * parts) {
        const uint4 v = *reinterpret_cast<const uint4*>(Ar + c);
        const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&v);
        const float4 x0 = *reinterpret_cast<const float4*>(xs + c);
        const float4 x1 = *reinterpret_cast<const float4*>(xs + c + 4);
        float2 f = __bfloat1622float2(h[0]);
        a0 = fmaf(f.x, x0.x, a0); a1 = fmaf(f.y, x0.y, a1);
        f = __bfloat1622float2(h[1]);
        a0 = fmaf(f.x, x0.z, a0); a1 = fmaf(f.y, x0.w, a1);
        f = __bfloat1622float2(h[2]);
        a0 = fmaf(f.x, x1.x, a0); a1 = fmaf(f.y, x1.y, a1);
        f = __bfloat1622float2(h[3]);
        a0 = fmaf(f.x, x1.z, a0); a1 = fmaf(f.y, x1.w, a1);
    }
    const float sum = warp_sumf(a0 + a1);
    return lane == 0 ? (double)sum : 0.0;
}

// One element of a stored local-inverse row, in the store's arithmetic (the same
// rounding as the row_dot forms above: fp64, or fp32 for the fp32 and bf16 stores).
__device__ __forceinline__ double store_elem(const double* p) { return __ldg(p); }
__device__ __forceinline__ float store_elem(const float* p) { return __ldg(p); }
__device__ __forceinline__ float store_elem(const __nv_bfloat16* p) { return __bfloat162float(__ldg(p)); }
__device__ __forceinline__ double fma_x(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float fma_x(float a, float b, float c) { return fmaf(a, b, c); }

// What the P phase needs of one run (contiguous rows of one subdomain's local
// inverse), staged in shared memory at kernel start.
// One pair row of the symmetric store (rows m and n-1-m of the lower triangle of an
// n x n fp32 local inverse A, the diagonal entries halved, see sym_ld) against the staged
// r' in x (zero past n): lane l keeps the sums of columns 128 t + 4 l .. + 3 in acc[t].
// Each entry a_mk of row m adds a_mk x_m to column k (the upper triangle's share of row
// k), and the row's own sum_{k <= m} a_mk x_k goes to rsum[m]; the halved diagonal enters
// both, so once every pair of the subdomain is done, rsum[j] plus column j is
// sum_k a_jk x_k over the whole row j.
template <int TT>
__device__ __forceinline__ void sym_pair(const float* A, const float* x, int n, int m, int lane,
                                         float4 (&acc)[TT], float* rsum) {
    const int b = n - 1 - m;
    const int la = (m + 4) & ~3;
    const float xm = x[m], xb = x[b];
    float dA = 0.f, dB = 0.f;
#pragma unroll
    for (int t = 0; t < TT; ++t) {
        const int c = 128 * t + 4 * lane;
        if (128 * t < la && c < la) {
            const float4 u = *reinterpret_cast<const float4*>(A + c);
            const float4 v = *reinterpret_cast<const float4*>(x + c);
            dA = fmaf(u.x, v.x, dA); dA = fmaf(u.y, v.y, dA);
            dA = fmaf(u.z, v.z, dA); dA = fmaf(u.w, v.w, dA);
            acc[t].x = fmaf(u.x, xm, acc[t].x); acc[t].y = fmaf(u.y, xm, acc[t].y);
            acc[t].z = fmaf(u.z, xm, acc[t].z); acc[t].w = fmaf(u.w, xm, acc[t].w);
        }
        if (b != m && 128 * t <= b && c <= b) {
            const float4 u = *reinterpret_cast<const float4*>(A + la + c);
            const float4 v = *reinterpret_cast<const float4*>(x + c);
            dB = fmaf(u.x, v.x, dB); dB = fmaf(u.y, v.y, dB);
            dB = fmaf(u.z, v.z, dB); dB = fmaf(u.w, v.w, dB);
            acc[t].x = fmaf(u.x, xb, acc[t].x); acc[t].y = fmaf(u.y, xb, acc[t].y);
            acc[t].z = fmaf(u.z, xb, acc[t].z); acc[t].w = fmaf(u.w, xb, acc[t].w);
        }
    }
    dA = warp_sumf(dA);
    dB = warp_sumf(dB);
    if (lane == 0) {
        rsum[m] = dA;
        if (b != m) rsum[b] = dB;
    }
}

struct RunDesc {
    int64_t mat_off;      // element offset of the block in the store
    int64_t in_off;       // first DOF of the block's subdomain
    int32_t row_begin, row_end, ld, ncols, block, pair_begin, pair_count;
    int32_t ord;          // position of the run's first row in the CTA's row sequence
};

// Rows of the CTA's elements of y = K x, warp per element, with x read from the
// CTA-local staging xn (index: local element l * NP + j): lane (i, g) sums
// columns g, g + G, ... of the element's column-major block-row panel.
template <int NP, typename F>
__device__ __forceinline__ void local_rows(const int32_t* __restrict__ row_ptr,
                                           const int32_t* __restrict__ col_local,
                                           const double* __restrict__ val, const double* xn,
                                           int64_t e0, int64_t e1, F&& emit) {
    constexpr int G = 32 / NP;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int g = (lane < G * NP) ? lane / NP : G;
    const int i = lane - (lane / NP) * NP;
    for (int64_t e = e0 + warp; e < e1; e += nw) {
        const int32_t b0 = row_ptr[e];
        const int ncol = (row_ptr[e + 1] - b0) * NP;
        const double* V = val + (int64_t)b0 * NP * NP;
        const int32_t* cl = col_local + b0;
        double acc8[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) acc8[u] = 0.0;
        int c = g;
        for (; c + 7 * G < ncol; c += 8 * G) {
            double vv[8], xv[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int cu = c + u * G, su = cu / NP;
                vv[u] = __ldg(V + (int64_t)cu * NP + i);
                xv[u] = xn[__ldg(cl + su) * NP + (cu - su * NP)];
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) acc8[u] = fma(vv[u], xv[u], acc8[u]);
        }
        for (; c < ncol; c += G) {
            const int sa = c / NP;
            acc8[0] = fma(__ldg(V + (int64_t)c * NP + i), xn[__ldg(cl + sa) * NP + (c - sa * NP)], acc8[0]);
        }
        const double a0 = (acc8[0] + acc8[4]) + (acc8[2] + acc8[6]);
        const double a1 = (acc8[1] + acc8[5]) + (acc8[3] + acc8[7]);
        const double acc = a0 + a1;
        double tot = acc;
#pragma unroll
        for (int k = 1; k < G; ++k) tot += __shfl_down_sync(0xffffffffu, acc, k * NP);
        if (lane < NP) emit(e, i, tot);
    }
}

// Rows of one element of y = K x from its block-row panel V in shared memory (nb
// column-major NP x NP blocks, as in local_rows), with x read from the CTA-local staging
// xn.  Block s's local element id is in lane s of clv (nb <= 32); lane (i, g) sums
// columns g, g + G, ... and lanes i < NP return row i's total.
template <int NP>
__device__ __forceinline__ double panel_rows(const double* V, int clv, int nb, const double* xn, int lane) {
    constexpr int G = 32 / NP;
    const int g = (lane < G * NP) ? lane / NP : G;   // the spare lanes are not summed
    const int i = lane - (lane / NP) * NP;
    const int ncol = nb * NP;
    double a0 = 0.0, a1 = 0.0;
    for (int cb = 0; cb < ncol; cb += 2 * G) {        // the same trip count in every lane
        const int c0 = cb + g, c1 = cb + G + g;
        const int s0 = min(c0, ncol - 1) / NP, s1 = min(c1, ncol - 1) / NP;
        const int k0 = __shfl_sync(0xffffffffu, clv, s0);
        const int k1 = __shfl_sync(0xffffffffu, clv, s1);
        if (c0 < ncol) a0 = fma(V[c0 * NP + i], xn[k0 * NP + (c0 - s0 * NP)], a0);
        if (c1 < ncol) a1 = fma(V[c1 * NP + i], xn[k1 * NP + (c1 - s1 * NP)], a1);
    }
    const double acc = a0 + a1;
    double tot = acc;
#pragma unroll
    for (int k = 1; k < G; ++k) tot += __shfl_down_sync(0xffffffffu, acc, k * NP);
    return tot;
}

}  // namespace polydg
