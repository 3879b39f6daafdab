// Linear-algebra kernels of libpolydg on the PCG hot path (Sec. 4, Eq. prec, PCG).
// One PCG iteration is four kernels (graph nodes):
//   K1 precond_kernel   x += alpha p, r -= alpha q (double-buffered), then per
//                       subdomain the ragged GEMV z_loc = K_i^{-1} r_i (fp64/fp32/bf16
//                       store) and the coarse restriction R_0 r (fp64), with
//                       |r|^2, r.z_loc, z_loc.q and the stopping test;
//   K2 coarse_kernel    y0 = K_0^{-1} r0 (fp64), r.z = r.z_loc + r0.y0, beta;
//   K3 direction_kernel p = z_loc + R_0^T y0 + beta p;
//   K4 matvec_kernel    q = K_h p (fp64, warp per element), p.q, alpha.
// The identities r.(R_0^T y0) = (R_0 r).y0 and z.q = z_loc.q + y0.(R_0 q) let
// the dot products close before the prolongation, so K3 needs no reduction.
// Also here: setup kernels (batched Cholesky inversion of K_i and K_0).
#include <type_traits>

#include <cuda_runtime.h>
#include <cuda_bf16.h>

#include "device.cuh"
#include "kernels.h"

namespace polydg {

// ------------------------------------------------------------------ matvec
// Two warps per element e (warp h = 0, 1 of a pair).  Row e of K_h holds m_e
// blocks (diagonal first) stored consecutively, each column-major, so the row
// is an [m_e * NP columns][NP rows] column-major panel.  Lane (i, g), i < NP,
// g < G = 32 / NP, of warp h accumulates row i over columns g + h G, g + 3 G,
// ... : each warp load reads G * NP consecutive doubles.  The pair's partial
// rows are summed through shared memory.
//   MODE_PLAIN: y = K x.
//   MODE_PCG:   q = K p; p.q -> alpha = (r.z)/(p.q).
//   MODE_RESID: r = b - K x; |b|^2, |r|^2, first stopping test; zeroes p, q.
//   MODE_RHS:   y = Kminus x + c1 v1 + c2 [t^{k+1/2} < t_stim] v2.
constexpr int kElemsPerCta = kBlock / 64;

template <int NP, int MODE>
__global__ void __launch_bounds__(kBlock)
matvec_kernel(const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
              const double* __restrict__ val, const double* __restrict__ x,
              double* __restrict__ y, int64_t nc, const double* __restrict__ v1,
              const double* __restrict__ v2, double c1, double c2, PcgScalars* sc,
              double* partials, const SimScalars* ss, double dt, double stim_duration,
              double* __restrict__ zero1, double* __restrict__ zero2) {
    constexpr int G = 32 / NP;
    __shared__ double sh[32];
    __shared__ double half[kElemsPerCta][32];
    __shared__ bool last;
    if (MODE == MODE_PCG || MODE == MODE_RESID) {
        if (sc->done) return;
    }
    if (ss && ss->failed) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, h = warp & 1, slot = warp >> 1;
    const int64_t e = (int64_t)blockIdx.x * kElemsPerCta + slot;
    const int g = (lane < G * NP) ? lane / NP : 2 * G;
    const int i = lane - (lane / NP) * NP;
    double acc0 = 0.0, acc1 = 0.0;
    const bool valid = e < nc;
    if (valid) {
        const int32_t b0 = row_ptr[e];
        const int ncol = (row_ptr[e + 1] - b0) * NP;
        const double* V = val + (int64_t)b0 * NP * NP;
        const int32_t* cl = col + b0;
        int c = g + h * G;
        for (; c + 2 * G < ncol; c += 4 * G) {
            const int c2 = c + 2 * G;
            const int s1 = c / NP, s2 = c2 / NP;
            const double v1 = __ldg(V + (int64_t)c * NP + i), v2 = __ldg(V + (int64_t)c2 * NP + i);
            const double x1 = __ldg(x + (int64_t)__ldg(cl + s1) * NP + (c - s1 * NP));
            const double x2 = __ldg(x + (int64_t)__ldg(cl + s2) * NP + (c2 - s2 * NP));
            acc0 = fma(v1, x1, acc0);
            acc1 = fma(v2, x2, acc1);
        }
        if (c < ncol) {
            const int s1 = c / NP;
            acc0 = fma(__ldg(V + (int64_t)c * NP + i), __ldg(x + (int64_t)__ldg(cl + s1) * NP + (c - s1 * NP)), acc0);
        }
    }
    double acc = acc0 + acc1;
    {   // lane i < NP sums the partials of lanes i + k NP (k < G), which are < G NP <= 32
        double tot = acc;
#pragma unroll
        for (int k = 1; k < G; ++k) tot += __shfl_down_sync(0xffffffffu, acc, k * NP);
        acc = tot;
    }
    if (h == 1) half[slot][lane] = acc;
    __syncthreads();
    if (h == 0) acc += half[slot][lane];
    const bool owner = valid && h == 0 && lane < NP;
    const int64_t t = e * NP + i;
    double d0 = 0.0, d1 = 0.0;
    if (owner) {
        if (MODE == MODE_PLAIN) {
            y[t] = acc;
        } else if (MODE == MODE_PCG) {
            y[t] = acc;
            d0 = x[t] * acc;
        } else if (MODE == MODE_RESID) {
            const double bv = v1[t];
            const double rv = bv - acc;
            y[t] = rv;
            zero1[t] = 0.0;
            zero2[t] = 0.0;
            d0 = bv * bv;
            d1 = rv * rv;
        } else {
            const double tmid = ((double)ss->k + 0.5) * dt;
            const double on = (tmid < stim_duration) ? 1.0 : 0.0;
            y[t] = acc + c1 * v1[t] + c2 * on * v2[t];
        }
    }
    if (MODE == MODE_PCG) {
        const double s = block_sum(d0, sh);
        if (publish_partials(partials, &s, 1, &sc->ticket[T_MATVEC], &last)) {
            const double pq = sum_partials(partials, gridDim.x, sh);
            if (threadIdx.x == 0) {
                sc->pq = pq;
                sc->ticket[T_MATVEC] = 0;
                if (!(pq > 0.0) || !finite(pq)) {
                    sc->status = kEBREAKDOWN;
                    sc->done = 1;
                } else {
                    sc->alpha = sc->rz / pq;
                    sc->alpha_valid = 1;
                }
            }
        }
    } else if (MODE == MODE_RESID) {
        double s[2];
        s[0] = block_sum(d0, sh);
        s[1] = block_sum(d1, sh);
        if (publish_partials(partials, s, 2, &sc->ticket[T_INIT], &last)) {
            const double bb = sum_partials(partials, gridDim.x, sh);
            const double rr = sum_partials(partials + kMaxPartials, gridDim.x, sh);
            if (threadIdx.x == 0) {
                sc->ticket[T_INIT] = 0;
                sc->bb = bb;
                sc->rr = rr;
                sc->it = 0;
                sc->pass = 0;
                sc->alpha = 0.0;
                sc->alpha_valid = 0;
                sc->beta = 0.0;
                sc->status = kOK;
                if (!finite(bb) || !finite(rr)) {
                    sc->status = kENONFINITE;
                    sc->done = 1;
                    sc->relres = rr;
                } else if (bb == 0.0) {
                    sc->relres = 0.0;
                    sc->done = 2;           // b = 0: the solution is x = 0
                } else {
                    sc->relres = sqrt(rr / bb);
                    if (rr <= sc->rtol2 * bb) sc->done = 1;
                }
            }
        }
    }
}

// ---------------------------------------------------- K1: update + precond
// One CTA per tile (rows [row0, row0 + rows) of one LOCAL block).  Thread 0
// starts a single bulk copy (cp.async.bulk, completion on an mbarrier) of the
// tile's rows of K_i^{-1} into shared memory; meanwhile the CTA stages the
// block's input r' = r - alpha q (fp64 for the fp64 store, fp32 otherwise).
// Each warp then reduces rows from shared memory.  A second pass over the
// tile's own rows commits x and r into the other parity buffer and adds the
// |r'|^2, r'.z and z.q terms.  RESTRICT tiles (the n_q rows of R_0 on one
// (agglomerate, subdomain) pair, fp64) read their rows directly.
constexpr uint32_t kMaxSpin = 1u << 22;   // bounded mbarrier polls (~0.1-1 s)

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void bulk_copy_g2s(void* dst, const void* src, uint32_t bytes,
                                              uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
            "r"(smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait on phase 0 of `bar`; false if the copy did not land in time.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar) {
    for (uint32_t k = 0; k < kMaxSpin; ++k)
        if (mbar_try_wait(bar, 0)) return true;
    return false;
}

__device__ __forceinline__ double dot_row64(const double* __restrict__ Ar, const double* xs, int ld,
                                            int lane) {
    double a0 = 0.0, a1 = 0.0;
    for (int c = 2 * lane; c < ld; c += 64) {
        const double2 u = *reinterpret_cast<const double2*>(Ar + c);
        a0 = fma(u.x, xs[c], a0);
        a1 = fma(u.y, xs[c + 1], a1);
    }
    return warp_sum(a0 + a1);
}

__device__ __forceinline__ float dot_row32(const float* Ar, const float* xs, int ld, int lane) {
    float a0 = 0.f, a1 = 0.f;
    for (int c = 4 * lane; c < ld; c += 128) {
        const float4 u = *reinterpret_cast<const float4*>(Ar + c);
        const float4 v = *reinterpret_cast<const float4*>(xs + c);
        a0 = fmaf(u.x, v.x, a0); a1 = fmaf(u.y, v.y, a1);
        a0 = fmaf(u.z, v.z, a0); a1 = fmaf(u.w, v.w, a1);
    }
    return warp_sumf(a0 + a1);
}

__device__ __forceinline__ float dot_row16(const __nv_bfloat16* Ar, const float* xs, int ld, int lane) {
    float a0 = 0.f, a1 = 0.f;
    for (int c = 8 * lane; c < ld; c += 256) {
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
    return warp_sumf(a0 + a1);
}

// Shared-memory layout of a LOCAL tile: [rows x ld store elements][ld staged
// inputs][rows doubles z].  Returns the byte offsets.
template <int DT>
struct TileLayout {
    using T = typename std::conditional<DT == 0, double, typename std::conditional<DT == 1, float, __nv_bfloat16>::type>::type;
    using X = typename std::conditional<DT == 0, double, float>::type;
};

template <int DT>
__global__ void __launch_bounds__(kBlock)
precond_kernel(K1Args a) {
    using T = typename TileLayout<DT>::T;
    using X = typename TileLayout<DT>::X;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ double sh[32];
    __shared__ bool last;
    __shared__ __align__(8) uint64_t bar;
    PcgScalars* sc = a.sc;
    if (sc && sc->done) {
        if (a.use_cond && blockIdx.x == 0 && threadIdx.x == 0) cudaGraphSetConditional(a.cond, 0);
        return;
    }
    const int par = sc ? (sc->pass & 1) : 0;
    const double* __restrict__ xin = a.x[par];
    const double* __restrict__ rin = a.r[par];
    double* __restrict__ xout = a.x[par ^ 1];
    double* __restrict__ rout = a.r[par ^ 1];
    const double alpha = (sc && sc->alpha_valid) ? sc->alpha : 0.0;
    const bool flexible = sc && sc->flexible;
    const GemvTile tile = a.tiles[blockIdx.x];
    const GemvBlock B = a.blocks[tile.block];
    const double* __restrict__ ri = rin + B.in_off;
    const double* __restrict__ qi = a.q ? a.q + B.in_off : nullptr;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    double prr = 0.0, prz = 0.0, pzq = 0.0;
    if (B.kind == KIND_RESTRICT) {
        double* rs = reinterpret_cast<double*>(smem);
        double* qs = rs + B.ld;
        for (int j = threadIdx.x; j < B.ld; j += blockDim.x) {
            const bool in = j < B.ncols;
            const double qv = (in && qi) ? qi[j] : 0.0;
            rs[j] = in ? fma(-alpha, qv, ri[j]) : 0.0;
            qs[j] = flexible ? qv : 0.0;
        }
        __syncthreads();
        const double* R = a.st64 + B.mat_off;
        for (int row = warp; row < B.nrows; row += nw) {
            const double* Rr = R + (int64_t)row * B.ld;
            const double yr = dot_row64(Rr, rs, B.ld, lane);
            const double yq = flexible ? dot_row64(Rr, qs, B.ld, lane) : 0.0;
            if (lane == 0) {
                a.r0p[B.out_off + row] = yr;
                a.q0p[B.out_off + row] = yq;
            }
        }
    } else if (B.kind == KIND_LOCAL) {
        const int nrt = min(a.rows, B.nrows - tile.row0);          // rows of this tile
        const T* gsrc = reinterpret_cast<const T*>(DT == 0 ? (const void*)a.st64
                                                           : DT == 1 ? (const void*)a.st32
                                                                     : (const void*)a.st16) +
                        B.mat_off + (int64_t)tile.row0 * B.ld;
        T* As = reinterpret_cast<T*>(smem);
        const size_t abytes = (((size_t)a.rows * B.ld * sizeof(T)) + 15) & ~(size_t)15;
        X* xs = reinterpret_cast<X*>(smem + abytes);
        double* zs = reinterpret_cast<double*>(smem + abytes + (((size_t)B.ld * sizeof(X) + 15) & ~(size_t)15));
        const uint32_t bytes = (uint32_t)((size_t)nrt * B.ld * sizeof(T));
        if (threadIdx.x == 0) {
            mbar_init(&bar, 1);
            mbar_expect_tx(&bar, bytes);
            bulk_copy_g2s(As, gsrc, bytes, &bar);
        }
        for (int j = threadIdx.x; j < B.ld; j += blockDim.x)
            xs[j] = (j < B.ncols) ? (X)(qi ? fma(-alpha, qi[j], ri[j]) : ri[j]) : (X)0;
        __syncthreads();                       // xs staged, mbarrier initialised
        const bool landed = mbar_wait_bounded(&bar);
        if (!landed) {
            // The copy did not complete in time: flag it and wait once more (bounded)
            // for the copy in flight.  The tile still takes part in the reductions,
            // so the last CTA ends the solve with an error status.
            if (threadIdx.x == 0 && a.err) atomicExch(a.err, 1);
            mbar_wait_bounded(&bar);
        }
        for (int rr = warp; rr < nrt; rr += nw) {
            if (!landed) {
                if (lane == 0) zs[rr] = 0.0;
                continue;
            }
            double zr;
            if (DT == 0) zr = dot_row64(reinterpret_cast<const double*>(As) + (size_t)rr * B.ld,
                                        reinterpret_cast<const double*>(xs), B.ld, lane);
            else if (DT == 1) zr = (double)dot_row32(reinterpret_cast<const float*>(As) + (size_t)rr * B.ld,
                                                     reinterpret_cast<const float*>(xs), B.ld, lane);
            else zr = (double)dot_row16(reinterpret_cast<const __nv_bfloat16*>(As) + (size_t)rr * B.ld,
                                        reinterpret_cast<const float*>(xs), B.ld, lane);
            if (lane == 0) zs[rr] = zr;
        }
        __syncthreads();
        for (int rr = threadIdx.x; rr < nrt; rr += blockDim.x) {
            const int row = tile.row0 + rr;
            const int64_t t = B.in_off + row;
            const double zr = zs[rr];
            a.z[t] = zr;
            if (sc) {
                const double qv = qi ? qi[row] : 0.0;
                const double rp = fma(-alpha, qv, ri[row]);
                rout[t] = rp;
                xout[t] = fma(alpha, a.p[t], xin[t]);
                prr = fma(rp, rp, prr);
                prz = fma(rp, zr, prz);
                if (flexible) pzq = fma(zr, qv, pzq);
            }
        }
    } else {  // KIND_IDENTITY: z = r'
        const int rend = min(tile.row0 + a.rows, B.nrows);
        for (int row = tile.row0 + threadIdx.x; row < rend; row += blockDim.x) {
            const int64_t t = B.in_off + row;
            const double qv = qi ? qi[row] : 0.0;
            const double rp = fma(-alpha, qv, ri[row]);
            a.z[t] = rp;
            if (sc) {
                rout[t] = rp;
                xout[t] = fma(alpha, a.p[t], xin[t]);
                prr = fma(rp, rp, prr);
                prz = fma(rp, rp, prz);
                if (flexible) pzq = fma(rp, qv, pzq);
            }
        }
    }
    if (!sc) return;
    double s[3];
    s[0] = block_sum(prr, sh);
    s[1] = block_sum(prz, sh);
    s[2] = block_sum(pzq, sh);
    if (publish_partials(a.partials, s, 3, &sc->ticket[T_K1], &last)) {
        const double rr = sum_partials(a.partials, gridDim.x, sh);
        const double rz = sum_partials(a.partials + kMaxPartials, gridDim.x, sh);
        const double zq = sum_partials(a.partials + 2 * kMaxPartials, gridDim.x, sh);
        if (threadIdx.x == 0) {
            sc->ticket[T_K1] = 0;
            sc->rr = rr;
            sc->rz_loc = rz;
            sc->zq_loc = zq;
            sc->it += sc->alpha_valid;
            sc->alpha_valid = 0;
            sc->pass += 1;
            sc->relres = sqrt(rr / sc->bb);
            if (a.err && *a.err) {
                sc->status = kEDEVICE;
                sc->done = 1;
            } else if (!finite(rr) || !finite(rz)) {
                sc->status = kENONFINITE;
                sc->done = 1;
            } else if (rr <= sc->rtol2 * sc->bb) {
                sc->status = kOK;
                sc->done = 1;
            } else if (sc->it >= sc->maxit) {
                sc->status = kENOTCONV;
                sc->done = 1;
            }
            if (sc->done && a.use_cond) cudaGraphSetConditional(a.cond, 0);
        }
    }
}

// ------------------------------------------------------------ K2: coarse
// r0 and q0 are assembled from the (agglomerate, subdomain) partial sums in
// fixed order; warp per row of K_0^{-1}: y0 = K_0^{-1} r0.  Then
// r.z = r.z_loc + r0.y0, z.q = z_loc.q + q0.y0 and the new beta.
__device__ __forceinline__ void finish_beta(PcgScalars* sc, double rz, double zq) {
    if (!finite(rz) || !finite(zq)) {
        sc->status = kENONFINITE;
        sc->done = 1;
        return;
    }
    if (sc->it == 0) {
        sc->beta = 0.0;
    } else if (sc->flexible) {
        // z_{k+1}.(r_{k+1} - r_k) = -alpha_k z_{k+1}.q_k  (r_{k+1} = r_k - alpha_k q_k)
        sc->beta = -sc->alpha * zq / sc->rz;
    } else {
        sc->beta = rz / sc->rz;
    }
    sc->rz = rz;
    sc->zq = zq;
    if (!finite(sc->beta) || rz == 0.0) {
        sc->status = kEBREAKDOWN;
        sc->done = 1;
    }
}

__global__ void __launch_bounds__(kBlock)
coarse_kernel(K2Args a) {
    extern __shared__ double cs[];
    __shared__ double sh[32];
    __shared__ bool last;
    PcgScalars* sc = a.sc;
    if (sc && sc->done) return;
    const int n0 = a.n0;
    double* r0s = cs;
    double* q0s = cs + n0;
    const bool flexible = sc && sc->flexible;
    for (int idx = threadIdx.x; idx < n0; idx += blockDim.x) {
        const int J = idx / a.nq, k = idx - J * a.nq;
        double sr = 0.0, sq = 0.0;
        for (int64_t pp = a.pair_ptr[J]; pp < a.pair_ptr[J + 1]; ++pp) {
            sr += a.r0p[pp * a.nq + k];
            if (flexible) sq += a.q0p[pp * a.nq + k];
        }
        r0s[idx] = sr;
        q0s[idx] = sq;
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    double pr = 0.0, pq = 0.0;
    const int row = blockIdx.x * (blockDim.x >> 5) + warp;       // warp per row of K_0^{-1}
    if (row < n0) {
        const double* Kr = a.K0inv + (int64_t)row * a.ld0;
        double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
        int c = lane;
        for (; c + 96 < n0; c += 128) {
            a0 = fma(__ldg(Kr + c), r0s[c], a0);
            a1 = fma(__ldg(Kr + c + 32), r0s[c + 32], a1);
            a2 = fma(__ldg(Kr + c + 64), r0s[c + 64], a2);
            a3 = fma(__ldg(Kr + c + 96), r0s[c + 96], a3);
        }
        for (; c < n0; c += 32) a0 = fma(__ldg(Kr + c), r0s[c], a0);
        const double acc = warp_sum((a0 + a1) + (a2 + a3));
        if (lane == 0) {
            a.y0[row] = acc;
            pr = acc * r0s[row];
            pq = acc * q0s[row];
        }
    }
    if (!sc) return;
    double s[2];
    s[0] = block_sum(pr, sh);
    s[1] = block_sum(pq, sh);
    if (publish_partials(a.partials, s, 2, &sc->ticket[T_COARSE], &last)) {
        const double r0y = sum_partials(a.partials, gridDim.x, sh);
        const double q0y = sum_partials(a.partials + kMaxPartials, gridDim.x, sh);
        if (threadIdx.x == 0) {
            sc->ticket[T_COARSE] = 0;
            finish_beta(sc, sc->rz_loc + r0y, sc->zq_loc + q0y);
        }
    }
}

// --------------------------------------------------------- K3: direction
// p = z_loc + T_e y0_{J(e)} + beta p   (z = z_loc + R_0^T y0, Eq. prec).
// With sc == nullptr it writes out = z_loc + R_0^T y0 instead (asm_apply).
template <int NQ>
__global__ void __launch_bounds__(kBlock)
direction_kernel(double* __restrict__ p, const double* __restrict__ zl, const double* __restrict__ T,
                 const int32_t* __restrict__ agg, const double* __restrict__ y0, int64_t nc, int np,
                 const PcgScalars* sc, double* __restrict__ out) {
    if (sc && sc->done) return;
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nc * np) return;
    double v = zl[t];
    if (T) {
        const int64_t e = t / np;
        const double* Tr = T + t * NQ;
        const double* y = y0 + (int64_t)agg[e] * NQ;
#pragma unroll
        for (int k = 0; k < NQ; ++k) v = fma(Tr[k], y[k], v);
    }
    if (sc) p[t] = fma(sc->beta, p[t], v);
    else out[t] = v;
}

// ------------------------------------------------------------ permutations
// dst[internal e][j] = src[caller c][j]  (to_internal = 1), or the reverse.
// With sc != nullptr the internal source is the parity buffer src2[pass & 1]
// and b = 0 (done == 2) yields zeros.
__global__ void permute_kernel(const double* __restrict__ src, const double* __restrict__ src_odd,
                               double* __restrict__ dst, const int64_t* __restrict__ to_caller,
                               int64_t nc, int np, int to_internal, const PcgScalars* sc) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nc * np) return;
    const int64_t e = t / np, j = t - e * np, c = to_caller[e];
    if (to_internal) {
        dst[t] = src[c * np + j];
    } else {
        const double* s = (sc && (sc->pass & 1)) ? src_odd : src;
        dst[c * np + j] = (sc && sc->done == 2) ? 0.0 : s[t];
    }
}

__global__ void copy_kernel(const double* __restrict__ src, double* __restrict__ dst, int64_t n,
                            const SimScalars* ss) {
    if (ss && ss->failed) return;
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n) dst[t] = src[t];
}

// --------------------------------------------------------- setup: S1 kernels
// Dense K_i = R_i K_h R_i^T from the block-sparse rows of subdomain i.
__global__ void extract_local_kernel(const int32_t* __restrict__ row_ptr,
                                     const int32_t* __restrict__ col,
                                     const double* __restrict__ val,
                                     const int64_t* __restrict__ sub_ptr,
                                     const int64_t* __restrict__ mat_off,
                                     const int32_t* __restrict__ ld, double* __restrict__ dense,
                                     int np) {
    const int s = blockIdx.x;
    const int64_t e0 = sub_ptr[s], e1 = sub_ptr[s + 1];
    double* D = dense + mat_off[s];
    const int L = ld[s];
    for (int64_t e = e0; e < e1; ++e) {
        for (int32_t bi = row_ptr[e]; bi < row_ptr[e + 1]; ++bi) {
            const int64_t f = col[bi];
            if (f < e0 || f >= e1) continue;
            for (int k = threadIdx.x; k < np * np; k += blockDim.x) {
                const int i = k / np, j = k - i * np;
                // blocks are stored column-major: entry (i, j) at j * np + i
                D[((e - e0) * np + i) * L + (f - e0) * np + j] = val[(int64_t)bi * np * np + j * np + i];
            }
        }
    }
}

// In-place inverse of SPD matrices by Cholesky (one CTA per matrix):
//   1. A = L L^T (right-looking, lower triangle of A);
//   2. W = L^{-1}, stored transposed (Wt[j][k] = W[k][j]) in a zeroed workspace;
//   3. A^{-1} = W^T W, written to the full A.
// A non-positive pivot sets status[m] = ENOTSPD and leaves A undefined.
__global__ void __launch_bounds__(1024)
chol_inverse_kernel(double* __restrict__ store, const int64_t* __restrict__ mat_off,
                    const int32_t* __restrict__ nrow, const int32_t* __restrict__ ld,
                    double* __restrict__ work, const int64_t* __restrict__ work_off,
                    const int32_t* __restrict__ wld, int* __restrict__ status) {
    extern __shared__ double shm[];   // max(n) doubles
    __shared__ double tile_a[32][33], tile_b[32][33];
    __shared__ int fail;
    const int m = blockIdx.x;
    double* A = store + mat_off[m];
    double* Wt = work + work_off[m];
    const int n = nrow[m], L = ld[m], WL = wld[m];
    const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
    if (tid == 0) fail = 0;
    __syncthreads();
    // 1. Cholesky
    for (int k = 0; k < n; ++k) {
        if (tid == 0) {
            const double d = A[(int64_t)k * L + k];
            if (!(d > 0.0) || !isfinite(d)) fail = 1;
            else A[(int64_t)k * L + k] = sqrt(d);
        }
        __syncthreads();
        if (fail) break;
        const double lkk = A[(int64_t)k * L + k];
        for (int i = k + 1 + tid; i < n; i += nt) {
            const double v = A[(int64_t)i * L + k] / lkk;
            A[(int64_t)i * L + k] = v;
            shm[i] = v;
        }
        __syncthreads();
        for (int i = k + 1 + warp; i < n; i += nw) {
            const double lik = shm[i];
            double* Ai = A + (int64_t)i * L;
            for (int j = k + 1 + lane; j <= i; j += 32) Ai[j] = fma(-lik, shm[j], Ai[j]);
        }
        __syncthreads();
    }
    if (fail) {
        if (tid == 0) status[m] = kENOTSPD;
        return;
    }
    // 2. Wt = (L^{-1})^T: row j of Wt is column j of W, owned by one thread.
    for (int i = 0; i < n; ++i) {
        for (int k = tid; k <= i; k += nt) shm[k] = A[(int64_t)i * L + k];
        __syncthreads();
        for (int j = tid; j <= i; j += nt) {
            if (j == i) {
                Wt[(int64_t)i * WL + i] = 1.0 / shm[i];
            } else {
                const double* wj = Wt + (int64_t)j * WL;
                double s = 0.0;
                for (int k = j; k < i; ++k) s = fma(shm[k], wj[k], s);
                Wt[(int64_t)j * WL + i] = -s / shm[i];
            }
        }
        __syncthreads();
    }
    // 3. A^{-1}[i][j] = sum_k Wt[i][k] Wt[j][k]  (32x32 tiles, upper tiles mirrored)
    const int nb = (n + 31) / 32;
    const int tx = tid & 31, ty = tid >> 5;
    for (int I = 0; I < nb; ++I)
        for (int J = I; J < nb; ++J) {
            double acc = 0.0;
            for (int k0 = J * 32; k0 < nb * 32; k0 += 32) {
                if (ty < 32) {
                    tile_a[ty][tx] = Wt[(int64_t)(I * 32 + ty) * WL + k0 + tx];
                    tile_b[ty][tx] = Wt[(int64_t)(J * 32 + ty) * WL + k0 + tx];
                }
                __syncthreads();
                if (ty < 32) {
#pragma unroll 8
                    for (int kk = 0; kk < 32; ++kk) acc = fma(tile_a[ty][kk], tile_b[tx][kk], acc);
                }
                __syncthreads();
            }
            const int i = I * 32 + ty, j = J * 32 + tx;
            if (ty < 32 && i < n && j < n) {
                if (I == J) {
                    if (j >= i) {
                        A[(int64_t)i * L + j] = acc;
                        A[(int64_t)j * L + i] = acc;
                    }
                } else {
                    A[(int64_t)i * L + j] = acc;
                    A[(int64_t)j * L + i] = acc;
                }
            }
            __syncthreads();
        }
    if (tid == 0) status[m] = 0;
}

// Copy an fp64 block into the fp32 or bf16 store (same ld, zero padding kept).
__global__ void cast_store_kernel(const double* __restrict__ src, float* __restrict__ d32,
                                  __nv_bfloat16* __restrict__ d16, int64_t n) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n;
         t += (int64_t)gridDim.x * blockDim.x) {
        if (d32) d32[t] = (float)src[t];
        else d16[t] = __float2bfloat16_rn((float)src[t]);
    }
}

// ------------------------------------------------------------ launchers
#define NP_SWITCH(np, ...)                                   \
    switch (np) {                                            \
        case 3: { constexpr int NP = 3; __VA_ARGS__; } break;  \
        case 6: { constexpr int NP = 6; __VA_ARGS__; } break;  \
        case 10: { constexpr int NP = 10; __VA_ARGS__; } break; \
        case 15: { constexpr int NP = 15; __VA_ARGS__; } break; \
        case 21: { constexpr int NP = 21; __VA_ARGS__; } break; \
        case 28: { constexpr int NP = 28; __VA_ARGS__; } break; \
        default: return cudaErrorInvalidValue;                \
    }

static inline unsigned grid_for(int64_t n) { return (unsigned)((n + kBlock - 1) / kBlock); }

cudaError_t launch_matvec(int mode, int np, const DeviceMatrix& K, const double* val,
                          const double* x, double* y, const double* v1, const double* v2,
                          double c1, double c2, PcgScalars* sc, double* partials,
                          const SimScalars* ss, double dt, double stim_duration, double* zero1,
                          double* zero2, cudaStream_t s) {
    const unsigned g = (unsigned)((K.nc + kElemsPerCta - 1) / kElemsPerCta);
    if (g > (unsigned)kMaxPartials) return cudaErrorInvalidValue;
#define MV(M)                                                                                  \
    NP_SWITCH(np, matvec_kernel<NP, M><<<g, kBlock, 0, s>>>(K.row_ptr, K.col, val, x, y, K.nc, v1, \
                                                            v2, c1, c2, sc, partials, ss, dt,      \
                                                            stim_duration, zero1, zero2))
    switch (mode) {
        case MODE_PLAIN: MV(MODE_PLAIN); break;
        case MODE_PCG: MV(MODE_PCG); break;
        case MODE_RESID: MV(MODE_RESID); break;
        default: MV(MODE_RHS); break;
    }
#undef MV
    return cudaGetLastError();
}

cudaError_t launch_precond(const K1Args& a, int dtype, int ntiles, size_t smem, cudaStream_t s) {
    if (ntiles > kMaxPartials) return cudaErrorInvalidValue;
    if (dtype == 0) precond_kernel<0><<<ntiles, kBlock, smem, s>>>(a);
    else if (dtype == 1) precond_kernel<1><<<ntiles, kBlock, smem, s>>>(a);
    else precond_kernel<2><<<ntiles, kBlock, smem, s>>>(a);
    return cudaGetLastError();
}

// The opt-in shared-memory limits only grow, so graphs captured for earlier
// preconditioners stay launchable.
static size_t g_precond_smem = 0, g_coarse_smem = 0;

cudaError_t set_precond_smem(size_t smem) {
    if (smem <= g_precond_smem) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(precond_kernel<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(precond_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(precond_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) g_precond_smem = smem;
    return e;
}

cudaError_t launch_coarse(const K2Args& a, cudaStream_t s) {
    const int rows_per_cta = kBlock / 32;
    const int grid = a.n0 > 0 ? (a.n0 + rows_per_cta - 1) / rows_per_cta : 1;
    const size_t smem = 2 * (size_t)a.n0 * sizeof(double);
    coarse_kernel<<<grid, kBlock, smem, s>>>(a);
    return cudaGetLastError();
}

cudaError_t set_coarse_smem(size_t smem) {
    if (smem <= g_coarse_smem) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(coarse_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e == cudaSuccess) g_coarse_smem = smem;
    return e;
}

cudaError_t launch_direction(int nq, double* p, const double* zl, const double* T,
                             const int32_t* agg, const double* y0, int64_t nc, int np,
                             const PcgScalars* sc, double* out, cudaStream_t s) {
    const unsigned g = grid_for(nc * np);
    if (T == nullptr) nq = 3;
    switch (nq) {
        case 3: direction_kernel<3><<<g, kBlock, 0, s>>>(p, zl, T, agg, y0, nc, np, sc, out); break;
        case 4: direction_kernel<4><<<g, kBlock, 0, s>>>(p, zl, T, agg, y0, nc, np, sc, out); break;
        case 6: direction_kernel<6><<<g, kBlock, 0, s>>>(p, zl, T, agg, y0, nc, np, sc, out); break;
        case 10: direction_kernel<10><<<g, kBlock, 0, s>>>(p, zl, T, agg, y0, nc, np, sc, out); break;
        case 15: direction_kernel<15><<<g, kBlock, 0, s>>>(p, zl, T, agg, y0, nc, np, sc, out); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_permute(const double* src, const double* src_odd, double* dst,
                           const int64_t* to_caller, int64_t nc, int np, int to_internal,
                           const PcgScalars* sc, cudaStream_t s) {
    permute_kernel<<<grid_for(nc * np), kBlock, 0, s>>>(src, src_odd, dst, to_caller, nc, np,
                                                        to_internal, sc);
    return cudaGetLastError();
}

cudaError_t launch_copy(const double* src, double* dst, int64_t n, const SimScalars* ss,
                        cudaStream_t s) {
    copy_kernel<<<grid_for(n), kBlock, 0, s>>>(src, dst, n, ss);
    return cudaGetLastError();
}

cudaError_t launch_extract_local(const DeviceMatrix& K, const int64_t* sub_ptr, int n_sub,
                                 const int64_t* mat_off, const int32_t* ld, double* dense,
                                 int np, cudaStream_t s) {
    extract_local_kernel<<<n_sub, 256, 0, s>>>(K.row_ptr, K.col, K.val, sub_ptr, mat_off, ld,
                                              dense, np);
    return cudaGetLastError();
}

cudaError_t launch_chol_inverse(double* store, const int64_t* mat_off, const int32_t* nrow,
                                const int32_t* ld, double* work, const int64_t* work_off,
                                const int32_t* wld, int* status, int nmat, int max_n,
                                cudaStream_t s) {
    const size_t shm = (size_t)max_n * sizeof(double);
    cudaError_t e = cudaFuncSetAttribute(chol_inverse_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm);
    if (e != cudaSuccess) return e;
    chol_inverse_kernel<<<nmat, 1024, shm, s>>>(store, mat_off, nrow, ld, work, work_off, wld,
                                                status);
    return cudaGetLastError();
}

cudaError_t launch_cast_store(const double* src, float* d32, __nv_bfloat16* d16, int64_t n,
                              cudaStream_t s) {
    cast_store_kernel<<<1024, kBlock, 0, s>>>(src, d32, d16, n);
    return cudaGetLastError();
}

}  // namespace polydg
