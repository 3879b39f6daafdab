// Persistent PCG kernel (Sec. 4 and 5: PCG with the two-level additive Schwarz
// preconditioner of Eq. prec, stopping on |r|_2 <= rtol |b|_2).
//
// One cooperative launch runs the whole solve: one CTA per SM, each owning a
// fixed share of every phase.  With w = K z and the recurrences
//     p_k = z_k + beta p_{k-1},   q_k = w_k + beta q_{k-1}  (= K p_k),
//     p_{k+1}.q_{k+1} = z.w + 2 beta z.q_k + beta^2 p_k.q_k    (K symmetric),
// the matvec no longer waits for beta, and one iteration is two phases:
//   P   p_k, q_k, x += alpha p_k, r' = r - alpha q_k (r, p, q double-buffered);
//       z_loc = K_i^{-1} r'_i on the CTA's rows of the local inverses, streamed by
//       cp.async.bulk into a shared-memory ring prefetched across phases and
//       iterations (the inverses are constant); R_0 r' for the subdomains the
//       CTA stages first; partial |r'|^2                     -> barrier, test
//   CM  y0 = K_0^{-1} R_0 r' for the agglomerates the CTA's elements touch
//       (redundantly per CTA; a distributed coarse phase with one more barrier
//       when the coarse space is large), z = z_loc + R_0^T y0 for its elements
//       and their face neighbours in shared memory, w = K z on its elements
//       (fp64); partial r'.z, z.q_k, z.w                      -> barrier, beta, alpha
// Every CTA sums the per-CTA partials in the same order, so all CTAs hold
// bit-identical scalars and take the same branches; the result is deterministic.
// Waits (grid barriers, mbarriers) are bounded: on timeout the kernel raises an
// error flag, waits (bounded) for its own copies in flight and stops.
#include <type_traits>

#include <cuda_runtime.h>
#include <cuda_bf16.h>

#include "device.cuh"
#include "kernels.h"

namespace polydg {

constexpr uint32_t kSpinLimit = 1u << 22;     // bounded polls for every wait

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

__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    const uint64_t pol = evict_first_policy();
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

// Block-wide sums of N values at once (results valid in every thread).
template <int N>
__device__ __forceinline__ void block_sum_n(double (&v)[N]) {
    __shared__ double shn[N][32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int k = 0; k < N; ++k) v[k] = warp_sum(v[k]);
    __syncthreads();
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < N; ++k) shn[k][w] = v[k];
    __syncthreads();
#pragma unroll
    for (int k = 0; k < N; ++k) {
        double t = (lane < nw) ? shn[k][lane] : 0.0;
        v[k] = warp_sum(t);
    }
    __syncthreads();
}

// Grid barrier over all CTAs of a cooperative launch.  gs->count starts at 0 for
// the launch and only grows: barrier number k completes when it reaches
// (k + 1) * gridDim.x, so no CTA has to reset or flip anything.  The arrive is a
// fire-and-forget release reduction after a fence that publishes the CTA's
// writes; waiters poll with acquire loads.  `target` lives in thread 0.
// Returns false (and raises *err) if the other CTAs did not arrive in time.
__device__ bool grid_barrier(GridSync* gs, unsigned& target, int* err) {
    __shared__ int ok_sh;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        target += gridDim.x;
        __threadfence();
        asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(&gs->count) : "memory");
        uint32_t k = 0;
        while ((int)(ld_acquire(&gs->count) - target) < 0) {
            if (++k > kSpinLimit) { ok = 0; atomicExch(err, 1); break; }
        }
        ok_sh = ok && (*((volatile int*)err) == 0);
    }
    __syncthreads();
    return ok_sh != 0;
}

// Grid barrier that also sums N values over all CTAs: every CTA publishes its
// block sums before the barrier and afterwards adds all CTAs' partials in CTA
// order, so every CTA obtains the same bit-identical, deterministic sums.
template <int N>
__device__ bool barrier_sum(GridSync* gs, unsigned& gen, int* err, double* partials,
                            double* /*bcast*/, double (&v)[N]) {
    block_sum_n<N>(v);
    if (threadIdx.x == 0)
#pragma unroll
        for (int k = 0; k < N; ++k) partials[(size_t)k * gridDim.x + blockIdx.x] = v[k];
    const bool ok = grid_barrier(gs, gen, err);
#pragma unroll
    for (int k = 0; k < N; ++k) v[k] = 0.0;
    for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x)
#pragma unroll
        for (int k = 0; k < N; ++k) v[k] += __ldcg(partials + (size_t)k * gridDim.x + i);
    block_sum_n<N>(v);
    return ok;
}

template <int DT>
struct StoreType {
    using T = typename std::conditional<DT == 0, double,
              typename std::conditional<DT == 1, float, __nv_bfloat16>::type>::type;
    using X = typename std::conditional<DT == 0, double, float>::type;
};

// Row dot products from shared memory (row Ar of ld entries, staged input xs),
// over the column chunks part, part + parts, ... of 32 lanes x vector width.
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
    return (double)warp_sumf(a0 + a1);
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
    return (double)warp_sumf(a0 + a1);
}

// What the P phase needs of one tile, staged in shared memory at kernel start.
struct TileDesc {
    int64_t src_off;      // element offset of the tile's first row in the store
    int64_t in_off;       // first DOF of the tile's subdomain
    int32_t row0, nrt, ld, ncols, block, pair_begin, pair_count;
    uint32_t bytes;       // bulk-copy size
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

template <int DT, int NP>
__global__ void __launch_bounds__(kPersistThreads, 1)
pcg_persistent_kernel(PersistArgs a) {
    using T = typename StoreType<DT>::T;
    using X = typename StoreType<DT>::X;
    extern __shared__ __align__(128) unsigned char smem[];
    constexpr int S = kStages;
    __shared__ __align__(8) uint64_t bars[S];

    const int cta = blockIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    PcgScalars* sc = a.sc;
    if (sc->done) return;             // a failed earlier step: nothing to do (uniform)
    const bool flexible = sc->flexible != 0;
    const double rtol2 = sc->rtol2;
    const int maxit = sc->maxit;
    unsigned gen = 0;                 // barrier target of thread 0 (gs->count is 0 at launch)

    auto buf = [&](int k) { return reinterpret_cast<T*>(smem + (size_t)k * a.buf_bytes); };
    X* xs = reinterpret_cast<X*>(smem + a.xs_off);                 // r' in the store's arithmetic
    double* rp = reinterpret_cast<double*>(smem + a.rp_off);       // r' (fp64)
    double* zs = reinterpret_cast<double*>(smem + a.zs_off);       // [S][rows]
    double* r0s = reinterpret_cast<double*>(smem + a.r0_off);      // [n0]
    double* y0l = reinterpret_cast<double*>(smem + a.y0_off);      // y0 of the CTA's agglomerates
    double* pn = reinterpret_cast<double*>(smem + a.pn_off);       // x or z of the needed elements
    TileDesc* td = reinterpret_cast<TileDesc*>(smem + a.td_off);   // this CTA's tiles
    __shared__ double zpart[kPersistThreads / 32];                 // split-row partial dots

    const int64_t e0 = a.elem_ptr[cta], e1 = a.elem_ptr[cta + 1];
    const int n_own = (int)(e1 - e0);
    const int32_t* need = a.need + a.need_ptr[cta];
    const int32_t* needj = a.need_aggl + a.need_ptr[cta];
    const int n_need = a.need_ptr[cta + 1] - a.need_ptr[cta];
    const int32_t* aggs = a.need_agg + a.need_agg_ptr[cta];
    const int n_aggs = a.need_agg_ptr[cta + 1] - a.need_agg_ptr[cta];
    const int t0 = a.tile_ptr[cta], nt = a.tile_ptr[cta + 1] - t0;
    const int c0 = a.crow_ptr[cta], c1 = a.crow_ptr[cta + 1];
    const bool coarse = a.n0 > 0;

    // ---- init: r = b - K x on own elements; p, q, z, w = 0; |b|^2, |r|^2
    for (int idx = threadIdx.x; idx < n_need * NP; idx += blockDim.x) {
        const int l = idx / NP;
        pn[idx] = __ldcg(a.x + (int64_t)need[l] * NP + (idx - l * NP));
    }
    for (int64_t t = e0 * NP + threadIdx.x; t < e1 * NP; t += blockDim.x) {
        a.p[0][t] = 0.0; a.p[1][t] = 0.0; a.q[0][t] = 0.0; a.q[1][t] = 0.0;
        a.z[t] = 0.0; a.w[t] = 0.0;
    }
    __syncthreads();
    double v2[2] = {0.0, 0.0};
    local_rows<NP>(a.row_ptr, a.col_local, a.val, pn, e0, e1, [&](int64_t e, int i, double kx) {
        const int64_t t = e * NP + i;
        const double bv = a.b[t], rv = bv - kx;
        a.r[0][t] = rv;
        v2[0] = fma(bv, bv, v2[0]);
        v2[1] = fma(rv, rv, v2[1]);
    });
    uint32_t seq = 0;                 // tiles consumed so far (all iterations)
    for (int k = threadIdx.x; k < nt; k += blockDim.x) {
        const GemvTile tl = a.tiles[t0 + k];
        const GemvBlock B = a.blocks[tl.block];
        TileDesc d;
        d.src_off = B.mat_off + (int64_t)tl.row0 * B.ld;
        d.in_off = B.in_off;
        d.row0 = tl.row0;
        d.nrt = min(a.rows, B.nrows - tl.row0);
        d.ld = B.ld;
        d.ncols = B.ncols;
        d.block = tl.block;
        d.pair_begin = B.pair_begin;
        d.pair_count = B.pair_count;
        d.bytes = (uint32_t)((size_t)d.nrt * B.ld * sizeof(T));
        td[k] = d;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int k = 0; k < S; ++k) mbar_init(&bars[k]);
        for (int k = 0; k < S && nt > 0; ++k) {   // the inverses do not depend on the iterate
            const TileDesc& d = td[k % nt];
            bulk_load(buf(k), reinterpret_cast<const T*>(a.store) + d.src_off, d.bytes, &bars[k]);
        }
    }
    bool ok = barrier_sum<2>(a.gs, gen, a.err, a.partials, a.bcast, v2);
    const double bb = v2[0];
    double rr = v2[1];
    int status = kOK, it = 0, done = 0, par = 0, pp = 0;
    double alpha = 0.0, beta = 0.0, rz = 0.0, pq = 0.0, relres = 0.0;
    int pending = 0;                  // alpha p_k / alpha q_k not yet committed to x, r
    if (!ok) { status = kEDEVICE; done = 1; }
    else if (!isfinite(bb) || !isfinite(rr)) { status = kENONFINITE; done = 1; }
    else if (bb == 0.0) { done = 2; }
    else { relres = sqrt(rr / bb); if (rr <= rtol2 * bb) done = 1; }

    while (!done) {
        // ---------------------------------------------------------------- P
        const double* rin = a.r[par];
        double* rout = a.r[par ^ 1];
        const double* pold = a.p[pp];
        const double* qold = a.q[pp];
        double* pnew = a.p[pp ^ 1];
        double* qnew = a.q[pp ^ 1];
        const double al = pending ? alpha : 0.0, be = beta;
        double v1[1] = {0.0};                     // |r'|^2
        if (a.identity) {
            for (int64_t t = e0 * NP + threadIdx.x; t < e1 * NP; t += blockDim.x) {
                const double pk = fma(be, pold[t], a.z[t]), qk = fma(be, qold[t], a.w[t]);
                pnew[t] = pk;
                qnew[t] = qk;
                a.x[t] = fma(al, pk, a.x[t]);
                const double r_ = fma(-al, qk, rin[t]);
                rout[t] = r_;
                a.zl[t] = r_;
                v1[0] = fma(r_, r_, v1[0]);
            }
        } else {
            int staged = -1;
            const int parts = (a.rows < nw && nw % a.rows == 0) ? nw / a.rows : 1;
            for (int k = 0; k < nt; ++k, ++seq) {
                const TileDesc& tl = td[k];
                const int nrt = tl.nrt;
                if (tl.block != staged) {
                    __syncthreads();
                    for (int j = threadIdx.x; j < tl.ld; j += blockDim.x) {
                        double r_ = 0.0;
                        if (j < tl.ncols) {
                            const int64_t t = tl.in_off + j;
                            const double qk = fma(be, __ldcg(qold + t), __ldcg(a.w + t));
                            r_ = fma(-al, qk, __ldcg(rin + t));
                        }
                        rp[j] = r_;
                        if (DT != 0) xs[j] = (X)r_;
                    }
                    staged = tl.block;
                    __syncthreads();
                }
                // operands of the commit, fetched before the tile lands
                const int64_t tr = tl.in_off + tl.row0 + threadIdx.x;
                double zv = 0.0, wv = 0.0, pv = 0.0, qv = 0.0, xv = 0.0;
                if ((int)threadIdx.x < nrt) {
                    zv = __ldcg(a.z + tr); wv = __ldcg(a.w + tr);
                    pv = __ldcg(pold + tr); qv = __ldcg(qold + tr);
                    xv = a.x[tr];
                }
                const int bi = seq % S;
                if (!mbar_wait(&bars[bi], (seq / S) & 1)) {
                    if (threadIdx.x == 0) atomicExch(a.err, 1);
                }
                double* zt = zs + bi * a.rows;
                const T* As = buf(bi);
                const X* xin = (DT == 0) ? reinterpret_cast<const X*>(rp) : xs;
                if (parts == 1) {
                    for (int r_ = warp; r_ < nrt; r_ += nw) {
                        const double zr = row_dot(As + (size_t)r_ * tl.ld, xin, tl.ld, lane, 0, 1);
                        if (lane == 0) zt[r_] = zr;
                    }
                    __syncthreads();
                } else {                  // rows < warps: each row split over `parts` warps
                    const int r_ = warp % a.rows, part = warp / a.rows;
                    const double zr = (r_ < nrt) ? row_dot(As + (size_t)r_ * tl.ld, xin, tl.ld, lane, part, parts) : 0.0;
                    if (lane == 0) zpart[warp] = zr;
                    __syncthreads();
                    if ((int)threadIdx.x < nrt) {
                        double sum = 0.0;
                        for (int pt = 0; pt < parts; ++pt) sum += zpart[pt * a.rows + threadIdx.x];
                        zt[threadIdx.x] = sum;
                    }
                    __syncthreads();
                }
                if (threadIdx.x == 0) {   // buffer bi is free: prefetch S tiles ahead (cyclic)
                    const TileDesc& tn = td[(k + S) % nt];
                    bulk_load(buf(bi), reinterpret_cast<const T*>(a.store) + tn.src_off, tn.bytes, &bars[bi]);
                }
                if ((int)threadIdx.x < nrt) {
                    const double pk = fma(be, pv, zv), qk = fma(be, qv, wv);
                    const double r_ = rp[tl.row0 + threadIdx.x];
                    pnew[tr] = pk;
                    qnew[tr] = qk;
                    a.x[tr] = fma(al, pk, xv);
                    rout[tr] = r_;
                    a.zl[tr] = zt[threadIdx.x];
                    v1[0] = fma(r_, r_, v1[0]);
                }
                if (tl.row0 == 0 && coarse) {   // this CTA stages the subdomain first: R_0 r'
                    for (int pi = 0; pi < tl.pair_count; ++pi) {
                        const GemvBlock R = a.blocks[a.sub_pairs[tl.pair_begin + pi]];
                        const double* Rm = a.st64 + R.mat_off;
                        for (int row = warp; row < R.nrows; row += nw) {
                            const double* Rr = Rm + (int64_t)row * R.ld;
                            double s0 = 0.0, s1 = 0.0;
                            int j = lane;
                            for (; j + 32 < R.ncols; j += 64) {
                                s0 = fma(__ldg(Rr + j), rp[j], s0);
                                s1 = fma(__ldg(Rr + j + 32), rp[j + 32], s1);
                            }
                            if (j < R.ncols) s0 = fma(__ldg(Rr + j), rp[j], s0);
                            const double sv = warp_sum(s0 + s1);
                            if (lane == 0) a.r0p[R.out_off + row] = sv;
                        }
                    }
                }
            }
        }
        if (threadIdx.x == 0 && n_own > 0) {     // K_h rows of the CM phase into L2
            const char* lo = reinterpret_cast<const char*>(a.val + (int64_t)a.row_ptr[e0] * NP * NP);
            const char* hi = reinterpret_cast<const char*>(a.val + (int64_t)a.row_ptr[e1] * NP * NP);
            for (const char* c = lo; c < hi; c += 65536)
                prefetch_l2(c, (uint32_t)min((int64_t)65536, (int64_t)(hi - c)));
        }
        ok = barrier_sum<1>(a.gs, gen, a.err, a.partials, a.bcast, v1);
        rr = v1[0];
        it += pending;
        pending = 0;
        par ^= 1;
        pp ^= 1;
        relres = sqrt(rr / bb);
        if (!ok) { status = kEDEVICE; break; }
        if (!isfinite(rr)) { status = kENONFINITE; break; }
        if (rr <= rtol2 * bb) { status = kOK; break; }
        if (it >= maxit) { status = kENOTCONV; break; }
        const double* rk = a.r[par];              // r_{k+1}
        const double* qk = a.q[pp];               // q_k
        // ---------------------------------------------------------------- coarse
        if (coarse) {
            if (a.redundant || c1 > c0) {
                for (int idx = threadIdx.x; idx < a.n0; idx += blockDim.x) {
                    const int J = idx / a.nq, kq = idx - J * a.nq;
                    double s_r = 0.0;
                    for (int64_t p2 = a.pair_ptr[J]; p2 < a.pair_ptr[J + 1]; ++p2)
                        s_r += __ldcg(a.r0p + p2 * a.nq + kq);
                    r0s[idx] = s_r;
                }
                __syncthreads();
            }
            auto coarse_row = [&](int row) {
                const double* Kr = a.K0inv + (int64_t)row * a.ld0;
                double s0 = 0.0, s1 = 0.0;
                int c = lane;
                for (; c + 32 < a.n0; c += 64) {
                    s0 = fma(__ldg(Kr + c), r0s[c], s0);
                    s1 = fma(__ldg(Kr + c + 32), r0s[c + 32], s1);
                }
                if (c < a.n0) s0 = fma(__ldg(Kr + c), r0s[c], s0);
                return warp_sum(s0 + s1);
            };
            if (a.redundant) {                    // y0 of this CTA's agglomerates only
                for (int w2 = warp; w2 < n_aggs * a.nq; w2 += nw) {
                    const int jl = w2 / a.nq, kq = w2 - jl * a.nq;
                    const double y = coarse_row(aggs[jl] * a.nq + kq);
                    if (lane == 0) y0l[w2] = y;
                }
            } else {                              // distributed coarse rows, then a barrier
                for (int row = c0 + warp; row < c1; row += nw) {
                    const double y = coarse_row(row);
                    if (lane == 0) a.y0[row] = y;
                }
                ok = grid_barrier(a.gs, gen, a.err);
                if (!ok) { status = kEDEVICE; break; }
            }
            __syncthreads();
        }
        // ---------------------------------------------------------------- CM
        // z = z_loc + R_0^T y0 for own and neighbour elements; w = K z on own elements
        for (int idx = threadIdx.x; idx < n_need * NP; idx += blockDim.x) {
            const int l = idx / NP, j = idx - l * NP;
            const int64_t e = need[l], t = e * NP + j;
            double v = __ldcg(a.zl + t);
            if (coarse) {
                const double* Tr = a.T + t * a.nq;
                if (a.redundant) {
                    const double* y = y0l + needj[l] * a.nq;
                    for (int kq = 0; kq < a.nq; ++kq) v = fma(__ldg(Tr + kq), y[kq], v);
                } else {
                    const double* y = a.y0 + (int64_t)a.agg[e] * a.nq;
                    for (int kq = 0; kq < a.nq; ++kq) v = fma(__ldg(Tr + kq), __ldcg(y + kq), v);
                }
            }
            pn[idx] = v;
            if (l < n_own) a.z[t] = v;
        }
        __syncthreads();
        double v3[3] = {0.0, 0.0, 0.0};           // r.z, z.q_k, z.w
        local_rows<NP>(a.row_ptr, a.col_local, a.val, pn, e0, e1, [&](int64_t e, int i, double kz) {
            const int64_t t = e * NP + i;
            const double zv = pn[(e - e0) * NP + i];
            a.w[t] = kz;
            v3[0] = fma(__ldcg(rk + t), zv, v3[0]);
            v3[1] = fma(zv, __ldcg(qk + t), v3[1]);
            v3[2] = fma(zv, kz, v3[2]);
        });
        ok = barrier_sum<3>(a.gs, gen, a.err, a.partials, a.bcast, v3);
        if (!ok) { status = kEDEVICE; break; }
        const double rz_new = v3[0], zq = v3[1], zw = v3[2];
        if (!isfinite(rz_new) || !isfinite(zq) || !isfinite(zw)) { status = kENONFINITE; break; }
        double bnew;
        if (it == 0) bnew = 0.0;
        else if (flexible) bnew = -alpha * zq / rz;   // z_{k+1}.(r_{k+1} - r_k) = -alpha_k z_{k+1}.q_k
        else bnew = rz_new / rz;
        if (!isfinite(bnew) || rz_new == 0.0) { status = kEBREAKDOWN; break; }
        const double pq_new = zw + 2.0 * bnew * zq + bnew * bnew * pq;
        if (!(pq_new > 0.0) || !isfinite(pq_new)) { status = kEBREAKDOWN; break; }
        beta = bnew;
        rz = rz_new;
        pq = pq_new;
        alpha = rz / pq;
        pending = 1;
    }
    if (done == 2) {            // b = 0: the solution is x = 0
        for (int64_t t = e0 * NP + threadIdx.x; t < e1 * NP; t += blockDim.x) a.x[t] = 0.0;
    }
    // wait (bounded) for this CTA's copies still in flight before leaving
    if (!a.identity && nt > 0) {
        for (uint32_t s2 = seq; s2 < seq + S; ++s2) mbar_wait(&bars[s2 % S], (s2 / S) & 1);
    }
    if (cta == 0 && threadIdx.x == 0) {
        sc->bb = bb;
        sc->rr = rr;
        sc->relres = relres;
        sc->it = it;
        sc->status = status;
        sc->done = done ? done : 1;
        sc->pass = 0;
    }
}

template <int DT>
static cudaError_t launch_dt(int np, const PersistArgs& a, size_t smem, cudaStream_t s) {
    void* args[] = {(void*)&a};
    const void* fn = nullptr;
    switch (np) {
        case 3: fn = (const void*)pcg_persistent_kernel<DT, 3>; break;
        case 6: fn = (const void*)pcg_persistent_kernel<DT, 6>; break;
        case 10: fn = (const void*)pcg_persistent_kernel<DT, 10>; break;
        case 15: fn = (const void*)pcg_persistent_kernel<DT, 15>; break;
        default: return cudaErrorInvalidValue;
    }
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    return cudaLaunchCooperativeKernel(fn, dim3(a.grid), dim3(kPersistThreads), args, smem, s);
}

cudaError_t launch_pcg_persistent(int dtype, int np, const PersistArgs& a, size_t smem,
                                  cudaStream_t s) {
    if (a.grid > kMaxPartials) return cudaErrorInvalidValue;
    switch (dtype) {
        case 0: return launch_dt<0>(np, a, smem, s);
        case 1: return launch_dt<1>(np, a, smem, s);
        default: return launch_dt<2>(np, a, smem, s);
    }
}

cudaError_t persistent_occupancy(int dtype, int np, size_t smem, int* blocks_per_sm) {
    const void* fn = nullptr;
#define PICK(DT)                                                               \
    switch (np) {                                                              \
        case 3: fn = (const void*)pcg_persistent_kernel<DT, 3>; break;         \
        case 6: fn = (const void*)pcg_persistent_kernel<DT, 6>; break;         \
        case 10: fn = (const void*)pcg_persistent_kernel<DT, 10>; break;       \
        case 15: fn = (const void*)pcg_persistent_kernel<DT, 15>; break;       \
        default: return cudaErrorInvalidValue;                                 \
    }
    if (dtype == 0) { PICK(0) } else if (dtype == 1) { PICK(1) } else { PICK(2) }
#undef PICK
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, fn, kPersistThreads, smem);
}

}  // namespace polydg
