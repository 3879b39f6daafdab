// Linear-algebra kernels of libpolydg on the PCG hot path (Sec. 4, Eq. prec, PCG):
//   * block-sparse SIP-DG matvec q = K_h p (float64; Eq. coer + mass, Sec. 3),
//     fused with the PCG dot products and coefficient updates;
//   * ragged batched dense GEMV with the local inverses K_i^{-1} (fp64/fp32/bf16
//     store) and the coarse inverse K_0^{-1} (fp64) in one launch;
//   * coarse restriction R_0 r and prolongation R_0^T y (L2-projection blocks T_K);
//   * fused PCG vector updates with deterministic last-CTA reductions;
//   * setup: batched Cholesky factorisation and inversion of K_i and K_0.
#include <cuda_runtime.h>
#include <cuda_bf16.h>

#include "device.cuh"
#include "kernels.h"

namespace polydg {

// ------------------------------------------------------------------ matvec
// Thread per DOF row (e, i); row e of K_h holds blocks row_ptr[e]..row_ptr[e+1]-1
// (n_p x n_p, row-major).  MODE_PLAIN: y = K x.  MODE_PCG: q = K p, then
// alpha = (r.z)/(p.q).  MODE_RESID: r = b - K x, |b|^2, |r|^2, first
// convergence test.  MODE_RHS: y = Kminus x + c1 v1 + c2(t) v2.
template <int NP, int MODE>
__global__ void __launch_bounds__(kBlock)
bsr_matvec_kernel(const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
                  const double* __restrict__ val, const double* __restrict__ x,
                  double* __restrict__ y, int64_t nc, const double* __restrict__ v1,
                  const double* __restrict__ v2, double c1, double c2, PcgScalars* sc,
                  double* partials, const SimScalars* ss, double dt, double stim_duration) {
    __shared__ double sh[32];
    __shared__ bool last;
    if (MODE == MODE_PCG || MODE == MODE_RESID) {
        if (sc->done) return;
    }
    if (ss && ss->failed) return;
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t n = nc * NP;
    double acc = 0.0, xr = 0.0, vr = 0.0;
    if (t < n) {
        const int64_t e = t / NP;
        const int i = (int)(t - e * NP);
        const int32_t b0 = row_ptr[e], b1 = row_ptr[e + 1];
        for (int32_t bi = b0; bi < b1; ++bi) {
            const double* B = val + (int64_t)bi * NP * NP + i * NP;
            const double* xc = x + (int64_t)col[bi] * NP;
#pragma unroll
            for (int j = 0; j < NP; ++j) acc = fma(__ldg(B + j), __ldg(xc + j), acc);
        }
        if (MODE == MODE_PLAIN) {
            y[t] = acc;
        } else if (MODE == MODE_PCG) {
            y[t] = acc;
            xr = x[t];
        } else if (MODE == MODE_RESID) {
            vr = v1[t];
            acc = vr - acc;
            y[t] = acc;
        } else {  // MODE_RHS
            const double tmid = ((double)ss->k + 0.5) * dt;
            const double on = (tmid < stim_duration) ? 1.0 : 0.0;
            y[t] = acc + c1 * v1[t] + c2 * on * v2[t];
        }
    }
    if (MODE == MODE_PCG) {
        const double s = block_sum(xr * acc, sh);
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
                }
            }
        }
    } else if (MODE == MODE_RESID) {
        double s[2];
        s[0] = block_sum(vr * vr, sh);
        s[1] = block_sum(acc * acc, sh);
        if (publish_partials(partials, s, 2, &sc->ticket[T_INIT], &last)) {
            const double bb = sum_partials(partials, gridDim.x, sh);
            const double rr = sum_partials(partials + kMaxPartials, gridDim.x, sh);
            if (threadIdx.x == 0) {
                sc->ticket[T_INIT] = 0;
                sc->bb = bb;
                sc->rr = rr;
                sc->it = 0;
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

// ------------------------------------------------------------- PCG vectors
// x += alpha p; r -= alpha q; |r|^2 -> convergence test (Euclidean norm of the
// relative residual, Sec. 5).  Last kernel of the loop body: ends the device
// loop through the graph's conditional handle when done.
__global__ void __launch_bounds__(kBlock)
pcg_update_kernel(double* __restrict__ x, double* __restrict__ r, const double* __restrict__ p,
                  const double* __restrict__ q, int64_t n, PcgScalars* sc, double* partials,
                  cudaGraphConditionalHandle cond, int use_cond) {
    __shared__ double sh[32];
    __shared__ bool last;
    if (sc->done) {
        if (use_cond && blockIdx.x == 0 && threadIdx.x == 0) cudaGraphSetConditional(cond, 0);
        return;
    }
    const double alpha = sc->alpha;
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double rn = 0.0;
    if (t < n) {
        x[t] = fma(alpha, p[t], x[t]);
        rn = fma(-alpha, q[t], r[t]);
        r[t] = rn;
    }
    const double s = block_sum(rn * rn, sh);
    if (publish_partials(partials, &s, 1, &sc->ticket[T_UPDATE], &last)) {
        const double rr = sum_partials(partials, gridDim.x, sh);
        if (threadIdx.x == 0) {
            sc->ticket[T_UPDATE] = 0;
            sc->rr = rr;
            sc->it += 1;
            sc->relres = sqrt(rr / sc->bb);
            if (!finite(rr)) {
                sc->status = kENONFINITE;
                sc->done = 1;
            } else if (rr <= sc->rtol2 * sc->bb) {
                sc->status = kOK;
                sc->done = 1;
            } else if (sc->it >= sc->maxit) {
                sc->status = kENOTCONV;
                sc->done = 1;
            }
            if (sc->done && use_cond) cudaGraphSetConditional(cond, 0);
        }
    }
}

// p = z + beta p (beta = 0 on the first iteration).
__global__ void __launch_bounds__(kBlock)
pcg_direction_kernel(double* __restrict__ p, const double* __restrict__ z, int64_t n,
                     const PcgScalars* sc) {
    if (sc->done) return;
    const double beta = sc->beta;
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n) p[t] = fma(beta, p[t], z[t]);
}

// Shared tail of the preconditioner kernels: given r.z and z.q sums, form beta.
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
    sc->rz_old = sc->rz;
    sc->rz = rz;
    sc->zq = zq;
    if (!finite(sc->beta) || rz == 0.0) {
        sc->status = kEBREAKDOWN;
        sc->done = 1;
    }
}

// Unpreconditioned CG: z = r (the direction kernel reads r); r.r and r.q.
__global__ void __launch_bounds__(kBlock)
identity_dots_kernel(const double* __restrict__ r, const double* __restrict__ q, int64_t n,
                     PcgScalars* sc, double* partials) {
    __shared__ double sh[32];
    __shared__ bool last;
    if (sc->done) return;
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double a = 0.0, b = 0.0;
    const bool use_q = sc->it > 0 && sc->flexible;   // q = K p_{k-1} exists from k = 1
    if (t < n) {
        const double rv = r[t];
        a = rv * rv;
        if (use_q) b = rv * q[t];
    }
    double s[2];
    s[0] = block_sum(a, sh);
    s[1] = block_sum(b, sh);
    if (publish_partials(partials, s, 2, &sc->ticket[T_IDENT], &last)) {
        const double rz = sum_partials(partials, gridDim.x, sh);
        const double zq = sum_partials(partials + kMaxPartials, gridDim.x, sh);
        if (threadIdx.x == 0) {
            sc->ticket[T_IDENT] = 0;
            finish_beta(sc, rz, zq);
        }
    }
}

// ------------------------------------------------------ coarse restriction
// r0[J*NQ + a] = sum_{e in J} sum_i T_e[i][a] r[e*NP + i]   (R_0 = (R_0^T)^T).
// One warp per agglomerate; lanes stride over its (cell, i) pairs.
template <int NP, int NQ>
__global__ void restrict_kernel(const double* __restrict__ r, const double* __restrict__ T,
                                const int64_t* __restrict__ agg_ptr,
                                const int32_t* __restrict__ agg_cells, int n_agg,
                                double* __restrict__ r0, const int* done) {
    if (done && *done) return;
    const int warp = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
    if (warp >= n_agg) return;
    double acc[NQ];
#pragma unroll
    for (int a = 0; a < NQ; ++a) acc[a] = 0.0;
    const int64_t p0 = agg_ptr[warp], cnt = (agg_ptr[warp + 1] - p0) * NP;
    for (int64_t idx = lane; idx < cnt; idx += 32) {
        const int64_t e = agg_cells[p0 + idx / NP];
        const int i = (int)(idx % NP);
        const double rv = r[e * NP + i];
        const double* Tr = T + (e * NP + i) * NQ;
#pragma unroll
        for (int a = 0; a < NQ; ++a) acc[a] = fma(Tr[a], rv, acc[a]);
    }
#pragma unroll
    for (int a = 0; a < NQ; ++a) {
        const double s = warp_sum(acc[a]);
        if (lane == 0) r0[(int64_t)warp * NQ + a] = s;
    }
}

// z[e][i] += sum_a T_e[i][a] y0[J(e)][a]; with sc != nullptr also r.z and z.q
// (q = K p of the previous iteration) and the new beta.
template <int NP, int NQ>
__global__ void __launch_bounds__(kBlock)
prolong_kernel(double* __restrict__ z, const double* __restrict__ T, const int32_t* __restrict__ agg,
               const double* __restrict__ y0, int64_t nc, const double* __restrict__ r,
               const double* __restrict__ q, PcgScalars* sc, double* partials) {
    __shared__ double sh[32];
    __shared__ bool last;
    if (sc && sc->done) return;
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double a = 0.0, b = 0.0;
    if (t < nc * NP) {
        const int64_t e = t / NP;
        double zt = z[t];
        if (T) {
            const double* Tr = T + t * NQ;
            const double* y = y0 + (int64_t)agg[e] * NQ;
#pragma unroll
            for (int k = 0; k < NQ; ++k) zt = fma(Tr[k], y[k], zt);
            z[t] = zt;
        }
        if (sc) {
            a = r[t] * zt;
            if (sc->it > 0 && sc->flexible) b = zt * q[t];   // q = K p_{k-1} exists from k = 1
        }
    }
    if (!sc) return;
    double s[2];
    s[0] = block_sum(a, sh);
    s[1] = block_sum(b, sh);
    if (publish_partials(partials, s, 2, &sc->ticket[T_PROLONG], &last)) {
        const double rz = sum_partials(partials, gridDim.x, sh);
        const double zq = sum_partials(partials + kMaxPartials, gridDim.x, sh);
        if (threadIdx.x == 0) {
            sc->ticket[T_PROLONG] = 0;
            finish_beta(sc, rz, zq);
        }
    }
}

// ------------------------------------------------------------- ragged GEMV
// One CTA per tile of `rows` rows of one dense block.  The block's input
// vector is staged in shared memory (converted to the accumulation type and
// zero-padded to ld); each warp streams whole rows with 16-byte loads.
template <typename TA>
__device__ __forceinline__ TA dot16(const double* a, const TA* x) {
    const double2 v = *reinterpret_cast<const double2*>(a);
    return (TA)(v.x * (double)x[0] + v.y * (double)x[1]);
}

__device__ __forceinline__ float dot16f(const float* a, const float* x) {
    const float4 v = __ldg(reinterpret_cast<const float4*>(a));
    return v.x * x[0] + v.y * x[1] + v.z * x[2] + v.w * x[3];
}

__device__ __forceinline__ float dot16b(const __nv_bfloat16* a, const float* x) {
    const uint4 v = __ldg(reinterpret_cast<const uint4*>(a));
    const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&v);
    float s = 0.0f;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const float2 f = __bfloat1622float2(h[k]);
        s = fmaf(f.x, x[2 * k], s);
        s = fmaf(f.y, x[2 * k + 1], s);
    }
    return s;
}

__global__ void __launch_bounds__(kBlock)
ragged_gemv_kernel(const GemvBlock* __restrict__ blocks, const GemvTile* __restrict__ tiles,
                   int rows, const double* __restrict__ st64, const float* __restrict__ st32,
                   const __nv_bfloat16* __restrict__ st16, const double* __restrict__ r,
                   const double* __restrict__ r0, double* __restrict__ z, double* __restrict__ y0,
                   const int* done) {
    extern __shared__ double xs_raw[];
    if (done && *done) return;
    const GemvTile tile = tiles[blockIdx.x];
    const GemvBlock B = blocks[tile.block];
    const double* in = (B.sel ? r0 : r) + B.in_off;
    double* out = (B.sel ? y0 : z) + B.out_off;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int rend = min(tile.row0 + rows, B.n);
    if (B.dtype == 0) {
        double* xs = xs_raw;
        for (int j = threadIdx.x; j < B.ld; j += blockDim.x) xs[j] = (j < B.n) ? in[j] : 0.0;
        __syncthreads();
        const double* A = st64 + B.mat_off;
        for (int row = tile.row0 + warp; row < rend; row += nw) {
            const double* Ar = A + (int64_t)row * B.ld;
            double acc = 0.0;
            for (int c = 2 * lane; c < B.ld; c += 64) {
                const double2 v = __ldg(reinterpret_cast<const double2*>(Ar + c));
                acc = fma(v.x, xs[c], acc);
                acc = fma(v.y, xs[c + 1], acc);
            }
            acc = warp_sum(acc);
            if (lane == 0) out[row] = acc;
        }
    } else {
        float* xs = reinterpret_cast<float*>(xs_raw);
        for (int j = threadIdx.x; j < B.ld; j += blockDim.x) xs[j] = (j < B.n) ? (float)in[j] : 0.0f;
        __syncthreads();
        if (B.dtype == 1) {
            const float* A = st32 + B.mat_off;
            for (int row = tile.row0 + warp; row < rend; row += nw) {
                const float* Ar = A + (int64_t)row * B.ld;
                float acc = 0.0f;
                for (int c = 4 * lane; c < B.ld; c += 128) acc += dot16f(Ar + c, xs + c);
                acc = warp_sumf(acc);
                if (lane == 0) out[row] = (double)acc;
            }
        } else {
            const __nv_bfloat16* A = st16 + B.mat_off;
            for (int row = tile.row0 + warp; row < rend; row += nw) {
                const __nv_bfloat16* Ar = A + (int64_t)row * B.ld;
                float acc = 0.0f;
                for (int c = 8 * lane; c < B.ld; c += 256) acc += dot16b(Ar + c, xs + c);
                acc = warp_sumf(acc);
                if (lane == 0) out[row] = (double)acc;
            }
        }
    }
}

// ------------------------------------------------------------ permutations
// dst[internal e][j] = src[caller c][j] (to_internal = false reverses).
__global__ void permute_kernel(const double* __restrict__ src, double* __restrict__ dst,
                               const int64_t* __restrict__ to_caller, int64_t nc, int np,
                               int to_internal, const PcgScalars* zero_if_b0) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nc * np) return;
    const int64_t e = t / np, j = t - e * np, c = to_caller[e];
    if (to_internal) {
        dst[t] = src[c * np + j];
    } else {
        dst[c * np + j] = (zero_if_b0 && zero_if_b0->done == 2) ? 0.0 : src[t];
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
                D[((e - e0) * np + i) * L + (f - e0) * np + j] = val[(int64_t)bi * np * np + k];
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
                          const SimScalars* ss, double dt, double stim_duration,
                          cudaStream_t s) {
    const unsigned g = grid_for(K.nc * np);
    if (g > (unsigned)kMaxPartials) return cudaErrorInvalidValue;
    switch (mode) {
        case MODE_PLAIN:
            NP_SWITCH(np, bsr_matvec_kernel<NP, MODE_PLAIN><<<g, kBlock, 0, s>>>(
                K.row_ptr, K.col, val, x, y, K.nc, v1, v2, c1, c2, sc, partials, ss, dt, stim_duration));
            break;
        case MODE_PCG:
            NP_SWITCH(np, bsr_matvec_kernel<NP, MODE_PCG><<<g, kBlock, 0, s>>>(
                K.row_ptr, K.col, val, x, y, K.nc, v1, v2, c1, c2, sc, partials, ss, dt, stim_duration));
            break;
        case MODE_RESID:
            NP_SWITCH(np, bsr_matvec_kernel<NP, MODE_RESID><<<g, kBlock, 0, s>>>(
                K.row_ptr, K.col, val, x, y, K.nc, v1, v2, c1, c2, sc, partials, ss, dt, stim_duration));
            break;
        default:
            NP_SWITCH(np, bsr_matvec_kernel<NP, MODE_RHS><<<g, kBlock, 0, s>>>(
                K.row_ptr, K.col, val, x, y, K.nc, v1, v2, c1, c2, sc, partials, ss, dt, stim_duration));
            break;
    }
    return cudaGetLastError();
}

cudaError_t launch_update(double* x, double* r, const double* p, const double* q, int64_t n,
                          PcgScalars* sc, double* partials, cudaGraphConditionalHandle cond,
                          int use_cond, cudaStream_t s) {
    const unsigned g = grid_for(n);
    if (g > (unsigned)kMaxPartials) return cudaErrorInvalidValue;
    pcg_update_kernel<<<g, kBlock, 0, s>>>(x, r, p, q, n, sc, partials, cond, use_cond);
    return cudaGetLastError();
}

cudaError_t launch_direction(double* p, const double* z, int64_t n, const PcgScalars* sc,
                             cudaStream_t s) {
    pcg_direction_kernel<<<grid_for(n), kBlock, 0, s>>>(p, z, n, sc);
    return cudaGetLastError();
}

cudaError_t launch_identity_dots(const double* r, const double* q, int64_t n, PcgScalars* sc,
                                 double* partials, cudaStream_t s) {
    const unsigned g = grid_for(n);
    if (g > (unsigned)kMaxPartials) return cudaErrorInvalidValue;
    identity_dots_kernel<<<g, kBlock, 0, s>>>(r, q, n, sc, partials);
    return cudaGetLastError();
}

#define NQ_SWITCH(nq, ...)                                  \
    switch (nq) {                                           \
        case 3: { constexpr int NQ = 3; __VA_ARGS__; } break; \
        case 6: { constexpr int NQ = 6; __VA_ARGS__; } break; \
        case 10: { constexpr int NQ = 10; __VA_ARGS__; } break; \
        default: return cudaErrorInvalidValue;               \
    }

cudaError_t launch_restrict(int np, int nq, const double* r, const double* T,
                            const int64_t* agg_ptr, const int32_t* agg_cells, int n_agg,
                            double* r0, const int* done, cudaStream_t s) {
    const unsigned g = (unsigned)((n_agg * 32 + kBlock - 1) / kBlock);
    NP_SWITCH(np, NQ_SWITCH(nq, restrict_kernel<NP, NQ><<<g, kBlock, 0, s>>>(
                                    r, T, agg_ptr, agg_cells, n_agg, r0, done)));
    return cudaGetLastError();
}

cudaError_t launch_prolong(int np, int nq, double* z, const double* T, const int32_t* agg,
                           const double* y0, int64_t nc, const double* r, const double* q,
                           PcgScalars* sc, double* partials, cudaStream_t s) {
    const unsigned g = grid_for(nc * np);
    if (g > (unsigned)kMaxPartials) return cudaErrorInvalidValue;
    if (T == nullptr) nq = 3;   // no coarse space: only the dot products
    NP_SWITCH(np, NQ_SWITCH(nq, prolong_kernel<NP, NQ><<<g, kBlock, 0, s>>>(
                                    z, T, agg, y0, nc, r, q, sc, partials)));
    return cudaGetLastError();
}

cudaError_t launch_gemv(const GemvBlock* blocks, const GemvTile* tiles, int ntiles, int rows,
                        int max_ld, const double* st64, const float* st32,
                        const __nv_bfloat16* st16, const double* r, const double* r0,
                        double* z, double* y0, const int* done, cudaStream_t s) {
    if (ntiles == 0) return cudaSuccess;
    const size_t shm = (size_t)max_ld * sizeof(double);
    ragged_gemv_kernel<<<ntiles, kBlock, shm, s>>>(blocks, tiles, rows, st64, st32, st16, r, r0,
                                                   z, y0, done);
    return cudaGetLastError();
}

cudaError_t set_gemv_smem(int max_ld) {
    return cudaFuncSetAttribute(ragged_gemv_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)(max_ld * sizeof(double)));
}

cudaError_t launch_permute(const double* src, double* dst, const int64_t* to_caller, int64_t nc,
                           int np, int to_internal, const PcgScalars* zero_if_b0,
                           cudaStream_t s) {
    permute_kernel<<<grid_for(nc * np), kBlock, 0, s>>>(src, dst, to_caller, nc, np, to_internal,
                                                        zero_if_b0);
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
