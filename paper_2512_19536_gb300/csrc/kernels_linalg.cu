// Linear-algebra kernels of libpolydg outside the persistent PCG kernel: the
// block-sparse matvec y = K_h x (polydg_matvec) and the right-hand side of a time step
// (Eq. fully-discrete-1), the caller <-> internal permutations, and the setup kernels
// (extraction of the dense K_i, batched Cholesky inversion of K_i and K_0, the reduced-
// precision copies of the local inverses).  The PCG iteration itself -- matvec, local
// and coarse solves, vector algebra -- runs in kernels_pcg.cu.
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
//   MODE_RHS:   y = Kminus x + c1 v1 + c2 [t^{k+1/2} < t_stim] v2.
constexpr int kElemsPerCta = kBlock / 64;

template <int NP, int MODE>
__global__ void __launch_bounds__(kBlock)
matvec_kernel(const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
              const double* __restrict__ val, const double* __restrict__ x,
              double* __restrict__ y, int64_t nc, const double* __restrict__ v1,
              const double* __restrict__ v2, double c1, double c2, const SimScalars* ss,
              double dt, double stim_duration) {
    constexpr int G = 32 / NP;
    __shared__ double half[kElemsPerCta][32];
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
            const double w1 = __ldg(V + (int64_t)c * NP + i), w2 = __ldg(V + (int64_t)c2 * NP + i);
            const double x1 = __ldg(x + (int64_t)__ldg(cl + s1) * NP + (c - s1 * NP));
            const double x2 = __ldg(x + (int64_t)__ldg(cl + s2) * NP + (c2 - s2 * NP));
            acc0 = fma(w1, x1, acc0);
            acc1 = fma(w2, x2, acc1);
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
    if (valid && h == 0 && lane < NP) {
        const int64_t t = e * NP + i;
        if (MODE == MODE_PLAIN) {
            y[t] = acc;
        } else {
            const double tmid = ((double)ss->k + 0.5) * dt;
            const double on = (tmid < stim_duration) ? 1.0 : 0.0;
            y[t] = acc + c1 * v1[t] + c2 * on * v2[t];
        }
    }
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
                          double c1, double c2, const SimScalars* ss, double dt,
                          double stim_duration, cudaStream_t s) {
    const unsigned g = (unsigned)((K.nc + kElemsPerCta - 1) / kElemsPerCta);
#define MV(M)                                                                                  \
    NP_SWITCH(np, matvec_kernel<NP, M><<<g, kBlock, 0, s>>>(K.row_ptr, K.col, val, x, y, K.nc, v1, \
                                                            v2, c1, c2, ss, dt, stim_duration))
    if (mode == MODE_PLAIN) {
        MV(MODE_PLAIN);
    } else {
        MV(MODE_RHS);
    }
#undef MV
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
