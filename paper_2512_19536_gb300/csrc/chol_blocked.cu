// Blocked FP64 Cholesky factorisation and inversion of a large SPD matrix on the device
// (the coarse matrix K_0 of Sec. 4, Eq. prec, when the coarse space has thousands of
// DOFs: one CTA per matrix, as chol_inverse_kernel does for the local matrices, would take
// minutes there).
//
// The matrix is copied into an N x N work array, N = n rounded up to 64, with the identity
// on the padded diagonal, and processed in 64 x 64 tiles:
//   1. A = L L^T, right-looking: per block column k, the diagonal tile (one CTA), the
//      panel below it (L_ik = A_ik L_kk^{-T}, a CTA per tile) and the trailing update
//      A_ij -= L_ik L_jk^T (a CTA per tile of the lower triangle);
//   2. Y = L^{-1} by forward substitution on the identity, block row after block row:
//      Y_kJ = L_kk^{-1} Y_kJ (J <= k), then Y_iJ -= L_ik Y_kJ (i > k, J <= k);
//   3. X = L^{-T} Y by backward substitution, lower tiles only (A^{-1} is symmetric):
//      X_kJ = L_kk^{-T} X_kJ (J <= k), then X_iJ -= L_ki^T X_kJ (J <= i < k);
//   4. the strict upper triangle mirrored from the lower one.
// Each step is one launch on the stream; the tile products are FP64 SIMT GEMMs (GB300's
// FP64 tensor rate is no higher than its FP64 CUDA-core rate).  A non-positive pivot
// sets *status and leaves the result undefined.
#include <cstdint>

#include <cuda_runtime.h>

#include "kernels.h"

namespace polydg {

namespace {

constexpr int kTb = 64;            // tile order
constexpr int kTp = kTb + 1;       // padded shared-memory row (bank spread of doubles)
constexpr int kTt = 256;           // threads per CTA

__device__ __forceinline__ void load_tile(double (*s)[kTp], const double* A, int64_t lda, int ti, int tj) {
    const double* src = A + (int64_t)ti * kTb * lda + (int64_t)tj * kTb;
    for (int q = threadIdx.x; q < kTb * kTb; q += kTt) {
        const int r = q / kTb, c = q - r * kTb;
        s[r][c] = src[(int64_t)r * lda + c];
    }
}

__device__ __forceinline__ void store_tile(const double (*s)[kTp], double* A, int64_t lda, int ti, int tj) {
    double* dst = A + (int64_t)ti * kTb * lda + (int64_t)tj * kTb;
    for (int q = threadIdx.x; q < kTb * kTb; q += kTt) {
        const int r = q / kTb, c = q - r * kTb;
        dst[(int64_t)r * lda + c] = s[r][c];
    }
}

// Cholesky of diagonal tile k in place (lower triangle; the strict upper one zeroed).
__global__ void __launch_bounds__(kTt) potrf_tile_kernel(double* A, int64_t lda, int k, int* status) {
    __shared__ double s[kTb][kTp];
    __shared__ int bad;
    load_tile(s, A, lda, k, k);
    if (threadIdx.x == 0) bad = 0;
    __syncthreads();
    for (int j = 0; j < kTb; ++j) {
        if (threadIdx.x == 0) {
            const double d = s[j][j];
            if (!(d > 0.0)) bad = 1;
            s[j][j] = sqrt(fmax(d, 0.0));
        }
        __syncthreads();
        if (bad) break;
        const double ljj = s[j][j];
        for (int i = j + 1 + (int)threadIdx.x; i < kTb; i += kTt) s[i][j] /= ljj;
        __syncthreads();
        // trailing update of the tile: s[i][c] -= s[i][j] s[c][j], j < c <= i
        for (int q = threadIdx.x; q < kTb * kTb; q += kTt) {
            const int i = q / kTb, c = q - i * kTb;
            if (c > j && c <= i) s[i][c] -= s[i][j] * s[c][j];
        }
        __syncthreads();
    }
    if (bad) {
        if (threadIdx.x == 0) atomicExch(status, 1);
        return;
    }
    for (int q = threadIdx.x; q < kTb * kTb; q += kTt) {
        const int r = q / kTb, c = q - r * kTb;
        if (c > r) s[r][c] = 0.0;
    }
    __syncthreads();
    store_tile(s, A, lda, k, k);
}

// L_ik = A_ik L_kk^{-T} for the tiles i = k + 1 + blockIdx.x: row r of the tile solves
// L_kk x^T = a^T by forward substitution (one thread per row).
__global__ void __launch_bounds__(kTt) trsm_panel_kernel(double* A, int64_t lda, int k) {
    __shared__ double L[kTb][kTp], X[kTb][kTp];
    const int i = k + 1 + blockIdx.x;
    load_tile(L, A, lda, k, k);
    load_tile(X, A, lda, i, k);
    __syncthreads();
    const int r = threadIdx.x;
    if (r < kTb) {
        for (int c = 0; c < kTb; ++c) {
            double v = X[r][c];
            for (int m = 0; m < c; ++m) v -= X[r][m] * L[c][m];
            X[r][c] = v / L[c][c];
        }
    }
    __syncthreads();
    store_tile(X, A, lda, i, k);
}

// Forward step of Y = L^{-1}: Y_kJ = L_kk^{-1} Y_kJ for J = blockIdx.x <= k (column c of
// the tile by one thread: L_kk x = y by forward substitution).
__global__ void __launch_bounds__(kTt) trsm_fwd_kernel(const double* Lm, int64_t ldl, double* Y, int64_t ldy,
                                                       int k) {
    __shared__ double L[kTb][kTp], X[kTb][kTp];
    const int J = blockIdx.x;
    load_tile(L, Lm, ldl, k, k);
    load_tile(X, Y, ldy, k, J);
    __syncthreads();
    const int c = threadIdx.x;
    if (c < kTb) {
        for (int r = 0; r < kTb; ++r) {
            double v = X[r][c];
            for (int m = 0; m < r; ++m) v -= L[r][m] * X[m][c];
            X[r][c] = v / L[r][r];
        }
    }
    __syncthreads();
    store_tile(X, Y, ldy, k, J);
}

// Backward step of X = L^{-T} Y: X_kJ = L_kk^{-T} X_kJ for J = blockIdx.x <= k (L_kk^T x =
// y by backward substitution, one thread per column).
__global__ void __launch_bounds__(kTt) trsm_bwd_kernel(const double* Lm, int64_t ldl, double* Y, int64_t ldy,
                                                       int k) {
    __shared__ double L[kTb][kTp], X[kTb][kTp];
    const int J = blockIdx.x;
    load_tile(L, Lm, ldl, k, k);
    load_tile(X, Y, ldy, k, J);
    __syncthreads();
    const int c = threadIdx.x;
    if (c < kTb) {
        for (int r = kTb - 1; r >= 0; --r) {
            double v = X[r][c];
            for (int m = r + 1; m < kTb; ++m) v -= L[m][r] * X[m][c];
            X[r][c] = v / L[r][r];
        }
    }
    __syncthreads();
    store_tile(X, Y, ldy, k, J);
}

enum TileMode { TM_SYRK = 0, TM_FWD = 1, TM_BWD = 2 };

// C -= op(A) op(B) over the tiles of one step (a CTA per tile, thread (ty, tx) of a 16 x 16
// grid computes rows 4 ty .. 4 ty + 3 and columns 4 tx .. 4 tx + 3):
//   TM_SYRK  C = W_ij  -= L_ik L_jk^T  for k < j <= i < nt      (W holds L in its lower part)
//   TM_FWD   C = Y_iJ  -= L_ik Y_kJ    for k < i < nt, J <= k
//   TM_BWD   C = Y_iJ  -= L_ki^T Y_kJ  for J <= i < k
__global__ void __launch_bounds__(kTt) tile_update_kernel(const double* Lm, int64_t ldl, double* C, int64_t ldc,
                                                          int k, int nt, int mode) {
    __shared__ double As[kTb][kTp], Bs[kTb][kTp];
    int ti, tj, ai, aj, bi, bj;
    const int b = blockIdx.x;
    if (mode == TM_SYRK) {                 // lower-triangle tiles of [k+1, nt)^2, row by row
        int i = 0;
        while ((i + 1) * (i + 2) / 2 <= b) ++i;
        const int j = b - i * (i + 1) / 2;
        ti = k + 1 + i; tj = k + 1 + j;
        ai = ti; aj = k; bi = tj; bj = k;
    } else if (mode == TM_FWD) {           // (i, J), i in (k, nt), J in [0, k]
        const int i = b / (k + 1), J = b - i * (k + 1);
        ti = k + 1 + i; tj = J;
        ai = ti; aj = k; bi = k; bj = J;
    } else {                               // (i, J), J <= i < k: lower-triangle tiles of [0, k)^2
        int i = 0;
        while ((i + 1) * (i + 2) / 2 <= b) ++i;
        const int J = b - i * (i + 1) / 2;
        ti = i; tj = J;
        ai = k; aj = i; bi = k; bj = J;
    }
    load_tile(As, Lm, ldl, ai, aj);
    load_tile(Bs, mode == TM_SYRK ? Lm : C, mode == TM_SYRK ? ldl : ldc, bi, bj);
    __syncthreads();
    const int ty = threadIdx.x >> 4, tx = threadIdx.x & 15;
    double acc[4][4] = {};
    for (int m = 0; m < kTb; ++m) {
        double a[4], bb[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int r = 4 * ty + u, c = 4 * tx + u;
            a[u] = mode == TM_BWD ? As[m][r] : As[r][m];          // op(A)[r][m]
            bb[u] = mode == TM_SYRK ? Bs[c][m] : Bs[m][c];        // op(B)[m][c]
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int v = 0; v < 4; ++v) acc[u][v] = fma(a[u], bb[v], acc[u][v]);
    }
    double* dst = C + (int64_t)ti * kTb * ldc + (int64_t)tj * kTb;
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            const int r = 4 * ty + u, c = 4 * tx + v;
            dst[(int64_t)r * ldc + c] -= acc[u][v];
        }
}

// Padded copy: W (N x N) = [A 0; 0 I], Y = I.
__global__ void pad_copy_kernel(const double* A, int64_t lda, int n, double* W, double* Y, int N) {
    const int64_t total = (int64_t)N * N;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
        const int r = (int)(q / N), c = (int)(q - (int64_t)r * N);
        W[q] = (r < n && c < n) ? A[(int64_t)r * lda + c] : (r == c ? 1.0 : 0.0);
        Y[q] = r == c ? 1.0 : 0.0;
    }
}

// Out (n x n, leading dimension ldo) = the inverse: lower tiles of Y, the upper part mirrored.
__global__ void unpad_sym_kernel(const double* Y, int N, double* out, int64_t ldo, int n) {
    const int64_t total = (int64_t)n * n;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
        const int r = (int)(q / n), c = (int)(q - (int64_t)r * n);
        const bool lower = (r / kTb) >= (c / kTb);     // tiles J <= i were computed
        out[(int64_t)r * ldo + c] = lower ? Y[(int64_t)r * N + c] : Y[(int64_t)c * N + r];
    }
}

}  // namespace

int64_t chol_blocked_work_doubles(int n) {
    const int64_t N = (int64_t)(n + kTb - 1) / kTb * kTb;
    return 2 * N * N;
}

cudaError_t launch_chol_blocked_inverse(const double* A, int64_t lda, int n, double* out, int64_t ldo,
                                        double* work, int* status, cudaStream_t s) {
    const int nt = (n + kTb - 1) / kTb, N = nt * kTb;
    double* W = work;
    double* Y = work + (int64_t)N * N;
    pad_copy_kernel<<<1024, 256, 0, s>>>(A, lda, n, W, Y, N);
    for (int k = 0; k < nt; ++k) {
        potrf_tile_kernel<<<1, kTt, 0, s>>>(W, N, k, status);
        const int m = nt - k - 1;
        if (m > 0) {
            trsm_panel_kernel<<<m, kTt, 0, s>>>(W, N, k);
            tile_update_kernel<<<m * (m + 1) / 2, kTt, 0, s>>>(W, N, W, N, k, nt, TM_SYRK);
        }
    }
    for (int k = 0; k < nt; ++k) {
        trsm_fwd_kernel<<<k + 1, kTt, 0, s>>>(W, N, Y, N, k);
        if (k + 1 < nt) tile_update_kernel<<<(nt - k - 1) * (k + 1), kTt, 0, s>>>(W, N, Y, N, k, nt, TM_FWD);
    }
    for (int k = nt - 1; k >= 0; --k) {
        trsm_bwd_kernel<<<k + 1, kTt, 0, s>>>(W, N, Y, N, k);
        if (k > 0) tile_update_kernel<<<k * (k + 1) / 2, kTt, 0, s>>>(W, N, Y, N, k, nt, TM_BWD);
    }
    unpad_sym_kernel<<<1024, 256, 0, s>>>(Y, N, out, ldo, n);
    return cudaGetLastError();
}

}  // namespace polydg
