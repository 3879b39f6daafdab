// Device-side data structures and helpers of libpolydg (sm_103a).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>
#include <cuda_bf16.h>

namespace polydg {

constexpr int kBlock = 256;            // threads per CTA of the streaming kernels
constexpr int kPersistThreads = 512;   // threads per CTA of the persistent PCG kernel
constexpr int kMaxPartials = 1 << 15;  // partial sums per reduction (>= max grid)

// Scalars of one PCG solve, resident in device memory.  Reductions write
// per-CTA partials; the last CTA of a launch (ticket counter) sums them in
// CTA order, so every result is deterministic.
struct PcgScalars {
    double bb;        // |b|^2
    double rr;        // |r_k|^2
    double rz;        // r_k . z_k
    double rz_loc;    // r_k . (sum_i R_i^T K_i^{-1} R_i r_k)   (local part of r.z)
    double zq;        // z_{k+1} . q_k (flexible beta)
    double zq_loc;
    double pq;        // p_k . K p_k
    double alpha, beta;
    double rtol2;     // rtol^2
    double relres;
    int32_t it;       // committed iterations
    int32_t maxit, status, done, flexible;
    int32_t pass;     // loop passes; x and r live in buffer (pass & 1)
    int32_t alpha_valid;
    int32_t pad;
    uint32_t ticket[8];
};

enum Ticket { T_MATVEC = 0, T_K1 = 1, T_COARSE = 2, T_INIT = 3 };

// status values mirrored from polydg.h
constexpr int kOK = 0, kEDEVICE = -3, kENOTSPD = -4, kENOTCONV = -5, kEBREAKDOWN = -6, kENONFINITE = -7;

// One dense block of the ragged preconditioner kernel (Eq. prec).
//   LOCAL:    rows [0, nrows) of K_i^{-1}; in = out = the subdomain's DOF range.
//   RESTRICT: the n_q rows of R_0 restricted to the DOFs of one (agglomerate,
//             subdomain) pair; out_off indexes the pair's partial sums.
//   IDENTITY: z = r on a DOF range (unpreconditioned CG).
// Matrices are row-major with leading dimension ld (zero-padded to a multiple
// of 8 columns); mat_off counts elements of the store of the block's dtype.
enum TileKind { KIND_LOCAL = 0, KIND_RESTRICT = 1, KIND_IDENTITY = 2 };

struct GemvBlock {
    int64_t mat_off;
    int64_t in_off, out_off;
    int32_t nrows, ncols, ld;
    int32_t kind;
    int32_t dtype;        // 0 fp64, 1 fp32, 2 bf16
    int32_t pair_begin;   // LOCAL: first entry of its RESTRICT blocks in the sub_pairs list
    int32_t pair_count;   // LOCAL: number of (agglomerate, subdomain) pairs of this subdomain
    int32_t sym_off;      // LOCAL, fp32 stores: first float of its pair rows in the symmetric store
};

// Symmetric pair-row store of an n x n local inverse (the P phase of the persistent PCG
// kernel with fp32 stores): pair m < (n + 1) / 2 holds row m of the lower triangle
// (columns 0..m, zero-padded to a multiple of 4), then row n - 1 - m (columns 0..n-1-m,
// zero-padded likewise; empty when n - 1 - m == m), diagonal entries halved.  Pair rows sit sym_ld(n) floats
// apart; a copy of pair m carries sym_len(n, m) floats (16-byte multiples throughout).
__host__ __device__ __forceinline__ int sym_ld(int n) { return (n + 10) & ~3; }
__host__ __device__ __forceinline__ int sym_len(int n, int m) {
    return ((m + 4) & ~3) + (n - 1 - m != m ? ((n - m + 3) & ~3) : 0);
}
constexpr int kSymT = 5;                      // float4 column groups per lane: n <= 128 kSymT

struct GemvTile {
    int32_t block;
    int32_t row0;
};

// Rows [row_begin, row_end) of one LOCAL block, streamed by one CTA of the
// persistent PCG kernel in tiles of `rows` rows.
struct GemvRun {
    int32_t block;
    int32_t row_begin, row_end;
    int32_t pad;
};

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ float warp_sumf(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Sum over the CTA; result valid in every thread.  `sh` holds >= 32 doubles.
__device__ __forceinline__ double block_sum(double v, double* sh) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    v = warp_sum(v);
    __syncthreads();
    if (lane == 0) sh[w] = v;
    __syncthreads();
    double t = (threadIdx.x < nw) ? sh[threadIdx.x] : 0.0;
    if (w == 0) t = warp_sum(t);
    if (threadIdx.x == 0) sh[0] = t;
    __syncthreads();
    const double r = sh[0];
    __syncthreads();
    return r;
}

// Publish this CTA's partial(s) and return true in the last CTA to arrive.
// In the last CTA, partials of all CTAs are visible after the call.
__device__ __forceinline__ bool publish_partials(double* partials, const double* mine, int k,
                                                 uint32_t* ticket, bool* sh_last) {
    if (threadIdx.x == 0) {
        for (int i = 0; i < k; ++i) partials[i * kMaxPartials + blockIdx.x] = mine[i];
        __threadfence();
        const uint32_t t = atomicAdd(ticket, 1u);
        *sh_last = (t == gridDim.x - 1);
    }
    __syncthreads();
    const bool last = *sh_last;
    if (last) __threadfence();
    return last;
}

// Deterministic sum of partials[0..n) by one CTA (fixed order).
__device__ __forceinline__ double sum_partials(const double* partials, int n, double* sh) {
    double v = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) v += __ldcg(partials + i);
    return block_sum(v, sh);
}

__device__ __forceinline__ bool finite(double x) { return isfinite(x); }

}  // namespace polydg
