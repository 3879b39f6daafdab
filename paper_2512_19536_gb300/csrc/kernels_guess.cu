// Learned PCG initial guess: per-element network, its training, and the safeguard.
//
// Features of element e from the last three solutions (own values, elementwise mean and
// max over the face neighbours, cell size, time step, neighbour count: 9 n_p + 3 inputs),
// two ReLU hidden layers of width kGuessHidden, a linear output of n_p values o; the
// proposal is x0 = U^k + s_d o, kept only if |b - K x0|_2 < |b - K U^k|_2.  Training
// minimises the mean squared error to (U^{k+1} - U^k) / s_d with Adam.
//
// Inference: guess_tc.cu (tensor cores, FP16 operands, FP32 accumulation).
// Training: fp32 weights (master copy), activations and gradients; per-CTA partial
// gradients summed in CTA order (deterministic), then one Adam update per parameter.
#include <algorithm>

#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "device.cuh"
#include "guess_features.cuh"
#include "kernels.h"

namespace polydg {

constexpr int kGT = 32;                   // elements (samples) per tile
constexpr int kGThreads = 256;
constexpr int kH = kGuessHidden;          // 128
constexpr int kHP = kH + 1;               // padded row stride of transposed weights

// Offsets of the parameter groups in the flat (canonical) layout.
struct ParamOffsets {
    int w1, b1, w2, b2, w3, b3, total;
};
__host__ __device__ inline ParamOffsets param_offsets(int np) {
    const int F = guess_inputs(np);
    ParamOffsets o;
    o.w1 = 0;
    o.b1 = o.w1 + kH * F;
    o.w2 = o.b1 + kH;
    o.b2 = o.w2 + kH * kH;
    o.w3 = o.b2 + kH;
    o.b3 = o.w3 + np * kH;
    o.total = o.b3 + np;
    return o;
}

int guess_param_count(int np) { return param_offsets(np).total; }

// Shared-memory image of the weights: transposed, rows padded to kHP (conflict-free
// both for the forward pass, thread j reading W[j][i], and the backward pass, thread i
// reading W[j][i]):  W1t[i * kHP + j] = W1[j][i] (i < F),  W2t[i * kHP + j] = W2[j][i],
// W3t[i * n_p + c] = W3[c][i]; biases as is.
__host__ __device__ inline size_t guess_weights_bytes16(int np) {
    const int F = guess_inputs(np);
    return ((size_t)(F * kHP + kH * kHP + kH * np) * 2 + 15) / 16 * 16;
}

template <typename W, typename S>
__device__ __forceinline__ void stage_weights(const S* __restrict__ src, int np, W* w1t, W* w2t, W* w3t,
                                              float* b1, float* b2, float* b3) {
    const ParamOffsets o = param_offsets(np);
    const int F = guess_inputs(np);
    for (int q = threadIdx.x; q < kH * F; q += blockDim.x) {      // W1[j][i], q = j F + i
        const int j = q / F, i = q - j * F;
        w1t[i * kHP + j] = (W)(float)src[o.w1 + q];
    }
    for (int q = threadIdx.x; q < kH * kH; q += blockDim.x) {
        const int j = q / kH, i = q - j * kH;
        w2t[i * kHP + j] = (W)(float)src[o.w2 + q];
    }
    for (int q = threadIdx.x; q < np * kH; q += blockDim.x) {     // W3[c][i]
        const int c = q / kH, i = q - c * kH;
        w3t[i * np + c] = (W)(float)src[o.w3 + q];
    }
    for (int q = threadIdx.x; q < kH; q += blockDim.x) {
        b1[q] = (float)src[o.b1 + q];
        b2[q] = (float)src[o.b2 + q];
    }
    for (int q = threadIdx.x; q < np; q += blockDim.x) b3[q] = (float)src[o.b3 + q];
}

// Dense layer out[s][j] = act(b[j] + sum_i Wt[i * kHP + j] in[s][i]) for the tile's
// kGT samples: thread (j, half) computes 16 samples of hidden unit j.
template <typename W, bool RELU>
__device__ __forceinline__ void hidden_layer(const W* wt, const float* b, const float* in, int n_in,
                                             float* out) {
    const int j = threadIdx.x & (kH - 1), s0 = (threadIdx.x >> 7) * 16;
    float acc[16];
#pragma unroll
    for (int s = 0; s < 16; ++s) acc[s] = b[j];
    for (int i = 0; i < n_in; ++i) {
        const float w = (float)wt[i * kHP + j];
#pragma unroll
        for (int s = 0; s < 16; ++s) acc[s] = fmaf(w, in[(s0 + s) * n_in + i], acc[s]);
    }
#pragma unroll
    for (int s = 0; s < 16; ++s) out[(s0 + s) * kH + j] = RELU ? fmaxf(acc[s], 0.f) : acc[s];
}

// o[s * NP + c] = b3[c] + sum_i W3[c][i] h2[s][i].
template <typename W, int NP>
__device__ __forceinline__ void output_layer(const W* w3t, const float* b3, const float* h2, float* o) {
    for (int q = threadIdx.x; q < kGT * NP; q += blockDim.x) {
        const int s = q / NP, c = q - s * NP;
        float acc = b3[c];
        for (int i = 0; i < kH; ++i) acc = fmaf((float)w3t[i * NP + c], h2[s * kH + i], acc);
        o[q] = acc;
    }
}

// ------------------------------------------------------------------ safeguard
// |b - K xg|^2 and |b - K U^k|^2 (warp per element, K_h read once), then the last CTA
// (ticket) keeps the guess if its residual is strictly smaller.
template <int NP>
__global__ void __launch_bounds__(kBlock)
guess_select_kernel(const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
                    const double* __restrict__ val, const double* __restrict__ b,
                    const double* __restrict__ xg, const double* __restrict__ uk, int64_t nc,
                    double* partials, SimScalars* ss, int policy) {
    if (ss->failed || ss->k < 2) return;
    if (policy == 1) {                            // start from every proposal
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            ss->theta = 1.0;
            ss->use_guess = 1;
            ss->guesses_taken += 1;
        }
        return;
    }
    const bool damped = policy == 2;
    __shared__ double sh[32];
    __shared__ bool last;
    constexpr int G = 32 / NP;
    const int lane = threadIdx.x & 31;
    const int64_t e = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int g = (lane < G * NP) ? lane / NP : G;
    const int i = lane - (lane / NP) * NP;
    double ag = 0.0, a0 = 0.0;
    if (e < nc) {
        const int32_t b0 = row_ptr[e];
        const int ncol = (row_ptr[e + 1] - b0) * NP;
        const double* V = val + (int64_t)b0 * NP * NP;
        for (int c = g; c < ncol; c += G) {
            const int sblk = c / NP;
            const int64_t xi = (int64_t)__ldg(col + b0 + sblk) * NP + (c - sblk * NP);
            const double v = __ldg(V + (int64_t)c * NP + i);
            ag = fma(v, __ldg(xg + xi), ag);
            a0 = fma(v, __ldg(uk + xi), a0);
        }
    }
    double tg = ag, t0 = a0;
#pragma unroll
    for (int k = 1; k < G; ++k) {
        tg += __shfl_down_sync(0xffffffffu, ag, k * NP);
        t0 += __shfl_down_sync(0xffffffffu, a0, k * NP);
    }
    double dg = 0.0, d0 = 0.0, dx = 0.0;
    if (e < nc && lane < NP) {
        const double bv = b[e * NP + i];
        dg = (bv - tg) * (bv - tg);
        d0 = (bv - t0) * (bv - t0);
        dx = (bv - t0) * (bv - tg);
    }
    double s[3];
    s[0] = block_sum(dg, sh);
    s[1] = block_sum(d0, sh);
    s[2] = block_sum(dx, sh);
    if (publish_partials(partials, s, 3, &ss->guess_ticket, &last)) {
        const double rg = sum_partials(partials, gridDim.x, sh);
        const double r0 = sum_partials(partials + kMaxPartials, gridDim.x, sh);
        const double rx = sum_partials(partials + 2 * kMaxPartials, gridDim.x, sh);
        if (threadIdx.x == 0) {
            ss->guess_ticket = 0;
            if (damped) {
                // x0 = U^k + theta (xg - U^k); with K d = r0 - rg the residual b - K x0 =
                // r0 - theta K d is smallest at theta = r0.Kd / Kd.Kd (never above |r0|)
                const double kd2 = r0 - 2.0 * rx + rg, r0kd = r0 - rx;
                const double th = (kd2 > 0.0 && isfinite(kd2) && isfinite(r0kd)) ? r0kd / kd2 : 0.0;
                ss->theta = th;
                ss->use_guess = th != 0.0 ? 1 : 0;
                ss->guesses_taken += th != 0.0 ? 1 : 0;
            } else {
                ss->theta = 1.0;
                ss->use_guess = (rg < r0) ? 1 : 0;
                ss->guesses_taken += (rg < r0) ? 1 : 0;
            }
        }
    }
}

// x0 = U^k + theta (guess - U^k) if the guess was kept, else U^k.
__global__ void select_copy_kernel(const double* __restrict__ uk, const double* __restrict__ xg,
                                   double* __restrict__ x0, int64_t n, const SimScalars* ss) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (ss->failed || t >= n) return;
    x0[t] = ss->use_guess ? fma(ss->theta, xg[t] - uk[t], uk[t]) : uk[t];
}

// ------------------------------------------------------------------ subspace guess
// Policy 3: x0 = U^k + sum_d theta_d v_d over the directions v_0 = xg - U^k (the learned
// proposal, from k = 2 on, when a model is attached) and v_j = D_{k-j+1} for the last m
// solution increments D_i = U^i - U^{i-1}, theta the Galerkin projection of the correction
// onto their span (minimum of the K-norm of the error x* - x0, the norm CG minimises):
// V^T K V theta = V^T r0 with r0 = b - K U^k.  K v_j needs no pass over K_h: each step
// multiplies its newest increment D_k once and keeps K D_k in a second ring (slot k mod
// kHistRing, like U^k).  The increment is formed exactly (the difference of two nearby
// doubles), so its product carries only the product's own rounding, unlike a difference
// of the products K U^i.  m = min(kHistDirs, hist_len - 1, kd_len).  The direction list
// depends only on (k, hist_len, kd_len, model attached): every kernel after the ring
// update rebuilds the same list.
struct SubDirs {
    const double* a[kSubMaxDirs];        // v_d = a_d - b_d
    const double* b[kSubMaxDirs];
    const double* kv[kSubMaxDirs];       // K v_d
};

__device__ __forceinline__ int subspace_dirs(const SimScalars* ss, const double* U, const double* xg,
                                             const double* ring, const double* kdring, const double* kxg,
                                             int64_t n, SubDirs& D) {
    const int64_t k = ss->k;
    const int m = min(min(kHistDirs, ss->hist_len - 1), ss->kd_len);
    int nd = 0;
    if (xg != nullptr && k >= 2) { D.a[nd] = xg; D.b[nd] = U; D.kv[nd] = kxg; ++nd; }
    for (int j = 1; j <= m; ++j) {
        D.a[nd] = (j == 1) ? U : ring + ((k - j + 1) % kHistRing) * n;
        D.b[nd] = ring + ((k - j) % kHistRing) * n;
        D.kv[nd] = kdring + ((k - j + 1) % kHistRing) * n;
        ++nd;
    }
    return nd;
}

// y_v = K (x_v - w_v) for up to NV vectors (w_v may be null), warp per element row block;
// the differences are formed per entry before the product.
template <int NP, int NV>
__device__ __forceinline__ void multi_matvec_row(const int32_t* __restrict__ row_ptr,
                                                 const int32_t* __restrict__ col,
                                                 const double* __restrict__ val, int64_t e,
                                                 const double* const* x, const double* const* w,
                                                 int nv, double* t) {
    constexpr int G = 32 / NP;
    const int lane = threadIdx.x & 31;
    const int g = lane / NP, i = lane - g * NP;
    double a[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) a[v] = 0.0;
    const int32_t b0 = row_ptr[e];
    const int ncol = (row_ptr[e + 1] - b0) * NP;
    const double* V = val + (int64_t)b0 * NP * NP;
    if (g < G)
        for (int c = g; c < ncol; c += G) {
            const int sblk = c / NP;
            const int64_t xi = (int64_t)__ldg(col + b0 + sblk) * NP + (c - sblk * NP);
            const double kv = __ldg(V + (int64_t)c * NP + i);
#pragma unroll
            for (int v = 0; v < NV; ++v)
                if (v < nv) a[v] = fma(kv, __ldcg(x[v] + xi) - (w[v] ? __ldcg(w[v] + xi) : 0.0), a[v]);
        }
#pragma unroll
    for (int v = 0; v < NV; ++v) {
        double s = a[v];
#pragma unroll
        for (int k = 1; k < G; ++k) s += __shfl_down_sync(0xffffffffu, a[v], k * NP);
        t[v] = s;
    }
}

// W[0] = r0 = b - K U^k, K D_k = K (U^k - U^{k-1}) into the increment-product ring (slot k,
// from k = 1 on), W[1] = K (xg - U^k) (with a model).
template <int NP>
__global__ void __launch_bounds__(kBlock)
subspace_rows_kernel(const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
                     const double* __restrict__ val, const double* __restrict__ b,
                     const double* __restrict__ U, const double* xg, const double* ring,
                     double* __restrict__ kdring, double* __restrict__ W, int64_t n, int64_t nc,
                     SimScalars* ss) {
    if (ss->failed) return;
    const int64_t k = ss->k;
    const bool inc = ss->hist_len >= 2;          // U^{k-1} is in the ring
    const int lane = threadIdx.x & 31;
    const int64_t e = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (e < nc) {
        const double* Um1 = ring + ((k + kHistRing - 1) % kHistRing) * n;
        const double* x[3] = {U, inc ? U : U, xg};
        const double* w[3] = {nullptr, inc ? Um1 : nullptr, U};
        int nv = 1;
        double t[3];
        if (inc) nv = 2;
        if (xg != nullptr) { x[nv] = xg; w[nv] = U; ++nv; }
        multi_matvec_row<NP, 3>(row_ptr, col, val, e, x, w, nv, t);
        if (lane < NP) {
            const int64_t r = e * NP + lane;
            W[r] = b[r] - t[0];
            if (inc) kdring[(k % kHistRing) * n + r] = t[1];
            if (xg != nullptr) W[n + r] = t[nv - 1];
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {      // the product ring now reaches step k
        ss->kd_len = !inc ? 0 : (ss->kd_step == k - 1 ? min(ss->kd_len + 1, kHistDirs) : 1);
        ss->kd_step = k;
    }
}

// Restored history: K D_{k-h} = K (U^{k-h} - U^{k-h-1}) for h = 1 .. hist_len - 2 into the
// increment-product ring (the step's own rows kernel adds K D_k).
template <int NP>
__global__ void __launch_bounds__(kBlock)
history_products_kernel(const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
                        const double* __restrict__ val, const double* __restrict__ ring,
                        double* __restrict__ kdring, int64_t n, int64_t nc, SimScalars* ss) {
    const int64_t k = ss->k;
    const int np_ = max(0, ss->hist_len - 2);      // increments D_{k-1} .. D_{k-np_}
    const int lane = threadIdx.x & 31;
    const int64_t e = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (e < nc && np_ > 0) {
        const double* x[kHistDirs];
        const double* w[kHistDirs];
        for (int h = 0; h < kHistDirs; ++h) {
            const int hh = 1 + min(h, np_ - 1);
            x[h] = ring + ((k - hh) % kHistRing) * n;
            w[h] = ring + ((k - hh - 1) % kHistRing) * n;
        }
        double t[kHistDirs];
        multi_matvec_row<NP, kHistDirs>(row_ptr, col, val, e, x, w, np_, t);
        if (lane < NP) {
            const int64_t r = e * NP + lane;
#pragma unroll
            for (int h = 0; h < kHistDirs; ++h)
                if (h < np_) kdring[((k - 1 - h) % kHistRing) * n + r] = t[h];
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {   // as if steps k-np_ .. k-1 had stored theirs
        ss->kd_len = np_;
        ss->kd_step = k - 1;
    }
}

// The dot products c_d = v_d . r0 and H_ij = v_i . K v_j (i <= j), per-CTA partial sums in
// fixed row order; the last CTA adds them in CTA order and solves for theta by elimination
// on the directions whose Schur-complement pivots stay above 1e-13 of the largest diagonal
// (greedy, largest pivot first), the others left at zero.  The guess is used when it
// lowers the K-norm of the error (gain c.theta > 0).
constexpr int kGramThreads = 512;       // one thread per (i <= j) pair and per c_i: up to 350
constexpr int kGramRows = 64;           // rows per shared-memory tile

__global__ void __launch_bounds__(kGramThreads)
subspace_gram_kernel(const double* __restrict__ W, const double* U, const double* xg,
                     const double* ring, const double* kdring, int64_t n, double* gram,
                     SimScalars* ss) {
    __shared__ double tile[2 * kSubMaxDirs + 1][kGramRows + 1];   // r0, K v_d, v_d
    __shared__ double Gs[kSubMaxPairs];
    __shared__ SubDirs D;
    __shared__ int snd;
    __shared__ bool last;
    if (ss->failed) return;
    if (threadIdx.x == 0) snd = subspace_dirs(ss, U, xg, ring, kdring, W + n, n, D);
    __syncthreads();
    const int nd = snd;
    if (nd == 0) {
        if (blockIdx.x == 0 && threadIdx.x == 0) ss->use_guess = 0;
        return;
    }
    const int npair = nd + nd * (nd + 1) / 2;
    int pi = 0, pj = 0;                  // tile rows multiplied by thread p
    if (threadIdx.x < npair) {
        int p = threadIdx.x;
        if (p < nd) {                    // c_p = v_p . r0
            pi = 1 + nd + p;
            pj = 0;
        } else {                         // H_ij = v_i . K v_j, i <= j
            p -= nd;
            int i2 = 0;
            while (p >= nd - i2) { p -= nd - i2; ++i2; }
            pi = 1 + nd + i2;
            pj = 1 + i2 + p;
        }
    }
    double acc = 0.0;
    const int nrow = 1 + 2 * nd;
    for (int64_t r0 = (int64_t)blockIdx.x * kGramRows; r0 < n; r0 += (int64_t)gridDim.x * kGramRows) {
        for (int idx = threadIdx.x; idx < nrow * kGramRows; idx += kGramThreads) {
            const int v = idx / kGramRows, q = idx - v * kGramRows;
            const int64_t r = r0 + q;
            double x = 0.0;
            if (r < n) {
                if (v == 0) x = __ldcg(W + r);
                else if (v <= nd) x = __ldcg(D.kv[v - 1] + r);
                else x = __ldcg(D.a[v - 1 - nd] + r) - __ldcg(D.b[v - 1 - nd] + r);
            }
            tile[v][q] = x;
        }
        __syncthreads();
        if (threadIdx.x < npair)
            for (int q = 0; q < kGramRows; ++q) acc = fma(tile[pi][q], tile[pj][q], acc);
        __syncthreads();
    }
    if (threadIdx.x < npair) gram[threadIdx.x * kSubMaxCtas + blockIdx.x] = acc;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(&ss->guess_ticket, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!last) return;
    __threadfence();
    if (threadIdx.x < npair) {           // eight independent chains, combined in a fixed order
        double part[8] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
        const double* src = gram + threadIdx.x * kSubMaxCtas;
        unsigned c = 0;
        for (; c + 8 <= gridDim.x; c += 8)
#pragma unroll
            for (int q = 0; q < 8; ++q) part[q] += __ldcg(src + c + q);
        for (; c < gridDim.x; ++c) part[0] += __ldcg(src + c);
        Gs[threadIdx.x] = ((part[0] + part[1]) + (part[2] + part[3])) + ((part[4] + part[5]) + (part[6] + part[7]));
    }
    __syncthreads();
    // Symmetric elimination with greedy diagonal pivoting on H = V^T K V, c = V^T r0, all
    // threads sharing each pivot's rank-one update; the pivot rows as eliminated give
    // theta by back substitution.  Directions never chosen as pivots keep theta = 0.
    __shared__ double sA[kSubMaxDirs][kSubMaxDirs + 1], sR[kSubMaxDirs][kSubMaxDirs + 1];
    __shared__ double sc[kSubMaxDirs], sc0[kSubMaxDirs], sD[kSubMaxDirs], sdmax;
    __shared__ int ssel[kSubMaxDirs], sused[kSubMaxDirs], sq, sok;
    auto pair = [&](int i, int j) { return nd + i * nd - i * (i - 1) / 2 + (j - i); };   // i <= j
    for (int idx = threadIdx.x; idx < nd * nd; idx += blockDim.x) {
        const int i = idx / nd, j = idx - i * nd;
        sA[i][j] = Gs[i <= j ? pair(i, j) : pair(j, i)];
    }
    if (threadIdx.x < nd) {
        sc[threadIdx.x] = sc0[threadIdx.x] = Gs[threadIdx.x];
        sused[threadIdx.x] = 0;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        ss->guess_ticket = 0;
        double dmax = 0.0;
        bool ok = true;
        for (int d = 0; d < nd; ++d) {
            dmax = fmax(dmax, sA[d][d]);
            ok = ok && isfinite(sA[d][d]) && isfinite(sc[d]);
        }
        sdmax = dmax;
        sok = (ok && isfinite(dmax) && dmax > 0.0) ? 1 : 0;
    }
    __syncthreads();
    int ns = 0;
    while (sok && ns < nd) {
        if (threadIdx.x == 0) {
            int q = -1;
            double best = 1e-13 * sdmax;
            for (int d = 0; d < nd; ++d)
                if (!sused[d] && sA[d][d] > best) { best = sA[d][d]; q = d; }
            sq = q;
            if (q >= 0) { sused[q] = 1; ssel[ns] = q; sD[ns] = sA[q][q]; }
        }
        __syncthreads();
        const int q = sq;
        if (q < 0) break;
        for (int j = threadIdx.x; j < nd; j += blockDim.x) sR[ns][j] = sA[q][j];
        __syncthreads();
        const double inv = 1.0 / sD[ns], cq = sc[q];
        for (int idx = threadIdx.x; idx < nd * nd; idx += blockDim.x) {
            const int i = idx / nd, j = idx - i * nd;
            if (!sused[i] && !sused[j]) sA[i][j] -= sR[ns][i] * sR[ns][j] * inv;
        }
        if (threadIdx.x < nd && !sused[threadIdx.x]) sc[threadIdx.x] -= sR[ns][threadIdx.x] * cq * inv;
        ++ns;
        __syncthreads();
    }
    if (threadIdx.x != 0) return;
    double th[kSubMaxDirs];
    for (int d = 0; d < kSubMaxDirs; ++d) th[d] = 0.0;
    for (int t = ns - 1; t >= 0; --t) {
        const int q = ssel[t];
        double v = sc[q];
        for (int u = t + 1; u < ns; ++u) v -= sR[t][ssel[u]] * th[ssel[u]];
        th[q] = v / sD[t];
    }
    double gain = 0.0;
    for (int d = 0; d < nd; ++d) gain += sc0[d] * th[d];
    const bool use = sok && ns > 0 && isfinite(gain) && gain > 0.0;
    for (int d = 0; d < kSubMaxDirs; ++d) ss->theta_sub[d] = (use && d < nd) ? th[d] : 0.0;
    ss->sub_dirs = use ? nd : 0;
    ss->use_guess = use ? 1 : 0;
    ss->guesses_taken += use ? 1 : 0;
}

// x0 = U^k + sum_d theta_d v_d when the subspace guess is used, else U^k.
__global__ void subspace_copy_kernel(const double* __restrict__ U, const double* xg,
                                     const double* ring, const double* kdring, const double* kxg,
                                     double* __restrict__ x0, int64_t n, const SimScalars* ss) {
    __shared__ SubDirs D;
    __shared__ int snd;
    if (ss->failed) return;
    if (threadIdx.x == 0) snd = ss->use_guess ? subspace_dirs(ss, U, xg, ring, kdring, kxg, n, D) : 0;
    __syncthreads();
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    double x = U[t];
    for (int d = 0; d < snd; ++d) x = fma(ss->theta_sub[d], __ldcg(D.a[d] + t) - __ldcg(D.b[d] + t), x);
    x0[t] = x;
}

// New potentials from the caller: the ring restarts from U^k (and U^{k-1}).
__global__ void history_reset_kernel(double* __restrict__ ring, const double* __restrict__ U,
                                     const double* __restrict__ Uprev, int64_t n, SimScalars* ss) {
    const int64_t k = ss->k;
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n) {
        ring[(k % kHistRing) * n + t] = U[t];
        if (k >= 1) ring[((k - 1) % kHistRing) * n + t] = Uprev[t];
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) ss->hist_len = k >= 1 ? 2 : 1;
}

// count caller-order solutions hist[h] = U^{k-h} into the ring (internal order), U, Uprev, Uprev2.
__global__ void history_set_kernel(const double* __restrict__ hist, int count, double* __restrict__ ring,
                                   double* __restrict__ U, double* __restrict__ Uprev, double* Uprev2,
                                   const int64_t* __restrict__ to_caller, int64_t nc, int np,
                                   SimScalars* ss) {
    const int64_t k = ss->k;
    const int cnt = (int)min((int64_t)min(count, kHistRing), k + 1);
    const int64_t n = nc * np;
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n) {
        const int64_t e = t / np, j = t - e * np;
        const int64_t src = to_caller[e] * np + j;
        for (int h = 0; h < cnt; ++h) {
            const double v = hist[h * n + src];
            ring[((k - h) % kHistRing) * n + t] = v;
            if (h == 0) U[t] = v;
            if (h == 1) Uprev[t] = v;
            if (h == 2 && Uprev2) Uprev2[t] = v;
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) ss->hist_len = cnt;
}

// ------------------------------------------------------------------ training
// One minibatch: forward, MSE loss and backward for tiles of kGT samples; CTA c adds
// its tiles' gradients into part[c * P + .] (its first tile stores) and its loss sum
// into lpart[c].  Sample q is (state k, caller cell id) in samples[2 q], [2 q + 1].
template <int NP>
__global__ void __launch_bounds__(kGThreads)
guess_train_kernel(GuessFeat f, const float* __restrict__ w32, const double* __restrict__ traj,
                   int64_t n_dofs, const int64_t* __restrict__ samples, int64_t n_samples,
                   const int64_t* __restrict__ to_internal, const int64_t* __restrict__ to_caller,
                   float* __restrict__ part, double* __restrict__ lpart) {
    constexpr int F = guess_inputs(NP);
    const ParamOffsets po = param_offsets(NP);
    extern __shared__ __align__(16) unsigned char gsm[];
    float* w1t = reinterpret_cast<float*>(gsm);
    float* w2t = w1t + F * kHP;
    float* w3t = w2t + kH * kHP;
    float* b1 = w3t + kH * NP;
    float* b2 = b1 + kH;
    float* b3 = b2 + kH;
    float* xs = b3 + 16;
    float* h1 = xs + kGT * F;
    float* h2 = h1 + kGT * kH;
    float* dz2 = h2 + kGT * kH;
    float* dz1 = dz2 + kGT * kH;
    float* o = dz1 + kGT * kH;                 // then do
    float* tg = o + kGT * NP;
    __shared__ int64_t elems[kGT], kst[kGT];
    __shared__ double lsh[32];
    stage_weights(w32, NP, w1t, w2t, w3t, b1, b2, b3);
    float* g = part + (size_t)blockIdx.x * po.total;
    const float inv = 1.f / (float)((double)n_samples * NP);
    double lsum = 0.0;
    bool first = true;
    const int64_t n_tiles = (n_samples + kGT - 1) / kGT;
    for (int64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
        const int64_t q0 = tile * kGT;
        const int n = (int)min((int64_t)kGT, n_samples - q0);
        if (threadIdx.x < kGT) {
            const int s = threadIdx.x;
            elems[s] = s < n ? to_internal[samples[2 * (q0 + s) + 1]] : 0;
            kst[s] = s < n ? samples[2 * (q0 + s)] : 2;
        }
        __syncthreads();
        // features (per sample its own state k) and targets
        for (int s = threadIdx.x >> 5; s < kGT; s += blockDim.x >> 5) {
            if (s < n) {
                const double* Uk = traj + kst[s] * n_dofs;
                element_features<NP>(f, Uk, Uk - n_dofs, Uk - 2 * n_dofs, elems[s], xs + s * F,
                                     [&](int64_t c) { return to_caller[c] * NP; });
            } else {
                zero_row(xs + s * F, F);
            }
        }
        for (int q = threadIdx.x; q < kGT * NP; q += blockDim.x) {
            const int s = q / NP, c = q - s * NP;
            float t = 0.f;
            if (s < n) {
                const int64_t o_ = to_caller[elems[s]] * NP + c;
                const double* Uk = traj + kst[s] * n_dofs;
                t = (float)((Uk[n_dofs + o_] - Uk[o_]) / f.s_d);
            }
            tg[q] = t;
        }
        __syncthreads();
        hidden_layer<float, true>(w1t, b1, xs, F, h1);
        __syncthreads();
        hidden_layer<float, true>(w2t, b2, h1, kH, h2);
        __syncthreads();
        output_layer<float, NP>(w3t, b3, h2, o);
        __syncthreads();
        for (int q = threadIdx.x; q < kGT * NP; q += blockDim.x) {   // o <- dL/do
            const int s = q / NP;
            const float d = (s < n) ? o[q] - tg[q] : 0.f;
            lsum += (double)d * d;
            o[q] = 2.f * d * inv;
        }
        __syncthreads();
        {   // dz2 = (do W3) * [h2 > 0]
            const int j = threadIdx.x & (kH - 1), s0 = (threadIdx.x >> 7) * 16;
            for (int s = s0; s < s0 + 16; ++s) {
                float acc = 0.f;
#pragma unroll
                for (int c = 0; c < NP; ++c) acc = fmaf(o[s * NP + c], w3t[j * NP + c], acc);
                dz2[s * kH + j] = h2[s * kH + j] > 0.f ? acc : 0.f;
            }
        }
        __syncthreads();
        {   // dz1 = (dz2 W2) * [h1 > 0]: dh1[s][i] = sum_j W2[j][i] dz2[s][j]
            const int i = threadIdx.x & (kH - 1), s0 = (threadIdx.x >> 7) * 16;
            float acc[16];
#pragma unroll
            for (int s = 0; s < 16; ++s) acc[s] = 0.f;
            for (int j = 0; j < kH; ++j) {
                const float w = w2t[i * kHP + j];
#pragma unroll
                for (int s = 0; s < 16; ++s) acc[s] = fmaf(w, dz2[(s0 + s) * kH + j], acc[s]);
            }
#pragma unroll
            for (int s = 0; s < 16; ++s) dz1[(s0 + s) * kH + i] = h1[(s0 + s) * kH + i] > 0.f ? acc[s] : 0.f;
        }
        __syncthreads();
        // weight gradients of this tile, added into the CTA's partial (canonical layout)
        auto put = [&](int idx, float v) { g[idx] = first ? v : g[idx] + v; };
        for (int q = threadIdx.x; q < kH * F; q += blockDim.x) {     // W1[j][i]
            const int j = q / F, i = q - j * F;
            float acc = 0.f;
            for (int s = 0; s < kGT; ++s) acc = fmaf(dz1[s * kH + j], xs[s * F + i], acc);
            put(po.w1 + q, acc);
        }
        for (int q = threadIdx.x; q < kH * kH; q += blockDim.x) {    // W2[j][i]
            const int j = q / kH, i = q - j * kH;
            float acc = 0.f;
            for (int s = 0; s < kGT; ++s) acc = fmaf(dz2[s * kH + j], h1[s * kH + i], acc);
            put(po.w2 + q, acc);
        }
        for (int q = threadIdx.x; q < NP * kH; q += blockDim.x) {    // W3[c][i]
            const int c = q / kH, i = q - c * kH;
            float acc = 0.f;
            for (int s = 0; s < kGT; ++s) acc = fmaf(o[s * NP + c], h2[s * kH + i], acc);
            put(po.w3 + q, acc);
        }
        for (int q = threadIdx.x; q < kH; q += blockDim.x) {
            float a1 = 0.f, a2 = 0.f;
            for (int s = 0; s < kGT; ++s) { a1 += dz1[s * kH + q]; a2 += dz2[s * kH + q]; }
            put(po.b1 + q, a1);
            put(po.b2 + q, a2);
        }
        for (int q = threadIdx.x; q < NP; q += blockDim.x) {
            float a3 = 0.f;
            for (int s = 0; s < kGT; ++s) a3 += o[s * NP + q];
            put(po.b3 + q, a3);
        }
        first = false;
        __syncthreads();
    }
    const double lt = block_sum(lsum, lsh);
    if (threadIdx.x == 0) lpart[blockIdx.x] = lt;
}

// grad = sum over CTAs of the partials (CTA order); one Adam step of the fp32 master
// weights; fp16 copy for inference; loss = sum of the CTAs' loss sums / (samples n_p).
__global__ void guess_adam_kernel(const float* __restrict__ part, int ncta, int P,
                                  float* __restrict__ w32, float* __restrict__ m, float* __restrict__ v,
                                  __half* __restrict__ w16, float lr, float b1, float b2, float eps,
                                  float c1, float c2, const double* __restrict__ lpart, double inv_count,
                                  double* loss) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p == 0) {
        double l = 0.0;
        for (int c = 0; c < ncta; ++c) l += lpart[c];
        *loss = l * inv_count;
    }
    if (p >= P) return;
    float gsum = 0.f;
    for (int c = 0; c < ncta; ++c) gsum += part[(size_t)c * P + p];
    const float mm = b1 * m[p] + (1.f - b1) * gsum;
    const float vv = b2 * v[p] + (1.f - b2) * gsum * gsum;
    m[p] = mm;
    v[p] = vv;
    const float w = w32[p] - lr * (mm / c1) / (sqrtf(vv / c2) + eps);
    w32[p] = w;
    w16[p] = __float2half_rn(w);
}

__global__ void to_half_kernel(const float* __restrict__ w32, __half* __restrict__ w16, int P) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p < P) w16[p] = __float2half_rn(w32[p]);
}

// ------------------------------------------------------------------ launchers

size_t guess_train_smem(int np) {
    const int F = guess_inputs(np);
    return (size_t)(F * kHP + kH * kHP + kH * np + 2 * kH + 16 + kGT * F + 4 * kGT * kH + 2 * kGT * np) *
           sizeof(float);
}

// n_p <= 10: the training kernel keeps the whole network in shared memory
#define GUESS_NP_SWITCH(np, ...)                                \
    switch (np) {                                               \
        case 3: { constexpr int NP = 3; __VA_ARGS__; } break;   \
        case 6: { constexpr int NP = 6; __VA_ARGS__; } break;   \
        case 10: { constexpr int NP = 10; __VA_ARGS__; } break; \
        default: return cudaErrorInvalidValue;                  \
    }

// the K_h row kernels (history products, subspace rows) hold no network: every n_p of
// the block-sparse operator, including n_p = 15 (2D P4)
#define KROW_NP_SWITCH(np, ...)                                 \
    switch (np) {                                               \
        case 3: { constexpr int NP = 3; __VA_ARGS__; } break;   \
        case 6: { constexpr int NP = 6; __VA_ARGS__; } break;   \
        case 10: { constexpr int NP = 10; __VA_ARGS__; } break; \
        case 15: { constexpr int NP = 15; __VA_ARGS__; } break; \
        default: return cudaErrorInvalidValue;                  \
    }

// Raise the shared-memory limits of the inference and training kernels for n_p (once,
// before any launch, so that launches can be recorded into CUDA graphs).
cudaError_t guess_prepare(int np) {
    GUESS_NP_SWITCH(np, {
        cudaError_t e = guess_propose_tc_prepare(np);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(guess_train_kernel<NP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)guess_train_smem(np));
        return e;
    })
    return cudaSuccess;
}

cudaError_t launch_guess_select(int np, const DeviceMatrix& K, const double* b, const double* xg,
                                const double* uk, double* partials, SimScalars* ss, int policy,
                                cudaStream_t s) {
    const unsigned grid = policy == 1 ? 1u : (unsigned)((K.nc * 32 + kBlock - 1) / kBlock);
    if (grid > (unsigned)kMaxPartials) return cudaErrorInvalidValue;
    GUESS_NP_SWITCH(np, {
        guess_select_kernel<NP><<<grid, kBlock, 0, s>>>(K.row_ptr, K.col, K.val, b, xg, uk, K.nc,
                                                        partials, ss, policy);
    })
    return cudaGetLastError();
}

cudaError_t launch_select_copy(const double* uk, const double* xg, double* x0, int64_t n,
                               const SimScalars* ss, cudaStream_t s) {
    select_copy_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(uk, xg, x0, n, ss);
    return cudaGetLastError();
}

cudaError_t launch_guess_subspace(int np, const DeviceMatrix& K, const double* b, const double* U,
                                  const double* xg, const double* ring, double* kuring, double* W,
                                  double* gram, int64_t n, SimScalars* ss, cudaStream_t s) {
    const unsigned grid = (unsigned)((K.nc * 32 + kBlock - 1) / kBlock);
    KROW_NP_SWITCH(np, {
        subspace_rows_kernel<NP><<<grid, kBlock, 0, s>>>(K.row_ptr, K.col, K.val, b, U, xg, ring, kuring,
                                                         W, n, K.nc, ss);
    })
    const unsigned g2 = (unsigned)std::min<int64_t>(kSubMaxCtas, (n + kGramRows - 1) / kGramRows);
    subspace_gram_kernel<<<g2, kGramThreads, 0, s>>>(W, U, xg, ring, kuring, n, gram, ss);
    return cudaGetLastError();
}

cudaError_t launch_subspace_copy(const double* U, const double* xg, const double* ring,
                                 const double* kuring, const double* W, double* x0, int64_t n,
                                 const SimScalars* ss, cudaStream_t s) {
    subspace_copy_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(U, xg, ring, kuring, W + n, x0, n, ss);
    return cudaGetLastError();
}

cudaError_t launch_history_reset(int np, const DeviceMatrix& K, double* ring, double* kuring,
                                 const double* U, const double* Uprev, int64_t n, SimScalars* ss,
                                 cudaStream_t s) {
    history_reset_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(ring, U, Uprev, n, ss);
    const unsigned grid = (unsigned)((K.nc * 32 + kBlock - 1) / kBlock);
    KROW_NP_SWITCH(np, {
        history_products_kernel<NP><<<grid, kBlock, 0, s>>>(K.row_ptr, K.col, K.val, ring, kuring, n,
                                                            K.nc, ss);
    })
    return cudaGetLastError();
}

cudaError_t launch_history_set(const DeviceMatrix& K, const double* hist, int count, double* ring,
                               double* kuring, double* U, double* Uprev, double* Uprev2,
                               const int64_t* to_caller, int64_t nc, int np, SimScalars* ss,
                               cudaStream_t s) {
    history_set_kernel<<<(unsigned)((nc * np + 255) / 256), 256, 0, s>>>(hist, count, ring, U, Uprev,
                                                                       Uprev2, to_caller, nc, np, ss);
    const unsigned grid = (unsigned)((K.nc * 32 + kBlock - 1) / kBlock);
    KROW_NP_SWITCH(np, {
        history_products_kernel<NP><<<grid, kBlock, 0, s>>>(K.row_ptr, K.col, K.val, ring, kuring,
                                                            nc * np, K.nc, ss);
    })
    return cudaGetLastError();
}

cudaError_t launch_guess_train(int np, const GuessFeat& f, const float* w32, const double* traj,
                               int64_t n_dofs, const int64_t* samples, int64_t n_samples,
                               const int64_t* to_internal, const int64_t* to_caller, float* part,
                               double* lpart, int grid, cudaStream_t s) {
    const size_t smem = guess_train_smem(np);
    GUESS_NP_SWITCH(np, {
        guess_train_kernel<NP><<<grid, kGThreads, smem, s>>>(f, w32, traj, n_dofs, samples, n_samples,
                                                             to_internal, to_caller, part, lpart);
    })
    return cudaGetLastError();
}

cudaError_t launch_guess_adam(const float* part, int ncta, int P, float* w32, float* m, float* v,
                              __half* w16, float lr, float b1, float b2, float eps, float c1, float c2,
                              const double* lpart, double inv_count, double* loss, cudaStream_t s) {
    guess_adam_kernel<<<(unsigned)((P + 255) / 256), 256, 0, s>>>(part, ncta, P, w32, m, v, w16, lr, b1,
                                                                 b2, eps, c1, c2, lpart, inv_count, loss);
    return cudaGetLastError();
}

cudaError_t launch_to_half(const float* w32, __half* w16, int P, cudaStream_t s) {
    to_half_kernel<<<(unsigned)((P + 255) / 256), 256, 0, s>>>(w32, w16, P);
    return cudaGetLastError();
}

}  // namespace polydg
