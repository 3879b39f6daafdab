// Local solves shared by simulations that differ only in a scalar conductivity.
//
// On one mesh and partition with Sigma_K = sigma I, the SIP stiffness is linear in
// sigma (Eq. eta takes lambda_max(Sigma_K) = sigma; Eq. coer is linear in Sigma), so
// K_i(sigma) = chi_cm M_i + (dt sigma / 2) A_i with A_i the sigma = 1 stiffness.  With
// M_i = L_i L_i^T (one Cholesky factor per element) and L_i^{-1} A_i L_i^{-T} =
// Q_i diag(lam_i) Q_i^T,
//     K_i(sigma)^{-1} = L_i^{-T} Q_i diag(1 / (chi_cm + c lam_i)) Q_i^T L_i^{-1},  c = dt sigma/2,
// so one eigenbasis per subdomain serves every simulation on the mesh, and the R
// right-hand sides of R simulations take two passes over Q_i (as Q_i^T rows, then Q_i
// rows) instead of R passes over R different inverses.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <thread>
#include <vector>

#include "contexts.h"

namespace polydg {

struct RhsPtrs {
    const double* r[kMaxTcRhs];
    double* z[kMaxTcRhs];
    double c[kMaxTcRhs];    // dt sigma_s / 2
};

template <typename T>
__device__ __forceinline__ float to_f(T v) { return (float)v; }
template <>
__device__ __forceinline__ float to_f<__nv_bfloat16>(__nv_bfloat16 v) { return __bfloat162float(v); }

// One CTA per subdomain: X_s = L^{-1} r_s; Y_s = diag(1/(chi + c_s lam)) Q^T X_s;
// z_s = L^{-T} Q Y_s.  Warp per row of Q^T (pass 1) and of Q (pass 2), R dots per row.
template <typename T, int R>
__global__ void __launch_bounds__(512)
shared_local_apply_kernel(const SharedBlock* __restrict__ blocks, const T* __restrict__ q,
                          const float* __restrict__ lam, const double* __restrict__ linv, int np,
                          double chi, RhsPtrs p) {
    extern __shared__ __align__(16) float sm[];
    const SharedBlock B = blocks[blockIdx.x];
    const int n = B.n, ld = B.ld;
    float* X = sm;                 // [R][ld]
    float* Y = sm + R * ld;        // [R][ld]
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    // X_s = L^{-1} r_s, element by element (L^{-1} lower triangular, row-major n_p x n_p)
    for (int idx = threadIdx.x; idx < R * ld; idx += blockDim.x) {
        const int s = idx / ld, k = idx - s * ld;
        float v = 0.f;
        if (k < n) {
            const int el = k / np, i = k - el * np;
            const double* Li = linv + ((int64_t)(B.cell0 + el) * np + i) * np;
            const double* rs = p.r[s] + B.in_off + (int64_t)el * np;
            double acc = 0.0;
            for (int j = 0; j <= i; ++j) acc = fma(Li[j], rs[j], acc);
            v = (float)acc;
        }
        X[idx] = v;
    }
    __syncthreads();
    const T* Qt = q + B.q_off;
    const T* Qr = Qt + (int64_t)n * ld;
    const float* lm = lam + B.lam_off;
    for (int j = warp; j < n; j += nw) {                 // pass 1: rows of Q^T
        const T* row = Qt + (int64_t)j * ld;
        float acc[R];
#pragma unroll
        for (int s = 0; s < R; ++s) acc[s] = 0.f;
        for (int k = lane; k < n; k += 32) {
            const float a = to_f(row[k]);
#pragma unroll
            for (int s = 0; s < R; ++s) acc[s] = fmaf(a, X[s * ld + k], acc[s]);
        }
#pragma unroll
        for (int s = 0; s < R; ++s) {
            const float v = warp_sumf(acc[s]);
            if (lane == 0) Y[s * ld + j] = (float)((double)v / (chi + p.c[s] * (double)lm[j]));
        }
    }
    __syncthreads();
    for (int k = warp; k < n; k += nw) {                 // pass 2: rows of Q, into X
        const T* row = Qr + (int64_t)k * ld;
        float acc[R];
#pragma unroll
        for (int s = 0; s < R; ++s) acc[s] = 0.f;
        for (int j = lane; j < n; j += 32) {
            const float a = to_f(row[j]);
#pragma unroll
            for (int s = 0; s < R; ++s) acc[s] = fmaf(a, Y[s * ld + j], acc[s]);
        }
#pragma unroll
        for (int s = 0; s < R; ++s) {
            const float v = warp_sumf(acc[s]);
            if (lane == 0) X[s * ld + k] = v;
        }
    }
    __syncthreads();
    // z_s = L^{-T} V_s: z[i] = sum_{j >= i} Linv[j][i] V[j] per element
    for (int idx = threadIdx.x; idx < R * n; idx += blockDim.x) {
        const int s = idx / n, k = idx - s * n;
        const int el = k / np, i = k - el * np;
        const double* L0 = linv + (int64_t)(B.cell0 + el) * np * np;
        const float* V = X + s * ld + el * np;
        double acc = 0.0;
        for (int j = i; j < np; ++j) acc = fma(L0[j * np + i], (double)V[j], acc);
        p.z[s][B.in_off + k] = acc;
    }
}

// Caller order <-> internal order for the R vectors of one application in one launch
// (grid.y = vector): to_internal dst[k][t] = src[k][c n_p + j], else the reverse, with
// element e = t / n_p of internal order at caller cell c = to_caller[e].
struct PermPtrs {
    const double* src[kMaxTcRhs];
    double* dst[kMaxTcRhs];
};

__global__ void permute_many_kernel(PermPtrs p, const int64_t* __restrict__ to_caller, int64_t nc, int np,
                                    int to_internal) {
    const int k = blockIdx.y;
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nc * np) return;
    const int64_t e = t / np, j = t - e * np, c = to_caller[e];
    if (to_internal) p.dst[k][t] = p.src[k][c * np + j];
    else p.dst[k][c * np + j] = p.src[k][t];
}

static cudaError_t launch_permute_many(const PermPtrs& p, int nvec, const int64_t* to_caller, int64_t nc,
                                       int np, int to_internal, cudaStream_t s) {
    const dim3 grid((unsigned)((nc * np + 255) / 256), (unsigned)nvec);
    permute_many_kernel<<<grid, 256, 0, s>>>(p, to_caller, nc, np, to_internal);
    return cudaGetLastError();
}

}  // namespace polydg

namespace polydg {

// lower Cholesky factor of a small SPD matrix and its inverse (row-major n x n)
static bool small_chol_inv(int n, const double* a, double* linv) {
    std::vector<double> L(n * n, 0.0);
    for (int j = 0; j < n; ++j) {
        double d = a[j * n + j];
        for (int k = 0; k < j; ++k) d -= L[j * n + k] * L[j * n + k];
        if (!(d > 0.0)) return false;
        L[j * n + j] = std::sqrt(d);
        for (int i = j + 1; i < n; ++i) {
            double v = a[i * n + j];
            for (int k = 0; k < j; ++k) v -= L[i * n + k] * L[j * n + k];
            L[i * n + j] = v / L[j * n + j];
        }
    }
    for (int i = 0; i < n * n; ++i) linv[i] = 0.0;
    for (int c = 0; c < n; ++c) {                  // solve L x = e_c
        for (int i = c; i < n; ++i) {
            double v = (i == c) ? 1.0 : 0.0;
            for (int k = c; k < i; ++k) v -= L[i * n + k] * linv[k * n + c];
            linv[i * n + c] = v / L[i * n + i];
        }
    }
    return true;
}

}  // namespace polydg

extern "C" {

int shared_local_setup(polydg_ctx* c, int precision, shared_local** out) {
    if (!c || !out || (precision != POLYDG_FP32 && precision != POLYDG_BF16)) {
        set_error("shared_local_setup: need a context, an output pointer and POLYDG_FP32 or POLYDG_BF16");
        return POLYDG_EINVAL;
    }
    *out = nullptr;
    const HostSetup& H = c->H;
    const int np = H.n_p;
    const double s0 = H.sigma[0];
    const int d = H.dim;
    for (int64_t k = 0; k < H.nc; ++k) {
        const double* S = &H.sigma[(size_t)d * d * k];
        bool scalar = true;
        for (int i = 0; i < d; ++i)
            for (int j = 0; j < d; ++j) scalar = scalar && S[i * d + j] == (i == j ? s0 : 0.0);
        if (!scalar) {
            set_error("shared_local_setup: the conductivity must be the same scalar multiple of I on every cell");
            return POLYDG_EINVAL;
        }
    }
    shared_local* sl = new shared_local();
    sl->ctx = c;
    sl->precision = precision;
    sl->sigma_ref = s0;
    sl->n_sub = H.n_sub;
    auto fail = [&](int code) { shared_local_destroy(sl); return code; };
    // per element L_K^{-1}
    std::vector<double> linv((size_t)H.nc * np * np);
    for (int64_t e = 0; e < H.nc; ++e)
        if (!small_chol_inv(np, &H.Mblk[(size_t)e * np * np], &linv[(size_t)e * np * np])) {
            set_error("shared_local_setup: an element mass matrix is not positive definite");
            return fail(POLYDG_ENOTSPD);
        }
    // layout
    int64_t q_total = 0, lam_total = 0;
    sl->hblocks.resize(H.n_sub);
    for (int i = 0; i < H.n_sub; ++i) {
        SharedBlock& B = sl->hblocks[i];
        B.cell0 = (int32_t)H.sub_ptr[i];
        B.ncell = (int32_t)(H.sub_ptr[i + 1] - H.sub_ptr[i]);
        B.n = B.ncell * np;
        B.ld = (B.n + 7) / 8 * 8;
        B.in_off = H.sub_ptr[i] * np;
        B.q_off = q_total;
        B.lam_off = lam_total;
        q_total += 2 * (int64_t)B.n * B.ld;
        lam_total += B.n;
        sl->max_ld = std::max<int64_t>(sl->max_ld, B.ld);
    }
    const int esz = precision == POLYDG_FP32 ? 4 : 2;
    sl->store_bytes = q_total * esz;
    std::vector<float> q32(precision == POLYDG_FP32 ? q_total : 0), lam(lam_total);
    std::vector<__nv_bfloat16> q16(precision == POLYDG_BF16 ? q_total : 0);
    // C_i = L^{-1} A_i L^{-T} with A = (K - Kminus) / (dt sigma); eigendecomposition per subdomain
    const double scale = 1.0 / (H.dt * s0);
    std::atomic<int> next(0), bad(0);
    auto work = [&]() {
        std::vector<double> A, C, w, qt;
        for (int i = next++; i < H.n_sub; i = next++) {
            const SharedBlock& B = sl->hblocks[i];
            const int n = B.n;
            A.assign((size_t)n * n, 0.0);
            for (int el = 0; el < B.ncell; ++el) {
                const int64_t e = B.cell0 + el;
                for (int32_t bi = H.row_ptr[e]; bi < H.row_ptr[e + 1]; ++bi) {
                    const int64_t f = H.col[bi];
                    if (f < B.cell0 || f >= B.cell0 + B.ncell) continue;
                    const double* Kb = &H.Kval[(size_t)bi * np * np];
                    const double* Km = &H.Kminus_val[(size_t)bi * np * np];
                    for (int a = 0; a < np; ++a)
                        for (int b = 0; b < np; ++b)
                            A[(size_t)(el * np + a) * n + (f - B.cell0) * np + b] =
                                (Kb[a * np + b] - Km[a * np + b]) * scale;
                }
            }
            // C = Linv A Linv^T (block diagonal Linv): rows, then columns
            C.assign((size_t)n * n, 0.0);
            for (int el = 0; el < B.ncell; ++el) {
                const double* Li = &linv[(size_t)(B.cell0 + el) * np * np];
                for (int a = 0; a < np; ++a)
                    for (int k = 0; k <= a; ++k) {
                        const double l = Li[a * np + k];
                        const double* src = &A[(size_t)(el * np + k) * n];
                        double* dst = &C[(size_t)(el * np + a) * n];
                        for (int j = 0; j < n; ++j) dst[j] += l * src[j];
                    }
            }
            std::fill(A.begin(), A.end(), 0.0);
            for (int r = 0; r < n; ++r)
                for (int el = 0; el < B.ncell; ++el) {
                    const double* Li = &linv[(size_t)(B.cell0 + el) * np * np];
                    const double* src = &C[(size_t)r * n + el * np];
                    double* dst = &A[(size_t)r * n + el * np];
                    for (int b = 0; b < np; ++b) {
                        double acc = 0.0;
                        for (int k = 0; k <= b; ++k) acc += src[k] * Li[b * np + k];
                        dst[b] = acc;
                    }
                }
            for (int r = 0; r < n; ++r)                   // symmetrise the rounding
                for (int j = 0; j < r; ++j) {
                    const double v = 0.5 * (A[(size_t)r * n + j] + A[(size_t)j * n + r]);
                    A[(size_t)r * n + j] = A[(size_t)j * n + r] = v;
                }
            w.resize(n);
            qt.resize((size_t)n * n);
            if (!sym_eig(n, A.data(), w.data(), qt.data())) { bad = 1; continue; }
            for (int j = 0; j < n; ++j) lam[B.lam_off + j] = (float)w[j];
            const int64_t ldq = B.ld;
            for (int r = 0; r < n; ++r)
                for (int k = 0; k < ldq; ++k) {
                    const double vt = k < n ? qt[(size_t)r * n + k] : 0.0;   // Q^T[r][k]
                    const double vq = k < n ? qt[(size_t)k * n + r] : 0.0;   // Q[r][k]
                    const int64_t o1 = B.q_off + (int64_t)r * ldq + k;
                    const int64_t o2 = B.q_off + (int64_t)n * ldq + (int64_t)r * ldq + k;
                    if (precision == POLYDG_FP32) { q32[o1] = (float)vt; q32[o2] = (float)vq; }
                    else { q16[o1] = __float2bfloat16_rn((float)vt); q16[o2] = __float2bfloat16_rn((float)vq); }
                }
        }
    };
    const int nthr = std::max(1, std::min<int>((int)std::thread::hardware_concurrency(), H.n_sub));
    std::vector<std::thread> pool;
    for (int t = 1; t < nthr; ++t) pool.emplace_back(work);
    work();
    for (auto& t : pool) t.join();
    if (bad) { set_error("shared_local_setup: an eigendecomposition did not converge"); return fail(POLYDG_ENOTCONV); }
    int st;
    if (precision == POLYDG_BF16) {
        // tiles of tcgen05.mma: per subdomain the 128 x 64 tiles of Q^T (row j, column k) and
        // then of Q (row k, column j), zero-padded to 128 rows and 64 columns, element (r, c)
        // of a tile at byte (r/8) 1024 + (c/8) 128 + (r%8) 16 + (c%8) 2
        int64_t total = 0;
        sl->htc.resize(H.n_sub);
        for (int i = 0; i < H.n_sub; ++i) {
            const SharedBlock& B = sl->hblocks[i];
            TcBlock& T = sl->htc[i];
            T.n = B.n;
            T.mt = (B.n + 127) / 128;
            T.kt = (B.n + 63) / 64;
            T.cell0 = B.cell0;
            T.in_off = B.in_off;
            T.lam_off = B.lam_off;
            T.tile_off = total;
            total += 2 * (int64_t)T.mt * T.kt * 16384;
            sl->max_kpad = std::max(sl->max_kpad, T.kt * 64);
        }
    }
    if (precision == POLYDG_BF16 && sl->max_kpad <= 1024) {   // larger subdomains: SIMT passes only
        const int64_t total = sl->htc.back().tile_off + 2 * (int64_t)sl->htc.back().mt * sl->htc.back().kt * 16384;
        std::vector<__nv_bfloat16> tiles(total / 2, __float2bfloat16_rn(0.f));
        std::atomic<int> nx(0);
        auto tile_work = [&]() {
            for (int i = nx++; i < H.n_sub; i = nx++) {
                const SharedBlock& B = sl->hblocks[i];
                const TcBlock& T = sl->htc[i];
                for (int pass = 0; pass < 2; ++pass) {
                    const int64_t qbase = B.q_off + (pass ? (int64_t)B.n * B.ld : 0);   // Q^T, then Q
                    for (int row = 0; row < B.n; ++row)
                        for (int col = 0; col < B.n; ++col) {
                            const int mt = row / 128, kt = col / 64, r = row % 128, c = col % 64;
                            const int64_t tile = (int64_t)pass * T.mt * T.kt + (int64_t)mt * T.kt + kt;
                            const int64_t byte = T.tile_off + tile * 16384 + (r / 8) * 1024 + (c / 8) * 128 +
                                                 (r % 8) * 16 + (c % 8) * 2;
                            tiles[byte / 2] = q16[qbase + (int64_t)row * B.ld + col];
                        }
                }
            }
        };
        std::vector<std::thread> tpool;
        for (int tt = 1; tt < nthr; ++tt) tpool.emplace_back(tile_work);
        tile_work();
        for (auto& th : tpool) th.join();
        sl->tile_bytes = total;
        if ((st = upload(&sl->tc, sl->htc)) || (st = dalloc(&sl->d_err, 1))) return fail(st);
        if ((st = dalloc(&sl->tiles, total))) return fail(st);
        if (cudaMemcpy(sl->tiles, tiles.data(), total, cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemset(sl->d_err, 0, sizeof(int)) != cudaSuccess) {
            set_error("shared_local_setup: tile upload failed");
            return fail(POLYDG_ECUDA);
        }
    }
    if ((st = upload(&sl->blocks, sl->hblocks)) || (st = upload(&sl->lam, lam)) || (st = upload(&sl->linv, linv)))
        return fail(st);
    if (precision == POLYDG_FP32) { if ((st = upload(&sl->st32, q32))) return fail(st); }
    else if ((st = upload(&sl->st16, q16))) return fail(st);
    *out = sl;
    return POLYDG_OK;
}

int shared_local_info(const shared_local* sl, int64_t* store_bytes, double* sigma_ref) {
    if (!sl) { set_error("shared_local_info: null argument"); return POLYDG_EINVAL; }
    if (store_bytes) *store_bytes = sl->store_bytes;
    if (sigma_ref) *sigma_ref = sl->sigma_ref;
    return POLYDG_OK;
}

int shared_local_apply(shared_local* sl, int nrhs, const double* const* r_dev, double* const* z_dev,
                       const double* sigmas, void* stream) {
    const int max_rhs = (sl && sl->tiles) ? kMaxTcRhs : kMaxRhs;
    if (!sl || nrhs < 1 || nrhs > max_rhs || !r_dev || !z_dev || !sigmas) {
        set_error("shared_local_apply: need 1 <= nrhs <= 16 (BF16, subdomains <= 1024 DOFs) or 4 "
                  "vectors and conductivities");
        return POLYDG_EINVAL;
    }
    polydg_ctx* c = sl->ctx;
    const int np = c->H.n_p;
    const int64_t n = c->H.nc * np;
    cudaStream_t s = (cudaStream_t)stream;
    RhsPtrs p = {};
    PermPtrs pin = {}, pout = {};
    for (int k = 0; k < nrhs; ++k) {
        if (!(sigmas[k] > 0)) { set_error("shared_local_apply: conductivities must be > 0"); return POLYDG_EINVAL; }
        for (int t = 0; t < 2; ++t)
            if (!sl->tmp[2 * k + t])
                if (int st = dalloc(&sl->tmp[2 * k + t], n)) return st;
        pin.src[k] = r_dev[k];
        pin.dst[k] = sl->tmp[2 * k];
        pout.src[k] = sl->tmp[2 * k + 1];
        pout.dst[k] = z_dev[k];
        p.r[k] = sl->tmp[2 * k];
        p.z[k] = sl->tmp[2 * k + 1];
        p.c[k] = 0.5 * c->H.dt * sigmas[k];
    }
    CU(launch_permute_many(pin, nrhs, c->d_to_caller, c->H.nc, np, 1, s));
    const double chi = c->H.chi_cm;
    if (sl->tiles) {                         // tensor cores: both passes as tcgen05 BF16 GEMMs
        TcRhs tp = {};
        tp.nrhs = nrhs;
        for (int k = 0; k < nrhs; ++k) { tp.r[k] = p.r[k]; tp.z[k] = p.z[k]; tp.c[k] = p.c[k]; }
        int h_err = 0;
        CU(launch_shared_tc(sl->tc, sl->n_sub, sl->tiles, sl->lam, sl->linv, np, chi, tp, sl->max_kpad,
                            sl->d_err, s));
        CU(cudaMemcpyAsync(&h_err, sl->d_err, sizeof(int), cudaMemcpyDeviceToHost, s));
        CU(cudaStreamSynchronize(s));
        if (h_err) {
            cudaMemsetAsync(sl->d_err, 0, sizeof(int), s);
            set_error("shared_local_apply: a device-side wait timed out");
            return POLYDG_ECUDA;
        }
        CU(launch_permute_many(pout, nrhs, c->d_to_caller, c->H.nc, np, 0, s));
        return POLYDG_OK;
    }
    const size_t smem = 2 * (size_t)kMaxRhs * sl->max_ld * sizeof(float);
    const unsigned grid = (unsigned)sl->n_sub;
#define LAUNCH(T, R, Q)                                                                              \
    {                                                                                                \
        CU(cudaFuncSetAttribute(shared_local_apply_kernel<T, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)); \
        shared_local_apply_kernel<T, R><<<grid, 512, smem, s>>>(sl->blocks, Q, sl->lam, sl->linv, np, chi, p);     \
    }
    if (sl->precision == POLYDG_FP32) {
        switch (nrhs) {
            case 1: LAUNCH(float, 1, sl->st32) break;
            case 2: LAUNCH(float, 2, sl->st32) break;
            case 3: LAUNCH(float, 3, sl->st32) break;
            default: LAUNCH(float, 4, sl->st32) break;
        }
    } else {
        switch (nrhs) {
            case 1: LAUNCH(__nv_bfloat16, 1, sl->st16) break;
            case 2: LAUNCH(__nv_bfloat16, 2, sl->st16) break;
            case 3: LAUNCH(__nv_bfloat16, 3, sl->st16) break;
            default: LAUNCH(__nv_bfloat16, 4, sl->st16) break;
        }
    }
#undef LAUNCH
    CU(cudaGetLastError());
    CU(launch_permute_many(pout, nrhs, c->d_to_caller, c->H.nc, np, 0, s));
    return POLYDG_OK;
}

void shared_local_destroy(shared_local* sl) {
    if (!sl) return;
    dfree(sl->blocks); dfree(sl->st32); dfree(sl->st16); dfree(sl->lam); dfree(sl->linv);
    dfree(sl->tc); dfree(sl->tiles); dfree(sl->d_err);
    for (auto& t : sl->tmp) dfree(t);
    delete sl;
}

}  // extern "C"
