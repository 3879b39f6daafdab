// Lockstep PCG of up to four simulations that share a mesh, partition and coarse space
// and whose conductivities are scalar multiples of the identity (Sec. 4, Eq. prec), with
// the local solves of every subdomain taken from one shared eigenbasis:
//     K_i(sigma_s)^{-1} = L_i^{-T} Q_i diag(1 / (chi_cm + c_s lam_i)) Q_i^T L_i^{-1}.
// One CTA group runs the R solves at once; each CTA owns element-aligned row ranges
// ("pieces") of subdomains.  Per iteration:
//   P1  per piece: stage r'_s of the whole subdomain, commit the piece's rows of every
//       simulation, X_s = L^{-1} r'_s, R_0 r'_s (piece at row 0), pass 1 over the piece's
//       rows of Q_i^T: Y_s = D_s Q_i^T X_s (R dot products per streamed row) -> global
//                                                        -> barrier, |r'|^2, tests
//   P2  per piece: pass 2 over its rows of Q_i with the whole subdomain's Y_s, z_loc,s =
//       L^{-T} V_s; the coarse solves                    -> barrier
//   CM  z = z_loc + R_0^T y0, w = K_s z, dots per simulation   -> barrier, beta, alpha
// The rows stream through per-warp copy rings prefetched across phases and iterations.
// Each simulation keeps its own scalars and stopping test; one that has converged or
// failed drops out of the work while the others go on.
#include <cuda_runtime.h>
#include <cuda_bf16.h>

#include "device.cuh"
#include "kernels.h"
#include "pcg_device.cuh"

namespace polydg {

template <typename T>
__device__ __forceinline__ void load8(const T* p, float (&f)[8]);

template <>
__device__ __forceinline__ void load8<__nv_bfloat16>(const __nv_bfloat16* p, float (&f)[8]) {
    const uint4 v = *reinterpret_cast<const uint4*>(p);
    const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&v);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const float2 t = __bfloat1622float2(h[k]);
        f[2 * k] = t.x;
        f[2 * k + 1] = t.y;
    }
}

template <>
__device__ __forceinline__ void load8<float>(const float* p, float (&f)[8]) {
    const float4 a = *reinterpret_cast<const float4*>(p);
    const float4 b = *reinterpret_cast<const float4*>(p + 4);
    f[0] = a.x; f[1] = a.y; f[2] = a.z; f[3] = a.w;
    f[4] = b.x; f[5] = b.y; f[6] = b.z; f[7] = b.w;
}

// acc[s] = row . V_s for the live simulations (row: ld entries, a multiple of 8; V_s at
// V + s * stride in shared memory); warp-wide, result in every lane.
template <typename T>
__device__ __forceinline__ void row_dots(const T* row, const float* V, int stride, int ld, int live,
                                         int lane, float (&acc)[kMaxRhs]) {
#pragma unroll
    for (int s = 0; s < kMaxRhs; ++s) acc[s] = 0.f;
    for (int c = 8 * lane; c < ld; c += 256) {
        float f[8];
        load8(row + c, f);
#pragma unroll
        for (int s = 0; s < kMaxRhs; ++s) {
            if (!((live >> s) & 1)) continue;
            const float4 x0 = *reinterpret_cast<const float4*>(V + s * stride + c);
            const float4 x1 = *reinterpret_cast<const float4*>(V + s * stride + c + 4);
            float a = acc[s];
            a = fmaf(f[0], x0.x, a); a = fmaf(f[1], x0.y, a); a = fmaf(f[2], x0.z, a); a = fmaf(f[3], x0.w, a);
            a = fmaf(f[4], x1.x, a); a = fmaf(f[5], x1.y, a); a = fmaf(f[6], x1.z, a); a = fmaf(f[7], x1.w, a);
            acc[s] = a;
        }
    }
#pragma unroll
    for (int s = 0; s < kMaxRhs; ++s) acc[s] = warp_sumf(acc[s]);
}

// v[s] += x for the runtime index s (unrolled, so v stays in registers)
template <int N>
__device__ __forceinline__ void add_at(double (&v)[N], int s, double x) {
#pragma unroll
    for (int k = 0; k < N; ++k)
        if (k == s) v[k] += x;
}

// Per-simulation scalars of a group, uniform over the CTA: kept in shared memory
// (thread 0 writes them between CTA barriers) rather than replicated in registers.
struct GroupScalars {
    double alpha[kMaxRhs], beta[kMaxRhs], rz[kMaxRhs], pq[kMaxRhs], bb[kMaxRhs], rr[kMaxRhs];
    double rtol2[kMaxRhs];
    int it[kMaxRhs], pending[kMaxRhs], status[kMaxRhs], maxit[kMaxRhs], flex[kMaxRhs];
    int live, started;
};

template <typename T, int NP>
__device__ __forceinline__ void pcg_group_cta(const GroupArgs& a, const int cta, const unsigned G,
                                              unsigned char* smem) {
    constexpr int NW = kPersistThreads / 32;
    constexpr int MR = kMaxRhs;
    __shared__ __align__(8) uint64_t wbars[NW][kMaxWarpStages];
    __shared__ GroupScalars gsc;
    __shared__ double red[3 * kPersistThreads], outv[3 * MR];

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int R = a.R;
    if (threadIdx.x == 0) {
        int live = 0;
        for (int s = 0; s < MR; ++s) {
            const bool on = s < R && !a.sim[s].sc->done;
            if (on) live |= 1 << s;
            gsc.flex[s] = s < R && a.sim[s].sc->flexible != 0;
            gsc.rtol2[s] = s < R ? a.sim[s].sc->rtol2 : 0.0;
            gsc.maxit[s] = s < R ? a.sim[s].sc->maxit : 0;
            gsc.alpha[s] = gsc.beta[s] = gsc.rz[s] = gsc.pq[s] = 0.0;
            gsc.it[s] = gsc.pending[s] = 0;
            gsc.status[s] = kOK;
        }
        gsc.live = live;
        gsc.started = live;
    }
    __syncthreads();
    if (!gsc.live) return;
    unsigned gen = 0;
    const int S = a.wstages;
    const int ldm = (int)a.ld_max;
    auto slot = [&](int w, int k) { return reinterpret_cast<T*>(smem + ((size_t)w * S + k) * a.slot_bytes); };
    double* rp = reinterpret_cast<double*>(smem + a.rp_off);   // [MR][ldm] r' (fp64)
    float* X = reinterpret_cast<float*>(smem + a.x_off);       // [MR][ldm] L^{-1} r', then V
    float* Y = reinterpret_cast<float*>(smem + a.y_off);       // [MR][ldm] Q^T X of the subdomain
    double* r0s = reinterpret_cast<double*>(smem + a.r0_off);  // [n0], one simulation at a time
    double* pn = reinterpret_cast<double*>(smem + a.pn_off);   // z or x of a chunk's needed elements
    RunDesc* rd = reinterpret_cast<RunDesc*>(smem + a.td_off);

    const int64_t e0 = a.elem_ptr[cta], e1 = a.elem_ptr[cta + 1];
    const int ch0 = a.cta_chunk[cta], ch1 = a.cta_chunk[cta + 1];
    const int c0 = a.crow_ptr[cta], c1 = a.crow_ptr[cta + 1];
    const int pc0 = a.piece_ptr[cta], npieces = a.piece_ptr[cta + 1] - pc0;
    const bool coarse = a.n0 > 0;
    const float chi_f = (float)a.chi;

    // ---- init: per simulation r = b - K x on own elements; p, q, z, w = 0; |b|^2, |r|^2
    double v2[2 * MR];
#pragma unroll
    for (int k = 0; k < 2 * MR; ++k) v2[k] = 0.0;
    {
        const int live = gsc.live;
#pragma unroll
        for (int s = 0; s < MR; ++s) {
            if (!((live >> s) & 1)) continue;
            const GroupSim& sm = a.sim[s];
            for (int64_t t = e0 * NP + threadIdx.x; t < e1 * NP; t += blockDim.x) {
                sm.p[0][t] = 0.0; sm.p[1][t] = 0.0; sm.q[0][t] = 0.0; sm.q[1][t] = 0.0;
                sm.z[t] = 0.0; sm.w[t] = 0.0;
            }
            for (int ch = ch0; ch < ch1; ++ch) {
                const int64_t ce0 = a.chunk_elem[ch], ce1 = a.chunk_elem[ch + 1];
                const int32_t* need = a.need + a.need_ptr[ch];
                const int n_need = a.need_ptr[ch + 1] - a.need_ptr[ch];
                __syncthreads();
                for (int idx = threadIdx.x; idx < n_need * NP; idx += blockDim.x) {
                    const int l = idx / NP;
                    pn[idx] = __ldcg(sm.x + (int64_t)need[l] * NP + (idx - l * NP));
                }
                __syncthreads();
                local_rows<NP>(a.row_ptr, a.col_local, sm.val, pn, ce0, ce1, [&](int64_t e, int i, double kx) {
                    const int64_t t = e * NP + i;
                    const double bv = sm.b[t], rv = bv - kx;
                    sm.r[0][t] = rv;
                    v2[2 * s] = fma(bv, bv, v2[2 * s]);
                    v2[2 * s + 1] = fma(rv, rv, v2[2 * s + 1]);
                });
            }
        }
    }
    // ---- the CTA's rows: its pieces' rows of Q^T (pass 1), then the same rows of Q (pass 2)
    int n_rows = 0;
    for (int k = 0; k < 2 * npieces; ++k) {
        const int pi = k < npieces ? k : k - npieces;
        const GemvRun pz = a.pieces[pc0 + pi];
        const SharedBlock B = a.sblocks[pz.block];
        if ((k & (blockDim.x - 1)) == (int)threadIdx.x) {
            RunDesc d;
            d.mat_off = B.q_off + (k >= npieces ? (int64_t)B.n * B.ld : 0);
            d.in_off = B.in_off;
            d.row_begin = pz.row_begin;
            d.row_end = pz.row_end;
            d.ld = B.ld;
            d.ncols = B.n;
            d.block = pz.block;
            d.pair_begin = 0;
            d.pair_count = 0;
            d.ord = n_rows;
            rd[k] = d;
        }
        n_rows += pz.row_end - pz.row_begin;
    }
    const int nruns = 2 * npieces;
    const bool has_rows = warp < n_rows;
    uint32_t wseq = 0, n_done = 0, n_issued = 0;
    bool wfail = false;
    int iss_run = 0, iss_row = 0, first_run = 0, first_row = 0;
    __syncthreads();
    if (has_rows) {
        while (rd[first_run].ord + (rd[first_run].row_end - rd[first_run].row_begin) <= warp) ++first_run;
        first_row = rd[first_run].row_begin + (warp - rd[first_run].ord);
        iss_run = first_run;
        iss_row = first_row;
    }
    auto issue = [&](int k) {
        const RunDesc& d = rd[iss_run];
        bulk_load(slot(warp, k), reinterpret_cast<const T*>(a.qstore) + d.mat_off + (int64_t)iss_row * d.ld,
                  (uint32_t)((size_t)d.ld * sizeof(T)), &wbars[warp][k], evict_first_policy());
        iss_row += NW;
        while (iss_row >= rd[iss_run].row_end) {
            const int over = iss_row - rd[iss_run].row_end;
            if (iss_run + 1 == nruns) { iss_run = first_run; iss_row = first_row; break; }
            ++iss_run;
            iss_row = rd[iss_run].row_begin + over;
        }
    };
    if (has_rows) {
        if (lane == 0) {
            for (int k = 0; k < S; ++k) mbar_init(&wbars[warp][k]);
            for (int k = 0; k < S; ++k) issue(k);
        }
        n_issued = S;
    }
    // this warp's rows of run ri: f(row, acc) with the R dot products of the row with V
    auto rows_of = [&](int ri, const float* V, int live, auto&& f) {
        const RunDesc& rn = rd[ri];
        const int k0 = ((warp - rn.ord) % NW + NW) % NW;
        for (int row = rn.row_begin + k0; row < rn.row_end; row += NW, ++wseq) {
            const int k = wseq % S;
            if (!wfail && !mbar_wait(&wbars[warp][k], (wseq / S) & 1)) {
                wfail = true;
                if (lane == 0) atomicExch(a.err, 1);
            }
            if (wfail) continue;
            ++n_done;
            float acc[MR];
            row_dots(slot(warp, k), V, ldm, rn.ld, live, lane, acc);
            __syncwarp();
            if (lane == 0) {
                f(row, acc);
                issue(k);
            }
            ++n_issued;
        }
    };

    bool ok = barrier_sum<2 * MR>(a.gs, G, cta, gen, a.err, a.partials, v2, red, outv, [&](const double* sm) {
        int live = gsc.live;
        for (int s = 0; s < MR; ++s) {
            gsc.bb[s] = sm[2 * s];
            gsc.rr[s] = sm[2 * s + 1];
            if (!((live >> s) & 1)) continue;
            if (!isfinite(sm[2 * s]) || !isfinite(sm[2 * s + 1])) { gsc.status[s] = kENONFINITE; live &= ~(1 << s); }
            else if (sm[2 * s] == 0.0) live &= ~(1 << s);                 // b = 0: x = 0 below
            else if (sm[2 * s + 1] <= gsc.rtol2[s] * sm[2 * s]) live &= ~(1 << s);
        }
        gsc.live = live;
    });
    if (!ok) {
        if (threadIdx.x == 0) { for (int s = 0; s < MR; ++s) if ((gsc.live >> s) & 1) gsc.status[s] = kEDEVICE; gsc.live = 0; }
        __syncthreads();
    }
#pragma unroll
    for (int s = 0; s < MR; ++s)                       // b = 0: the solution is x = 0
        if (((gsc.started >> s) & 1) && gsc.bb[s] == 0.0)
            for (int64_t t = e0 * NP + threadIdx.x; t < e1 * NP; t += blockDim.x) a.sim[s].x[t] = 0.0;
    int par = 0, pp = 0;

    while (gsc.live) {
        const int live = gsc.live;
        // ---------------------------------------------------------------- P1
        // per piece: stage r' of the whole subdomain, commit the piece's rows, X = L^{-1} r',
        // R_0 r' (the piece that starts the subdomain), pass 1 over the piece's rows of Q^T
        double v1[MR];
#pragma unroll
        for (int s = 0; s < MR; ++s) v1[s] = 0.0;
        for (int pi = 0; pi < npieces; ++pi) {
            const RunDesc& rn = rd[pi];
            const SharedBlock B = a.sblocks[rn.block];
            const int n = B.n, ld = B.ld;
            __syncthreads();                      // the previous piece's readers are done
            for (int idx = threadIdx.x; idx < R * ld; idx += blockDim.x) {
                const int s = idx / ld, j = idx - s * ld;
                double r_ = 0.0;
                if (((live >> s) & 1) && j < n) {
                    const GroupSim& sm = a.sim[s];
                    const int64_t t = B.in_off + j;
                    const double al = gsc.pending[s] ? gsc.alpha[s] : 0.0, be = gsc.beta[s];
                    const double qk = fma(be, __ldcg(sm.q[pp] + t), __ldcg(sm.w + t));
                    r_ = fma(-al, qk, __ldcg(sm.r[par] + t));
                    if (j >= rn.row_begin && j < rn.row_end) {
                        const double pk = fma(be, __ldcg(sm.p[pp] + t), __ldcg(sm.z + t));
                        sm.p[pp ^ 1][t] = pk;
                        sm.q[pp ^ 1][t] = qk;
                        sm.x[t] = fma(al, pk, sm.x[t]);
                        sm.r[par ^ 1][t] = r_;
                        add_at(v1, s, r_ * r_);
                    }
                }
                rp[s * ldm + j] = r_;
            }
            __syncthreads();
            for (int idx = threadIdx.x; idx < R * ld; idx += blockDim.x) {
                const int s = idx / ld, k = idx - s * ld;
                float v = 0.f;
                if (((live >> s) & 1) && k < n) {
                    const int el = k / NP, ii = k - el * NP;
                    const double* Li = a.linv + ((int64_t)(B.cell0 + el) * NP + ii) * NP;
                    const double* r_ = rp + s * ldm + el * NP;
                    double acc = 0.0;
                    for (int j = 0; j <= ii; ++j) acc = fma(Li[j], r_[j], acc);
                    v = (float)acc;
                }
                X[s * ldm + k] = v;
            }
            if (coarse && rn.row_begin == 0) {
                const int pb = a.pair_begin[rn.block], pc = a.pair_count[rn.block];
                const int items = R * pc * a.nq;
                for (int w2 = warp; w2 < items; w2 += nw) {
                    const int s = w2 / (pc * a.nq), rem = w2 - s * pc * a.nq;
                    const int pj = rem / a.nq, row = rem - pj * a.nq;
                    if (!((live >> s) & 1)) continue;
                    const GemvBlock Rb = a.blocks[a.sub_pairs[pb + pj]];
                    const double* Rr = a.st64 + Rb.mat_off + (int64_t)row * Rb.ld;
                    const double* r_ = rp + s * ldm;
                    double s0 = 0.0, s1 = 0.0;
                    int j = lane;
                    for (; j + 32 < Rb.ncols; j += 64) {
                        s0 = fma(__ldg(Rr + j), r_[j], s0);
                        s1 = fma(__ldg(Rr + j + 32), r_[j + 32], s1);
                    }
                    if (j < Rb.ncols) s0 = fma(__ldg(Rr + j), r_[j], s0);
                    const double sv = warp_sum(s0 + s1);
                    if (lane == 0) a.sim[s].r0p[Rb.out_off + row] = sv;
                }
            }
            __syncthreads();
            const float* lm = a.lam + B.lam_off;
            rows_of(pi, X, live, [&](int row, const float (&acc)[MR]) {
                const float l = lm[row];
#pragma unroll
                for (int s = 0; s < MR; ++s)
                    if ((live >> s) & 1) a.sim[s].yq[B.in_off + row] = acc[s] / (chi_f + (float)a.sim[s].c * l);
            });
        }
        // stopping tests by thread 0 (0 go on, 1 converged, 2 non-finite, 3 maxit)
        ok = barrier_sum<MR>(a.gs, G, cta, gen, a.err, a.partials, v1, red, outv, [&](const double* sm) {
            int lv = gsc.live;
            for (int s = 0; s < MR; ++s) {
                if (!((lv >> s) & 1)) continue;
                gsc.it[s] += gsc.pending[s];
                gsc.pending[s] = 0;
                gsc.rr[s] = sm[s];
                const double r2 = sm[s];
                const int code = !isfinite(r2) ? 2 : (r2 <= gsc.rtol2[s] * gsc.bb[s]) ? 1
                                 : (gsc.it[s] >= gsc.maxit[s]) ? 3 : 0;
                if (code == 2) { gsc.status[s] = kENONFINITE; lv &= ~(1 << s); }
                else if (code == 1) { gsc.status[s] = kOK; lv &= ~(1 << s); }
                else if (code == 3) { gsc.status[s] = kENOTCONV; lv &= ~(1 << s); }
            }
            gsc.live = lv;
        });
        par ^= 1;
        pp ^= 1;
        if (!ok) {
            if (threadIdx.x == 0) { for (int s = 0; s < MR; ++s) if ((live >> s) & 1) gsc.status[s] = kEDEVICE; gsc.live = 0; }
            __syncthreads();
            break;
        }
        const int live2 = gsc.live;
        if (!live2) break;
        // ---------------------------------------------------------------- P2 + coarse
        // pass 2 over the pieces' rows of Q with the whole subdomain's Y; z_loc = L^{-T} V
        for (int pi = 0; pi < npieces; ++pi) {
            const RunDesc& rn = rd[npieces + pi];
            const SharedBlock B = a.sblocks[rn.block];
            const int n = B.n, ld = B.ld;
            __syncthreads();
            for (int idx = threadIdx.x; idx < R * ld; idx += blockDim.x) {
                const int s = idx / ld, j = idx - s * ld;
                Y[s * ldm + j] = (((live2 >> s) & 1) && j < n) ? __ldcg(a.sim[s].yq + B.in_off + j) : 0.f;
            }
            __syncthreads();
            rows_of(npieces + pi, Y, live2, [&](int row, const float (&acc)[MR]) {
#pragma unroll
                for (int s = 0; s < MR; ++s)
                    if ((live2 >> s) & 1) X[s * ldm + row] = acc[s];
            });
            __syncthreads();
            const int len = rn.row_end - rn.row_begin;    // element-aligned
            for (int idx = threadIdx.x; idx < R * len; idx += blockDim.x) {
                const int s = idx / len, k = rn.row_begin + (idx - s * len);
                if (!((live2 >> s) & 1)) continue;
                const int el = k / NP, ii = k - el * NP;
                const double* L0 = a.linv + (int64_t)(B.cell0 + el) * NP * NP;
                const float* V = X + s * ldm + el * NP;
                double acc = 0.0;
                for (int j = ii; j < NP; ++j) acc = fma(L0[j * NP + ii], (double)V[j], acc);
                a.sim[s].zl[B.in_off + k] = acc;
            }
        }
        // coarse solves, each row once (rows [c0, c1) of this CTA, to global memory); the
        // barrier below then completes y0 and the neighbours' z_loc for the CM phase
#pragma unroll
        for (int s = 0; s < MR; ++s) {
            if (!coarse || !((live2 >> s) & 1) || c1 <= c0) continue;
            const GroupSim& sm = a.sim[s];
            __syncthreads();                      // r0s of the previous simulation is done
            for (int idx = threadIdx.x; idx < a.n0; idx += blockDim.x) {
                const int J = idx / a.nq, kq = idx - J * a.nq;
                double s_r = 0.0;
                for (int64_t p2 = a.pair_ptr[J]; p2 < a.pair_ptr[J + 1]; ++p2)
                    s_r += __ldcg(sm.r0p + p2 * a.nq + kq);
                r0s[idx] = s_r;
            }
            __syncthreads();
            for (int row = c0 + warp; row < c1; row += nw) {
                const double* Kr = sm.K0inv + (int64_t)row * a.ld0;
                double s0 = 0.0, s1 = 0.0;
                int c = lane;
                for (; c + 32 < a.n0; c += 64) {
                    s0 = fma(__ldg(Kr + c), r0s[c], s0);
                    s1 = fma(__ldg(Kr + c + 32), r0s[c + 32], s1);
                }
                if (c < a.n0) s0 = fma(__ldg(Kr + c), r0s[c], s0);
                const double y = warp_sum(s0 + s1);
                if (lane == 0) sm.y0[row] = y;
            }
        }
        ok = grid_barrier(a.gs, G, gen, a.err);
        if (!ok) {
            if (threadIdx.x == 0) { for (int s = 0; s < MR; ++s) if ((live2 >> s) & 1) gsc.status[s] = kEDEVICE; gsc.live = 0; }
            __syncthreads();
            break;
        }
        // ---------------------------------------------------------------- CM
        double v3[3 * MR];
#pragma unroll
        for (int k = 0; k < 3 * MR; ++k) v3[k] = 0.0;
#pragma unroll
        for (int s = 0; s < MR; ++s) {
            if (!((live2 >> s) & 1)) continue;
            const GroupSim& sm = a.sim[s];
            const double* rk = sm.r[par];
            const double* qk = sm.q[pp];
            for (int ch = ch0; ch < ch1; ++ch) {
                const int64_t ce0 = a.chunk_elem[ch], ce1 = a.chunk_elem[ch + 1];
                const int n_chunk = (int)(ce1 - ce0);
                const int32_t* need = a.need + a.need_ptr[ch];
                const int n_need = a.need_ptr[ch + 1] - a.need_ptr[ch];
                __syncthreads();
                for (int idx = threadIdx.x; idx < n_need * NP; idx += blockDim.x) {
                    const int l = idx / NP, j = idx - l * NP;
                    const int64_t e = need[l], t = e * NP + j;
                    double v = __ldcg(sm.zl + t);
                    if (coarse) {
                        const double* Tr = a.T + t * a.nq;
                        const double* y = sm.y0 + (int64_t)a.agg[e] * a.nq;
                        for (int kq = 0; kq < a.nq; ++kq) v = fma(__ldg(Tr + kq), __ldcg(y + kq), v);
                    }
                    pn[idx] = v;
                    if (l < n_chunk) sm.z[t] = v;
                }
                __syncthreads();
                local_rows<NP>(a.row_ptr, a.col_local, sm.val, pn, ce0, ce1, [&](int64_t e, int ii, double kz) {
                    const int64_t t = e * NP + ii;
                    const double zv = pn[(e - ce0) * NP + ii];
                    sm.w[t] = kz;
                    v3[3 * s] = fma(__ldcg(rk + t), zv, v3[3 * s]);
                    v3[3 * s + 1] = fma(zv, __ldcg(qk + t), v3[3 * s + 1]);
                    v3[3 * s + 2] = fma(zv, kz, v3[3 * s + 2]);
                });
            }
        }
        // beta, p.q, alpha per simulation by thread 0 (2 non-finite, 4 breakdown)
        ok = barrier_sum<3 * MR>(a.gs, G, cta, gen, a.err, a.partials, v3, red, outv, [&](const double* sm) {
            int lv = gsc.live;
            for (int s = 0; s < MR; ++s) {
                if (!((lv >> s) & 1)) continue;
                const double rz_new = sm[3 * s], zq = sm[3 * s + 1], zw = sm[3 * s + 2];
                if (!isfinite(rz_new) || !isfinite(zq) || !isfinite(zw)) { gsc.status[s] = kENONFINITE; lv &= ~(1 << s); continue; }
                double bnew;
                if (gsc.it[s] == 0) bnew = 0.0;
                else if (gsc.flex[s]) bnew = -gsc.alpha[s] * zq / gsc.rz[s];
                else bnew = rz_new / gsc.rz[s];
                const double pq_new = zw + 2.0 * bnew * zq + bnew * bnew * gsc.pq[s];
                if (!isfinite(bnew) || rz_new == 0.0 || !(pq_new > 0.0) || !isfinite(pq_new)) {
                    gsc.status[s] = kEBREAKDOWN; lv &= ~(1 << s); continue;
                }
                gsc.rz[s] = rz_new;
                gsc.alpha[s] = rz_new / pq_new;
                gsc.beta[s] = bnew;
                gsc.pq[s] = pq_new;
                gsc.pending[s] = 1;
            }
            gsc.live = lv;
        });
        if (!ok) {
            if (threadIdx.x == 0) { for (int s = 0; s < MR; ++s) if ((live2 >> s) & 1) gsc.status[s] = kEDEVICE; gsc.live = 0; }
            __syncthreads();
            break;
        }
    }
    if (has_rows) {                       // bounded wait for this warp's copies still in flight
        for (uint32_t c = n_done; c < n_issued; ++c)
            if (!mbar_wait(&wbars[warp][c % S], (c / S) & 1)) break;
    }
    if (cta == 0 && threadIdx.x == 0) {
        for (int s = 0; s < MR; ++s) {
            if (!((gsc.started >> s) & 1)) continue;
            PcgScalars* sc = a.sim[s].sc;
            sc->bb = gsc.bb[s];
            sc->rr = gsc.rr[s];
            sc->relres = gsc.bb[s] > 0.0 ? sqrt(gsc.rr[s] / gsc.bb[s]) : 0.0;
            sc->it = gsc.it[s];
            sc->status = gsc.status[s];
            sc->done = 1;
            sc->pass = 0;                 // x is single-buffered here
        }
    }
}

template <typename T, int NP>
__global__ void __launch_bounds__(kPersistThreads, 1)
pcg_group_kernel(const GroupArgs* __restrict__ args, const int2* __restrict__ map) {
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(16) GroupArgs ga;
    const int2 m = map[blockIdx.x];
    {
        static_assert(sizeof(GroupArgs) % 8 == 0, "GroupArgs is copied as 8-byte words");
        const uint64_t* src = reinterpret_cast<const uint64_t*>(args + m.x);
        uint64_t* dst = reinterpret_cast<uint64_t*>(&ga);
        for (int k = threadIdx.x; k < (int)(sizeof(GroupArgs) / 8); k += blockDim.x) dst[k] = src[k];
    }
    __syncthreads();
    pcg_group_cta<T, NP>(ga, m.y, (unsigned)ga.grid, smem);
}

static const void* group_fn(int qdtype, int np) {
    if (qdtype == 1) {
        switch (np) {
            case 3: return (const void*)pcg_group_kernel<float, 3>;
            case 6: return (const void*)pcg_group_kernel<float, 6>;
            case 10: return (const void*)pcg_group_kernel<float, 10>;
            default: return nullptr;
        }
    }
    switch (np) {
        case 3: return (const void*)pcg_group_kernel<__nv_bfloat16, 3>;
        case 6: return (const void*)pcg_group_kernel<__nv_bfloat16, 6>;
        case 10: return (const void*)pcg_group_kernel<__nv_bfloat16, 10>;
        default: return nullptr;
    }
}

cudaError_t launch_pcg_groups(int qdtype, int np, const GroupArgs* args_dev, const int2* map_dev,
                              int n_cta, size_t smem, cudaStream_t s) {
    // the shared-memory limit was raised by group_occupancy at set-up (graph capture)
    const void* fn = group_fn(qdtype, np);
    if (!fn || n_cta < 1) return cudaErrorInvalidValue;
    void* args[] = {(void*)&args_dev, (void*)&map_dev};
    return cudaLaunchCooperativeKernel(fn, dim3(n_cta), dim3(kPersistThreads), args, smem, s);
}

cudaError_t group_occupancy(int qdtype, int np, size_t smem, int* blocks_per_sm) {
    const void* fn = group_fn(qdtype, np);
    if (!fn) return cudaErrorInvalidValue;
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, fn);
    if (e != cudaSuccess) return e;
    if ((size_t)fa.maxDynamicSharedSizeBytes < smem) {
        e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, fn, kPersistThreads, smem);
}

}  // namespace polydg
