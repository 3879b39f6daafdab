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
//       iterations (the inverses are constant; a fraction of their lines, chosen by
//       the plan, stays in L2 as evict-last); R_0 r' for the subdomains the
//       CTA stages first; partial |r'|^2                     -> barrier, test
//   CM  y0 = K_0^{-1} R_0 r' for the agglomerates the CTA's elements touch
//       (redundantly per CTA; a distributed coarse phase with one more barrier
//       when the coarse space is large), z = z_loc + R_0^T y0 for its elements
//       and their face neighbours in shared memory, w = K z on its elements
//       (fp64); partial r'.z, z.q_k, z.w                      -> barrier, beta, alpha
// Every CTA sums the per-CTA partials in the same order, so all CTAs hold
// bit-identical scalars and take the same branches; the result is deterministic.
// Waits (grid barriers, mbarriers) are bounded: on timeout the kernel raises an
// error flag, waits (bounded) for its own copies in flight and stops.  A grid
// barrier gives up after a.wait_limit polls.
// With a.apply_only the launch applies the preconditioner once, z = B_ad^{-1} b: r = b,
// one P phase (alpha = beta = 0, so r' = r), the coarse solve and the z part of the CM
// phase, then it stops -- the same code that every PCG iteration runs.
#include <type_traits>

#include <cuda_runtime.h>
#include <cuda_bf16.h>

#include "device.cuh"
#include "kernels.h"
#include "pcg_device.cuh"

namespace polydg {

// The whole solve as seen by CTA `cta` of the G CTAs working on it.
template <int DT, int NP, bool CMS>
__device__ __forceinline__ void pcg_solve_cta(const PersistArgs& a, const int cta, const unsigned G,
                                              unsigned char* smem) {
    using T = typename StoreType<DT>::T;
    using X = typename StoreType<DT>::X;
    constexpr int NW = kPersistThreads / 32;
    __shared__ __align__(8) uint64_t wbars[NW][kMaxWarpStages];
    __shared__ __align__(8) uint64_t cmbars[NW][kMaxCmStages];
    __shared__ double scal[3];            // alpha, beta, pq from thread 0
    __shared__ int scode;                 // thread 0's verdict after a grid sum
    __shared__ double red[3 * kPersistThreads], outv[3];   // grid-sum scratch

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    PcgScalars* sc = a.sc;
    if (sc->done) return;             // a failed earlier step: nothing to do (uniform)
    const bool flexible = sc->flexible != 0;
    const double rtol2 = sc->rtol2;
    const int maxit = sc->maxit;
    const bool apply = a.apply_only != 0;
    const bool sym = DT == 1 && CMS && a.sym_bufld > 0;   // P phase from the symmetric pair-row store
    const uint32_t wl = a.wait_limit;
    // Pipelined PCG (sc->flexible == 2; Ghysels and Vanroose's rearrangement): per iteration
    // the P phase applies the local solves to w and sums gamma = r.u, delta = w.u and |r|^2 in
    // the same pass (the one reduction, at the first barrier: stopping test, alpha, beta);
    // the CM phase forms m = B w, n = K m and updates z = n + beta z, q = m + beta q,
    // s = w + beta s, p = u + beta p, x += alpha p, r -= alpha s, u -= alpha q, w -= alpha z
    // on its own rows, then a plain barrier.  The first pass forms u = B r and w = K u.
    // Roles of the buffers: r = r[0], u = r[1], w = w, p = p[0], s = p[1], q = q[0],
    // z = q[1], B's local part = zl.
    const bool pipe = sc->flexible == 2 && !apply;
    bool pinit = pipe;
    double gam_old = 0.0, alp_old = 0.0;        // thread 0: gamma and alpha of the last iteration
    unsigned gen = 0;                 // barrier target of thread 0 (gs->count is 0 at launch)

    const int S = a.wstages;                                       // copy slots per warp
    auto slot = [&](int w, int k) { return reinterpret_cast<T*>(smem + ((size_t)w * S + k) * a.slot_bytes); };
    X* xs = reinterpret_cast<X*>(smem + a.xs_off);                 // r' in the store's arithmetic
    double* rp = reinterpret_cast<double*>(smem + a.rp_off);       // r' (fp64)
    double* r0s = reinterpret_cast<double*>(smem + a.r0_off);      // [n0]
    double* y0l = reinterpret_cast<double*>(smem + a.y0_off);      // y0 of the CTA's agglomerates
    double* pn = reinterpret_cast<double*>(smem + a.pn_off);       // x or z of the needed elements
    RunDesc* rd = reinterpret_cast<RunDesc*>(smem + a.td_off);     // this CTA's runs

    const int64_t e0 = a.elem_ptr[cta], e1 = a.elem_ptr[cta + 1];
    const int n_own = (int)(e1 - e0);
    const int ch0 = a.cta_chunk[cta], ch1 = a.cta_chunk[cta + 1];
    const int32_t* aggs = a.need_agg + a.need_agg_ptr[cta];
    const int n_aggs = a.need_agg_ptr[cta + 1] - a.need_agg_ptr[cta];
    const int run0 = a.run_ptr[cta], nruns = a.run_ptr[cta + 1] - run0;
    const int c0 = a.crow_ptr[cta], c1 = a.crow_ptr[cta + 1];
    const bool coarse = a.n0 > 0;

    // ---- init: r = b - K x on own elements; p, q, z, w = 0; |b|^2, |r|^2
    for (int64_t t = e0 * NP + threadIdx.x; t < e1 * NP; t += blockDim.x) {
        a.p[0][t] = 0.0; a.p[1][t] = 0.0; a.q[0][t] = 0.0; a.q[1][t] = 0.0;
        a.z[t] = 0.0; a.w[t] = 0.0;
    }
    double v2[2] = {0.0, 0.0};
    if (apply) {                                // r = b: the preconditioner's input
        for (int64_t t = e0 * NP + threadIdx.x; t < e1 * NP; t += blockDim.x) {
            const double bv = a.b[t];
            a.r[0][t] = bv;
            v2[0] = fma(bv, bv, v2[0]);
        }
        v2[1] = v2[0];
    }
    for (int ch = ch0; ch < (apply ? ch0 : ch1); ++ch) {        // chunks of the CTA's elements
        const int64_t ce0 = a.chunk_elem[ch], ce1 = a.chunk_elem[ch + 1];
        const int32_t* need = a.need + a.need_ptr[ch];
        const int n_need = a.need_ptr[ch + 1] - a.need_ptr[ch];
        __syncthreads();
        for (int idx = threadIdx.x; idx < n_need * NP; idx += blockDim.x) {
            const int l = idx / NP;
            pn[idx] = __ldcg(a.x + (int64_t)need[l] * NP + (idx - l * NP));
        }
        __syncthreads();
        local_rows<NP>(a.row_ptr, a.col_local, a.val, pn, ce0, ce1, [&](int64_t e, int i, double kx) {
            const int64_t t = e * NP + i;
            const double bv = a.b[t], rv = bv - kx;
            a.r[0][t] = rv;
            v2[0] = fma(bv, bv, v2[0]);
            v2[1] = fma(rv, rv, v2[1]);
        });
    }
    // The CTA's rows of the local inverses, run after run, are dealt to the warps in
    // turn: warp w owns the rows at positions w, w + NW, ... of that sequence and
    // streams them, one row per copy, through its own ring of S slots.
    int n_rows = 0;
    for (int k = 0; k < (a.small ? 0 : nruns); ++k) {   // small subdomains: no run table, no copies
        const GemvRun rn = a.runs[run0 + k];
        if ((k & (blockDim.x - 1)) == (int)threadIdx.x) {
            const GemvBlock B = a.blocks[rn.block];
            RunDesc d;
            d.mat_off = B.mat_off;
            d.in_off = B.in_off;
            d.row_begin = rn.row_begin;
            d.row_end = rn.row_end;
            d.ld = B.ld;
            d.ncols = B.ncols;
            d.block = rn.block;
            d.pair_begin = B.pair_begin;
            d.pair_count = B.pair_count;
            if (sym) {                            // whole subdomain: its pair rows
                d.mat_off = B.sym_off;
                d.row_begin = 0;
                d.row_end = (B.ncols + 1) / 2;
                d.ld = sym_ld(B.ncols);
            }
            d.ord = n_rows;
            rd[k] = d;
        }
        n_rows += sym ? (rn.row_end - rn.row_begin + 1) / 2 : rn.row_end - rn.row_begin;
    }
    const bool has_rows = warp < n_rows;
    const int rows_w = has_rows ? (n_rows - 1 - warp) / NW + 1 : 0;   // this warp's rows per P phase
    uint32_t wseq = 0;                // rows this warp consumed so far (all iterations)
    uint32_t n_done = 0, n_issued = 0;  // copies seen complete / issued (copy c: slot c % S)
    int iss_left = 0;                 // rows of the current P phase not yet issued
    bool wfail = false;               // a copy wait timed out: no more waits or copies
    // issue side (lane 0): run and row of the warp's next copy; after the CTA's last
    // run it starts over at the warp's first row (the next P phase's first copy).  With
    // the CM ring (CMS) the copies stop at the end of each P phase, which leaves the
    // slots to the CM phase, and the next P phase's first ones go out when it ends.
    int iss_run = 0, iss_row = 0, first_run = 0, first_row = 0;
    __syncthreads();
    if (has_rows) {
        while (rd[first_run].ord + (rd[first_run].row_end - rd[first_run].row_begin) <= warp) ++first_run;
        first_row = rd[first_run].row_begin + (warp - rd[first_run].ord);
        iss_run = first_run;
        iss_row = first_row;
    }
    const uint64_t l2pol = stream_policy(a.l2_keep);
    auto issue = [&](int k) {
        const RunDesc& d = rd[iss_run];
        if (sym)
            bulk_load(slot(warp, k), reinterpret_cast<const float*>(a.store) + d.mat_off + (int64_t)iss_row * d.ld,
                      (uint32_t)(sym_len(d.ncols, iss_row) * sizeof(float)), &wbars[warp][k], l2pol);
        else
            bulk_load(slot(warp, k), reinterpret_cast<const T*>(a.store) + d.mat_off + (int64_t)iss_row * d.ld,
                      (uint32_t)((size_t)d.ld * sizeof(T)), &wbars[warp][k], l2pol);
        iss_row += NW;
        while (iss_row >= rd[iss_run].row_end) {
            const int over = iss_row - rd[iss_run].row_end;
            if (iss_run + 1 == nruns) { iss_run = first_run; iss_row = first_row; break; }
            ++iss_run;
            iss_row = rd[iss_run].row_begin + over;
        }
    };
    // lane 0: the first copies of a P phase (at most S, at most the warp's rows)
    auto issue_first = [&]() {
        const int m = min(S, rows_w);
        if (lane == 0)
            for (int j = 0; j < m; ++j) issue((int)((n_issued + j) % S));
        n_issued += m;
        iss_left = rows_w - m;
    };
    if (has_rows) {
        if (lane == 0)
            for (int k = 0; k < S; ++k) mbar_init(&wbars[warp][k]);
        if (CMS) {
            issue_first();
        } else {                      // no CM ring: the copies run on into the next P phase
            if (lane == 0)
                for (int k = 0; k < S; ++k) issue(k);
            n_issued = S;
        }
    }
    bool p_armed = true;              // the coming P phase's first copies are in flight
    // CM phase: this warp's elements (chunk by chunk: ce0 + warp, + NW, ...) stream their
    // K_h block-row panels through CS slots of cm_slot_bytes in [0, y0_off)
    const int CS = CMS ? a.cm_stages : 1;     // (1: a divisor for the dead code of CMS = false)
    uint32_t cm_base = 0;             // panels of the earlier CM phases (all consumed)
    bool cmfail = false;
    // lane 0: element e's panel into slot k (from the 16-byte boundary at or below it;
    // the values array carries two doubles of slack past its end)
    auto cm_issue = [&](int k, int64_t e) {
        const int64_t b0 = a.row_ptr[e], b1 = a.row_ptr[e + 1];
        const uintptr_t src = reinterpret_cast<uintptr_t>(a.val + b0 * NP * NP);
        const uintptr_t s16 = src & ~(uintptr_t)15;
        const uint32_t bytes = (uint32_t)(((uintptr_t)(b1 - b0) * NP * NP * 8 + (src - s16) + 15) & ~(uintptr_t)15);
        bulk_load(smem + ((size_t)warp * CS + k) * a.cm_slot_bytes, reinterpret_cast<const void*>(s16), bytes,
                  &cmbars[warp][k], evict_first_policy());
    };
    if (CMS && CS > 0 && lane == 0)
        for (int k = 0; k < CS; ++k) mbar_init(&cmbars[warp][k]);
    bool ok = barrier_sum<2>(a.gs, G, cta, gen, a.err, a.partials, v2, red, outv, [](const double*) {}, wl);
    const double bb = v2[0];
    double rr = v2[1];
    int status = kOK, it = 0, done = 0, par = 0, pp = 0;
    double alpha = 0.0, beta = 0.0, rz = 0.0, pq = 0.0, relres = 0.0;
    int pending = 0;                  // alpha p_k / alpha q_k not yet committed to x, r
    if (!ok) { status = kEDEVICE; done = 1; }
    else if (!isfinite(bb) || !isfinite(rr)) { status = kENONFINITE; done = 1; }
    else if (apply) { relres = 1.0; }          // one application: no stopping test
    else if (bb == 0.0) { done = 2; }
    else { relres = sqrt(rr / bb); if (rr <= rtol2 * bb) done = 1; }

    // per-CTA work time of the P and the coarse + CM phases (thread 0, SM cycles), for
    // the tile-partition autotuner; the clock reads are skipped unless requested
    const bool timing = a.cta_cycles != nullptr;
    long long cyc_p = 0, cyc_cm = 0, t_mark = 0;
    while (!done) {
        // ---------------------------------------------------------------- P
        if (timing && threadIdx.x == 0) t_mark = clock64();
        if (CMS && !p_armed && has_rows && !wfail) issue_first();
        p_armed = true;
        const double* rin = a.r[par];
        double* rout = a.r[par ^ 1];
        const double* pold = a.p[pp];
        const double* qold = a.q[pp];
        double* pnew = a.p[pp ^ 1];
        double* qnew = a.q[pp ^ 1];
        const double al = pending ? alpha : 0.0, be = beta;
        double v1[1] = {0.0};                     // |r'|^2
        double vp[3] = {0.0, 0.0, 0.0};           // pipelined: r.u, w.u, r.r on own rows
        const double* vin = pinit ? a.r[0] : a.w; // pipelined: the input of the local solves
        auto pdots = [&](int64_t t) {
            const double rt = __ldcg(a.r[0] + t), ut = __ldcg(a.r[1] + t), wt = __ldcg(a.w + t);
            vp[0] = fma(rt, ut, vp[0]);
            vp[1] = fma(wt, ut, vp[1]);
            vp[2] = fma(rt, rt, vp[2]);
        };
        if (a.identity && pipe) {
            for (int64_t t = e0 * NP + threadIdx.x; t < e1 * NP; t += blockDim.x) {
                a.zl[t] = __ldcg(vin + t);
                if (!pinit) pdots(t);
            }
        } else if (a.identity) {
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
        } else if (a.small) {
            // whole subdomains of at most 32 DOFs, one per warp at a time: lane j commits
            // DOF j (p_k, q_k, x, r'), then computes row j of K_i^{-1} r' and row j of each
            // restriction block with r' broadcast by shuffles (no CTA barrier, no copies)
            for (int k = warp; k < nruns; k += nw) {
                const GemvRun rn = a.runs[run0 + k];
                const GemvBlock B = a.blocks[rn.block];
                const int n = B.ncols;
                const int64_t t = B.in_off + lane;
                double r_ = 0.0;
                if (lane < n && pipe) {
                    r_ = __ldcg(vin + t);
                    if (!pinit) pdots(t);
                } else if (lane < n) {
                    const double qk = fma(be, __ldcg(qold + t), __ldcg(a.w + t));
                    r_ = fma(-al, qk, __ldcg(rin + t));
                    const double pk = fma(be, __ldcg(pold + t), __ldcg(a.z + t));
                    pnew[t] = pk;
                    qnew[t] = qk;
                    a.x[t] = fma(al, pk, a.x[t]);
                    rout[t] = r_;
                    v1[0] = fma(r_, r_, v1[0]);
                }
                const X xr = (X)r_;
                const T* Ar = reinterpret_cast<const T*>(a.store) + B.mat_off + (int64_t)min(lane, n - 1) * B.ld;
                X acc = (X)0;
                for (int c = 0; c < n; ++c) acc = fma_x(store_elem(Ar + c), __shfl_sync(0xffffffffu, xr, c), acc);
                if (lane < n) a.zl[t] = (double)acc;
                if (coarse) {
                    for (int pi = 0; pi < B.pair_count; ++pi) {
                        const GemvBlock R = a.blocks[a.sub_pairs[B.pair_begin + pi]];
                        const double* Rr = a.st64 + R.mat_off + (int64_t)min(lane, R.nrows - 1) * R.ld;
                        double sv = 0.0;
                        for (int c = 0; c < R.ncols; ++c) sv = fma(__ldg(Rr + c), __shfl_sync(0xffffffffu, r_, c), sv);
                        if (lane < R.nrows) a.r0p[R.out_off + lane] = sv;
                    }
                }
            }
        } else {
            for (int ri = 0; ri < nruns; ++ri) {
                const RunDesc& rn = rd[ri];
                // r' of the run's subdomain (all its DOFs: the product's input), and
                // the commit of the run's own rows: p_k, q_k, x += alpha p_k, r'
                __syncthreads();                  // the previous run's readers of xs / rp are done
                // (symmetric store: the run is the whole subdomain, every DOF its own)
                const int xlen = sym ? (rn.ncols + 3) & ~3 : rn.ld;
                for (int j = threadIdx.x; j < xlen; j += blockDim.x) {
                    double r_ = 0.0;
                    const bool own = sym || (j >= rn.row_begin && j < rn.row_end);
                    if (j < rn.ncols && pipe) {
                        const int64_t t = rn.in_off + j;
                        r_ = __ldcg(vin + t);
                        if (!pinit && own) pdots(t);
                    } else if (j < rn.ncols) {
                        const int64_t t = rn.in_off + j;
                        const double qk = fma(be, __ldcg(qold + t), __ldcg(a.w + t));
                        r_ = fma(-al, qk, __ldcg(rin + t));
                        if (own) {
                            const double pk = fma(be, __ldcg(pold + t), __ldcg(a.z + t));
                            pnew[t] = pk;
                            qnew[t] = qk;
                            a.x[t] = fma(al, pk, a.x[t]);
                            rout[t] = r_;
                            v1[0] = fma(r_, r_, v1[0]);
                        }
                    }
                    rp[j] = r_;
                    if (DT != 0) xs[j] = (X)r_;
                }
                __syncthreads();
                if (rn.row_begin == 0 && coarse) {   // this CTA streams the subdomain's first rows: R_0 r'
                    for (int pi = 0; pi < rn.pair_count; ++pi) {
                        const GemvBlock R = a.blocks[a.sub_pairs[rn.pair_begin + pi]];
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
                // this warp's rows of the run: z_loc = row . r'
                const X* xin = (DT == 0) ? reinterpret_cast<const X*>(rp) : xs;
                const int k0 = ((warp - rn.ord) % NW + NW) % NW;
                if constexpr (DT == 1 && CMS) {
                    if (sym) {                    // pair rows; column sums in registers
                        float4 cacc[kSymT];
                        // row sums: one per row, each written once (after the warps' buffers)
                        float* rsum = reinterpret_cast<float*>(smem + a.r0_off) + NW * a.sym_bufld;
#pragma unroll
                        for (int t = 0; t < kSymT; ++t) cacc[t] = make_float4(0.f, 0.f, 0.f, 0.f);
                        for (int row = k0; row < rn.row_end; row += NW, ++wseq) {
                            const int k = wseq % S;
                            if (!wfail && !mbar_wait(&wbars[warp][k], (wseq / S) & 1)) {
                                wfail = true;
                                if (lane == 0) atomicExch(a.err, 1);
                            }
                            if (wfail) continue;
                            ++n_done;
                            sym_pair(reinterpret_cast<const float*>(slot(warp, k)), xs, rn.ncols, row, lane, cacc,
                                     rsum);
                            __syncwarp();         // every lane is done with the slot
                            if (!CMS || iss_left > 0) {
                                if (lane == 0) issue(k);
                                ++n_issued;
                                --iss_left;
                            }
                        }
                        // z_loc: the row sum and the warps' column sums in warp order
                        // (deterministic); the buffers are in r0s, idle until the coarse phase
                        float* buf = reinterpret_cast<float*>(smem + a.r0_off);
                        __syncthreads();
#pragma unroll
                        for (int t = 0; t < kSymT; ++t)
                            if (128 * t < rn.ncols)
                                *reinterpret_cast<float4*>(buf + warp * a.sym_bufld + 128 * t + 4 * lane) = cacc[t];
                        __syncthreads();
                        for (int j = threadIdx.x; j < rn.ncols; j += blockDim.x) {
                            float sv = rsum[j];
                            for (int w = 0; w < NW; ++w) sv += buf[w * a.sym_bufld + j];
                            a.zl[rn.in_off + j] = (double)sv;
                        }
                        continue;
                    }
                }
                for (int row = rn.row_begin + k0; row < rn.row_end; row += NW, ++wseq) {
                    const int k = wseq % S;
                    if (!wfail && !mbar_wait(&wbars[warp][k], (wseq / S) & 1)) {
                        wfail = true;
                        if (lane == 0) atomicExch(a.err, 1);
                    }
                    if (wfail) continue;          // the solve stops with an error at the next barrier
                    ++n_done;
                    const double zr = row_dot(slot(warp, k), xin, rn.ld, lane, 0, 1);
                    __syncwarp();                 // every lane is done with the slot
                    if (lane == 0) a.zl[rn.in_off + row] = zr;
                    if (!CMS || iss_left > 0) {
                        if (lane == 0) issue(k);
                        ++n_issued;
                        --iss_left;
                    }
                }
            }
        }
        p_armed = false;
        if (threadIdx.x == 0 && n_own > 0) {     // K_h rows of the CM phase's first chunk into L2
            const int64_t pe1 = a.chunk_elem[ch0 + 1];
            // a bulk prefetch takes a 16-byte aligned address and a multiple of 16 bytes;
            // an n_p x n_p fp64 block is 8 bytes short of that for odd n_p (3, 15), so both
            // ends are rounded down (val itself is 256-byte aligned: lo stays inside it)
            const uintptr_t lo = reinterpret_cast<uintptr_t>(a.val + (int64_t)a.row_ptr[e0] * NP * NP) & ~(uintptr_t)15;
            const uintptr_t hi = reinterpret_cast<uintptr_t>(a.val + (int64_t)a.row_ptr[pe1] * NP * NP) & ~(uintptr_t)15;
            for (uintptr_t c = lo; c < hi; c += 65536)
                prefetch_l2(reinterpret_cast<const void*>(c), (uint32_t)min((uintptr_t)65536, hi - c));
        }
        // stopping test by thread 0: 0 go on, 1 converged, 2 non-finite, 3 maxit
        if (timing) {
            __syncthreads();
            if (threadIdx.x == 0) cyc_p += clock64() - t_mark;
        }
        int code = 0;
        if (pipe && pinit) {
            ok = grid_barrier(a.gs, G, gen, a.err, wl);
        } else if (pipe) {
            // the iteration's one reduction: stopping test on |r_k|, then beta and alpha
            ok = barrier_sum<3>(a.gs, G, cta, gen, a.err, a.partials, vp, red, outv, [&](const double* sm) {
                const double gam = sm[0], del = sm[1], r2 = sm[2];
                if (!isfinite(gam) || !isfinite(del) || !isfinite(r2)) { scode = 2; return; }
                if (r2 <= rtol2 * bb) { scode = 1; return; }
                if (it >= maxit) { scode = 3; return; }
                double bt = 0.0, den = del;
                if (it > 0) {
                    bt = gam / gam_old;
                    den = del - bt * gam / alp_old;
                }
                const double al_ = gam / den;
                if (!(den > 0.0) || !isfinite(al_) || !isfinite(bt) || gam == 0.0) { scode = 4; return; }
                scal[0] = al_;
                scal[1] = bt;
                scode = 0;
                if (a.trace && cta == 0) {        // alpha_k and beta_{k-1}, as the textbook form's
                    if (it < a.trace_cap) a.trace[it] = al_;
                    if (it > 0 && it - 1 < a.trace_cap) a.trace[a.trace_cap + it - 1] = bt;
                }
                gam_old = gam;
                alp_old = al_;
            }, wl);
            rr = vp[2];
            code = scode;
        } else {
            ok = barrier_sum<1>(a.gs, G, cta, gen, a.err, a.partials, v1, red, outv, [&](const double* sm) {
                const double r2 = sm[0];
                scode = !isfinite(r2) ? 2 : apply ? 0 : (r2 <= rtol2 * bb) ? 1 : (it + pending >= maxit) ? 3 : 0;
            }, wl);
            rr = v1[0];
            it += pending;
            pending = 0;
            par ^= 1;
            pp ^= 1;
            code = scode;
        }
        if (!ok) { status = kEDEVICE; break; }
        if (code == 2) { status = kENONFINITE; break; }
        if (code == 1) { status = kOK; break; }
        if (code == 3) { status = kENOTCONV; break; }
        if (code == 4) { status = kEBREAKDOWN; break; }
        const double pal = pipe ? scal[0] : 0.0, pbe = pipe ? scal[1] : 0.0;
        const double* rk = a.r[par];              // r_{k+1}
        const double* qk = a.q[pp];               // q_k
        if (timing && threadIdx.x == 0) t_mark = clock64();
        // ---------------------------------------------------------------- coarse
        if (coarse) {
            // R_0 r' = the pair partials summed per coarse DOF, by groups of L lanes (L =
            // pair_lanes, a power of 2) and a shuffle tree, in one fixed order (the same
            // bits wherever a sum is formed).  Split mode: this CTA sums its slice of the
            // coarse DOFs into r0g, a grid barrier, then the CTAs that need R_0 r' load it;
            // otherwise every such CTA sums all of them.
            const int L = a.pair_lanes, gl = lane & (L - 1);
            const int per_pass = (int)blockDim.x / L;
            auto pair_sums = [&](int i0, int i1, double* out) {
                for (int base = i0; base < i1; base += per_pass) {
                    const int idx = base + (int)threadIdx.x / L;
                    double s_r = 0.0;
                    if (idx < i1) {
                        const int J = idx / a.nq, kq = idx - J * a.nq;
                        for (int64_t p2 = a.pair_ptr[J] + gl; p2 < a.pair_ptr[J + 1]; p2 += L)
                            s_r += __ldcg(a.r0p + p2 * a.nq + kq);
                    }
                    for (int o = L >> 1; o > 0; o >>= 1) s_r += __shfl_xor_sync(0xffffffffu, s_r, o);
                    if (idx < i1 && gl == 0) out[idx] = s_r;
                }
            };
            if (a.r0_split) {
                pair_sums((int)(((int64_t)a.n0 * cta) / G), (int)(((int64_t)a.n0 * (cta + 1)) / G), a.r0g);
                ok = grid_barrier(a.gs, G, gen, a.err, wl);
                if (!ok) { status = kEDEVICE; break; }
                if (a.redundant || c1 > c0) {
                    for (int idx = threadIdx.x; idx < a.n0; idx += blockDim.x) r0s[idx] = __ldcg(a.r0g + idx);
                    __syncthreads();
                }
            } else if (a.redundant || c1 > c0) {
                pair_sums(0, a.n0, r0s);
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
                // eight rows per warp, four lanes per row: two shuffle levels per row
                // instead of a 32-lane butterfly (fp64 adds are scarce on this GPU)
                const int sub = lane >> 2, l4 = lane & 3, nrows = n_aggs * a.nq;
                for (int base = warp * 8; base < nrows; base += nw * 8) {
                    const int w2 = base + sub;
                    double acc = 0.0;
                    if (w2 < nrows) {
                        const int jl = w2 / a.nq, kq = w2 - jl * a.nq;
                        const double* Kr = a.K0inv + (int64_t)(aggs[jl] * a.nq + kq) * a.ld0;
                        for (int c = l4; c < a.n0; c += 4) acc = fma(__ldg(Kr + c), r0s[c], acc);
                    }
                    acc += __shfl_xor_sync(0xffffffffu, acc, 1);
                    acc += __shfl_xor_sync(0xffffffffu, acc, 2);
                    if (l4 == 0 && w2 < nrows) y0l[w2] = acc;
                }
            } else {                              // distributed coarse rows, then a barrier
                for (int row = c0 + warp; row < c1; row += nw) {
                    const double y = coarse_row(row);
                    if (lane == 0) a.y0[row] = y;
                }
                ok = grid_barrier(a.gs, G, gen, a.err, wl);
                if (!ok) { status = kEDEVICE; break; }
            }
            __syncthreads();
        }
        // ---------------------------------------------------------------- CM
        // z = z_loc + R_0^T y0 for own and neighbour elements; w = K z on own elements,
        // chunk by chunk of the CTA's elements
        double v3[3] = {0.0, 0.0, 0.0};           // r.z, z.q_k, z.w
        const bool cm_stream = CMS && CS > 0 && !apply;
        // this phase's panels: consumed, seen complete, issued (panel j: slot (cm_base + j) % CS)
        uint32_t cm_seq = 0, cm_done = 0, cm_issued = 0;
        int cm_ch = ch1;                  // issue side: chunk and element of the next panel
        int64_t cm_e = 0;
        auto cm_norm = [&]() {
            while (cm_ch < ch1 && cm_e >= a.chunk_elem[cm_ch + 1]) {
                ++cm_ch;
                if (cm_ch < ch1) cm_e = a.chunk_elem[cm_ch] + warp;
            }
        };
        if (cm_stream) {
            // the ring's region ([0, y0_off): P slots and staging, r0s) is free once every
            // thread is past the coarse phase; the first CS panels fly during the z staging
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            __syncthreads();
            cm_ch = ch0;
            cm_e = ch0 < ch1 ? a.chunk_elem[ch0] + warp : 0;
            cm_norm();
            for (int m = 0; m < CS && cm_ch < ch1; ++m) {
                if (lane == 0) cm_issue((int)((cm_base + cm_issued) % CS), cm_e);
                ++cm_issued;
                cm_e += NW;
                cm_norm();
            }
        }
        for (int ch = ch0; ch < ch1; ++ch) {
            const int64_t ce0 = a.chunk_elem[ch], ce1 = a.chunk_elem[ch + 1];
            const int n_chunk = (int)(ce1 - ce0);
            const int32_t* need = a.need + a.need_ptr[ch];
            const int32_t* needj = a.need_aggl + a.need_ptr[ch];
            const int n_need = a.need_ptr[ch + 1] - a.need_ptr[ch];
            if (ch > ch0) __syncthreads();        // the previous chunk's readers of pn are done
            for (int idx = threadIdx.x; idx < n_need * NP; idx += blockDim.x) {
                const int l = idx / NP, j = idx - l * NP;
                const int64_t e = need[l], t = e * NP + j;
                double v = __ldcg(a.zl + t);
                if (coarse) {
                    const double* Tr = a.T + t * a.nq;
                    if (a.redundant) {
                        const double* y = y0l + needj[l] * a.nq;
                        for (int kq = 0; kq < a.nq; ++kq) v = fma(__ldg(Tr + kq), y[kq], v);
                    } else {                      // needj: the element's agglomerate
                        const double* y = a.y0 + (int64_t)needj[l] * a.nq;
                        for (int kq = 0; kq < a.nq; ++kq) v = fma(__ldg(Tr + kq), __ldcg(y + kq), v);
                    }
                }
                pn[idx] = v;
                if (l < n_chunk) a.z[t] = v;
            }
            __syncthreads();
            if (apply) continue;                  // z is the result: no matvec
            auto emit = [&](int64_t e, int i, double kz) {
                const int64_t t = e * NP + i;
                const double zv = pn[(e - ce0) * NP + i];
                if (pipe) {                       // zv = m (u on the first pass), kz = K m
                    if (pinit) {
                        a.r[1][t] = zv;
                        a.w[t] = kz;
                        return;
                    }
                    const double zn = fma(pbe, a.q[1][t], kz);
                    const double qn = fma(pbe, a.q[0][t], zv);
                    const double sn = fma(pbe, a.p[1][t], a.w[t]);
                    const double pn_ = fma(pbe, a.p[0][t], a.r[1][t]);
                    a.q[1][t] = zn;
                    a.q[0][t] = qn;
                    a.p[1][t] = sn;
                    a.p[0][t] = pn_;
                    a.x[t] = fma(pal, pn_, a.x[t]);
                    a.r[0][t] = fma(-pal, sn, a.r[0][t]);
                    a.r[1][t] = fma(-pal, qn, a.r[1][t]);
                    a.w[t] = fma(-pal, zn, a.w[t]);
                    return;
                }
                a.w[t] = kz;
                v3[0] = fma(__ldcg(rk + t), zv, v3[0]);
                v3[1] = fma(zv, __ldcg(qk + t), v3[1]);
                v3[2] = fma(zv, kz, v3[2]);
            };
            if (!cm_stream) {
                local_rows<NP>(a.row_ptr, a.col_local, a.val, pn, ce0, ce1, emit);
            } else {
                // the same elements in the same order as the issue side: panel cm_seq is in
                // slot cm_seq % CS; once read, the slot takes the warp's panel CS further on
                for (int64_t e = ce0 + warp; e < ce1; e += NW) {
                    const uint32_t g = cm_base + cm_seq;
                    const int k = (int)(g % CS);
                    const int32_t b0 = a.row_ptr[e];
                    const int nb = a.row_ptr[e + 1] - b0;
                    const int clv = lane < nb ? __ldg(a.col_local + b0 + lane) : 0;
                    if (!cmfail && !__all_sync(0xffffffffu, mbar_wait(&cmbars[warp][k], (g / CS) & 1))) {
                        cmfail = true;
                        if (lane == 0) atomicExch(a.err, 1);
                        // bounded wait for the panels still in flight, before anything else
                        // may reuse their slots
                        for (uint32_t c = cm_done; c < cm_issued; ++c)
                            if (!mbar_wait(&cmbars[warp][(cm_base + c) % CS], ((cm_base + c) / CS) & 1)) break;
                    }
                    double kz = 0.0;
                    if (!cmfail) {                // else the solve stops at the next barrier
                        ++cm_done;
                        const double* V = reinterpret_cast<const double*>(smem + ((size_t)warp * CS + k) * a.cm_slot_bytes) +
                                          (((int64_t)b0 * NP * NP) & 1);
                        kz = panel_rows<NP>(V, clv, nb, pn, lane);
                        __syncwarp();             // every lane is done with the slot
                        if (cm_ch < ch1) {
                            if (lane == 0) cm_issue(k, cm_e);
                            ++cm_issued;
                            cm_e += NW;
                            cm_norm();
                        }
                    }
                    ++cm_seq;
                    if (lane < NP) emit(e, lane, kz);
                }
            }
        }
        cm_base += cm_seq;
        if (apply) break;                         // status kOK: z = B_ad^{-1} b is complete
        // beta, p.q and alpha by thread 0: code 0 go on, 2 non-finite, 4 breakdown
        if (timing) {
            __syncthreads();
            if (threadIdx.x == 0) cyc_cm += clock64() - t_mark;
        }
        if (cm_stream) {
            // every warp is done with its panels: the next P phase's first rows fly
            // during the grid reduction (their slots overlap the CM ring)
            __syncthreads();
            if (has_rows && !wfail && !cmfail) {
                issue_first();
                p_armed = true;
            }
        }
        if (pipe) {                               // the own rows are updated: a plain barrier
            ok = grid_barrier(a.gs, G, gen, a.err, wl);
            if (!ok) { status = kEDEVICE; break; }
            if (!pinit) ++it;
            pinit = false;
            continue;
        }
        ok = barrier_sum<3>(a.gs, G, cta, gen, a.err, a.partials, v3, red, outv, [&](const double* sm) {
            const double rz_new = sm[0], zq = sm[1], zw = sm[2];
            if (!isfinite(rz_new) || !isfinite(zq) || !isfinite(zw)) { scode = 2; return; }
            double bnew;
            if (it == 0) bnew = 0.0;
            else if (flexible) bnew = -alpha * zq / rz;   // z_{k+1}.(r_{k+1} - r_k) = -alpha_k z_{k+1}.q_k
            else bnew = rz_new / rz;
            const double pq_new = zw + 2.0 * bnew * zq + bnew * bnew * pq;
            if (!isfinite(bnew) || rz_new == 0.0 || !(pq_new > 0.0) || !isfinite(pq_new)) { scode = 4; return; }
            scal[0] = rz_new / pq_new;
            scal[1] = bnew;
            scal[2] = pq_new;
            scode = 0;
            if (a.trace && cta == 0) {            // alpha_k and beta_{k-1} for Lanczos estimates
                if (it < a.trace_cap) a.trace[it] = scal[0];
                if (it > 0 && it - 1 < a.trace_cap) a.trace[a.trace_cap + it - 1] = bnew;
            }
        }, wl);
        if (!ok) { status = kEDEVICE; break; }
        const int code3 = scode;
        if (code3 == 2) { status = kENONFINITE; break; }
        if (code3 == 4) { status = kEBREAKDOWN; break; }
        rz = v3[0];
        alpha = scal[0];
        beta = scal[1];
        pq = scal[2];
        pending = 1;
    }
    if (done == 2) {            // b = 0: the solution is x = 0
        for (int64_t t = e0 * NP + threadIdx.x; t < e1 * NP; t += blockDim.x) a.x[t] = 0.0;
    }
    // wait (bounded) for this CTA's copies still in flight before leaving
    if (!a.identity && has_rows) {      // bounded wait for this warp's copies still in flight
        for (uint32_t c = n_done; c < n_issued; ++c)
            if (!mbar_wait(&wbars[warp][c % S], (c / S) & 1)) break;
    }

    if (timing && threadIdx.x == 0) {
        a.cta_cycles[cta] = cyc_p;
        a.cta_cycles[G + cta] = cyc_cm;
    }
    if (cta == 0 && threadIdx.x == 0) {
        relres = bb > 0.0 ? sqrt(rr / bb) : 0.0;
        sc->bb = bb;
        sc->rr = rr;
        sc->relres = relres;
        sc->it = it;
        sc->status = status;
        sc->done = done ? done : 1;
        sc->pass = 0;
    }
}

// The symmetric pair-row store (sym_ld / sym_len) of the fp32 local inverses, block
// blockIdx.y: the lower triangles of the stored rows (the inverse is symmetric; its lower
// triangle defines it), the diagonal entries halved (exact: the P phase adds each of them
// twice, once in its row's sum and once in its column's).
__global__ void sym_pack_kernel(const GemvBlock* __restrict__ blocks, const float* __restrict__ st32,
                                float* __restrict__ sym) {
    const GemvBlock B = blocks[blockIdx.y];
    const int n = B.ncols, ld = sym_ld(n), npair = (n + 1) / 2;
    const int64_t total = (int64_t)npair * ld;
    float* dst = sym + B.sym_off;
    const float* src = st32 + B.mat_off;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int m = (int)(i / ld), c = (int)(i % ld);
        const int la = (m + 4) & ~3, b = n - 1 - m;
        float v = 0.f;
        if (c < la) {
            if (c <= m) v = src[(int64_t)m * B.ld + c] * (c == m ? 0.5f : 1.f);
        } else if (b != m && c - la <= b) {
            v = src[(int64_t)b * B.ld + (c - la)] * (c - la == b ? 0.5f : 1.f);
        }
        dst[i] = v;
    }
}

cudaError_t launch_sym_pack(const GemvBlock* blocks, int n_local, const float* st32, float* sym,
                            cudaStream_t s) {
    if (n_local < 1 || n_local > 65535) return cudaErrorInvalidValue;
    sym_pack_kernel<<<dim3(32, n_local), 256, 0, s>>>(blocks, st32, sym);
    return cudaGetLastError();
}

// One solve on all CTAs of the launch.
template <int DT, int NP>
__global__ void __launch_bounds__(kPersistThreads, 1)
pcg_persistent_kernel(const __grid_constant__ PersistArgs a) {
    extern __shared__ __align__(128) unsigned char smem[];
    pcg_solve_cta<DT, NP, true>(a, blockIdx.x, gridDim.x, smem);
}

// Independent solves of several simulations in one launch: CTA b works on
// simulation map[b].x as its CTA map[b].y of args[map[b].x].grid.  Each group
// has its own scalars, barrier counter and stopping test, so a simulation that
// converges early leaves the others undisturbed.
template <int DT, int NP>
__global__ void __launch_bounds__(kPersistThreads, 1)
pcg_batched_kernel(const PersistArgs* __restrict__ args, const int2* __restrict__ map) {
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(16) PersistArgs sa;
    const int2 m = map[blockIdx.x];
    {
        static_assert(sizeof(PersistArgs) % 8 == 0, "PersistArgs is copied as 8-byte words");
        const uint64_t* src = reinterpret_cast<const uint64_t*>(args + m.x);
        uint64_t* dst = reinterpret_cast<uint64_t*>(&sa);
        for (int k = threadIdx.x; k < (int)(sizeof(PersistArgs) / 8); k += blockDim.x) dst[k] = src[k];
    }
    __syncthreads();
    pcg_solve_cta<DT, NP, false>(sa, m.y, (unsigned)sa.grid, smem);
}

template <int DT>
static const void* kernel_fn(int np, bool batched) {
    switch (np) {
        case 3: return batched ? (const void*)pcg_batched_kernel<DT, 3> : (const void*)pcg_persistent_kernel<DT, 3>;
        case 6: return batched ? (const void*)pcg_batched_kernel<DT, 6> : (const void*)pcg_persistent_kernel<DT, 6>;
        case 10: return batched ? (const void*)pcg_batched_kernel<DT, 10> : (const void*)pcg_persistent_kernel<DT, 10>;
        case 15: return batched ? (const void*)pcg_batched_kernel<DT, 15> : (const void*)pcg_persistent_kernel<DT, 15>;
        default: return nullptr;
    }
}

static const void* pick(int dtype, int np, bool batched) {
    return dtype == 0 ? kernel_fn<0>(np, batched) : dtype == 1 ? kernel_fn<1>(np, batched)
                                                              : kernel_fn<2>(np, batched);
}

cudaError_t launch_pcg_persistent(int dtype, int np, const PersistArgs& a, size_t smem,
                                  cudaStream_t s) {
    if (a.grid > kMaxPartials) return cudaErrorInvalidValue;
    const void* fn = pick(dtype, np, false);
    if (!fn) return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    void* args[] = {(void*)&a};
    return cudaLaunchCooperativeKernel(fn, dim3(a.grid), dim3(kPersistThreads), args, smem, s);
}

cudaError_t launch_pcg_batched(int dtype, int np, const PersistArgs* args_dev, const int2* map_dev,
                               int n_cta, size_t smem, cudaStream_t s) {
    // the shared-memory limit was raised by persistent_occupancy(.., batched = 1) at set-up
    // (this launch may be recorded into a CUDA graph)
    const void* fn = pick(dtype, np, true);
    if (!fn || n_cta < 1) return cudaErrorInvalidValue;
    void* args[] = {(void*)&args_dev, (void*)&map_dev};
    return cudaLaunchCooperativeKernel(fn, dim3(n_cta), dim3(kPersistThreads), args, smem, s);
}

cudaError_t persistent_occupancy(int dtype, int np, size_t smem, int* blocks_per_sm, int batched) {
    const void* fn = pick(dtype, np, batched != 0);
    if (!fn) return cudaErrorInvalidValue;
    cudaError_t e;
    if (batched) {      // only ever raised, so every batch created earlier can still launch
        cudaFuncAttributes fa;
        if ((e = cudaFuncGetAttributes(&fa, fn)) != cudaSuccess) return e;
        if ((size_t)fa.maxDynamicSharedSizeBytes < smem)
            e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    } else {
        e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    }
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, fn, kPersistThreads, smem);
}

}  // namespace polydg
