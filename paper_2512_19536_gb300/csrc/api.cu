// C ABI of libpolydg (include/polydg.h): contexts, device buffers, the work
// plan of the persistent PCG kernel and the launch sequence of a time step.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <limits>
#include <map>
#include <string>
#include <utility>
#include <vector>

#include <cuda_runtime.h>
#include <cuda_bf16.h>

#include "contexts.h"
#include "internal.h"
#include "ionic_model.cuh"
#include "kernels.h"
#include "polydg.h"

namespace polydg {

static thread_local std::string g_error;
void set_error(const std::string& msg) { g_error = msg; }

// Polls of a grid barrier of the persistent PCG kernels before they give up
// (polydg_set_wait_limit); read when a launch's arguments are built.
constexpr uint32_t kDefaultWaitPolls = 1u << 22;
static std::atomic<uint32_t> g_wait_limit{kDefaultWaitPolls};

}  // namespace polydg

using namespace polydg;

namespace polydg {

// Cut the plan's tile sequence into G contiguous runs of about equal cost (tile cost,
// plus the stage cost of a tile that starts a subdomain within a run): greedy packing
// under a per-CTA budget, the smallest budget that fits in G runs found by bisection.
// Gives each CTA's tiles as runs of consecutive rows of one block.
static int partition_tiles(Plan& P, const asm_ctx* pc, int G, const std::vector<double>& tcost,
                           const std::vector<double>& tstage, std::vector<int32_t>& run_ptr,
                           std::vector<GemvRun>& runs) {
    const std::vector<GemvTile>& tiles = P.h_tiles;
    const int rows = P.rows;
    auto pack = [&](double budget, std::vector<int32_t>* ptr) {
        int used = 0;
        size_t k = 0;
        while (k < tiles.size()) {
            if (ptr) (*ptr)[used] = (int32_t)k;
            ++used;
            double acc = 0.0;
            const size_t first = k;
            while (k < tiles.size()) {
                const bool stage = (k == first) || tiles[k].block != tiles[k - 1].block;
                const double c = tcost[k] + (stage ? tstage[k] : 0.0);
                if (k > first && acc + c > budget) break;
                acc += c;
                ++k;
            }
        }
        return used;
    };
    double lo = 0.0, hi = 0.0;
    for (size_t k = 0; k < tiles.size(); ++k) hi += tcost[k] + tstage[k];
    for (int it = 0; it < 60; ++it) {
        const double mid = 0.5 * (lo + hi);
        if (pack(mid, nullptr) <= G) hi = mid; else lo = mid;
    }
    std::vector<int32_t> tile_ptr(G + 1, (int32_t)tiles.size());
    const int used = tiles.empty() ? 0 : pack(hi, &tile_ptr);
    for (int g = used; g <= G; ++g) tile_ptr[g] = (int32_t)tiles.size();
    P.est_seconds = tiles.empty() ? 0.0 : hi;
    P.h_tile_ptr = tile_ptr;
    run_ptr.assign(G + 1, 0);
    runs.clear();
    for (int g = 0; g < G; ++g) {
        run_ptr[g] = (int32_t)runs.size();
        for (int32_t k = tile_ptr[g]; k < tile_ptr[g + 1]; ++k) {
            const GemvTile& t = tiles[k];
            const int32_t end = std::min<int32_t>(t.row0 + rows, pc->blocks[t.block].nrows);
            if ((int32_t)runs.size() > run_ptr[g] && runs.back().block == t.block && runs.back().row_end == t.row0)
                runs.back().row_end = end;
            else
                runs.push_back({t.block, t.row0, end, 0});
        }
        if (!P.small && (int32_t)runs.size() - run_ptr[g] > 128) {
            set_error("pcg: a CTA would stream more than 128 subdomains; too many subdomains for the CTAs");
            return POLYDG_EINVAL;
        }
    }
    run_ptr[G] = (int32_t)runs.size();
    return POLYDG_OK;
}

// Split the work of one PCG iteration over `grid` CTAs: LOCAL tiles (rows of the
// local inverses) as contiguous runs balanced by bytes, elements and coarse rows
// evenly; per CTA the elements whose p its matvec rows need (own range first,
// then face neighbours) and the CTA-local column index of every block.
static int build_plan(polydg_ctx* c, asm_ctx* pc, int G, Plan& P, int batched = 0,
                      const std::vector<int64_t>* elem_split = nullptr) {
    const HostSetup& H = c->H;
    const int np = H.n_p;
    P.grid = G;
    P.dtype = pc ? pc->precision : 0;
    const int esz = P.dtype == 0 ? 8 : P.dtype == 1 ? 4 : 2;
    const int xsz = P.dtype == 0 ? 0 : 4;        // fp64 stores read r' from the fp64 copy
    int64_t max_ld = 8;
    std::vector<int> local_ids;
    std::vector<int32_t> sub_pairs;
    if (pc)
        for (int b = 0; b < (int)pc->blocks.size(); ++b)
            if (pc->blocks[b].kind == KIND_LOCAL) {
                local_ids.push_back(b);
                max_ld = std::max<int64_t>(max_ld, pc->blocks[b].ld);
            }
    const int64_t n0 = (pc && pc->has_coarse) ? pc->n0 : 0;
    // elements: an even split over the CTAs, each CTA's range cut into chunks of
    // at most kChunk elements; per chunk the elements whose z its matvec rows need
    // (the chunk first, then face neighbours outside it)
    constexpr int64_t kChunk = 64;
    std::vector<int64_t> elem_ptr(G + 1), chunk_elem;
    std::vector<int32_t> cta_chunk(G + 1, 0);
    for (int g = 0; g <= G; ++g) elem_ptr[g] = (H.nc * g) / G;
    if (elem_split && (int)elem_split->size() == G + 1) elem_ptr = *elem_split;
    for (int g = 0; g < G; ++g) {
        cta_chunk[g] = (int32_t)chunk_elem.size();
        const int64_t n_own = elem_ptr[g + 1] - elem_ptr[g];
        const int64_t nch = (n_own + kChunk - 1) / kChunk;
        for (int64_t k = 0; k < nch; ++k) chunk_elem.push_back(elem_ptr[g] + (n_own * k) / nch);
    }
    cta_chunk[G] = (int32_t)chunk_elem.size();
    chunk_elem.push_back(H.nc);
    const int n_chunks = cta_chunk[G];
    std::vector<int32_t> need_ptr(n_chunks + 1, 0), need, col_local(H.col.size());
    int max_need = 0;
    for (int ch = 0; ch < n_chunks; ++ch) {
        const int64_t e0 = chunk_elem[ch], e1 = chunk_elem[ch + 1];
        std::vector<int32_t> nb;
        for (int64_t e = e0; e < e1; ++e)
            for (int32_t bi = H.row_ptr[e]; bi < H.row_ptr[e + 1]; ++bi)
                if (H.col[bi] < e0 || H.col[bi] >= e1) nb.push_back(H.col[bi]);
        std::sort(nb.begin(), nb.end());
        nb.erase(std::unique(nb.begin(), nb.end()), nb.end());
        need_ptr[ch] = (int32_t)need.size();
        for (int64_t e = e0; e < e1; ++e) need.push_back((int32_t)e);
        need.insert(need.end(), nb.begin(), nb.end());
        for (int64_t e = e0; e < e1; ++e)
            for (int32_t bi = H.row_ptr[e]; bi < H.row_ptr[e + 1]; ++bi) {
                const int32_t f = H.col[bi];
                col_local[bi] = (f >= e0 && f < e1)
                                    ? (int32_t)(f - e0)
                                    : (int32_t)((e1 - e0) + (std::lower_bound(nb.begin(), nb.end(), f) - nb.begin()));
            }
        max_need = std::max(max_need, (int)((e1 - e0) + nb.size()));
    }
    need_ptr[n_chunks] = (int32_t)need.size();
    // agglomerates touched by each CTA's needed elements (coarse rows it solves redundantly)
    const int nq = (pc && pc->has_coarse) ? pc->nq : 1;
    std::vector<int32_t> agg_internal(H.nc, 0);
    if (pc && pc->has_coarse) {
        std::vector<int32_t> tmp(H.nc);
        cudaMemcpy(tmp.data(), pc->d_agg, H.nc * sizeof(int32_t), cudaMemcpyDeviceToHost);
        agg_internal = tmp;
    }
    std::vector<int32_t> need_aggl(need.size(), 0), need_agg_ptr(G + 1, 0), need_agg;
    int max_aggs = 0;
    for (int g = 0; g < G; ++g) {
        const int32_t k0 = need_ptr[cta_chunk[g]], k1 = need_ptr[cta_chunk[g + 1]];
        std::vector<int32_t> js;
        for (int32_t k = k0; k < k1; ++k) js.push_back(agg_internal[need[k]]);
        std::sort(js.begin(), js.end());
        js.erase(std::unique(js.begin(), js.end()), js.end());
        need_agg_ptr[g] = (int32_t)need_agg.size();
        for (int32_t k = k0; k < k1; ++k)
            need_aggl[k] = (int32_t)(std::lower_bound(js.begin(), js.end(), agg_internal[need[k]]) - js.begin());
        need_agg.insert(need_agg.end(), js.begin(), js.end());
        max_aggs = std::max(max_aggs, (int)js.size());
    }
    need_agg_ptr[G] = (int32_t)need_agg.size();
    // coarse rows solved redundantly per CTA while that costs little (<= 8k fp64 FMA per CTA);
    // otherwise distributed over the CTAs with one more grid barrier per iteration
    P.redundant = ((int64_t)max_aggs * nq * n0 <= 8192) ? 1 : 0;
    // distributed coarse rows: per needed element its agglomerate itself (read beside the
    // element id instead of through it)
    if (!P.redundant)
        for (size_t k = 0; k < need.size(); ++k) need_aggl[k] = agg_internal[need[k]];
    P.max_need = max_need;
    P.max_aggs = max_aggs;
    // fp32 stores with enough subdomains for every CTA to take whole ones: the P phase
    // streams the symmetric pair-row store (half the bytes), each CTA summing the upper
    // triangle's share of its subdomains' rows itself
    const int NWp = kPersistThreads / 32;
    P.sym = (pc && !batched && P.dtype == 1 && pc->d_sym && (int64_t)local_ids.size() >= 4 * (int64_t)G) ? 1 : 0;
    P.sym_bufld = P.sym ? (pc->sym_max_n + 127) / 128 * 128 : 0;
    // shared memory: 2 tile buffers, staged r' (store type), r' and q (fp64), z (2 x rows),
    // r0/q0, p of the needed elements
    auto r128 = [](size_t x) { return (x + 127) & ~(size_t)127; };
    // r0s doubles as the symmetric P phase's column-sum buffer (idle there)
    const size_t r0_bytes = std::max((size_t)n0 * 8, (size_t)(NWp + 1) * P.sym_bufld * 4);
    const size_t cap = 208 * 1024;              // + ~15 KB static shared memory of the kernel
    constexpr int kMaxRuns = 128;                // run descriptors (48 bytes) per CTA
    const size_t td_reserve = r128(kMaxRuns * 48);
    const size_t fixed = r128((size_t)max_ld * xsz) + r128((size_t)max_ld * 8) + r128(r0_bytes) +
                         r128((size_t)max_aggs * nq * 8) + r128((size_t)max_need * np * 8) + td_reserve;
    // per warp, as many one-row copy slots (up to kMaxWarpStages) as the rest leaves room for
    const int NW = kPersistThreads / 32;
    const size_t slot = !pc ? 0 : P.sym ? (size_t)sym_ld(pc->sym_max_n) * 4 : r128((size_t)max_ld * esz);
    const int64_t wst = (pc && fixed < cap) ? (int64_t)((cap - fixed) / (NW * slot)) : (pc ? 0 : 1);
    if (wst < 1) {
        set_error("pcg: a subdomain or coarse space is too large for the shared-memory plan");
        return POLYDG_EINVAL;
    }
    P.wstages = (int)std::min<int64_t>(kMaxWarpStages, wst);
    P.slot_bytes = slot;
    // subdomains of at most 32 DOFs (one element each in the massively parallel case,
    // T_S = T_h): whole subdomains go to warps, one lane per row, and the CTA reads its
    // runs from global memory (no shared-memory run table, no bulk row copies)
    P.small = 0;
    if (pc && !local_ids.empty()) {
        int max_rows = 0;
        for (int b : local_ids) max_rows = std::max(max_rows, (int)pc->blocks[b].nrows);
        P.small = max_rows <= 32 ? 1 : 0;
    }
    // R_0 r' = per coarse DOF, the sum of its pairs' partials.  Lane groups of L (a power
    // of 2) split each sum so that no lane adds more than 16 partials in sequence; the
    // shuffle tree costs L log2 L fp64 adds per coarse DOF, so L stays as small as that
    // allows.  When all the sums together exceed 8192 adds, the CTAs sum slices of the
    // coarse DOFs into a global vector behind one more grid barrier instead of every
    // CTA adding all of them (GB300's fp64 pipe retires ~2 FMA per clock per SM).
    P.pair_lanes = 1;
    P.r0_split = 0;
    if (pc && pc->has_coarse) {
        while (P.pair_lanes < 32 && P.pair_lanes * 16 < pc->max_pairs) P.pair_lanes *= 2;
        P.r0_split = (int64_t)pc->n_pairs * pc->nq > 8192 ? 1 : 0;
    }
    P.rows = P.small ? 32 : P.sym ? (1 << 30) : 16;   // partition granularity (rows per tile)
    const int rows = P.rows;
    P.xs_off = (size_t)NW * P.wstages * slot;
    P.rp_off = P.xs_off + r128((size_t)max_ld * xsz);
    P.r0_off = P.rp_off + r128((size_t)max_ld * 8);
    P.y0_off = P.r0_off + r128(r0_bytes);
    P.pn_off = P.y0_off + r128((size_t)max_aggs * nq * 8);
    P.td_off = P.pn_off + r128((size_t)max_need * np * 8);
    P.smem = P.td_off + td_reserve;
    // CM phase: each element's block-row panel of K_h is copied into a per-warp ring that
    // reuses [0, y0_off) -- the P phase's slots and staging and r0s, all idle by then --
    // when at least one slot per warp fits and no row has more than 32 blocks
    {
        int max_nb = 0;
        for (int64_t e = 0; e < H.nc; ++e) max_nb = std::max(max_nb, (int)(H.row_ptr[e + 1] - H.row_ptr[e]));
        P.cm_slot_bytes = r128((size_t)max_nb * np * np * 8 + 16);
        const int64_t cst = (int64_t)(P.y0_off / ((size_t)NW * P.cm_slot_bytes));
        P.cm_stages = (max_nb <= 32) ? (int)std::min<int64_t>(kMaxCmStages, cst) : 0;
    }
    // LOCAL tiles balanced by bytes
    std::vector<GemvTile> tiles;
    std::vector<int64_t> tbytes;
    for (int b : local_ids) {
        const GemvBlock& B = pc->blocks[b];
        for (int r0 = 0; r0 < B.nrows; r0 += rows) {
            tiles.push_back({b, r0});
            if (P.sym) {
                int64_t sb = 0;
                for (int q = 0; q < (B.ncols + 1) / 2; ++q) sb += 4 * (int64_t)sym_len(B.ncols, q);
                tbytes.push_back(sb);
            } else {
                tbytes.push_back((int64_t)std::min(rows, B.nrows - r0) * B.ld * esz);
            }
        }
    }
    // Split the tile sequence into G contiguous runs of about equal estimated time:
    // the tile's bytes at the per-SM share of HBM bandwidth, a fixed per-tile cost,
    // a re-stage of r' whenever a run enters a new subdomain, and the restriction
    // rows for the run that holds a subdomain's first tile.
    const double bw_sm = 6.0e12 / c->n_sm;               // bytes/s per SM (about HBM / SMs)
    const double c_tile = 0.1e-6, c_stage = 1.5e-6, c_pair = 2.0e-6;
    std::vector<double> tcost(tiles.size()), tstage(tiles.size());
    for (size_t k = 0; k < tiles.size(); ++k) {
        const GemvBlock& B = pc->blocks[tiles[k].block];
        tcost[k] = tbytes[k] / bw_sm + c_tile + (tiles[k].row0 == 0 ? c_pair * B.pair_count : 0.0);
        tstage[k] = c_stage;
    }
    P.h_tiles = tiles;
    P.h_cost = tcost;
    P.h_stage = tstage;
    std::vector<int32_t> run_ptr;
    std::vector<GemvRun> runs;
    if (int st = partition_tiles(P, pc, G, tcost, tstage, run_ptr, runs)) return st;
    if (pc) sub_pairs = pc->sub_pairs;
    std::vector<int32_t> crow_ptr(G + 1);
    for (int g = 0; g <= G; ++g) crow_ptr[g] = (int32_t)((n0 * g) / G);
    int st;
    if ((st = upload(&P.run_ptr, run_ptr)) || (st = upload(&P.runs, runs)) ||
        (st = upload(&P.sub_pairs, sub_pairs)) || (st = upload(&P.elem_ptr, elem_ptr)) ||
        (st = upload(&P.crow_ptr, crow_ptr)) || (st = upload(&P.need_ptr, need_ptr)) ||
        (st = upload(&P.need, need)) || (st = upload(&P.col_local, col_local)) ||
        (st = upload(&P.need_aggl, need_aggl)) || (st = upload(&P.need_agg_ptr, need_agg_ptr)) ||
        (st = upload(&P.need_agg, need_agg)) || (st = upload(&P.cta_chunk, cta_chunk)) ||
        (st = upload(&P.chunk_elem, chunk_elem)))
        return st;
    // L2 residency of the local inverses: what 60 % of L2 holds beside K_h (single
    // solves only; the autotuner sweeps the fraction)
    P.l2_keep = 0.f;
    if (pc && !batched && pc->store_bytes > 0) {
        int l2 = 0;
        cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, c->device);
        const double kh = 8.0 * np * np * (double)H.col.size();
        const double keep = (0.6 * l2 - kh) / (double)(P.sym ? pc->sym_bytes : pc->store_bytes);
        P.l2_keep = (float)std::max(0.0, std::min(1.0, keep));
    }
    int occ = 0;
    CU(persistent_occupancy(P.dtype, np, P.smem, &occ, batched));
    if (occ < 1) { set_error("pcg: the persistent kernel does not fit on an SM"); return POLYDG_ECUDA; }
    return POLYDG_OK;
}

// Arguments of one persistent PCG solve of K x = b on the vectors of w (internal
// order; x holds x0) under plan P.
static PersistArgs persist_args(polydg_ctx* c, asm_ctx* pc, const Plan& P, PcgWork& w) {
    const bool coarse = pc && pc->has_coarse;
    PersistArgs a = {};
    a.grid = P.grid;
    a.wstages = P.wstages;
    a.identity = pc ? 0 : 1;
    a.n0 = coarse ? (int)pc->n0 : 0;
    a.ld0 = coarse ? (int)pc->ld0 : 0;
    a.nq = coarse ? pc->nq : 1;
    a.nc = c->H.nc;
    a.slot_bytes = P.slot_bytes;
    a.sym_bufld = P.sym ? P.sym_bufld : 0;
    a.redundant = P.redundant;
    a.small = P.small;
    a.pair_lanes = P.pair_lanes;
    a.r0_split = P.r0_split;
    a.r0g = coarse ? pc->d_r0g : nullptr;
    a.l2_keep = P.l2_keep;
    a.xs_off = P.xs_off;
    a.rp_off = P.rp_off;
    a.r0_off = P.r0_off;
    a.y0_off = P.y0_off;
    a.pn_off = P.pn_off;
    a.td_off = P.td_off;
    a.cm_stages = P.cm_stages;
    a.cm_slot_bytes = (int)P.cm_slot_bytes;
    a.row_ptr = c->K.row_ptr;
    a.val = c->K.val;
    a.cta_chunk = P.cta_chunk;
    a.chunk_elem = P.chunk_elem;
    a.need_ptr = P.need_ptr;
    a.need = P.need;
    a.need_aggl = P.need_aggl;
    a.need_agg_ptr = P.need_agg_ptr;
    a.need_agg = P.need_agg;
    a.col_local = P.col_local;
    a.elem_ptr = P.elem_ptr;
    a.blocks = pc ? pc->d_blocks : nullptr;
    a.runs = P.runs;
    a.run_ptr = P.run_ptr;
    a.sub_pairs = P.sub_pairs;
    a.store = pc ? (P.dtype == 0 ? (const void*)pc->st64
                    : P.dtype == 1 ? (P.sym ? (const void*)pc->d_sym : (const void*)pc->st32)
                                   : (const void*)pc->st16)
                 : nullptr;
    a.st64 = pc ? pc->st64 : nullptr;
    a.K0inv = coarse ? pc->st64 + pc->off0 : nullptr;
    a.pair_ptr = coarse ? pc->d_pair_ptr : c->d_zero_ptr;
    a.T = coarse ? pc->d_T : nullptr;
    a.agg = coarse ? pc->d_agg : nullptr;
    a.crow_ptr = P.crow_ptr;
    a.b = w.b;
    a.x = w.x[0];
    a.r[0] = w.r[0];
    a.r[1] = w.r[1];
    a.p[0] = w.p;
    a.p[1] = w.p2;
    a.q[0] = w.q;
    a.q[1] = w.q2;
    a.z = w.z;
    a.zl = w.zl;
    a.w = w.w;
    a.r0p = pc ? pc->d_r0p : nullptr;
    a.y0 = pc ? pc->d_y0 : nullptr;
    a.sc = w.sc;
    a.partials = w.partials;
    a.bcast = w.bcast;
    a.gs = w.gs;
    a.err = w.err;
    a.wait_limit = g_wait_limit.load();
    return a;
}

// Enqueue one persistent PCG solve of K x = b on the vectors of w (internal
// order; x holds x0).  The scalars in w.sc must hold rtol2, maxit, flexible and done = 0.
static int run_pcg(polydg_ctx* c, asm_ctx* pc, PcgWork& w, cudaStream_t s, double* trace = nullptr,
                   int trace_cap = 0) {
    const Plan& P = pc ? pc->plan : c->id_plan;
    PersistArgs a = persist_args(c, pc, P, w);
    a.trace = trace;
    a.trace_cap = trace_cap;
    CU(cudaMemsetAsync(&w.gs->count, 0, sizeof(unsigned), s));
    CU(launch_pcg_persistent(P.dtype, c->H.n_p, a, P.smem, s));
    return POLYDG_OK;
}

static int check_ctx(const polydg_ctx* c, const char* fn) {
    if (!c) { set_error(std::string(fn) + ": null context"); return POLYDG_EINVAL; }
    return POLYDG_OK;
}

static inline int64_t round_up(int64_t x, int64_t m) { return (x + m - 1) / m * m; }
// coarse spaces larger than this are factorised and inverted by the blocked tile kernels
constexpr int64_t kHostCoarseDofs = 2048;

}  // namespace polydg

// ================================================================== C ABI
extern "C" {

const char* polydg_last_error(void) { return g_error.c_str(); }

// Device side of polydg_setup / polydg_setup3d once c->H holds the host assembly.
static int setup_device(polydg_ctx* c, polydg_ctx** out) {
    int st;
    auto fail = [&](int code) { polydg_destroy(c); return code; };
    if (cudaGetDevice(&c->device) != cudaSuccess) { set_error("polydg_setup: no CUDA device"); return fail(POLYDG_ECUDA); }
    const HostSetup& H = c->H;
    c->K.nc = H.nc;
    c->K.nblk = (int64_t)H.col.size();
    // device layout: every n_p x n_p block column-major, so that a row of blocks
    // is one column-major panel (coalesced warp loads in the matvec kernel)
    const int np = H.n_p;
    // K_h values plus two doubles: a panel copy of the CM phase starts on the 16-byte
    // boundary at or below its first block and may end up to 15 bytes past its last
    std::vector<double> Kt(H.Kval.size() + 2, 0.0), Kmt(H.Kminus_val.size());
    for (int64_t bi = 0; bi < c->K.nblk; ++bi)
        for (int i = 0; i < np; ++i)
            for (int j = 0; j < np; ++j) {
                Kt[bi * np * np + j * np + i] = H.Kval[bi * np * np + i * np + j];
                Kmt[bi * np * np + j * np + i] = H.Kminus_val[bi * np * np + i * np + j];
            }
    std::vector<GemvBlock> idb;
    std::vector<GemvTile> idt;
    {
        GemvBlock B = {};
        B.in_off = B.out_off = 0;
        B.nrows = B.ncols = (int32_t)(H.nc * np);
        B.kind = KIND_IDENTITY;
        idb.push_back(B);
        for (int64_t r0 = 0; r0 < H.nc * np; r0 += 256) idt.push_back({0, (int32_t)r0});
        c->n_id_tiles = (int)idt.size();
    }
    std::vector<int64_t> zero_ptr(2, 0);
    if ((st = upload(&c->K.row_ptr, H.row_ptr)) || (st = upload(&c->K.col, H.col)) ||
        (st = upload(&c->K.val, Kt)) || (st = upload(&c->K.val_minus, Kmt)) ||
        (st = upload(&c->d_id_blocks, idb)) || (st = upload(&c->d_id_tiles, idt)) ||
        (st = upload(&c->d_zero_ptr, zero_ptr)) ||
        (st = upload(&c->d_to_caller, H.to_caller)) || (st = upload(&c->d_node_ptr, H.node_ptr)) ||
        (st = upload(&c->d_node_w, H.node_w)) || (st = upload(&c->d_node_phi, H.node_phi)) ||
        (st = upload(&c->d_node_pos, H.node_to_caller_pos)) ||
        (st = upload(&c->d_to_internal, H.to_internal)))
        return fail(st);
    c->ionic_lpc = ionic_lanes_per_cell(H.node_ptr.data(), H.nc);
    {
        std::vector<double> diam(H.nc);
        for (int64_t e = 0; e < H.nc; ++e) diam[e] = H.diam[H.to_caller[e]];
        if ((st = upload(&c->d_diam, diam))) return fail(st);
    }
    if ((st = c->work.alloc(H.nc * H.n_p))) return fail(st);
    if (cudaMallocHost((void**)&c->h_sc, sizeof(PcgScalars)) != cudaSuccess) {
        set_error("polydg_setup: pinned allocation failed");
        return fail(POLYDG_ENOMEM);
    }
    if (cudaDeviceGetAttribute(&c->n_sm, cudaDevAttrMultiProcessorCount, c->device) != cudaSuccess ||
        c->n_sm < 1) {
        set_error("polydg_setup: cannot query the SM count");
        return fail(POLYDG_ECUDA);
    }
    if ((st = build_plan(c, nullptr, c->n_sm, c->id_plan))) return fail(st);
    *out = c;
    return POLYDG_OK;
}


int polydg_setup(const polydg_mesh* mesh, int p, const int32_t* subdomain_of_cell,
                 double chi_cm, double dt, double eta0, polydg_ctx** out) {
    if (!out) { set_error("polydg_setup: null output"); return POLYDG_EINVAL; }
    *out = nullptr;
    polydg_ctx* c = new polydg_ctx();
    int st = host_setup(mesh, p, subdomain_of_cell, chi_cm, dt, eta0, c->H);
    if (st) { delete c; return st; }
    return setup_device(c, out);
}

int polydg_setup3d(const polydg_mesh3d* mesh, int p, const int32_t* subdomain_of_cell,
                   double chi_cm, double dt, double eta0, polydg_ctx** out) {
    if (!out) { set_error("polydg_setup3d: null output"); return POLYDG_EINVAL; }
    *out = nullptr;
    polydg_ctx* c = new polydg_ctx();
    int st = host_setup3d(mesh, p, subdomain_of_cell, chi_cm, dt, eta0, c->H);
    if (st) { delete c; return st; }
    return setup_device(c, out);
}
int polydg_get_info(const polydg_ctx* c, polydg_info* out) {
    if (int st = check_ctx(c, "polydg_get_info")) return st;
    if (!out) { set_error("polydg_get_info: null output"); return POLYDG_EINVAL; }
    const HostSetup& H = c->H;
    out->n_cells = H.nc;
    out->n_dofs = H.nc * H.n_p;
    out->n_faces = (int64_t)H.f_plus.size();
    out->n_blocks = (int64_t)H.col.size();
    out->n_nodes = (int64_t)H.node_w.size();
    out->p = H.p;
    out->n_p = H.n_p;
    out->n_subdomains = H.n_sub;
    int64_t mx = 0;
    for (int i = 0; i < H.n_sub; ++i) mx = std::max(mx, (H.sub_ptr[i + 1] - H.sub_ptr[i]) * H.n_p);
    out->max_subdomain_dofs = (int32_t)mx;
    return POLYDG_OK;
}

int polydg_get_faces(const polydg_ctx* c, int64_t* plus, int64_t* minus) {
    if (int st = check_ctx(c, "polydg_get_faces")) return st;
    if (!plus || !minus) { set_error("polydg_get_faces: null output"); return POLYDG_EINVAL; }
    std::copy(c->H.f_plus.begin(), c->H.f_plus.end(), plus);
    std::copy(c->H.f_minus.begin(), c->H.f_minus.end(), minus);
    return POLYDG_OK;
}

int polydg_matvec(polydg_ctx* c, const double* x_dev, double* y_dev, void* stream) {
    if (int st = check_ctx(c, "polydg_matvec")) return st;
    if (!x_dev || !y_dev || x_dev == y_dev) { set_error("polydg_matvec: null or aliased vectors"); return POLYDG_EINVAL; }
    cudaStream_t s = (cudaStream_t)stream;
    const int np = c->H.n_p;
    CU(launch_permute(x_dev, nullptr, c->work.p, c->d_to_caller, c->H.nc, np, 1, nullptr, s));
    CU(launch_matvec(MODE_PLAIN, np, c->K, c->K.val, c->work.p, c->work.q, nullptr, nullptr, 0, 0,
                     nullptr, 0, 0, s));
    CU(launch_permute(c->work.q, nullptr, y_dev, c->d_to_caller, c->H.nc, np, 0, nullptr, s));
    return POLYDG_OK;
}

int asm_setup(polydg_ctx* c, const int32_t* coarse_of_cell, int q, int precision, asm_ctx** out) {
    if (int st = check_ctx(c, "asm_setup")) return st;
    if (!out) { set_error("asm_setup: null output"); return POLYDG_EINVAL; }
    *out = nullptr;
    if (precision < POLYDG_FP64 || precision > POLYDG_BF16) { set_error("asm_setup: bad precision"); return POLYDG_EINVAL; }
    const HostSetup& H = c->H;
    const int np = H.n_p;
    CoarseSetup C;
    if (coarse_of_cell) {
        if (int st = coarse_setup(H, coarse_of_cell, q, C)) return st;
        if (C.n_q != 3 && C.n_q != 4 && C.n_q != 6 && C.n_q != 10 && !(C.n_q == 15 && H.dim == 2)) {
            set_error("asm_setup: coarse degree q must be 1..4 (2D) or 1..2 (3D)");
            return POLYDG_EINVAL;
        }
    }
    asm_ctx* pc = new asm_ctx();
    pc->ctx = c;
    pc->precision = precision;
    auto fail = [&](int code) { asm_destroy(pc); return code; };
    int st;
    pc->has_coarse = coarse_of_cell != nullptr;
    // dense blocks: N local (K_i) + 1 coarse (K_0)
    struct Mat { int64_t n, ld, off, wld, woff; };
    std::vector<Mat> mats;
    int64_t off = 0, woff = 0, max_n = 0;
    for (int i = 0; i < H.n_sub; ++i) {
        const int64_t n = (H.sub_ptr[i + 1] - H.sub_ptr[i]) * np, ld = round_up(n, 8), wld = round_up(n, 32);
        mats.push_back({n, ld, off, wld, woff});
        off += n * ld;
        woff += wld * wld;
        max_n = std::max(max_n, n);
    }
    const int64_t n0 = pc->has_coarse ? (int64_t)C.n_agg * C.n_q : 0;
    if (pc->has_coarse) {
        const int64_t ld = round_up(n0, 8), wld = round_up(n0, 32);
        mats.push_back({n0, ld, off, wld, woff});
        off += n0 * ld;
        if (n0 <= kHostCoarseDofs) woff += wld * wld;
        max_n = std::max(max_n, n0);
    }
    const int nmat = (int)mats.size();
    double* work = nullptr;
    int64_t *d_off = nullptr, *d_woff = nullptr, *d_subptr = nullptr;
    int32_t *d_n = nullptr, *d_ld = nullptr, *d_wld = nullptr;
    int* d_status = nullptr;
    auto cleanup = [&]() {
        dfree(work); dfree(d_off); dfree(d_woff); dfree(d_subptr); dfree(d_n); dfree(d_ld);
        dfree(d_wld); dfree(d_status);
    };
    {
        std::vector<int64_t> vo, vwo;
        std::vector<int32_t> vn, vld, vwld;
        for (auto& m : mats) {
            vo.push_back(m.off); vwo.push_back(m.woff); vn.push_back((int32_t)m.n);
            vld.push_back((int32_t)m.ld); vwld.push_back((int32_t)m.wld);
        }
        if ((st = dalloc(&pc->st64, off)) || (st = dalloc(&work, woff)) || (st = upload(&d_off, vo)) ||
            (st = upload(&d_woff, vwo)) || (st = upload(&d_n, vn)) || (st = upload(&d_ld, vld)) ||
            (st = upload(&d_wld, vwld)) || (st = upload(&d_subptr, H.sub_ptr)) ||
            (st = dalloc(&d_status, nmat))) {
            cleanup();
            return fail(st);
        }
    }
    auto cu = [&](cudaError_t e, const char* what) {
        if (e == cudaSuccess) return POLYDG_OK;
        set_error(std::string("asm_setup: ") + what + ": " + cudaGetErrorString(e));
        return e == cudaErrorMemoryAllocation ? POLYDG_ENOMEM : POLYDG_ECUDA;
    };
    // A large coarse matrix (3D: thousands of coarse DOFs) is factorised and inverted by
    // the blocked tile kernels (chol_blocked.cu): the batched kernel gives each matrix one CTA.
    const bool coarse_blocked = pc->has_coarse && n0 > kHostCoarseDofs;
    const int nmat_dev = coarse_blocked ? nmat - 1 : nmat;
    int64_t max_n_dev = 0;
    for (int m = 0; m < nmat_dev; ++m) max_n_dev = std::max(max_n_dev, mats[m].n);
    const double* coarse_src = C.K0.data();
    if ((st = cu(cudaMemset(pc->st64, 0, off * sizeof(double)), "memset")) ||
        (st = cu(cudaMemset(work, 0, woff * sizeof(double)), "memset")) ||
        (st = cu(cudaMemset(d_status, 0, nmat * sizeof(int)), "memset")) ||
        (st = cu(launch_extract_local(c->K, d_subptr, H.n_sub, d_off, d_ld, pc->st64, np, 0), "extract")) ||
        (pc->has_coarse &&
         (st = cu(cudaMemcpy2D(pc->st64 + mats.back().off, mats.back().ld * sizeof(double), coarse_src,
                               n0 * sizeof(double), n0 * sizeof(double), n0, cudaMemcpyHostToDevice),
                  "coarse upload"))) ||
        (st = cu(launch_chol_inverse(pc->st64, d_off, d_n, d_ld, work, d_woff, d_wld, d_status, nmat_dev,
                                     (int)max_n_dev, 0), "cholesky")) ||
        (st = cu(cudaDeviceSynchronize(), "cholesky sync"))) {
        cleanup();
        return fail(st);
    }
    if (coarse_blocked) {                    // status slot nmat - 1 belongs to K_0
        double* bw = nullptr;
        if ((st = dalloc(&bw, chol_blocked_work_doubles((int)n0)))) { cleanup(); return fail(st); }
        double* K0 = pc->st64 + mats.back().off;
        st = cu(launch_chol_blocked_inverse(K0, mats.back().ld, (int)n0, K0, mats.back().ld, bw,
                                            d_status + (nmat - 1), 0), "coarse cholesky");
        if (!st) st = cu(cudaDeviceSynchronize(), "coarse cholesky sync");
        dfree(bw);
        if (st) { cleanup(); return fail(st); }
    }
    {
        std::vector<int> hs(nmat, 0);
        cudaMemcpy(hs.data(), d_status, nmat * sizeof(int), cudaMemcpyDeviceToHost);
        for (int m = 0; m < nmat; ++m)
            if (hs[m] != 0) {
                cleanup();
                set_error(m < H.n_sub ? "asm_setup: a local matrix K_i is not positive definite"
                                      : "asm_setup: the coarse matrix K_0 is not positive definite");
                return fail(POLYDG_ENOTSPD);
            }
    }
    cleanup();
    // reduced-precision copies of the local inverses
    const int64_t local_elems = H.n_sub > 0 ? mats[H.n_sub - 1].off + mats[H.n_sub - 1].n * mats[H.n_sub - 1].ld : 0;
    if (precision == POLYDG_FP32) {
        if ((st = dalloc(&pc->st32, local_elems))) return fail(st);
        if ((st = cu(launch_cast_store(pc->st64, pc->st32, nullptr, local_elems, 0), "cast"))) return fail(st);
    } else if (precision == POLYDG_BF16) {
        if ((st = dalloc(&pc->st16, local_elems))) return fail(st);
        if ((st = cu(launch_cast_store(pc->st64, nullptr, pc->st16, local_elems, 0), "cast"))) return fail(st);
    }
    const int esz = precision == POLYDG_FP64 ? 8 : precision == POLYDG_FP32 ? 4 : 2;
    // LOCAL blocks: the dense K_i^{-1} of each subdomain
    for (int m = 0; m < H.n_sub; ++m) {
        GemvBlock B = {};
        B.mat_off = mats[m].off;
        B.nrows = B.ncols = (int32_t)mats[m].n;
        B.ld = (int32_t)mats[m].ld;
        B.kind = KIND_LOCAL;
        B.dtype = precision;
        B.in_off = B.out_off = H.sub_ptr[m] * np;
        pc->blocks.push_back(B);
        pc->store_bytes += (int64_t)B.nrows * B.ld * esz;
    }
    // RESTRICT blocks: rows of R_0 on the DOFs of each (agglomerate, subdomain)
    // pair, fp64, stored after the inverses in st64
    if (pc->has_coarse) {
        pc->q = C.q; pc->nq = C.n_q; pc->n_agg = C.n_agg;
        pc->n0 = n0;
        pc->ld0 = mats.back().ld;
        pc->off0 = mats.back().off;
        std::vector<int32_t> sub_of(H.nc);
        for (int i = 0; i < H.n_sub; ++i)
            for (int64_t e = H.sub_ptr[i]; e < H.sub_ptr[i + 1]; ++e) sub_of[e] = i;
        std::vector<int64_t> pair_ptr(C.n_agg + 1, 0);
        std::vector<double> Rst;
        std::vector<GemvBlock> rblocks;
        for (int J = 0; J < C.n_agg; ++J) {
            int cur = -1;
            for (int64_t k = C.agg_ptr[J]; k < C.agg_ptr[J + 1]; ++k) {
                const int64_t e = C.agg_cells[k];          // ascending internal ids
                const int i = sub_of[e];
                if (i != cur) {
                    cur = i;
                    GemvBlock B = {};
                    B.nrows = C.n_q;
                    B.ncols = (int32_t)((H.sub_ptr[i + 1] - H.sub_ptr[i]) * np);
                    B.ld = (int32_t)round_up(B.ncols, 8);
                    B.kind = KIND_RESTRICT;
                    B.dtype = 0;
                    B.in_off = H.sub_ptr[i] * np;
                    B.out_off = (int64_t)rblocks.size() * C.n_q;
                    B.mat_off = off + (int64_t)Rst.size();
                    Rst.resize(Rst.size() + (size_t)B.nrows * B.ld, 0.0);
                    rblocks.push_back(B);
                    pair_ptr[J + 1]++;
                }
                GemvBlock& B = rblocks.back();
                double* R = Rst.data() + (B.mat_off - off);
                const int64_t c0 = (e - H.sub_ptr[i]) * np;
                for (int kk = 0; kk < np; ++kk)
                    for (int a = 0; a < C.n_q; ++a)
                        R[(int64_t)a * B.ld + c0 + kk] = C.T[(e * np + kk) * C.n_q + a];
            }
        }
        for (int J = 0; J < C.n_agg; ++J) pc->max_pairs = std::max(pc->max_pairs, (int)pair_ptr[J + 1]);
        for (int J = 0; J < C.n_agg; ++J) pair_ptr[J + 1] += pair_ptr[J];
        pc->n_pairs = (int)rblocks.size();
        // grow st64 to hold the R blocks
        double* grown = nullptr;
        if ((st = dalloc(&grown, off + Rst.size()))) return fail(st);
        if ((st = cu(cudaMemcpy(grown, pc->st64, off * sizeof(double), cudaMemcpyDeviceToDevice), "copy")) ||
            (st = cu(cudaMemcpy(grown + off, Rst.data(), Rst.size() * sizeof(double), cudaMemcpyHostToDevice), "copy"))) {
            dfree(grown);
            return fail(st);
        }
        dfree(pc->st64);
        pc->st64 = grown;
        for (auto& B : rblocks) {
            pc->blocks.push_back(B);
            pc->store_bytes += (int64_t)B.nrows * B.ld * 8;
        }
        pc->store_bytes += n0 * mats.back().ld * 8;
        if ((st = upload(&pc->d_pair_ptr, pair_ptr)) || (st = upload(&pc->d_T, C.T)) ||
            (st = upload(&pc->d_agg, C.agg_of_cell)))
            return fail(st);
    }
    // per subdomain (LOCAL block m = subdomain m): its restriction pairs
    for (int m = 0; m < H.n_sub; ++m) {
        GemvBlock& B = pc->blocks[m];
        B.pair_begin = (int32_t)pc->sub_pairs.size();
        for (int b = H.n_sub; b < (int)pc->blocks.size(); ++b)
            if (pc->blocks[b].kind == KIND_RESTRICT && pc->blocks[b].in_off == B.in_off)
                pc->sub_pairs.push_back(b);
        B.pair_count = (int32_t)pc->sub_pairs.size() - B.pair_begin;
    }
    // fp32 stores: the lower triangles again as pair rows (sym_ld), which the persistent
    // kernel streams instead of the full rows when every CTA can take whole subdomains
    int64_t sym_tot = 0;
    if (precision == POLYDG_FP32 && H.n_sub >= 1 && H.n_sub <= 65535) {
        int max_n = 0;
        for (int m = 0; m < H.n_sub; ++m) max_n = std::max(max_n, (int)mats[m].n);
        int64_t tot = 0, bytes = 0;
        for (int m = 0; m < H.n_sub; ++m) {
            const int n = (int)mats[m].n;
            pc->blocks[m].sym_off = (int32_t)std::min<int64_t>(tot, INT32_MAX);
            tot += (int64_t)((n + 1) / 2) * sym_ld(n);
            for (int q = 0; q < (n + 1) / 2; ++q) bytes += 4 * (int64_t)sym_len(n, q);
        }
        if (max_n > 32 && max_n <= 128 * kSymT && tot < INT32_MAX) {
            sym_tot = tot;
            pc->sym_bytes = bytes;
            pc->sym_max_n = max_n;
        }
    }
    pc->n_blocks = (int)pc->blocks.size();
    if ((st = upload(&pc->d_blocks, pc->blocks))) return fail(st);
    if (sym_tot > 0 &&
        ((st = dalloc(&pc->d_sym, sym_tot)) ||
         (st = cu(launch_sym_pack(pc->d_blocks, H.n_sub, pc->st32, pc->d_sym, 0), "sym pack")) ||
         (st = cu(cudaDeviceSynchronize(), "sym pack sync"))))
        return fail(st);
    const int64_t npairs = std::max<int64_t>(pc->n_pairs, 1) * std::max(pc->nq, 1);
    if ((st = dalloc(&pc->d_r0p, npairs)) || (st = dalloc(&pc->d_y0, std::max<int64_t>(n0, 1))) ||
        (st = dalloc(&pc->d_r0g, std::max<int64_t>(n0, 1))))
        return fail(st);
    if ((st = build_plan(c, pc, c->n_sm, pc->plan))) return fail(st);
    *out = pc;
    return POLYDG_OK;
}

int asm_autotune(asm_ctx* pc, int rounds, int iterations, double* gain) {
    if (!pc || rounds < 0 || iterations < 1) {
        set_error("asm_autotune: need a preconditioner, rounds >= 0 and iterations >= 1");
        return POLYDG_EINVAL;
    }
    polydg_ctx* c = pc->ctx;
    Plan& P = pc->plan;
    const int G = P.grid;
    const int64_t n = c->H.nc * c->H.n_p;
    PcgWork& w = c->work;
    // a fixed right-hand side (the cost of an iteration does not depend on the data)
    std::vector<double> hb(n);
    uint64_t st_rng = 0x9E3779B97F4A7C15ull;
    for (int64_t i = 0; i < n; ++i) {
        st_rng = st_rng * 6364136223846793005ull + 1442695040888963407ull;
        hb[i] = (double)(st_rng >> 11) * (1.0 / 9007199254740992.0) - 0.5;
    }
    long long* d_cyc = nullptr;
    if (int st = dalloc(&d_cyc, 2 * (size_t)G)) return st;
    struct Guard { long long*& p; ~Guard() { dfree(p); } } guard{d_cyc};
    CU(cudaMemcpy(w.b, hb.data(), n * sizeof(double), cudaMemcpyHostToDevice));
    cudaEvent_t e0, e1;
    CU(cudaEventCreate(&e0));
    CU(cudaEventCreate(&e1));
    std::vector<long long> cyc(2 * G);
    // one solve of exactly `iterations` iterations under the current plan
    auto run = [&](float* ms) -> int {
        PcgScalars init = {};
        init.rtol2 = 0.0;                     // never converges: runs to maxit
        init.maxit = iterations;
        init.flexible = pc->precision == POLYDG_FP64 ? 0 : 1;
        CU(cudaMemcpy(w.sc, &init, sizeof(init), cudaMemcpyHostToDevice));
        CU(cudaMemset(w.x[0], 0, n * sizeof(double)));
        CU(cudaMemset(w.err, 0, sizeof(int)));
        CU(cudaMemset(&w.gs->count, 0, sizeof(unsigned)));
        PersistArgs a = persist_args(c, pc, P, w);
        a.cta_cycles = d_cyc;
        CU(cudaEventRecord(e0, 0));
        CU(launch_pcg_persistent(P.dtype, c->H.n_p, a, P.smem, 0));
        CU(cudaEventRecord(e1, 0));
        CU(cudaEventSynchronize(e1));
        CU(cudaEventElapsedTime(ms, e0, e1));
        CU(cudaMemcpy(cyc.data(), d_cyc, 2 * G * sizeof(long long), cudaMemcpyDeviceToHost));
        return POLYDG_OK;
    };
    float t0 = 0.f, t_best = 0.f;
    if (int st = run(&t0)) return st;
    if (int st = run(&t0)) return st;         // the first launch warms caches and code
    t_best = t0;
    // (0) the fraction of the local-inverse lines kept in L2 (evict-last): five
    // candidates timed, the fastest kept, then re-timed for its per-CTA cycles
    {
        const float keep0 = P.l2_keep;
        float best_keep = keep0;
        for (float cand : {0.f, 0.25f, 0.5f, 0.75f, 1.f}) {
            P.l2_keep = cand;
            float t = 0.f;
            if (int st = run(&t)) { P.l2_keep = keep0; return st; }
            if (t < t_best) { t_best = t; best_keep = cand; }
        }
        P.l2_keep = best_keep;
        float tk = 0.f;
        if (int st = run(&tk)) return st;
    }
    std::vector<double> cost = P.h_cost, stage = P.h_stage;
    std::vector<int64_t> split(G + 1);
    CU(cudaMemcpy(split.data(), P.elem_ptr, (G + 1) * sizeof(int64_t), cudaMemcpyDeviceToHost));
    // Moves alternate: (a) re-cut the tile sequence with every CTA's tile costs rescaled
    // by its measured / modelled P-phase share; (b) re-split the elements so that every
    // CTA's measured CM cycles, spread evenly over its elements, are equal.  A move is
    // kept only if the timed iterations got faster; otherwise the previous plan returns
    // and is timed again (its per-CTA cycles feed the next move).
    for (int r = 0; r < 2 * rounds; ++r) {
        const bool tiles_move = (r % 2) == 0;
        Plan old = P;
        Plan fresh;
        std::vector<double> ncost = cost, nstage = stage;
        std::vector<int64_t> nsplit = split;
        const std::vector<int32_t> tp = P.h_tile_ptr;
        if (tiles_move) {
            double tot_m = 0.0, tot_t = 0.0;
            std::vector<double> m(G, 0.0);
            for (int g = 0; g < G; ++g) {
                for (int32_t k = tp[g]; k < tp[g + 1]; ++k) m[g] += cost[k] + stage[k];
                tot_m += m[g];
                tot_t += (double)cyc[g];
            }
            if (!(tot_m > 0.0 && tot_t > 0.0)) {   // nothing measured: re-time, same launch count
                float tx = 0.f;
                if (int st = run(&tx)) return st;
                if (int st = run(&tx)) return st;
                continue;
            }
            for (int g = 0; g < G; ++g) {
                if (m[g] <= 0.0 || cyc[g] <= 0) continue;
                const double f = ((double)cyc[g] / tot_t) / (m[g] / tot_m);
                for (int32_t k = tp[g]; k < tp[g + 1]; ++k) { ncost[k] *= f; nstage[k] *= f; }
            }
            fresh = P;                        // same arrays except the runs
            std::vector<int32_t> run_ptr;
            std::vector<GemvRun> runs;
            if (int st = partition_tiles(fresh, pc, G, ncost, nstage, run_ptr, runs)) return st;
            fresh.run_ptr = nullptr;
            fresh.runs = nullptr;
            if (int st = upload(&fresh.run_ptr, run_ptr)) return st;
            if (int st = upload(&fresh.runs, runs)) { dfree(fresh.run_ptr); return st; }
        } else {
            std::vector<double> pre(c->H.nc + 1, 0.0);
            for (int g = 0; g < G; ++g) {
                const int64_t a0 = split[g], a1 = split[g + 1];
                const double ce = (a1 > a0 && cyc[G + g] > 0) ? (double)cyc[G + g] / (double)(a1 - a0) : 0.0;
                for (int64_t e = a0; e < a1; ++e) pre[e + 1] = pre[e] + ce;
            }
            if (!(pre[c->H.nc] > 0.0)) {
                float tx = 0.f;
                if (int st = run(&tx)) return st;
                if (int st = run(&tx)) return st;
                continue;
            }
            int64_t e = 0;
            for (int g = 1; g < G; ++g) {
                const double target = pre[c->H.nc] * g / G;
                while (e < c->H.nc && pre[e + 1] <= target) ++e;
                nsplit[g] = std::max<int64_t>(nsplit[g - 1], e);
            }
            nsplit[0] = 0;
            nsplit[G] = c->H.nc;
            if (int st = build_plan(c, pc, G, fresh, 0, &nsplit)) { fresh.release(); return st; }
            fresh.l2_keep = P.l2_keep;
            std::vector<int32_t> run_ptr;
            std::vector<GemvRun> runs;
            if (int st = partition_tiles(fresh, pc, G, cost, stage, run_ptr, runs)) { fresh.release(); return st; }
            fresh.h_cost = cost;
            fresh.h_stage = stage;
            dfree(fresh.run_ptr);
            dfree(fresh.runs);
            if (int st = upload(&fresh.run_ptr, run_ptr)) { fresh.release(); return st; }
            if (int st = upload(&fresh.runs, runs)) { fresh.release(); return st; }
        }
        P = fresh;
        float t = 0.f;
        const int st = run(&t);
        if (st == POLYDG_OK && t < t_best) {   // keep the move: drop what the old plan alone owned
            t_best = t;
            if (tiles_move) { dfree(old.run_ptr); dfree(old.runs); }
            else old.release();
            cost = ncost;
            stage = nstage;
            split = nsplit;
        } else {                               // revert
            if (tiles_move) { dfree(fresh.run_ptr); dfree(fresh.runs); }
            else fresh.release();
            P = old;
            if (st) return st;
        }
        // re-time the kept plan (its per-CTA cycles feed the next move); every move is
        // two launches, so the autotuner always launches 8 + 4 rounds solves
        float t2 = 0.f;
        if (int st2 = run(&t2)) return st2;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (gain) *gain = t_best > 0.f ? (double)t0 / (double)t_best : 1.0;
    return POLYDG_OK;
}

int asm_get_info(const asm_ctx* pc, asm_info* out) {
    if (!pc || !out) { set_error("asm_get_info: null argument"); return POLYDG_EINVAL; }
    int64_t local = 0, restr = 0;
    for (const auto& B : pc->blocks) {
        const int esz = B.dtype == 0 ? 8 : B.dtype == 1 ? 4 : 2;
        if (B.kind == KIND_LOCAL) local += (int64_t)B.nrows * B.ld * esz;
        else if (B.kind == KIND_RESTRICT) restr += (int64_t)B.nrows * B.ld * 8;
    }
    out->local_store_bytes = pc->plan.sym ? pc->sym_bytes : local;
    out->coarse_bytes = pc->has_coarse ? pc->n0 * pc->ld0 * 8 : 0;
    out->restrict_bytes = restr;
    out->n_subdomains = pc->ctx->H.n_sub;
    out->n_coarse = (int32_t)pc->n0;
    out->precision = pc->precision;
    out->grid = pc->plan.grid;
    out->l2_keep_permille = (int32_t)std::lround(1000.0 * pc->plan.l2_keep);
    out->rows_per_tile = pc->plan.sym ? 2 : 1;   // rows per bulk copy (a pair of triangle rows)
    return POLYDG_OK;
}

int asm_apply(asm_ctx* pc, const double* r_dev, double* z_dev, void* stream) {
    if (!pc) { set_error("asm_apply: null preconditioner"); return POLYDG_EINVAL; }
    if (!r_dev || !z_dev || r_dev == z_dev) { set_error("asm_apply: null or aliased vectors"); return POLYDG_EINVAL; }
    polydg_ctx* c = pc->ctx;
    cudaStream_t s = (cudaStream_t)stream;
    const int np = c->H.n_p;
    // one launch of the persistent PCG kernel in its one-application mode: the P phase
    // and the coarse + z part of the CM phase of an iteration, on r = the input
    PcgScalars init = {};
    init.maxit = 1;
    *c->h_sc = init;
    CU(cudaMemcpyAsync(c->work.sc, c->h_sc, sizeof(PcgScalars), cudaMemcpyHostToDevice, s));
    CU(cudaMemsetAsync(c->work.err, 0, sizeof(int), s));
    CU(launch_permute(r_dev, nullptr, c->work.b, c->d_to_caller, c->H.nc, np, 1, nullptr, s));
    PersistArgs a = persist_args(c, pc, pc->plan, c->work);
    a.apply_only = 1;
    CU(cudaMemsetAsync(&c->work.gs->count, 0, sizeof(unsigned), s));
    CU(launch_pcg_persistent(pc->plan.dtype, np, a, pc->plan.smem, s));
    CU(launch_permute(c->work.z, nullptr, z_dev, c->d_to_caller, c->H.nc, np, 0, nullptr, s));
    CU(cudaMemcpyAsync(c->h_sc, c->work.sc, sizeof(PcgScalars), cudaMemcpyDeviceToHost, s));
    CU(cudaStreamSynchronize(s));
    const int st = c->h_sc->status;
    if (st != 0)
        set_error(st == POLYDG_ECUDA ? "asm_apply: a device-side wait timed out"
                                     : "asm_apply: non-finite value in r");
    return st;
}

int polydg_set_wait_limit(int64_t polls) {
    if (polls > (int64_t)UINT32_MAX) { set_error("polydg_set_wait_limit: at most 2^32 - 1 polls"); return POLYDG_EINVAL; }
    g_wait_limit.store(polls < 0 ? kDefaultWaitPolls : (uint32_t)polls);
    return POLYDG_OK;
}

int pcg_solve_trace(polydg_ctx* c, asm_ctx* pc, const double* b_dev, double* x_dev, double rtol,
                    int maxit, int flexible, void* stream, pcg_stats* stats, double* alphas,
                    double* betas, int capacity) {
    if (capacity < 0 || (capacity > 0 && (!alphas || !betas))) {
        set_error("pcg_solve_trace: capacity >= 0 and two host arrays of that length");
        return POLYDG_EINVAL;
    }
    if (int st = check_ctx(c, "pcg_solve")) return st;
    if (!b_dev || !x_dev || b_dev == x_dev) { set_error("pcg_solve_trace: null or aliased vectors"); return POLYDG_EINVAL; }
    if (!(rtol > 0) || maxit < 1) { set_error("pcg_solve_trace: rtol must be > 0 and maxit >= 1"); return POLYDG_EINVAL; }
    if (pc && pc->ctx != c) { set_error("pcg_solve_trace: preconditioner built on another context"); return POLYDG_EINVAL; }
    cudaStream_t s = (cudaStream_t)stream;
    const int np = c->H.n_p;
    PcgScalars init = {};
    init.rtol2 = rtol * rtol;
    init.maxit = maxit;
    init.flexible = flexible == 2 ? 2 : flexible ? 1 : 0;   // 2: pipelined
    *c->h_sc = init;
    CU(cudaMemcpyAsync(c->work.sc, c->h_sc, sizeof(PcgScalars), cudaMemcpyHostToDevice, s));
    CU(cudaMemsetAsync(c->work.err, 0, sizeof(int), s));
    CU(launch_permute(b_dev, nullptr, c->work.b, c->d_to_caller, c->H.nc, np, 1, nullptr, s));
    CU(launch_permute(x_dev, nullptr, c->work.x[0], c->d_to_caller, c->H.nc, np, 1, nullptr, s));
    double* d_trace = nullptr;
    if (capacity > 0)
        if (int st = dalloc(&d_trace, 2 * (size_t)capacity)) return st;
    struct Guard { double*& p; ~Guard() { dfree(p); } } guard{d_trace};
    if (capacity > 0) CU(cudaMemsetAsync(d_trace, 0, 2 * (size_t)capacity * sizeof(double), s));
    if (int st = run_pcg(c, pc, c->work, s, d_trace, capacity)) return st;
    CU(launch_permute(c->work.x[0], c->work.x[1], x_dev, c->d_to_caller, c->H.nc, np, 0, c->work.sc, s));
    CU(cudaMemcpyAsync(c->h_sc, c->work.sc, sizeof(PcgScalars), cudaMemcpyDeviceToHost, s));
    CU(cudaStreamSynchronize(s));
    if (capacity > 0) {
        CU(cudaMemcpy(alphas, d_trace, capacity * sizeof(double), cudaMemcpyDeviceToHost));
        CU(cudaMemcpy(betas, d_trace + capacity, capacity * sizeof(double), cudaMemcpyDeviceToHost));
    }
    const PcgScalars& r = *c->h_sc;
    if (stats) {
        stats->iterations = r.it;
        stats->status = r.status;
        stats->relres = r.relres;
        stats->bnorm = std::sqrt(r.bb);
    }
    if (r.status != 0) {
        set_error(r.status == POLYDG_ECUDA ? "pcg_solve_trace: a device-side wait timed out"
                  : r.status == POLYDG_ENOTCONV ? "pcg_solve_trace: maximum number of iterations reached"
                  : r.status == POLYDG_EBREAKDOWN ? "pcg_solve_trace: breakdown (p^T K p <= 0 or non-finite beta)"
                                                  : "pcg_solve_trace: non-finite value in b or the residual");
    }
    return r.status;
}

int pcg_solve(polydg_ctx* c, asm_ctx* pc, const double* b_dev, double* x_dev, double rtol,
              int maxit, int flexible, void* stream, pcg_stats* stats) {
    return pcg_solve_trace(c, pc, b_dev, x_dev, rtol, maxit, flexible, stream, stats, nullptr,
                           nullptr, 0);
}

// Number of eigenvalues of the symmetric tridiagonal (d, e) below x: the negative
// pivots of the LDL^T factorisation of T - x I (Sylvester's law of inertia), with a
// zero pivot replaced by -pivmin.
static int sturm_count(const std::vector<double>& d, const std::vector<double>& e2, double x,
                       double pivmin) {
    int neg = 0;
    double q = d[0] - x;
    if (std::fabs(q) < pivmin) q = -pivmin;
    if (q < 0.0) ++neg;
    for (size_t k = 1; k < d.size(); ++k) {
        q = d[k] - x - e2[k - 1] / q;
        if (std::fabs(q) < pivmin) q = -pivmin;
        if (q < 0.0) ++neg;
    }
    return neg;
}

int pcg_lanczos_extremes(const double* alphas, const double* betas, int m, double* lmin, double* lmax) {
    if (m < 1 || !alphas || !betas || !lmin || !lmax) {
        set_error("pcg_lanczos_extremes: need m >= 1 coefficients and output pointers");
        return POLYDG_EINVAL;
    }
    // T_kk = 1/alpha_k + beta_{k-1}/alpha_{k-1}, T_{k,k+1} = sqrt(beta_k)/alpha_k
    std::vector<double> d(m), e2(m > 1 ? m - 1 : 1, 0.0);
    for (int k = 0; k < m; ++k) {
        if (!(alphas[k] > 0.0) || (k < m - 1 && !(betas[k] >= 0.0)) || !std::isfinite(alphas[k])) {
            set_error("pcg_lanczos_extremes: alphas must be > 0 and betas >= 0");
            return POLYDG_EINVAL;
        }
        d[k] = 1.0 / alphas[k] + (k > 0 ? betas[k - 1] / alphas[k - 1] : 0.0);
        if (k < m - 1) e2[k] = betas[k] / (alphas[k] * alphas[k]);
    }
    // the two extreme eigenvalues by bisection on Sturm counts inside the Gershgorin
    // interval: O(m) per step, accurate to a few ulps of |T| (the tridiagonal is never
    // formed densely, so traces of many thousand iterations cost milliseconds)
    double lo = d[0], hi = d[0], tmax = 0.0;
    for (int k = 0; k < m; ++k) {
        const double r = (k > 0 ? std::sqrt(e2[k - 1]) : 0.0) + (k < m - 1 ? std::sqrt(e2[k]) : 0.0);
        lo = std::min(lo, d[k] - r);
        hi = std::max(hi, d[k] + r);
        tmax = std::max(tmax, std::fabs(d[k]) + r);
    }
    if (!std::isfinite(lo) || !std::isfinite(hi)) {
        set_error("pcg_lanczos_extremes: non-finite coefficients");
        return POLYDG_EINVAL;
    }
    const double eps = std::numeric_limits<double>::epsilon();
    const double pivmin = std::max(std::numeric_limits<double>::min(), eps * eps * tmax * tmax);
    auto bisect = [&](int target) {       // smallest x with count(x) >= target
        double a = lo - eps * tmax, b = hi + eps * tmax;
        for (int it = 0; it < 200 && b - a > 2.0 * eps * std::max(std::fabs(a), std::fabs(b)); ++it) {
            const double mid = 0.5 * (a + b);
            if (mid <= a || mid >= b) break;
            if (sturm_count(d, e2, mid, pivmin) >= target) b = mid; else a = mid;
        }
        return 0.5 * (a + b);
    };
    *lmin = bisect(1);
    *lmax = bisect(m);
    return POLYDG_OK;
}

int sim_set_ionic_form(sim_ctx* sm, int form) {
    if (!sm || (form != POLYDG_IONIC_NODAL && form != POLYDG_IONIC_MODAL)) {
        set_error("sim_set_ionic_form: need a simulation and form 0 (nodal) or 1 (modal)");
        return POLYDG_EINVAL;
    }
    if (sm->k != 0) {
        set_error("sim_set_ionic_form: the form is chosen before the first step");
        return POLYDG_EINVAL;
    }
    polydg_ctx* c = sm->ctx;
    const HostSetup& H = c->H;
    const int np = H.n_p;
    if (form == POLYDG_IONIC_NODAL) {
        if (sm->Ym) { dfree(sm->Ym); sm->Ym = nullptr; ++sm->version; }
        return POLYDG_OK;
    }
    if (sm->Ym) return POLYDG_OK;
    int st;
    if (!c->d_Minv) {
        std::vector<double> minv;
        if ((st = mass_inverse_blocks(H, minv))) return st;
        if ((st = upload(&c->d_Minv, minv))) return st;
    }
    if ((st = dalloc(&sm->Ym, 5 * H.nc * np))) return st;
    cudaError_t e = launch_init_modal(sm->Ym, H.nc, np, sm->d_y0, 0);
    if (e == cudaSuccess) e = cudaStreamSynchronize(0);
    if (e != cudaSuccess) {
        dfree(sm->Ym);
        sm->Ym = nullptr;
        set_error(std::string("sim_set_ionic_form: ") + cudaGetErrorString(e));
        return POLYDG_ECUDA;
    }
    ++sm->version;                      // batches re-record their step graph
    return POLYDG_OK;
}

int sim_create(polydg_ctx* c, asm_ctx* pc, const sim_params* prm, sim_ctx** out) {
    if (int st = check_ctx(c, "sim_create")) return st;
    if (!prm || !out) { set_error("sim_create: null argument"); return POLYDG_EINVAL; }
    *out = nullptr;
    if (!(prm->rtol > 0) || prm->maxit < 1 || !(prm->stim_width > 0)) {
        set_error("sim_create: rtol > 0, maxit >= 1 and stim_width > 0 required");
        return POLYDG_EINVAL;
    }
    if (pc && pc->ctx != c) { set_error("sim_create: preconditioner built on another context"); return POLYDG_EINVAL; }
    const HostSetup& H = c->H;
    const int np = H.n_p;
    if (np != 3 && np != 6 && np != 10 && np != 15) { set_error("sim_create: coupled steps need p <= 4"); return POLYDG_EINVAL; }
    sim_ctx* sm = new sim_ctx();
    sm->ctx = c;
    sm->pc = pc;
    sm->prm = *prm;
    auto fail = [&](int code) { sim_destroy(sm); return code; };
    const int64_t n = H.nc * np, nn = (int64_t)H.node_w.size();
    int st;
    if ((st = sm->work.alloc(n)) || (st = dalloc(&sm->U, n)) || (st = dalloc(&sm->Uprev, n)) ||
        (st = dalloc(&sm->Uprev2, n)) || (st = dalloc(&sm->xg, n)) ||
        (st = dalloc(&sm->I, n)) || (st = dalloc(&sm->y, 5 * nn)) || (st = dalloc(&sm->yc, 6 * nn)) || (st = dalloc(&sm->d_y0, 5)) ||
        (st = dalloc(&sm->d_ss, 1)) || (st = dalloc(&sm->ring, kHistRing * n)) ||
        (st = dalloc(&sm->kuring, kHistRing * n)) || (st = dalloc(&sm->subW, 2 * n)) || (st = dalloc(&sm->gram, kSubMaxPairs * kSubMaxCtas)))
        return fail(st);
    if (cudaMallocHost((void**)&sm->h_ss, sizeof(SimScalars)) != cudaSuccess) {
        set_error("sim_create: pinned allocation failed");
        return fail(POLYDG_ENOMEM);
    }
    // stimulus profile F_e[i] = sum_q w_q A exp(-|x_q - x0|^2 / (2 w^2)) phi_i(x_q)
    std::vector<double> F(n, 0.0), U0(n, 0.0);
    const double s2 = 2.0 * prm->stim_width * prm->stim_width;
    for (int64_t e = 0; e < H.nc; ++e) {
        U0[e * np] = prm->u0;   // constant u0: only the (0,0) mode
        for (int64_t qn = H.node_ptr[e]; qn < H.node_ptr[e + 1]; ++qn) {
            const double* xq = &H.node_x[(size_t)H.dim * qn];
            const double dx = xq[0] - prm->stim_x0, dy = xq[1] - prm->stim_y0;
            const double dz = H.dim == 3 ? xq[2] - prm->stim_z0 : 0.0;
            const double g = H.node_w[qn] * prm->stim_amplitude * std::exp(-(dx * dx + dy * dy + dz * dz) / s2);
            for (int i = 0; i < np; ++i) F[e * np + i] += g * H.node_phi[qn * np + i];
        }
    }
    double y0[5];
    bc::rest_state(prm->u0, y0);
    if ((st = upload(&sm->F, F))) return fail(st);
    auto cu = [&](cudaError_t e) {
        if (e == cudaSuccess) return POLYDG_OK;
        set_error(std::string("sim_create: ") + cudaGetErrorString(e));
        return POLYDG_ECUDA;
    };
    SimScalars ss = {};
    ss.hist_len = 1;                    // the ring holds U^0
    ss.kd_step = -2;                    // no increment products yet
    PcgScalars sc = {};
    sc.rtol2 = prm->rtol * prm->rtol;
    sc.maxit = prm->maxit;
    sc.flexible = prm->flexible == 2 ? 2 : prm->flexible ? 1 : 0;   // 2: pipelined
    if ((st = cu(cudaMemcpy(sm->U, U0.data(), n * sizeof(double), cudaMemcpyHostToDevice))) ||
        (st = cu(cudaMemcpy(sm->Uprev, U0.data(), n * sizeof(double), cudaMemcpyHostToDevice))) ||
        (st = cu(cudaMemcpy(sm->Uprev2, U0.data(), n * sizeof(double), cudaMemcpyHostToDevice))) ||
        (st = cu(cudaMemcpy(sm->ring, U0.data(), n * sizeof(double), cudaMemcpyHostToDevice))) ||
        (st = cu(cudaMemcpy(sm->d_y0, y0, 5 * sizeof(double), cudaMemcpyHostToDevice))) ||
        (st = cu(launch_init_y(sm->y, nn, sm->d_y0, 0))) ||
        (st = cu(cudaMemcpy(sm->d_ss, &ss, sizeof(ss), cudaMemcpyHostToDevice))) ||
        (st = cu(cudaMemcpy(sm->work.sc, &sc, sizeof(sc), cudaMemcpyHostToDevice))) ||
        (st = cu(cudaDeviceSynchronize())))
        return fail(st);
    *out = sm;
    return POLYDG_OK;
}


}  // extern "C"
namespace polydg {
// The parts of one Crank-Nicolson step (Eq. fully-discrete-1) before and after
// its PCG solve: ionic update at the nodes and the ion-current load,
// right-hand side, x0 = U^k; then the rotation of U and the step statistics.
static GuessFeat guess_features(const polydg_ctx* c, const guess_model* g) {
    GuessFeat f;
    f.row_ptr = c->K.row_ptr;
    f.col = c->K.col;
    f.diam = c->d_diam;
    f.u_rest = g->scales[0];
    f.s_u = g->scales[1];
    f.s_d = g->scales[2];
    f.h_ref = g->scales[3];
    f.dt_ref = g->scales[4];
    f.dt = c->H.dt;
    f.inv_s_u = 1.0 / f.s_u;
    f.inv_s_d = 1.0 / f.s_d;
    return f;
}

static int enqueue_step_pre(sim_ctx* sm, cudaStream_t s) {
    polydg_ctx* c = sm->ctx;
    const HostSetup& H = c->H;
    const int np = H.n_p;
    const int64_t n = H.nc * np, nn = (int64_t)H.node_w.size();
    PcgWork& w = sm->work;
    const double dt = H.dt;
    CU(launch_step_begin(w.sc, sm->d_ss, s));
    if (sm->Ym)
        CU(launch_ionic_modal(np, sm->U, sm->Uprev, c->d_node_ptr, c->d_node_w, c->d_node_phi, c->d_Minv,
                              sm->Ym, sm->y, nn, H.nc, dt, sm->I, sm->d_ss, s));
    else
        CU(launch_ionic(np, sm->U, sm->Uprev, c->d_node_ptr, c->d_node_w, c->d_node_phi, sm->y, sm->yc, nn,
                        H.nc, dt, sm->I, sm->d_ss, c->ionic_lpc, s));
    CU(launch_matvec(MODE_RHS, np, c->K, c->K.val_minus, sm->U, w.b, sm->I, sm->F, -H.chi_cm * dt,
                     dt, sm->d_ss, dt, sm->prm.stim_duration, s));
    if (sm->guess_policy == 3) {  // subspace of the learned proposal and the last increments
        const double* xg = nullptr;
        if (sm->guess) {
            const GuessFeat f = guess_features(c, sm->guess);
            CU(launch_guess_propose(np, f, sm->guess->img, sm->U, sm->Uprev, sm->Uprev2, sm->xg, H.nc,
                                    sm->d_ss, sm->gxt, sm->guess->d_err, sm->guess->n_sm, s));
            xg = sm->xg;
        }
        CU(launch_guess_subspace(np, c->K, w.b, sm->U, xg, sm->ring, sm->kuring, sm->subW, sm->gram, n,
                                 sm->d_ss, s));
        CU(launch_subspace_copy(sm->U, xg, sm->ring, sm->kuring, sm->subW, w.x[0], n, sm->d_ss, s));
    } else if (sm->guess) {     // from k = 2 on: learned proposal, kept if its residual is smaller
        const GuessFeat f = guess_features(c, sm->guess);
        CU(launch_guess_propose(np, f, sm->guess->img, sm->U, sm->Uprev, sm->Uprev2, sm->xg, H.nc,
                                sm->d_ss, sm->gxt, sm->guess->d_err, sm->guess->n_sm, s));
        CU(launch_guess_select(np, c->K, w.b, sm->xg, sm->U, w.partials, sm->d_ss, sm->guess_policy, s));
        CU(launch_select_copy(sm->U, sm->xg, w.x[0], n, sm->d_ss, s));
    } else {
        CU(launch_copy(sm->U, w.x[0], n, sm->d_ss, s));
    }
    return POLYDG_OK;
}

static int enqueue_step_post(sim_ctx* sm, cudaStream_t s) {
    const int64_t n = sm->ctx->H.nc * sm->ctx->H.n_p;
    PcgWork& w = sm->work;
    CU(launch_step_finish(sm->U, sm->Uprev, sm->Uprev2, w.x[0], w.x[1], n, w.sc, sm->d_ss, sm->ring, s));
    return POLYDG_OK;
}

static int enqueue_step(sim_ctx* sm, cudaStream_t s, cudaEvent_t ev_begin, cudaEvent_t ev_end) {
    if (int st = enqueue_step_pre(sm, s)) return st;
    if (ev_begin) CU(cudaEventRecord(ev_begin, s));
    if (int st = run_pcg(sm->ctx, sm->pc, sm->work, s)) return st;
    if (ev_end) CU(cudaEventRecord(ev_end, s));
    return enqueue_step_post(sm, s);
}

// One step of every simulation of a batch: the per-simulation kernels before the
// solves, one batched persistent launch for all solves, the kernels after.
static int enqueue_batch_step(batch_ctx* bt, cudaStream_t s) {
    for (sim_ctx* sm : bt->sims) {
        if (int st = enqueue_step_pre(sm, s)) return st;
        CU(cudaMemsetAsync(&sm->work.gs->count, 0, sizeof(unsigned), s));
    }
    if (bt->n_cta > 0)
        CU(launch_pcg_batched(bt->dtype, bt->np, bt->d_args, bt->d_map, bt->n_cta, bt->smem, s));
    if (bt->g_cta > 0)
        CU(launch_pcg_groups(bt->gq, bt->np, bt->d_gargs, bt->d_gmap, bt->g_cta, bt->gsmem, s));
    for (sim_ctx* sm : bt->sims)
        if (int st = enqueue_step_post(sm, s)) return st;
    return POLYDG_OK;
}

// Cut costs[0..n) into at most G contiguous runs minimising the largest run sum
// (bisection on the budget); ptr gets G + 1 boundaries (trailing runs empty).
static std::vector<int32_t> linear_partition(const std::vector<double>& costs, int G) {
    const int n = (int)costs.size();
    auto pack = [&](double budget, std::vector<int32_t>* ptr) {
        int runs = 0, k = 0;
        while (k < n) {
            if (ptr) (*ptr)[runs] = k;
            ++runs;
            double acc = 0.0;
            const int first = k;
            while (k < n && (k == first || acc + costs[k] <= budget)) acc += costs[k++];
        }
        return runs;
    };
    double lo = 0.0, hi = 0.0;
    for (double c : costs) hi += c;
    for (int it = 0; it < 60; ++it) {
        const double mid = 0.5 * (lo + hi);
        if (pack(mid, nullptr) <= G) hi = mid; else lo = mid;
    }
    std::vector<int32_t> ptr(G + 1, n);
    const int used = n ? pack(hi, &ptr) : 0;
    for (int g = used; g <= G; ++g) ptr[g] = n;
    return ptr;
}

// CTAs per unit: one at a time to the unit with the largest cost per CTA.
static std::vector<int> allocate_ctas(const std::vector<double>& cost, int n_cta) {
    std::vector<int> g(cost.size(), 1);
    for (int k = (int)cost.size(); k < n_cta; ++k) {
        int best = 0;
        for (int i = 1; i < (int)cost.size(); ++i)
            if (cost[i] / g[i] > cost[best] / g[best]) best = i;
        ++g[best];
    }
    return g;
}

// Plan and arguments of a lockstep group with `ctas` CTAs.
static int build_group(batch_ctx* bt, BatchGroup& gr, GroupArgs& ga) {
    sim_ctx* s0 = bt->sims[gr.members[0]];
    polydg_ctx* c = s0->ctx;
    asm_ctx* pc = s0->pc;
    shared_local* sl = s0->shared;
    const HostSetup& H = c->H;
    const int np = H.n_p, G = gr.ctas, R = (int)gr.members.size();
    if (int st = build_plan(c, pc, G, gr.plan, 1)) return st;
    const Plan& P = gr.plan;
    // element-aligned pieces of subdomains per CTA: tiles of two elements' rows, costed by
    // the bytes of Q_i^T and Q_i they stream, split into G contiguous runs of equal cost
    const int esz = sl->precision == POLYDG_FP32 ? 4 : 2;
    struct QT { int sub, r0, r1; };
    std::vector<QT> qt;
    std::vector<double> cost;
    const double bw_sm = 6.0e12 / c->n_sm;
    for (int i = 0; i < H.n_sub; ++i) {
        const SharedBlock& B = sl->hblocks[i];
        for (int r0 = 0; r0 < B.n; r0 += 2 * np) {
            const int r1 = std::min(B.n, r0 + 2 * np);
            qt.push_back({i, r0, r1});
            cost.push_back(2.0 * (r1 - r0) * B.ld * esz / bw_sm + 0.2e-6 + (r0 == 0 ? 3.0e-6 : 0.0));
        }
    }
    const std::vector<int32_t> tptr = linear_partition(cost, G);
    std::vector<GemvRun> pieces;
    std::vector<int32_t> piece_ptr(G + 1, 0);
    for (int g = 0; g < G; ++g) {
        piece_ptr[g] = (int32_t)pieces.size();
        for (int32_t k = tptr[g]; k < tptr[g + 1]; ++k) {
            if ((int32_t)pieces.size() > piece_ptr[g] && pieces.back().block == qt[k].sub &&
                pieces.back().row_end == qt[k].r0)
                pieces.back().row_end = qt[k].r1;
            else
                pieces.push_back({qt[k].sub, qt[k].r0, qt[k].r1, 0});
        }
        if ((int32_t)pieces.size() - piece_ptr[g] > 64) {
            set_error("batch_create: more than 64 subdomain pieces per CTA in a group");
            return POLYDG_EINVAL;
        }
    }
    piece_ptr[G] = (int32_t)pieces.size();
    std::vector<int32_t> pb(H.n_sub), pcnt(H.n_sub);
    for (int i = 0; i < H.n_sub; ++i) { pb[i] = pc->blocks[i].pair_begin; pcnt[i] = pc->blocks[i].pair_count; }
    int st;
    if ((st = upload(&gr.d_pieces, pieces)) || (st = upload(&gr.d_piece_ptr, piece_ptr)) ||
        (st = upload(&gr.d_pair_begin, pb)) || (st = upload(&gr.d_pair_count, pcnt)))
        return st;
    gr.yq.assign(R, nullptr);
    for (int k = 0; k < R; ++k)
        if ((st = dalloc(&gr.yq[k], (size_t)H.nc * np))) return st;
    // shared memory: per-warp slots of one row of Q, r' (fp64) and X, Y (fp32) of R
    // simulations, coarse and chunk staging, run descriptors
    auto r128 = [](size_t x) { return (x + 127) & ~(size_t)127; };
    const size_t ldm = (size_t)sl->max_ld;
    const int nq = pc->has_coarse ? pc->nq : 1;
    const size_t n0 = pc->has_coarse ? pc->n0 : 0;
    const size_t fixed = r128(kMaxRhs * ldm * 8) + 2 * r128(kMaxRhs * ldm * 4) + r128(n0 * 8) +
                         r128((size_t)P.max_need * np * 8) + r128(128 * 48);
    const size_t cap = 208 * 1024, slot = r128(ldm * esz);
    const int NW = kPersistThreads / 32;
    const int64_t wst = fixed < cap ? (int64_t)((cap - fixed) / (NW * slot)) : 0;
    if (wst < 1) { set_error("batch_create: a subdomain is too large for the shared-memory plan of a group"); return POLYDG_EINVAL; }
    ga = GroupArgs{};
    ga.grid = G;
    ga.R = R;
    ga.wstages = (int)std::min<int64_t>(kMaxWarpStages, wst);
    ga.n0 = (int)n0;
    ga.ld0 = pc->has_coarse ? (int)pc->ld0 : 0;
    ga.nq = nq;
    ga.redundant = P.redundant;
    ga.np_ = np;
    ga.nc = H.nc;
    ga.slot_bytes = slot;
    ga.ld_max = ldm;
    ga.rp_off = (size_t)NW * ga.wstages * slot;
    ga.x_off = ga.rp_off + r128(kMaxRhs * ldm * 8);
    ga.y_off = ga.x_off + r128(kMaxRhs * ldm * 4);
    ga.r0_off = ga.y_off + r128(kMaxRhs * ldm * 4);
    ga.y0_off = ga.r0_off + r128(n0 * 8);
    ga.pn_off = ga.y0_off;
    ga.td_off = ga.pn_off + r128((size_t)P.max_need * np * 8);
    const size_t smem = ga.td_off + r128(128 * 48);
    bt->gsmem = std::max(bt->gsmem, smem);
    ga.row_ptr = c->K.row_ptr;
    ga.cta_chunk = P.cta_chunk;
    ga.chunk_elem = P.chunk_elem;
    ga.need_ptr = P.need_ptr;
    ga.need = P.need;
    ga.need_aggl = P.need_aggl;
    ga.need_agg_ptr = P.need_agg_ptr;
    ga.need_agg = P.need_agg;
    ga.col_local = P.col_local;
    ga.elem_ptr = P.elem_ptr;
    ga.blocks = pc->d_blocks;
    ga.sub_pairs = P.sub_pairs;
    ga.pair_begin = gr.d_pair_begin;
    ga.pair_count = gr.d_pair_count;
    ga.st64 = pc->st64;
    ga.pair_ptr = pc->has_coarse ? pc->d_pair_ptr : c->d_zero_ptr;
    ga.T = pc->has_coarse ? pc->d_T : nullptr;
    ga.agg = pc->has_coarse ? pc->d_agg : nullptr;
    ga.crow_ptr = P.crow_ptr;
    ga.sblocks = sl->blocks;
    ga.qstore = sl->precision == POLYDG_FP32 ? (const void*)sl->st32 : (const void*)sl->st16;
    ga.lam = sl->lam;
    ga.linv = sl->linv;
    ga.pieces = gr.d_pieces;
    ga.piece_ptr = gr.d_piece_ptr;
    ga.chi = H.chi_cm;
    for (int k = 0; k < R; ++k) {
        sim_ctx* sm = bt->sims[gr.members[k]];
        PcgWork& w = sm->work;
        GroupSim& g = ga.sim[k];
        g.val = sm->ctx->K.val;
        g.K0inv = sm->pc->has_coarse ? sm->pc->st64 + sm->pc->off0 : nullptr;
        g.c = 0.5 * H.dt * sm->sigma;
        g.b = w.b;
        g.x = w.x[0];
        g.r[0] = w.r[0]; g.r[1] = w.r[1];
        g.p[0] = w.p; g.p[1] = w.p2;
        g.q[0] = w.q; g.q[1] = w.q2;
        g.z = w.z; g.zl = w.zl; g.w = w.w;
        g.r0p = sm->pc->d_r0p;
        g.y0 = sm->pc->d_y0;
        g.yq = gr.yq[k];
        g.sc = w.sc;
    }
    ga.partials = s0->work.partials;
    ga.gs = s0->work.gs;
    ga.err = s0->work.err;
    return POLYDG_OK;
}

// Zero the per-call counters of a simulation's scalars (host copy h).
static int reset_step_counters(sim_ctx* sm, SimScalars& h, cudaStream_t s) {
    CU(cudaMemcpyAsync(&h, sm->d_ss, sizeof(SimScalars), cudaMemcpyDeviceToHost, s));
    CU(cudaStreamSynchronize(s));
    h.steps_done = 0;
    h.total_its = 0;
    h.max_its = 0;
    h.last_relres = 0.0;
    h.guesses_taken = 0;
    CU(cudaMemcpyAsync(sm->d_ss, &h, sizeof(SimScalars), cudaMemcpyHostToDevice, s));
    return POLYDG_OK;
}

static void fill_stats(const SimScalars& h, double seconds, step_stats* st) {
    st->steps_done = h.steps_done;
    st->total_iterations = h.total_its;
    st->max_iterations = h.max_its;
    st->status = h.status;
    st->last_relres = h.last_relres;
    st->pcg_seconds = seconds;
    st->guesses_taken = h.guesses_taken;
}
}  // namespace polydg

extern "C" {

int monodomain_step(sim_ctx* sm, int nsteps, void* stream, step_stats* stats) {
    if (!sm) { set_error("monodomain_step: null simulation"); return POLYDG_EINVAL; }
    if (nsteps < 0) { set_error("monodomain_step: nsteps < 0"); return POLYDG_EINVAL; }
    cudaStream_t s = (cudaStream_t)stream;
    SimScalars& h = *sm->h_ss;
    if (int st = reset_step_counters(sm, h, s)) return st;
    while ((int)sm->ev.size() < 2 * nsteps) {
        cudaEvent_t e;
        CU(cudaEventCreate(&e));
        sm->ev.push_back(e);
    }
    for (int i = 0; i < nsteps; ++i)
        if (int st = enqueue_step(sm, s, sm->ev[2 * i], sm->ev[2 * i + 1])) return st;
    CU(cudaMemcpyAsync(&h, sm->d_ss, sizeof(SimScalars), cudaMemcpyDeviceToHost, s));
    CU(cudaStreamSynchronize(s));
    sm->k = h.k;
    if (stats) {
        double sec = 0.0;
        for (int i = 0; i < nsteps; ++i) {
            float ms = 0.f;
            if (cudaEventElapsedTime(&ms, sm->ev[2 * i], sm->ev[2 * i + 1]) == cudaSuccess) sec += 1e-3 * ms;
        }
        fill_stats(h, sec, stats);
    }
    if (h.status != 0) set_error("monodomain_step: a step's PCG solve failed");
    return h.status;
}

int sim_get_state(sim_ctx* sm, double* u_dev, double* y_dev, void* stream) {
    if (!sm || !u_dev) { set_error("sim_get_state: null argument"); return POLYDG_EINVAL; }
    polydg_ctx* c = sm->ctx;
    cudaStream_t s = (cudaStream_t)stream;
    CU(launch_permute(sm->U, nullptr, u_dev, c->d_to_caller, c->H.nc, c->H.n_p, 0, nullptr, s));
    if (y_dev) CU(launch_node_gather(sm->y, y_dev, c->d_node_pos, (int64_t)c->H.node_w.size(), s));
    return POLYDG_OK;
}

int sim_get_ionic_aux(sim_ctx* sm, double* aux_dev, void* stream) {
    if (!sm || !aux_dev) { set_error("sim_get_ionic_aux: null argument"); return POLYDG_EINVAL; }
    if (sm->Ym) { set_error("sim_get_ionic_aux: the modal form carries no per-node functions"); return POLYDG_EINVAL; }
    polydg_ctx* c = sm->ctx;
    CU(launch_node_gather(sm->yc, aux_dev, c->d_node_pos, (int64_t)c->H.node_w.size(), (cudaStream_t)stream, 6));
    return POLYDG_OK;
}

int sim_set_ionic_aux(sim_ctx* sm, const double* aux_dev, void* stream) {
    if (!sm || !aux_dev) { set_error("sim_set_ionic_aux: null argument"); return POLYDG_EINVAL; }
    if (sm->Ym) { set_error("sim_set_ionic_aux: the modal form carries no per-node functions"); return POLYDG_EINVAL; }
    polydg_ctx* c = sm->ctx;
    cudaStream_t s = (cudaStream_t)stream;
    CU(launch_node_scatter(aux_dev, sm->yc, c->d_node_pos, (int64_t)c->H.node_w.size(), s, 6));
    CU(launch_ionic_aux_valid(sm->d_ss, s));
    return POLYDG_OK;
}

int sim_set_potential(sim_ctx* sm, const double* u_dev, const double* uprev_dev, void* stream) {
    if (!sm || !u_dev) { set_error("sim_set_potential: null argument"); return POLYDG_EINVAL; }
    polydg_ctx* c = sm->ctx;
    cudaStream_t s = (cudaStream_t)stream;
    CU(launch_permute(u_dev, nullptr, sm->U, c->d_to_caller, c->H.nc, c->H.n_p, 1, nullptr, s));
    CU(launch_permute(uprev_dev ? uprev_dev : u_dev, nullptr, sm->Uprev, c->d_to_caller, c->H.nc,
                      c->H.n_p, 1, nullptr, s));
    CU(cudaMemcpyAsync(sm->Uprev2, sm->Uprev, c->H.nc * c->H.n_p * sizeof(double),
                       cudaMemcpyDeviceToDevice, s));
    CU(launch_history_reset(c->H.n_p, c->K, sm->ring, sm->kuring, sm->U, sm->Uprev, c->H.nc * c->H.n_p,
                            sm->d_ss, s));
    CU(launch_ionic_aux_valid(sm->d_ss, s, -1));  // the carried u^{k-1} no longer matches
    return POLYDG_OK;
}

int sim_set_history(sim_ctx* sm, const double* hist_dev, int count, void* stream) {
    if (!sm || !hist_dev || count < 1) { set_error("sim_set_history: need a simulation, a device array and count >= 1"); return POLYDG_EINVAL; }
    polydg_ctx* c = sm->ctx;
    CU(launch_history_set(c->K, hist_dev, count, sm->ring, sm->kuring, sm->U, sm->Uprev, sm->Uprev2,
                          c->d_to_caller, c->H.nc, c->H.n_p, sm->d_ss, (cudaStream_t)stream));
    CU(launch_ionic_aux_valid(sm->d_ss, (cudaStream_t)stream, -1));   // the carried u^{k-1} no longer matches
    return POLYDG_OK;
}

int sim_set_state(sim_ctx* sm, const double* y_dev, const double* Y_dev, int64_t k, void* stream) {
    if (!sm || k < 0) { set_error("sim_set_state: need a simulation and k >= 0"); return POLYDG_EINVAL; }
    if (sm->Ym ? !Y_dev : !y_dev) {
        set_error(sm->Ym ? "sim_set_state: the modal form needs the coefficients Y"
                         : "sim_set_state: the nodal form needs the nodal states y");
        return POLYDG_EINVAL;
    }
    polydg_ctx* c = sm->ctx;
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t nn = (int64_t)c->H.node_w.size(), n = c->H.nc * c->H.n_p;
    if (y_dev) CU(launch_node_scatter(y_dev, sm->y, c->d_node_pos, nn, s));
    if (sm->Ym)
        for (int l = 0; l < bc::kStates; ++l)
            CU(launch_permute(Y_dev + l * n, nullptr, sm->Ym + l * n, c->d_to_caller, c->H.nc, c->H.n_p, 1,
                              nullptr, s));
    CU(launch_set_step(sm->d_ss, k, s));
    sm->k = k;
    return POLYDG_OK;
}

int sim_get_ionic_coeffs(sim_ctx* sm, double* Y_dev, void* stream) {
    if (!sm || !Y_dev) { set_error("sim_get_ionic_coeffs: null argument"); return POLYDG_EINVAL; }
    if (!sm->Ym) { set_error("sim_get_ionic_coeffs: the simulation keeps its ionic state at the nodes"); return POLYDG_EINVAL; }
    polydg_ctx* c = sm->ctx;
    const int64_t n = c->H.nc * c->H.n_p;
    for (int l = 0; l < bc::kStates; ++l)
        CU(launch_permute(sm->Ym + l * n, nullptr, Y_dev + l * n, c->d_to_caller, c->H.nc, c->H.n_p, 0,
                          nullptr, (cudaStream_t)stream));
    return POLYDG_OK;
}

int64_t sim_step_index(const sim_ctx* sm) { return sm ? sm->k : -1; }

int batch_create(sim_ctx* const* sims, int n, batch_ctx** out) {
    if (!sims || n < 1 || !out) { set_error("batch_create: need n >= 1 simulations and an output pointer"); return POLYDG_EINVAL; }
    *out = nullptr;
    for (int i = 0; i < n; ++i) {
        if (!sims[i] || !sims[i]->pc) { set_error("batch_create: every simulation needs a preconditioner"); return POLYDG_EINVAL; }
        const sim_ctx* a = sims[i];
        const sim_ctx* b = sims[0];
        if (a->ctx->device != b->ctx->device || a->ctx->H.n_p != b->ctx->H.n_p) {
            set_error("batch_create: simulations must share the device and the degree");
            return POLYDG_EINVAL;
        }
        for (int j = 0; j < i; ++j)
            if (sims[j] == a || sims[j]->pc == a->pc) {
                set_error("batch_create: simulations must be distinct and have their own preconditioners");
                return POLYDG_EINVAL;
            }
    }
    batch_ctx* bt = new batch_ctx();
    bt->sims.assign(sims, sims + n);
    for (int i = 0; i < n; ++i) bt->shared_at_create.push_back(sims[i]->shared);
    bt->np = sims[0]->ctx->H.n_p;
    bt->device = sims[0]->ctx->device;
    bt->group.assign(n, 0);
    auto fail = [&](int code) { batch_destroy(bt); return code; };
    const int n_sm = sims[0]->ctx->n_sm;
    // simulations with shared local solves go into lockstep groups of <= kMaxRhs (in order)
    for (int i = 0; i < n; ++i) {
        sim_ctx* sm = sims[i];
        if (!sm->shared) { bt->solo.push_back(i); continue; }
        BatchGroup* g = nullptr;
        for (auto& gg : bt->groups)
            if (bt->sims[gg.members[0]]->shared == sm->shared && (int)gg.members.size() < kMaxRhs) g = &gg;
        if (!g) { bt->groups.emplace_back(); g = &bt->groups.back(); }
        g->members.push_back(i);
    }
    if ((int)bt->solo.size() > n_sm || (int)bt->groups.size() > n_sm) {
        set_error("batch_create: more simulations (or groups) than SMs");
        return fail(POLYDG_EINVAL);
    }
    for (auto& g : bt->groups) {
        const int q = bt->sims[g.members[0]]->shared->precision == POLYDG_FP32 ? 1 : 2;
        if (bt->gq && bt->gq != q) { set_error("batch_create: shared local solves of one batch need one precision"); return fail(POLYDG_EINVAL); }
        bt->gq = q;
    }
    // solo simulations: the per-simulation launch
    if (!bt->solo.empty()) {
        bt->dtype = sims[bt->solo[0]]->pc->precision;
        std::vector<double> cost;
        for (int i : bt->solo) {
            const sim_ctx* sm = sims[i];
            if (sm->pc->precision != bt->dtype) { set_error("batch_create: simulations must share the local precision"); return fail(POLYDG_EINVAL); }
            const int np = sm->ctx->H.n_p;
            cost.push_back((double)sm->pc->store_bytes + 8.0 * np * np * (double)sm->ctx->K.nblk +
                           96.0 * (double)(sm->ctx->H.nc * np));
        }
        const std::vector<int> g = allocate_ctas(cost, n_sm);
        bt->n_cta = n_sm;
        bt->plans.resize(bt->solo.size());
        std::vector<PersistArgs> args(bt->solo.size());
        std::vector<int2> map;
        for (size_t k = 0; k < bt->solo.size(); ++k) {
            sim_ctx* sm = sims[bt->solo[k]];
            bt->group[bt->solo[k]] = g[k];
            if (int st = build_plan(sm->ctx, sm->pc, g[k], bt->plans[k], 1)) return fail(st);
            bt->smem = std::max(bt->smem, bt->plans[k].smem);
            args[k] = persist_args(sm->ctx, sm->pc, bt->plans[k], sm->work);
            for (int j = 0; j < g[k]; ++j) map.push_back(make_int2((int)k, j));
        }
        int occ = 0;
        if (persistent_occupancy(bt->dtype, bt->np, bt->smem, &occ, 1) != cudaSuccess || occ < 1) {
            set_error("batch_create: the batched kernel does not fit on an SM");
            return fail(POLYDG_ECUDA);
        }
        int st;
        if ((st = upload(&bt->d_args, args)) || (st = upload(&bt->d_map, map))) return fail(st);
    }
    // lockstep groups: the group launch
    if (!bt->groups.empty()) {
        std::vector<double> cost;
        for (auto& gr : bt->groups) {
            const sim_ctx* s0 = bt->sims[gr.members[0]];
            const int np = s0->ctx->H.n_p;
            cost.push_back((double)s0->shared->store_bytes +
                           gr.members.size() * (8.0 * np * np * (double)s0->ctx->K.nblk +
                                                96.0 * (double)(s0->ctx->H.nc * np)));
        }
        const std::vector<int> g = allocate_ctas(cost, n_sm);
        std::vector<GroupArgs> gargs(bt->groups.size());
        std::vector<int2> map;
        for (size_t k = 0; k < bt->groups.size(); ++k) {
            BatchGroup& gr = bt->groups[k];
            gr.ctas = g[k];
            for (int i : gr.members) bt->group[i] = g[k];
            if (int st = build_group(bt, gr, gargs[k])) return fail(st);
            for (int j = 0; j < g[k]; ++j) map.push_back(make_int2((int)k, j));
        }
        bt->g_cta = n_sm;
        int occ = 0;
        if (group_occupancy(bt->gq, bt->np, bt->gsmem, &occ) != cudaSuccess || occ < 1) {
            set_error("batch_create: the group kernel does not fit on an SM");
            return fail(POLYDG_ECUDA);
        }
        int st;
        if ((st = upload(&bt->d_gargs, gargs)) || (st = upload(&bt->d_gmap, map))) return fail(st);
    }
    if (cudaStreamCreateWithFlags(&bt->cap, cudaStreamNonBlocking) != cudaSuccess ||
        cudaMallocHost((void**)&bt->h_ss, n * sizeof(SimScalars)) != cudaSuccess) {
        set_error("batch_create: CUDA setup failed");
        return fail(POLYDG_ECUDA);
    }
    *out = bt;
    return POLYDG_OK;
}

int sim_set_shared_local(sim_ctx* sm, shared_local* sl) {
    if (!sm) { set_error("sim_set_shared_local: null simulation"); return POLYDG_EINVAL; }
    if (sl) {
        const HostSetup& A = sm->ctx->H;
        const HostSetup& B = sl->ctx->H;
        if (A.nc != B.nc || A.n_p != B.n_p || A.sub_ptr != B.sub_ptr || A.to_caller != B.to_caller ||
            A.dt != B.dt || A.chi_cm != B.chi_cm || A.row_ptr != B.row_ptr || A.col != B.col) {
            set_error("sim_set_shared_local: the simulation's mesh, subdomains or time step differ");
            return POLYDG_EINVAL;
        }
        if (!sm->pc || !sm->pc->has_coarse || !sl->ctx) {
            set_error("sim_set_shared_local: the simulation needs a two-level preconditioner");
            return POLYDG_EINVAL;
        }
        const double s0 = A.sigma[0];
        for (int64_t k = 0; k < A.nc; ++k) {
            const double* S = &A.sigma[4 * k];
            if (S[1] != 0.0 || S[2] != 0.0 || S[0] != S[3] || S[0] != s0) {
                set_error("sim_set_shared_local: the simulation's conductivity is not one scalar multiple of I");
                return POLYDG_EINVAL;
            }
        }
        sm->sigma = s0;
    }
    if (sm->shared != sl) {
        sm->shared = sl;
        sm->version += 1;
    }
    return POLYDG_OK;
}

int batch_get_groups(const batch_ctx* bt, int32_t* ctas_of_sim) {
    if (!bt || !ctas_of_sim) { set_error("batch_get_groups: null argument"); return POLYDG_EINVAL; }
    for (size_t i = 0; i < bt->group.size(); ++i) ctas_of_sim[i] = bt->group[i];
    return POLYDG_OK;
}

int batch_step(batch_ctx* bt, int nsteps, void* stream, step_stats* per_sim, double* seconds) {
    if (!bt) { set_error("batch_step: null batch"); return POLYDG_EINVAL; }
    if (nsteps < 0) { set_error("batch_step: nsteps < 0"); return POLYDG_EINVAL; }
    cudaStream_t s = (cudaStream_t)stream;
    const int n = (int)bt->sims.size();
    for (int i = 0; i < n; ++i)
        if (bt->sims[i]->shared != bt->shared_at_create[i]) {
            set_error("batch_step: a simulation's shared local solves changed since batch_create");
            return POLYDG_EINVAL;
        }
    for (int i = 0; i < n; ++i)
        if (int st = reset_step_counters(bt->sims[i], bt->h_ss[i], s)) return st;
    bool stale = !bt->exec;
    for (int i = 0; i < n && !stale; ++i) stale = bt->versions[i] != bt->sims[i]->version;
    if (stale) {                        // (re)capture one step of all simulations
        if (bt->exec) { cudaGraphExecDestroy(bt->exec); bt->exec = nullptr; }
        if (bt->graph) { cudaGraphDestroy(bt->graph); bt->graph = nullptr; }
        bt->versions.resize(n);
        for (int i = 0; i < n; ++i) bt->versions[i] = bt->sims[i]->version;
        cudaGraph_t g = nullptr;
        CU(cudaStreamBeginCapture(bt->cap, cudaStreamCaptureModeThreadLocal));
        const int st = enqueue_batch_step(bt, bt->cap);
        const cudaError_t e = cudaStreamEndCapture(bt->cap, &g);
        if (st || e != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            if (!st) set_error(std::string("batch_step: graph capture failed: ") + cudaGetErrorString(e));
            return st ? st : POLYDG_ECUDA;
        }
        bt->graph = g;
        CU(cudaGraphInstantiate(&bt->exec, g, 0));
    }
    while ((int)bt->ev.size() < 2 * nsteps) {
        cudaEvent_t e;
        CU(cudaEventCreate(&e));
        bt->ev.push_back(e);
    }
    for (int k = 0; k < nsteps; ++k) {
        CU(cudaEventRecord(bt->ev[2 * k], s));
        CU(cudaGraphLaunch(bt->exec, s));
        CU(cudaEventRecord(bt->ev[2 * k + 1], s));
    }
    for (int i = 0; i < n; ++i)
        CU(cudaMemcpyAsync(&bt->h_ss[i], bt->sims[i]->d_ss, sizeof(SimScalars), cudaMemcpyDeviceToHost, s));
    CU(cudaStreamSynchronize(s));
    double sec = 0.0;
    for (int k = 0; k < nsteps; ++k) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, bt->ev[2 * k], bt->ev[2 * k + 1]) == cudaSuccess) sec += 1e-3 * ms;
    }
    if (seconds) *seconds = sec;
    int status = POLYDG_OK;
    for (int i = 0; i < n; ++i) {
        bt->sims[i]->k = bt->h_ss[i].k;
        if (per_sim) fill_stats(bt->h_ss[i], sec, &per_sim[i]);
        if (status == POLYDG_OK && bt->h_ss[i].status != 0) status = bt->h_ss[i].status;
    }
    if (status != POLYDG_OK) set_error("batch_step: a simulation's PCG solve failed");
    return status;
}

// the training kernel's shared-memory image of the network fits for n_p <= 10 (p <= 3)
static bool valid_np(int np) { return np == 3 || np == 6 || np == 10; }

int guess_n_params(int n_p) {
    if (!valid_np(n_p)) { set_error("guess_n_params: n_p must be 3, 6 or 10"); return POLYDG_EINVAL; }
    return guess_param_count(n_p);
}

int guess_create(int n_p, const double* params, const double* scales, guess_model** out) {
    if (!out || !params || !valid_np(n_p)) {
        set_error("guess_create: need n_p in {3, 6, 10}, parameters and an output pointer");
        return POLYDG_EINVAL;
    }
    *out = nullptr;
    guess_model* g = new guess_model();
    auto fail = [&](int code) { guess_destroy(g); return code; };
    g->np = n_p;
    g->P = guess_param_count(n_p);
    if (scales) {
        if (!(scales[1] > 0) || !(scales[2] > 0) || !(scales[3] > 0) || !(scales[4] > 0)) {
            set_error("guess_create: the scales s_u, s_d, h_ref, dt_ref must be > 0");
            return fail(POLYDG_EINVAL);
        }
        for (int k = 0; k < 5; ++k) g->scales[k] = scales[k];
    }
    if (cudaGetDevice(&g->device) != cudaSuccess) { set_error("guess_create: no CUDA device"); return fail(POLYDG_ECUDA); }
    int n_sm = 0;
    cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, g->device);
    g->grid_max = std::max(1, 2 * n_sm);
    std::vector<float> w(g->P);
    for (int k = 0; k < g->P; ++k) w[k] = (float)params[k];
    int st;
    if ((st = upload(&g->w32, w)) || (st = dalloc(&g->m, g->P)) || (st = dalloc(&g->v, g->P)) ||
        (st = dalloc(&g->w16, g->P)) || (st = dalloc(&g->part, (size_t)g->grid_max * g->P)) ||
        (st = dalloc(&g->lpart, g->grid_max)) || (st = dalloc(&g->loss, 1)) || (st = dalloc(&g->d_err, 1)) ||
        (st = dalloc(&g->img, guess_tc_image_bytes(n_p))))
        return fail(st);
    g->n_sm = std::max(1, n_sm);
    CU(cudaMemset(g->d_err, 0, sizeof(int)));
    CU(cudaMemset(g->m, 0, g->P * sizeof(float)));
    CU(cudaMemset(g->v, 0, g->P * sizeof(float)));
    CU(guess_prepare(n_p));
    CU(launch_to_half(g->w32, g->w16, g->P, 0));
    CU(launch_guess_tc_image(n_p, g->w16, g->img, 0));
    CU(cudaDeviceSynchronize());
    *out = g;
    return POLYDG_OK;
}

int guess_get_params(const guess_model* g, double* params, double* adam_m, double* adam_v,
                     int64_t* adam_t) {
    if (!g) { set_error("guess_get_params: null model"); return POLYDG_EINVAL; }
    std::vector<float> h(g->P);
    const float* src[3] = {g->w32, g->m, g->v};
    double* dst[3] = {params, adam_m, adam_v};
    for (int k = 0; k < 3; ++k) {
        if (!dst[k]) continue;
        CU(cudaMemcpy(h.data(), src[k], g->P * sizeof(float), cudaMemcpyDeviceToHost));
        for (int i = 0; i < g->P; ++i) dst[k][i] = h[i];
    }
    if (adam_t) *adam_t = g->t;
    return POLYDG_OK;
}

int guess_set_scales(guess_model* g, const double* scales) {
    if (!g || !scales || !(scales[1] > 0) || !(scales[2] > 0) || !(scales[3] > 0) || !(scales[4] > 0)) {
        set_error("guess_set_scales: need a model and scales with s_u, s_d, h_ref, dt_ref > 0");
        return POLYDG_EINVAL;
    }
    for (int k = 0; k < 5; ++k) g->scales[k] = scales[k];
    return POLYDG_OK;
}

int guess_propose(guess_model* g, polydg_ctx* c, const double* uk, const double* uk1,
                  const double* uk2, double* x_dev, void* stream) {
    if (!g || !c || !uk || !uk1 || !uk2 || !x_dev) { set_error("guess_propose: null argument"); return POLYDG_EINVAL; }
    if (g->np != c->H.n_p) { set_error("guess_propose: model and mesh differ in n_p"); return POLYDG_EINVAL; }
    cudaStream_t s = (cudaStream_t)stream;
    const int np = c->H.n_p;
    PcgWork& w = c->work;
    CU(launch_permute(uk, nullptr, w.r[0], c->d_to_caller, c->H.nc, np, 1, nullptr, s));
    CU(launch_permute(uk1, nullptr, w.r[1], c->d_to_caller, c->H.nc, np, 1, nullptr, s));
    CU(launch_permute(uk2, nullptr, w.b, c->d_to_caller, c->H.nc, np, 1, nullptr, s));
    const int64_t tiles = (c->H.nc + 127) / 128;
    if (tiles > g->xt_tiles) {
        CU(cudaStreamSynchronize(s));     // the previous call's tiles are no longer read
        dfree(g->xt);
        g->xt_tiles = 0;
        if (int st = dalloc(&g->xt, (size_t)tiles * guess_tc_tile_bytes(np))) return st;
        g->xt_tiles = tiles;
    }
    CU(launch_guess_propose(np, guess_features(c, g), g->img, w.r[0], w.r[1], w.b, w.z, c->H.nc,
                            nullptr, g->xt, g->d_err, g->n_sm, s));
    CU(launch_permute(w.z, nullptr, x_dev, c->d_to_caller, c->H.nc, np, 0, nullptr, s));
    int h_err = 0;
    CU(cudaMemcpyAsync(&h_err, g->d_err, sizeof(int), cudaMemcpyDeviceToHost, s));
    CU(cudaStreamSynchronize(s));
    if (h_err) {
        CU(cudaMemset(g->d_err, 0, sizeof(int)));
        set_error("guess_propose: a device-side wait timed out");
        return POLYDG_ECUDA;
    }
    return POLYDG_OK;
}

int guess_train_step(guess_model* g, polydg_ctx* c, const double* traj_dev, int64_t n_states,
                     const int64_t* samples, int64_t n_samples, double lr, double* loss,
                     void* stream) {
    if (!g || !c || !traj_dev || !samples || n_samples < 1 || !(lr >= 0)) {
        set_error("guess_train_step: need a model, a context, a trajectory, samples and lr >= 0");
        return POLYDG_EINVAL;
    }
    if (g->np != c->H.n_p) { set_error("guess_train_step: model and mesh differ in n_p"); return POLYDG_EINVAL; }
    for (int64_t q = 0; q < n_samples; ++q)
        if (samples[2 * q] < 2 || samples[2 * q] > n_states - 2 || samples[2 * q + 1] < 0 ||
            samples[2 * q + 1] >= c->H.nc) {
            set_error("guess_train_step: a sample needs 2 <= k <= n_states - 2 and a valid cell id");
            return POLYDG_EINVAL;
        }
    cudaStream_t s = (cudaStream_t)stream;
    if (n_samples > g->sample_cap) {
        dfree(g->samples);
        if (int st = dalloc(&g->samples, 2 * (size_t)n_samples)) return st;
        g->sample_cap = n_samples;
    }
    CU(cudaMemcpyAsync(g->samples, samples, 2 * n_samples * sizeof(int64_t), cudaMemcpyHostToDevice, s));
    const int64_t tiles = (n_samples + 31) / 32;
    const int grid = (int)std::min<int64_t>(tiles, g->grid_max);
    const int np = c->H.n_p;
    CU(launch_guess_train(np, guess_features(c, g), g->w32, traj_dev, c->H.nc * np, g->samples,
                          n_samples, c->d_to_internal, c->d_to_caller, g->part, g->lpart, grid, s));
    g->t += 1;
    const double b1 = 0.9, b2 = 0.999;
    const float c1 = (float)(1.0 - std::pow(b1, (double)g->t)), c2 = (float)(1.0 - std::pow(b2, (double)g->t));
    CU(launch_guess_adam(g->part, grid, g->P, g->w32, g->m, g->v, g->w16, (float)lr, (float)b1, (float)b2,
                         1e-8f, c1, c2, g->lpart, 1.0 / ((double)n_samples * np), g->loss, s));
    CU(launch_guess_tc_image(np, g->w16, g->img, s));       // the inference kernel's weight image
    double l = 0.0;
    CU(cudaMemcpyAsync(&l, g->loss, sizeof(double), cudaMemcpyDeviceToHost, s));
    CU(cudaStreamSynchronize(s));
    if (loss) *loss = l;
    return POLYDG_OK;
}

int sim_set_guess(sim_ctx* sm, guess_model* g, int policy) {
    if (!sm) { set_error("sim_set_guess: null simulation"); return POLYDG_EINVAL; }
    if (g && g->np != sm->ctx->H.n_p) { set_error("sim_set_guess: model and mesh differ in n_p"); return POLYDG_EINVAL; }
    if (policy < 0 || policy > 3) { set_error("sim_set_guess: policy must be 0, 1, 2 or 3"); return POLYDG_EINVAL; }
    if (!g && policy != 0 && policy != 3) { set_error("sim_set_guess: policies 1 and 2 need a model"); return POLYDG_EINVAL; }
    if (g && !sm->gxt) {
        const int64_t tiles = (sm->ctx->H.nc + 127) / 128;
        if (int st = dalloc(&sm->gxt, (size_t)tiles * guess_tc_tile_bytes(g->np))) return st;
    }
    if (sm->guess != g || sm->guess_policy != policy) {
        sm->guess = g;
        sm->guess_policy = policy;
        sm->version += 1;
    }
    return POLYDG_OK;
}

void guess_destroy(guess_model* g) {
    if (!g) return;
    dfree(g->w32); dfree(g->m); dfree(g->v); dfree(g->w16); dfree(g->d_err); dfree(g->img); dfree(g->xt); dfree(g->part); dfree(g->lpart);
    dfree(g->loss); dfree(g->samples);
    delete g;
}

void batch_destroy(batch_ctx* bt) {
    if (!bt) return;
    if (bt->exec) cudaGraphExecDestroy(bt->exec);
    if (bt->graph) cudaGraphDestroy(bt->graph);
    if (bt->cap) cudaStreamDestroy(bt->cap);
    for (auto e : bt->ev) cudaEventDestroy(e);
    for (auto& P : bt->plans) P.release();
    for (auto& g : bt->groups) g.release();
    dfree(bt->d_args); dfree(bt->d_map); dfree(bt->d_gargs); dfree(bt->d_gmap);
    if (bt->h_ss) cudaFreeHost(bt->h_ss);
    delete bt;
}

void sim_destroy(sim_ctx* sm) {
    if (!sm) return;
    for (auto e : sm->ev) cudaEventDestroy(e);
    sm->work.release();
    dfree(sm->U); dfree(sm->Uprev); dfree(sm->Uprev2); dfree(sm->xg); dfree(sm->I); dfree(sm->F); dfree(sm->y); dfree(sm->yc); dfree(sm->gxt); dfree(sm->d_y0);
    dfree(sm->Ym);
    dfree(sm->ring); dfree(sm->kuring); dfree(sm->subW); dfree(sm->gram);
    dfree(sm->d_ss);
    if (sm->h_ss) cudaFreeHost(sm->h_ss);
    delete sm;
}

void asm_destroy(asm_ctx* pc) {
    if (!pc) return;
    pc->plan.release();
    dfree(pc->d_blocks); dfree(pc->st64); dfree(pc->st32); dfree(pc->st16);
    dfree(pc->d_sym);
    dfree(pc->d_T); dfree(pc->d_agg); dfree(pc->d_pair_ptr); dfree(pc->d_r0p);
    dfree(pc->d_y0); dfree(pc->d_r0g);
    delete pc;
}

void polydg_destroy(polydg_ctx* c) {
    if (!c) return;
    c->id_plan.release();
    c->work.release();
    dfree(c->K.row_ptr); dfree(c->K.col); dfree(c->K.val); dfree(c->K.val_minus);
    dfree(c->d_to_caller); dfree(c->d_node_ptr); dfree(c->d_node_w); dfree(c->d_node_phi); dfree(c->d_Minv);
    dfree(c->d_node_pos); dfree(c->d_to_internal); dfree(c->d_diam); dfree(c->d_id_blocks); dfree(c->d_id_tiles); dfree(c->d_zero_ptr);
    if (c->h_sc) cudaFreeHost(c->h_sc);
    delete c;
}

}  // extern "C"
