// Library-internal context structures of libpolydg and the small device-memory
// helpers the entry points share (included by the translation units of the C ABI).
#pragma once

#include <string>
#include <vector>

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "internal.h"
#include "kernels.h"
#include "polydg.h"

namespace polydg {

#define CU(call)                                                                   \
    do {                                                                           \
        cudaError_t _e = (call);                                                   \
        if (_e != cudaSuccess) {                                                   \
            set_error(std::string(#call) + ": " + cudaGetErrorString(_e));         \
            return _e == cudaErrorMemoryAllocation ? POLYDG_ENOMEM : POLYDG_ECUDA;  \
        }                                                                          \
    } while (0)

template <typename T>
inline int dalloc(T** p, size_t count) {
    *p = nullptr;
    if (count == 0) count = 1;
    CU(cudaMalloc((void**)p, count * sizeof(T)));
    return POLYDG_OK;
}

template <typename T>
inline int upload(T** p, const std::vector<T>& v) {
    int st = dalloc(p, v.size());
    if (st) return st;
    if (!v.empty()) CU(cudaMemcpy(*p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
    return POLYDG_OK;
}

template <typename T>
inline void dfree(T*& p) {
    if (p) cudaFree((void*)p);
    p = nullptr;
}

// Vectors and scalars of one PCG solve (internal cell order).  The iterate
// and residual are double-buffered: after a solve they live in buffer
// (sc->pass & 1).
struct PcgWork {
    double *x[2] = {nullptr, nullptr}, *r[2] = {nullptr, nullptr};
    double *b = nullptr, *z = nullptr, *p = nullptr, *p2 = nullptr, *q = nullptr, *q2 = nullptr;
    double *zl = nullptr, *w = nullptr;
    PcgScalars* sc = nullptr;
    double* partials = nullptr;
    int* err = nullptr;                 // device-wait timeout flag of the kernels
    GridSync* gs = nullptr;             // grid-barrier state of the persistent kernel
    double* bcast = nullptr;            // grid sums broadcast by the barrier
    int alloc(int64_t n) {
        int st;
        if ((st = dalloc(&x[0], n)) || (st = dalloc(&x[1], n)) || (st = dalloc(&r[0], n)) ||
            (st = dalloc(&r[1], n)) || (st = dalloc(&b, n)) || (st = dalloc(&z, n)) ||
            (st = dalloc(&p, n)) || (st = dalloc(&p2, n)) || (st = dalloc(&q, n)) || (st = dalloc(&q2, n)) ||
            (st = dalloc(&zl, n)) || (st = dalloc(&w, n)) || (st = dalloc(&sc, 1)) ||
            (st = dalloc(&partials, 8 * (size_t)kMaxPartials)) || (st = dalloc(&err, 1)) ||
            (st = dalloc(&gs, 1)) || (st = dalloc(&bcast, 8)))
            return st;
        CU(cudaMemset(sc, 0, sizeof(PcgScalars)));
        CU(cudaMemset(err, 0, sizeof(int)));
        CU(cudaMemset(gs, 0, sizeof(GridSync)));
        return POLYDG_OK;
    }
    void release() {
        dfree(x[0]); dfree(x[1]); dfree(r[0]); dfree(r[1]); dfree(b); dfree(z); dfree(p); dfree(p2); dfree(q2); dfree(zl); dfree(w);
        dfree(q); dfree(sc); dfree(partials); dfree(err); dfree(gs); dfree(bcast);
    }
};

// Static work split of the persistent PCG kernel over its CTAs.
struct Plan {
    int grid = 0, rows = 1, dtype = 0;
    int redundant = 1;
    int wstages = 1;
    int small = 0;                      // every subdomain <= 32 DOFs: one warp per subdomain
    int pair_lanes = 1;                 // lanes summing one coarse DOF's pair partials
    int r0_split = 0;                   // pair partials summed by slices, one more barrier
    float l2_keep = 0.f;                // fraction of the local-inverse lines kept in L2
    size_t smem = 0, slot_bytes = 0, xs_off = 0, rp_off = 0, r0_off = 0, y0_off = 0,
           pn_off = 0, td_off = 0;
    int32_t *run_ptr = nullptr, *sub_pairs = nullptr, *crow_ptr = nullptr, *cta_chunk = nullptr;
    int64_t* chunk_elem = nullptr;
    int32_t *need_ptr = nullptr, *need = nullptr, *col_local = nullptr;
    int32_t *need_aggl = nullptr, *need_agg_ptr = nullptr, *need_agg = nullptr;
    GemvRun* runs = nullptr;
    int64_t* elem_ptr = nullptr;
    double est_seconds = 0.0;           // cost model: slowest CTA's P phase per iteration
    int max_need = 0, max_aggs = 0;     // staged elements per chunk, agglomerates per CTA
    int cm_stages = 0;                  // K_h panel slots per warp in the CM phase (0: loads)
    size_t cm_slot_bytes = 0;
    int sym = 0;                        // P phase from the symmetric pair-row store
    int sym_bufld = 0;                  // floats per warp of its column-sum buffer
    std::vector<GemvTile> h_tiles;      // the tile sequence and its modelled costs (autotuning)
    std::vector<double> h_cost, h_stage;
    std::vector<int32_t> h_tile_ptr;
    void release() {
        dfree(run_ptr); dfree(sub_pairs); dfree(crow_ptr); dfree(need_ptr); dfree(need);
        dfree(cta_chunk); dfree(chunk_elem);
        dfree(need_aggl); dfree(need_agg_ptr); dfree(need_agg);
        dfree(col_local); dfree(runs); dfree(elem_ptr);
    }
};

}  // namespace polydg

using namespace polydg;

struct polydg_ctx {
    HostSetup H;
    int device = 0;
    DeviceMatrix K;
    int64_t* d_to_caller = nullptr;
    int64_t* d_node_ptr = nullptr;
    int ionic_lpc = 32;             // lanes per cell of the ionic kernel (ionic_lanes_per_cell)
    double* d_node_w = nullptr;
    double* d_node_phi = nullptr;
    double* d_Minv = nullptr;           // [nc][n_p][n_p] inverse mass blocks (modal ionic state)
    int64_t* d_node_pos = nullptr;
    int64_t* d_to_internal = nullptr;   // caller -> internal cell id
    double* d_diam = nullptr;           // cell diameters, internal order
    // identity tiles (z = r) for unpreconditioned CG
    GemvBlock* d_id_blocks = nullptr;
    GemvTile* d_id_tiles = nullptr;
    int n_id_tiles = 0;
    int64_t* d_zero_ptr = nullptr;      // pair_ptr of an empty coarse space
    Plan id_plan;                       // persistent-kernel plan without preconditioner
    int n_sm = 0;
    PcgWork work;                       // pcg_solve / polydg_matvec buffers
    PcgScalars* h_sc = nullptr;         // pinned
};

struct asm_ctx {
    polydg_ctx* ctx = nullptr;
    int precision = POLYDG_FP64;
    int has_coarse = 0, q = 0, nq = 0, n_agg = 0, n_pairs = 0;
    int64_t n0 = 0, ld0 = 0, off0 = 0;
    int n_blocks = 0;
    Plan plan;                          // persistent-kernel plan with this preconditioner
    std::vector<int32_t> sub_pairs;     // RESTRICT block ids grouped by subdomain
    GemvBlock* d_blocks = nullptr;
    std::vector<GemvBlock> blocks;
    double* st64 = nullptr;
    float* st32 = nullptr;
    __nv_bfloat16* st16 = nullptr;
    double* d_T = nullptr;
    int32_t* d_agg = nullptr;
    int64_t* d_pair_ptr = nullptr;
    int max_pairs = 0;                  // most (agglomerate, subdomain) pairs of one agglomerate
    double* d_r0g = nullptr;            // R_0 r' summed by slices of the CTAs (split mode)
    double* d_r0p = nullptr;
    double* d_y0 = nullptr;
    int64_t store_bytes = 0;            // bytes of the dense stores read per apply
    float* d_sym = nullptr;             // fp32 stores: lower triangles as pair rows (sym_ld)
    int64_t sym_bytes = 0;              // bytes one apply copies from d_sym
    int sym_max_n = 0;                  // largest subdomain of d_sym
};

// Learned initial-guess network (fp32 master weights and Adam state, fp16 copy for
// inference) and its training buffers.
struct guess_model {
    int np = 0, P = 0, device = 0;
    double scales[5] = {-67.0, 50.0, 1.0, 1.0, 0.05};   // u_rest, s_u, s_d, h_ref, dt_ref
    float *w32 = nullptr, *m = nullptr, *v = nullptr, *part = nullptr;
    __half* w16 = nullptr;
    int* d_err = nullptr;               // raised by the inference kernel if a device wait ran out
    int n_sm = 1;
    unsigned char* img = nullptr;       // the weights as tensor-core operands (guess_tc.cu)
    unsigned char* xt = nullptr;        // feature tiles of guess_propose calls
    int64_t xt_tiles = 0;
    double *lpart = nullptr, *loss = nullptr;
    int64_t* samples = nullptr;
    int64_t sample_cap = 0;
    int grid_max = 0;
    int64_t t = 0;                      // Adam steps taken
};

struct sim_ctx {
    polydg_ctx* ctx = nullptr;
    asm_ctx* pc = nullptr;
    sim_params prm{};
    PcgWork work;
    guess_model* guess = nullptr;       // learned initial guess (nullptr: x0 = U^k)
    int guess_policy = 0;               // 0 keep the smaller residual, 1 always, 2 damped, 3 subspace
    shared_local* shared = nullptr;     // local solves shared with other simulations (batches)
    double sigma = 0.0;                 // its scalar conductivity when `shared` is set
    int64_t version = 0;                // bumped when the step's kernel sequence changes
    double *Uprev2 = nullptr, *xg = nullptr;
    double* ring = nullptr;             // [kHistRing][n] past solutions, slot k mod kHistRing = U^k
    double* kuring = nullptr;           // [kHistRing][n] products K (U^j - U^{j-1}), same slots as ring
    double* subW = nullptr;             // [2][n] r0 = b - K U^k and K (xg - U^k) of the subspace guess
    double* gram = nullptr;             // [kSubMaxPairs][kSubMaxCtas] Gram partial sums
    double *U = nullptr, *Uprev = nullptr, *I = nullptr, *F = nullptr, *y = nullptr;
    double* yc = nullptr;               // per node: E_Na, E_K, exp(-K_o/5), exp((25 - Na_i)/3),
                                        // u^{k-1}, exp(-u^{k-1}/720) (nodal form)
    unsigned char* gxt = nullptr;       // feature tiles of the learned guess (with a model)
    double* d_y0 = nullptr;
    double* Ym = nullptr;               // [5][n] modal ionic state (sim_set_ionic_form 1), or null
    SimScalars* d_ss = nullptr;
    SimScalars* h_ss = nullptr;         // pinned
    int64_t k = 0;
    std::vector<cudaEvent_t> ev;        // [2 * steps] around each step's PCG kernel
};

// Independent simulations advanced together: one cooperative launch per step in
// which simulation i owns CTAs [cta_begin[i], cta_begin[i] + group[i]).
// Local solves shared by simulations whose conductivity is a scalar multiple of I
// (shared_local.cu): per subdomain Q_i^T and Q_i (fp32 or bf16), lam_i, per element L_K^{-1}.
struct shared_local {
    polydg_ctx* ctx = nullptr;
    int precision = POLYDG_FP32;
    double sigma_ref = 1.0;
    int n_sub = 0;
    int64_t max_ld = 0, store_bytes = 0;
    std::vector<SharedBlock> hblocks;
    SharedBlock* blocks = nullptr;
    float* st32 = nullptr;
    __nv_bfloat16* st16 = nullptr;
    float* lam = nullptr;
    double* linv = nullptr;
    double* tmp[2 * kMaxTcRhs] = {};    // internal-order r and z of shared_local_apply
    // tensor-core tiles (BF16 store only): Q_i^T then Q_i of every subdomain, 16 KB tiles
    std::vector<TcBlock> htc;
    TcBlock* tc = nullptr;
    unsigned char* tiles = nullptr;
    int64_t tile_bytes = 0;
    int max_kpad = 0;
    int* d_err = nullptr;
};

// A lockstep group of a batch: simulations that share one shared_local.
struct BatchGroup {
    std::vector<int> members;           // indices into batch_ctx::sims
    Plan plan;                          // structure of the first member, for `ctas` CTAs
    int ctas = 0;
    int32_t *d_piece_ptr = nullptr, *d_pair_begin = nullptr, *d_pair_count = nullptr;
    GemvRun* d_pieces = nullptr;
    std::vector<float*> yq;             // per member: pass-1 output (one float per DOF)
    void release() {
        plan.release(); dfree(d_piece_ptr); dfree(d_pair_begin); dfree(d_pair_count); dfree(d_pieces);
        for (auto& y : yq) dfree(y);
    }
};

struct batch_ctx {
    std::vector<sim_ctx*> sims;
    // simulations with their own local inverses: one launch, a CTA group each
    std::vector<int> solo;              // indices into sims
    std::vector<Plan> plans;            // per solo simulation, for its CTA group
    std::vector<int> group;             // CTAs per simulation (group members: the group's)
    PersistArgs* d_args = nullptr;      // [solo]
    int2* d_map = nullptr;              // [n_cta] (solo index, CTA within its group)
    int n_cta = 0, dtype = 0, np = 0, device = 0;
    size_t smem = 0;
    // lockstep groups of simulations sharing local solves: a second launch
    std::vector<BatchGroup> groups;
    std::vector<shared_local*> shared_at_create;   // each simulation's shared local solves
    GroupArgs* d_gargs = nullptr;
    int2* d_gmap = nullptr;
    int g_cta = 0, gq = 0;
    size_t gsmem = 0;
    cudaStream_t cap = nullptr;         // stream the step is captured on
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    std::vector<int64_t> versions;      // the simulations' versions when the step was captured
    std::vector<cudaEvent_t> ev;        // [2 * steps] around each step's graph launch
    SimScalars* h_ss = nullptr;         // pinned [n]
};

