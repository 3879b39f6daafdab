// C ABI of libpolydg (include/polydg.h): contexts, device buffers, CUDA-graph
// capture of the PCG loop and of the monodomain step.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <utility>
#include <vector>

#include <cuda_runtime.h>
#include <cuda_bf16.h>

#include "internal.h"
#include "ionic_model.cuh"
#include "kernels.h"
#include "polydg.h"

namespace polydg {

static thread_local std::string g_error;
void set_error(const std::string& msg) { g_error = msg; }

#define CU(call)                                                                   \
    do {                                                                           \
        cudaError_t _e = (call);                                                   \
        if (_e != cudaSuccess) {                                                   \
            set_error(std::string(#call) + ": " + cudaGetErrorString(_e));         \
            return _e == cudaErrorMemoryAllocation ? POLYDG_ENOMEM : POLYDG_ECUDA;  \
        }                                                                          \
    } while (0)

template <typename T>
static int dalloc(T** p, size_t count) {
    *p = nullptr;
    if (count == 0) count = 1;
    CU(cudaMalloc((void**)p, count * sizeof(T)));
    return POLYDG_OK;
}

template <typename T>
static int upload(T** p, const std::vector<T>& v) {
    int st = dalloc(p, v.size());
    if (st) return st;
    if (!v.empty()) CU(cudaMemcpy(*p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
    return POLYDG_OK;
}

template <typename T>
static void dfree(T*& p) {
    if (p) cudaFree((void*)p);
    p = nullptr;
}

// Vectors and scalars of one PCG solve (internal cell order).
struct PcgWork {
    double *x = nullptr, *b = nullptr, *r = nullptr, *z = nullptr, *p = nullptr, *q = nullptr;
    PcgScalars* sc = nullptr;
    double* partials = nullptr;
    int alloc(int64_t n) {
        int st;
        if ((st = dalloc(&x, n)) || (st = dalloc(&b, n)) || (st = dalloc(&r, n)) ||
            (st = dalloc(&z, n)) || (st = dalloc(&p, n)) || (st = dalloc(&q, n)) ||
            (st = dalloc(&sc, 1)) || (st = dalloc(&partials, 2 * (size_t)kMaxPartials)))
            return st;
        CU(cudaMemset(sc, 0, sizeof(PcgScalars)));
        return POLYDG_OK;
    }
    void release() {
        dfree(x); dfree(b); dfree(r); dfree(z); dfree(p); dfree(q); dfree(sc); dfree(partials);
    }
};

struct Graph {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    void release() {
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        exec = nullptr;
        graph = nullptr;
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
    double* d_node_w = nullptr;
    double* d_node_phi = nullptr;
    int64_t* d_node_pos = nullptr;
    PcgWork work;                       // pcg_solve / polydg_matvec buffers
    PcgScalars* h_sc = nullptr;         // pinned
    cudaStream_t cap = nullptr, cap2 = nullptr;
    std::map<std::pair<const asm_ctx*, int>, Graph> graphs;
};

struct asm_ctx {
    polydg_ctx* ctx = nullptr;
    int precision = POLYDG_FP64;
    int has_coarse = 0, q = 0, nq = 0, n_agg = 0;
    int n_blocks = 0, ntiles = 0, rows = 32, max_ld = 0;
    GemvBlock* d_blocks = nullptr;
    GemvTile* d_tiles = nullptr;
    std::vector<GemvBlock> blocks;
    double* st64 = nullptr;
    float* st32 = nullptr;
    __nv_bfloat16* st16 = nullptr;
    double* d_T = nullptr;
    int32_t* d_agg = nullptr;
    int64_t* d_agg_ptr = nullptr;
    int32_t* d_agg_cells = nullptr;
    double* d_r0 = nullptr;
    double* d_y0 = nullptr;
    double* d_rin = nullptr;
    double* d_zout = nullptr;
    int64_t store_bytes = 0;            // bytes of the local-inverse store read per apply
};

struct sim_ctx {
    polydg_ctx* ctx = nullptr;
    asm_ctx* pc = nullptr;
    sim_params prm{};
    PcgWork work;
    double *U = nullptr, *Uprev = nullptr, *I = nullptr, *F = nullptr, *y = nullptr;
    double* d_y0 = nullptr;
    SimScalars* d_ss = nullptr;
    SimScalars* h_ss = nullptr;         // pinned
    Graph step;
    int64_t k = 0;
};

namespace polydg {

// ---------------------------------------------------------- graph capture
// Body of one PCG iteration (Saad Alg. 9.1 with the loop test at the end):
//   z = B r  (restrict, ragged GEMV, prolong + r.z, z.q, beta)
//   p = z + beta p;  q = K p, alpha;  x += alpha p, r -= alpha q, test.
static int capture_pcg_body(polydg_ctx* c, asm_ctx* pc, PcgWork& w, cudaStream_t s,
                            cudaGraphConditionalHandle cond) {
    const int np = c->H.n_p;
    const int64_t n = c->H.nc * np;
    const double* zsrc = w.r;
    if (pc) {
        if (pc->has_coarse)
            CU(launch_restrict(np, pc->nq, w.r, pc->d_T, pc->d_agg_ptr, pc->d_agg_cells,
                               pc->n_agg, pc->d_r0, &w.sc->done, s));
        CU(launch_gemv(pc->d_blocks, pc->d_tiles, pc->ntiles, pc->rows, pc->max_ld, pc->st64,
                       pc->st32, pc->st16, w.r, pc->d_r0, w.z, pc->d_y0, &w.sc->done, s));
        CU(launch_prolong(np, pc->has_coarse ? pc->nq : 3, w.z, pc->has_coarse ? pc->d_T : nullptr,
                          pc->d_agg, pc->d_y0, c->H.nc, w.r, w.q, w.sc, w.partials, s));
        zsrc = w.z;
    } else {
        CU(launch_identity_dots(w.r, w.q, n, w.sc, w.partials, s));
    }
    CU(launch_direction(w.p, zsrc, n, w.sc, s));
    CU(launch_matvec(MODE_PCG, np, c->K, c->K.val, w.p, w.q, nullptr, nullptr, 0, 0, w.sc,
                     w.partials, nullptr, 0, 0, s));
    CU(launch_update(w.x, w.r, w.p, w.q, n, w.sc, w.partials, cond, 1, s));
    return POLYDG_OK;
}

// Appends [r = b - K x; while (!done) body] to the capture running on c->cap.
static int capture_pcg_loop(polydg_ctx* c, asm_ctx* pc, PcgWork& w) {
    const int np = c->H.n_p;
    CU(launch_matvec(MODE_RESID, np, c->K, c->K.val, w.x, w.r, w.b, nullptr, 0, 0, w.sc,
                     w.partials, nullptr, 0, 0, c->cap));
    cudaStreamCaptureStatus cs;
    cudaGraph_t g;
    const cudaGraphNode_t* deps = nullptr;
    size_t ndeps = 0;
    CU(cudaStreamGetCaptureInfo(c->cap, &cs, nullptr, &g, &deps, nullptr, &ndeps));
    cudaGraphConditionalHandle cond;
    CU(cudaGraphConditionalHandleCreate(&cond, g, 1, cudaGraphCondAssignDefault));
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = cond;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t node;
    CU(cudaGraphAddNode(&node, g, deps, nullptr, ndeps, &cp));
    CU(cudaStreamUpdateCaptureDependencies(c->cap, &node, nullptr, 1,
                                           cudaStreamSetCaptureDependencies));
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    CU(cudaStreamBeginCaptureToGraph(c->cap2, body, nullptr, nullptr, 0,
                                     cudaStreamCaptureModeThreadLocal));
    int st = capture_pcg_body(c, pc, w, c->cap2, cond);
    cudaGraph_t body_out = nullptr;
    cudaError_t e = cudaStreamEndCapture(c->cap2, &body_out);
    if (st) return st;
    CU(e);
    return POLYDG_OK;
}

static int end_capture(polydg_ctx* c, Graph& G) {
    CU(cudaStreamEndCapture(c->cap, &G.graph));
    CU(cudaGraphInstantiate(&G.exec, G.graph, 0));
    return POLYDG_OK;
}

static void abort_capture(polydg_ctx* c) {
    cudaGraph_t g = nullptr;
    cudaStreamEndCapture(c->cap, &g);
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
}

static int pcg_graph(polydg_ctx* c, asm_ctx* pc, int flexible, Graph** out) {
    auto key = std::make_pair((const asm_ctx*)pc, flexible);
    auto it = c->graphs.find(key);
    if (it != c->graphs.end()) { *out = &it->second; return POLYDG_OK; }
    CU(cudaStreamBeginCapture(c->cap, cudaStreamCaptureModeThreadLocal));
    int st = capture_pcg_loop(c, pc, c->work);
    if (st) { abort_capture(c); return st; }
    Graph G;
    st = end_capture(c, G);
    if (st) { G.release(); return st; }
    auto res = c->graphs.emplace(key, G);
    *out = &res.first->second;
    return POLYDG_OK;
}

static int check_ctx(const polydg_ctx* c, const char* fn) {
    if (!c) { set_error(std::string(fn) + ": null context"); return POLYDG_EINVAL; }
    return POLYDG_OK;
}

static inline int64_t round_up(int64_t x, int64_t m) { return (x + m - 1) / m * m; }

}  // namespace polydg

// ================================================================== C ABI
extern "C" {

const char* polydg_last_error(void) { return g_error.c_str(); }

int polydg_setup(const polydg_mesh* mesh, int p, const int32_t* subdomain_of_cell,
                 double chi_cm, double dt, double eta0, polydg_ctx** out) {
    if (!out) { set_error("polydg_setup: null output"); return POLYDG_EINVAL; }
    *out = nullptr;
    polydg_ctx* c = new polydg_ctx();
    int st = host_setup(mesh, p, subdomain_of_cell, chi_cm, dt, eta0, c->H);
    if (st) { delete c; return st; }
    auto fail = [&](int code) { polydg_destroy(c); return code; };
    if (cudaGetDevice(&c->device) != cudaSuccess) { set_error("polydg_setup: no CUDA device"); return fail(POLYDG_ECUDA); }
    const HostSetup& H = c->H;
    c->K.nc = H.nc;
    c->K.nblk = (int64_t)H.col.size();
    if ((st = upload(&c->K.row_ptr, H.row_ptr)) || (st = upload(&c->K.col, H.col)) ||
        (st = upload(&c->K.val, H.Kval)) || (st = upload(&c->K.val_minus, H.Kminus_val)) ||
        (st = upload(&c->d_to_caller, H.to_caller)) || (st = upload(&c->d_node_ptr, H.node_ptr)) ||
        (st = upload(&c->d_node_w, H.node_w)) || (st = upload(&c->d_node_phi, H.node_phi)) ||
        (st = upload(&c->d_node_pos, H.node_to_caller_pos)))
        return fail(st);
    if ((st = c->work.alloc(H.nc * H.n_p))) return fail(st);
    if (cudaMallocHost((void**)&c->h_sc, sizeof(PcgScalars)) != cudaSuccess) {
        set_error("polydg_setup: pinned allocation failed");
        return fail(POLYDG_ENOMEM);
    }
    if (cudaStreamCreateWithFlags(&c->cap, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&c->cap2, cudaStreamNonBlocking) != cudaSuccess) {
        set_error("polydg_setup: stream creation failed");
        return fail(POLYDG_ECUDA);
    }
    *out = c;
    return POLYDG_OK;
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
    CU(launch_permute(x_dev, c->work.p, c->d_to_caller, c->H.nc, np, 1, nullptr, s));
    CU(launch_matvec(MODE_PLAIN, np, c->K, c->K.val, c->work.p, c->work.q, nullptr, nullptr, 0, 0,
                     nullptr, nullptr, nullptr, 0, 0, s));
    CU(launch_permute(c->work.q, y_dev, c->d_to_caller, c->H.nc, np, 0, nullptr, s));
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
        if (C.n_q != 3 && C.n_q != 6 && C.n_q != 10) { set_error("asm_setup: coarse degree q must be 1..3"); return POLYDG_EINVAL; }
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
        woff += wld * wld;
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
    if ((st = cu(cudaMemset(pc->st64, 0, off * sizeof(double)), "memset")) ||
        (st = cu(cudaMemset(work, 0, woff * sizeof(double)), "memset")) ||
        (st = cu(launch_extract_local(c->K, d_subptr, H.n_sub, d_off, d_ld, pc->st64, np, 0), "extract")) ||
        (pc->has_coarse &&
         (st = cu(cudaMemcpy2D(pc->st64 + mats.back().off, mats.back().ld * sizeof(double), C.K0.data(),
                               n0 * sizeof(double), n0 * sizeof(double), n0, cudaMemcpyHostToDevice),
                  "coarse upload"))) ||
        (st = cu(launch_chol_inverse(pc->st64, d_off, d_n, d_ld, work, d_woff, d_wld, d_status, nmat,
                                     (int)max_n, 0), "cholesky")) ||
        (st = cu(cudaDeviceSynchronize(), "cholesky sync"))) {
        cleanup();
        return fail(st);
    }
    {
        std::vector<int> hs(nmat);
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
    // block and tile tables
    std::vector<GemvTile> tiles;
    for (int m = 0; m < nmat; ++m) {
        GemvBlock B;
        B.mat_off = mats[m].off;
        B.n = (int32_t)mats[m].n;
        B.ld = (int32_t)mats[m].ld;
        const bool coarse = (m == H.n_sub);
        B.sel = coarse ? 1 : 0;
        B.dtype = coarse ? 0 : precision;
        B.in_off = coarse ? 0 : H.sub_ptr[m] * np;
        B.out_off = B.in_off;
        pc->blocks.push_back(B);
        pc->max_ld = std::max(pc->max_ld, B.ld);
        for (int r0 = 0; r0 < B.n; r0 += pc->rows) tiles.push_back({m, r0});
        pc->store_bytes += (int64_t)B.n * B.ld * (coarse ? 8 : esz);
    }
    pc->n_blocks = nmat;
    pc->ntiles = (int)tiles.size();
    if ((st = upload(&pc->d_blocks, pc->blocks)) || (st = upload(&pc->d_tiles, tiles)))
        return fail(st);
    if ((st = cu(set_gemv_smem(pc->max_ld), "gemv smem"))) return fail(st);
    if (pc->has_coarse) {
        pc->q = C.q; pc->nq = C.n_q; pc->n_agg = C.n_agg;
        if ((st = upload(&pc->d_T, C.T)) || (st = upload(&pc->d_agg, C.agg_of_cell)) ||
            (st = upload(&pc->d_agg_ptr, C.agg_ptr)) || (st = upload(&pc->d_agg_cells, C.agg_cells)))
            return fail(st);
    }
    if ((st = dalloc(&pc->d_r0, std::max<int64_t>(n0, 1))) || (st = dalloc(&pc->d_y0, std::max<int64_t>(n0, 1))) ||
        (st = dalloc(&pc->d_rin, H.nc * np)) || (st = dalloc(&pc->d_zout, H.nc * np)))
        return fail(st);
    *out = pc;
    return POLYDG_OK;
}

int asm_apply(asm_ctx* pc, const double* r_dev, double* z_dev, void* stream) {
    if (!pc) { set_error("asm_apply: null preconditioner"); return POLYDG_EINVAL; }
    if (!r_dev || !z_dev || r_dev == z_dev) { set_error("asm_apply: null or aliased vectors"); return POLYDG_EINVAL; }
    polydg_ctx* c = pc->ctx;
    cudaStream_t s = (cudaStream_t)stream;
    const int np = c->H.n_p;
    CU(launch_permute(r_dev, pc->d_rin, c->d_to_caller, c->H.nc, np, 1, nullptr, s));
    if (pc->has_coarse)
        CU(launch_restrict(np, pc->nq, pc->d_rin, pc->d_T, pc->d_agg_ptr, pc->d_agg_cells, pc->n_agg,
                           pc->d_r0, nullptr, s));
    CU(launch_gemv(pc->d_blocks, pc->d_tiles, pc->ntiles, pc->rows, pc->max_ld, pc->st64, pc->st32,
                   pc->st16, pc->d_rin, pc->d_r0, pc->d_zout, pc->d_y0, nullptr, s));
    if (pc->has_coarse)
        CU(launch_prolong(np, pc->nq, pc->d_zout, pc->d_T, pc->d_agg, pc->d_y0, c->H.nc, nullptr,
                          nullptr, nullptr, nullptr, s));
    CU(launch_permute(pc->d_zout, z_dev, c->d_to_caller, c->H.nc, np, 0, nullptr, s));
    return POLYDG_OK;
}

int pcg_solve(polydg_ctx* c, asm_ctx* pc, const double* b_dev, double* x_dev, double rtol,
              int maxit, int flexible, void* stream, pcg_stats* stats) {
    if (int st = check_ctx(c, "pcg_solve")) return st;
    if (!b_dev || !x_dev || b_dev == x_dev) { set_error("pcg_solve: null or aliased vectors"); return POLYDG_EINVAL; }
    if (!(rtol > 0) || maxit < 1) { set_error("pcg_solve: rtol must be > 0 and maxit >= 1"); return POLYDG_EINVAL; }
    if (pc && pc->ctx != c) { set_error("pcg_solve: preconditioner built on another context"); return POLYDG_EINVAL; }
    cudaStream_t s = (cudaStream_t)stream;
    Graph* G = nullptr;
    if (int st = pcg_graph(c, pc, flexible ? 1 : 0, &G)) return st;
    const int np = c->H.n_p;
    PcgScalars init = {};
    init.rtol2 = rtol * rtol;
    init.maxit = maxit;
    init.flexible = flexible ? 1 : 0;
    *c->h_sc = init;
    CU(cudaMemcpyAsync(c->work.sc, c->h_sc, sizeof(PcgScalars), cudaMemcpyHostToDevice, s));
    CU(launch_permute(b_dev, c->work.b, c->d_to_caller, c->H.nc, np, 1, nullptr, s));
    CU(launch_permute(x_dev, c->work.x, c->d_to_caller, c->H.nc, np, 1, nullptr, s));
    CU(cudaGraphLaunch(G->exec, s));
    CU(launch_permute(c->work.x, x_dev, c->d_to_caller, c->H.nc, np, 0, c->work.sc, s));
    CU(cudaMemcpyAsync(c->h_sc, c->work.sc, sizeof(PcgScalars), cudaMemcpyDeviceToHost, s));
    CU(cudaStreamSynchronize(s));
    const PcgScalars& r = *c->h_sc;
    if (stats) {
        stats->iterations = r.it;
        stats->status = r.status;
        stats->relres = r.relres;
        stats->bnorm = std::sqrt(r.bb);
    }
    if (r.status != 0) {
        set_error(r.status == POLYDG_ENOTCONV ? "pcg_solve: maximum number of iterations reached"
                  : r.status == POLYDG_EBREAKDOWN ? "pcg_solve: breakdown (p^T K p <= 0 or non-finite beta)"
                                                  : "pcg_solve: non-finite value in b or the residual");
    }
    return r.status;
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
        (st = dalloc(&sm->I, n)) || (st = dalloc(&sm->y, 5 * nn)) || (st = dalloc(&sm->d_y0, 5)) ||
        (st = dalloc(&sm->d_ss, 1)))
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
            const double dx = H.node_xy[2 * qn] - prm->stim_x0, dy = H.node_xy[2 * qn + 1] - prm->stim_y0;
            const double g = H.node_w[qn] * prm->stim_amplitude * std::exp(-(dx * dx + dy * dy) / s2);
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
    PcgScalars sc = {};
    sc.rtol2 = prm->rtol * prm->rtol;
    sc.maxit = prm->maxit;
    sc.flexible = prm->flexible ? 1 : 0;
    if ((st = cu(cudaMemcpy(sm->U, U0.data(), n * sizeof(double), cudaMemcpyHostToDevice))) ||
        (st = cu(cudaMemcpy(sm->Uprev, U0.data(), n * sizeof(double), cudaMemcpyHostToDevice))) ||
        (st = cu(cudaMemcpy(sm->d_y0, y0, 5 * sizeof(double), cudaMemcpyHostToDevice))) ||
        (st = cu(launch_init_y(sm->y, nn, sm->d_y0, 0))) ||
        (st = cu(cudaMemcpy(sm->d_ss, &ss, sizeof(ss), cudaMemcpyHostToDevice))) ||
        (st = cu(cudaMemcpy(sm->work.sc, &sc, sizeof(sc), cudaMemcpyHostToDevice))) ||
        (st = cu(cudaDeviceSynchronize())))
        return fail(st);
    // capture one step: ionic update, right-hand side, x0 = U^k, PCG loop, rotation
    if (cudaStreamBeginCapture(c->cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        set_error("sim_create: stream capture failed");
        return fail(POLYDG_ECUDA);
    }
    PcgWork& w = sm->work;
    const double dt = H.dt;
    if ((st = cu(launch_step_begin(w.sc, sm->d_ss, c->cap))) ||
        (st = cu(launch_ionic(np, sm->U, sm->Uprev, c->d_node_ptr, c->d_node_w, c->d_node_phi, sm->y,
                              nn, H.nc, dt, sm->I, sm->d_ss, c->cap))) ||
        (st = cu(launch_matvec(MODE_RHS, np, c->K, c->K.val_minus, sm->U, w.b, sm->I, sm->F,
                               -H.chi_cm * dt, dt, nullptr, nullptr, sm->d_ss, dt,
                               prm->stim_duration, c->cap))) ||
        (st = cu(launch_copy(sm->U, w.x, n, sm->d_ss, c->cap))) ||
        (st = capture_pcg_loop(c, pc, w)) ||
        (st = cu(launch_step_finish(sm->U, sm->Uprev, w.x, n, w.sc, sm->d_ss, c->cap)))) {
        abort_capture(c);
        return fail(st);
    }
    if ((st = end_capture(c, sm->step))) return fail(st);
    *out = sm;
    return POLYDG_OK;
}

int monodomain_step(sim_ctx* sm, int nsteps, void* stream, step_stats* stats) {
    if (!sm) { set_error("monodomain_step: null simulation"); return POLYDG_EINVAL; }
    if (nsteps < 0) { set_error("monodomain_step: nsteps < 0"); return POLYDG_EINVAL; }
    cudaStream_t s = (cudaStream_t)stream;
    SimScalars& h = *sm->h_ss;
    CU(cudaMemcpyAsync(&h, sm->d_ss, sizeof(SimScalars), cudaMemcpyDeviceToHost, s));
    CU(cudaStreamSynchronize(s));
    h.steps_done = 0;
    h.total_its = 0;
    h.max_its = 0;
    h.last_relres = 0.0;
    CU(cudaMemcpyAsync(sm->d_ss, &h, sizeof(SimScalars), cudaMemcpyHostToDevice, s));
    for (int i = 0; i < nsteps; ++i) CU(cudaGraphLaunch(sm->step.exec, s));
    CU(cudaMemcpyAsync(&h, sm->d_ss, sizeof(SimScalars), cudaMemcpyDeviceToHost, s));
    CU(cudaStreamSynchronize(s));
    sm->k = h.k;
    if (stats) {
        stats->steps_done = h.steps_done;
        stats->total_iterations = h.total_its;
        stats->max_iterations = h.max_its;
        stats->status = h.status;
        stats->last_relres = h.last_relres;
    }
    if (h.status != 0) set_error("monodomain_step: a step's PCG solve failed");
    return h.status;
}

int sim_get_state(sim_ctx* sm, double* u_dev, double* y_dev, void* stream) {
    if (!sm || !u_dev) { set_error("sim_get_state: null argument"); return POLYDG_EINVAL; }
    polydg_ctx* c = sm->ctx;
    cudaStream_t s = (cudaStream_t)stream;
    CU(launch_permute(sm->U, u_dev, c->d_to_caller, c->H.nc, c->H.n_p, 0, nullptr, s));
    if (y_dev) CU(launch_node_gather(sm->y, y_dev, c->d_node_pos, (int64_t)c->H.node_w.size(), s));
    return POLYDG_OK;
}

int sim_set_potential(sim_ctx* sm, const double* u_dev, const double* uprev_dev, void* stream) {
    if (!sm || !u_dev) { set_error("sim_set_potential: null argument"); return POLYDG_EINVAL; }
    polydg_ctx* c = sm->ctx;
    cudaStream_t s = (cudaStream_t)stream;
    CU(launch_permute(u_dev, sm->U, c->d_to_caller, c->H.nc, c->H.n_p, 1, nullptr, s));
    CU(launch_permute(uprev_dev ? uprev_dev : u_dev, sm->Uprev, c->d_to_caller, c->H.nc, c->H.n_p, 1,
                      nullptr, s));
    return POLYDG_OK;
}

int64_t sim_step_index(const sim_ctx* sm) { return sm ? sm->k : -1; }

void sim_destroy(sim_ctx* sm) {
    if (!sm) return;
    sm->step.release();
    sm->work.release();
    dfree(sm->U); dfree(sm->Uprev); dfree(sm->I); dfree(sm->F); dfree(sm->y); dfree(sm->d_y0);
    dfree(sm->d_ss);
    if (sm->h_ss) cudaFreeHost(sm->h_ss);
    delete sm;
}

void asm_destroy(asm_ctx* pc) {
    if (!pc) return;
    if (pc->ctx) {
        auto& g = pc->ctx->graphs;
        for (auto it = g.begin(); it != g.end();) {
            if (it->first.first == pc) { it->second.release(); it = g.erase(it); }
            else ++it;
        }
    }
    dfree(pc->d_blocks); dfree(pc->d_tiles); dfree(pc->st64); dfree(pc->st32); dfree(pc->st16);
    dfree(pc->d_T); dfree(pc->d_agg); dfree(pc->d_agg_ptr); dfree(pc->d_agg_cells);
    dfree(pc->d_r0); dfree(pc->d_y0); dfree(pc->d_rin); dfree(pc->d_zout);
    delete pc;
}

void polydg_destroy(polydg_ctx* c) {
    if (!c) return;
    for (auto& kv : c->graphs) kv.second.release();
    c->graphs.clear();
    c->work.release();
    dfree(c->K.row_ptr); dfree(c->K.col); dfree(c->K.val); dfree(c->K.val_minus);
    dfree(c->d_to_caller); dfree(c->d_node_ptr); dfree(c->d_node_w); dfree(c->d_node_phi);
    dfree(c->d_node_pos);
    if (c->h_sc) cudaFreeHost(c->h_sc);
    if (c->cap) cudaStreamDestroy(c->cap);
    if (c->cap2) cudaStreamDestroy(c->cap2);
    delete c;
}

}  // extern "C"
