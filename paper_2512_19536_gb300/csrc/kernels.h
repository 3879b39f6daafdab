// Launch wrappers of libpolydg's CUDA kernels (host-callable, no torch types).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "device.cuh"

namespace polydg {

enum MatvecMode { MODE_PLAIN = 0, MODE_RHS = 3 };

// Subspace initial guess (policy 3): the last kHistDirs solution increments, plus the
// learned proposal, combined by a Galerkin projection.  The solutions live in a ring
// of kHistRing vectors indexed by step (slot k mod kHistRing holds U^k).
constexpr int kHistDirs = 24;
constexpr int kHistRing = kHistDirs + 1;
constexpr int kSubMaxDirs = kHistDirs + 1;                       // + the learned proposal
constexpr int kSubMaxPairs = kSubMaxDirs + kSubMaxDirs * (kSubMaxDirs + 1) / 2;
constexpr int kSubMaxCtas = 1024;                                // Gram partial sums per pair

// Per-simulation scalars resident in device memory.
struct SimScalars {
    int64_t k;             // current step index (U holds U^k)
    int32_t failed;        // set once a step's solve failed: later steps do nothing
    int32_t max_its;
    int64_t steps_done;
    int64_t total_its;
    int32_t status;
    int32_t use_guess;     // this step's PCG starts from the learned guess
    double last_relres;
    int64_t guesses_taken; // steps (of this call) that started from the learned guess
    uint32_t guess_ticket; // last-CTA ticket of the guess selection
    uint32_t pad;
    double theta;          // x0 = U^k + theta (guess - U^k) when use_guess
    int32_t hist_len;      // consecutive solutions U^k, U^{k-1}, ... held by the ring (>= 1)
    int32_t sub_dirs;      // directions of this step's subspace guess
    double theta_sub[kSubMaxDirs];   // their coefficients
    int32_t kd_len;        // consecutive increment products K D_j held by their ring, up to kd_step
    int32_t yc_ok;         // the nodal ionic update's carried functions match: bit 0 those of
                           // the concentrations (the state), bit 1 those of u^{k-1}
    int64_t kd_step;
};

// Block-sparse K_h on the device (internal cell order).
struct DeviceMatrix {
    int64_t nc = 0, nblk = 0;
    int32_t* row_ptr = nullptr;
    int32_t* col = nullptr;
    double* val = nullptr;        // K_h
    double* val_minus = nullptr;  // chi_cm M - dt/2 A
};

// Grid-barrier state of a cooperative launch (count returns to 0 after each barrier).
struct GridSync {
    unsigned count;
    unsigned gen;
};

// Arguments of the persistent PCG kernel (kernels_pcg.cu).  Per-CTA work lists
// are CSR arrays indexed by blockIdx.x.
struct PersistArgs {
    int grid, wstages, identity, n0, ld0, nq, redundant;
    int small;                                 // every subdomain <= 32 DOFs: a warp per subdomain
    int pair_lanes;                            // lanes (power of 2) summing one coarse DOF's pairs
    int r0_split;                              // R_0 r' summed by slices into r0g, then a barrier
    double* r0g;                               // [n0] (r0_split)
    float l2_keep;                             // fraction of the local-inverse lines kept in L2
    int64_t nc;
    // shared-memory carve-up (byte offsets): wstages copy slots of slot_bytes per warp
    size_t slot_bytes, xs_off, rp_off, r0_off, y0_off, pn_off, td_off;
    // K_h (column-major blocks) and the per-CTA matvec plan.  Each CTA's elements
    // are cut into chunks; per chunk the elements whose z it needs (its own range
    // first, then face neighbours) and their agglomerates, and per block of K_h the
    // chunk-local index of its column element
    const int32_t* row_ptr;
    const double* val;
    const int32_t* cta_chunk;                  // [grid + 1] chunks of each CTA
    const int64_t* chunk_elem;                 // [n_chunks + 1] element range of each chunk
    const int32_t* need_ptr;                   // [n_chunks + 1]
    const int32_t* need;
    const int32_t* need_aggl;                  // per needed element: index into need_agg (redundant
                                               // coarse rows), else its agglomerate
    const int32_t* need_agg_ptr;               // [grid + 1]
    const int32_t* need_agg;                   // agglomerates of the needed elements
    const int32_t* col_local;                  // [n_blocks of K_h]
    const int64_t* elem_ptr;                   // [grid + 1] own element ranges
    // preconditioner
    const GemvBlock* blocks;
    const GemvRun* runs;                       // LOCAL row ranges streamed by each CTA
    const int32_t* run_ptr;                    // [grid + 1]
    const int32_t* sub_pairs;                  // RESTRICT block ids grouped by subdomain
    const void* store;                         // store of the local inverses (dtype)
    const double* st64;                        // fp64 store (restriction rows)
    const double* K0inv;
    const int64_t* pair_ptr;                   // [n_agg + 1] pairs of each agglomerate
    const double* T;
    const int32_t* agg;
    const int32_t* crow_ptr;                   // [grid + 1] coarse rows (distributed mode)
    // vectors (internal order)
    const double* b;
    double* x;
    double* r[2];
    double* p[2];
    double* q[2];
    double *z, *zl, *w;
    double *r0p, *y0;
    PcgScalars* sc;
    double* partials;
    double* bcast;
    GridSync* gs;
    int* err;
    long long* cta_cycles;                     // [2 * grid] P and CM work cycles per CTA, or null
    double* trace;                             // [2 * trace_cap]: alpha_k, then beta_k, or null
    int trace_cap;
    int apply_only;                            // 1: z = B_ad^{-1} b once (r = b, no solve)
    uint32_t wait_limit;                       // polls of a grid barrier before it gives up
    int cm_stages;                             // CM phase: K_h panel slots per warp (0: loads)
    int cm_slot_bytes;
    int sym_bufld;                             // > 0: the P phase streams the symmetric pair-row
                                               // store (fp32, whole subdomains per CTA; store
                                               // points at it); floats per warp of its
                                               // column-sum buffer at r0_off
};

constexpr int kMaxWarpStages = 4;              // copy slots per warp in the P phase
constexpr int kMaxCmStages = 4;                // K_h panel slots per warp in the CM phase

// Shared local solves (shared_local.cu): one subdomain's eigenbasis in the store.
struct SharedBlock {
    int64_t q_off;        // element offset of Q_i^T (n x ld) in the store; Q_i follows
    int64_t lam_off;      // offset of lam_i
    int64_t in_off;       // first DOF (internal order)
    int32_t n, ld, cell0, ncell;
};

constexpr int kMaxRhs = 4;                      // simulations sharing one eigenbasis pass

// Tensor-core form of the shared local solves (shared_local_tc.cu): per subdomain the
// 128 x 64 BF16 tiles of Q_i^T (pass 1) and then of Q_i (pass 2), each 16 KB in the
// core-matrix layout of tcgen05.mma, starting at byte tile_off of the tile store.
struct TcBlock {
    int64_t tile_off;      // bytes
    int64_t in_off;        // first DOF (internal order)
    int64_t lam_off;
    int32_t n, mt, kt, cell0;   // order, 128-row tiles, 64-column tiles, first cell
};
constexpr int kMaxTcRhs = 16;                   // right-hand sides of one tensor-core pass
struct TcRhs {
    const double* r[kMaxTcRhs];
    double* z[kMaxTcRhs];
    double c[kMaxTcRhs];                        // dt sigma_s / 2
    int nrhs;
    int pad;
};
size_t shared_tc_smem(int max_kpad, int nb);
cudaError_t launch_shared_tc(const TcBlock* blocks, int n_blocks, const unsigned char* tiles,
                             const float* lam, const double* linv, int np, double chi,
                             const TcRhs& p, int max_kpad, int* err, cudaStream_t s);

// One simulation of a lockstep group (kernels_group.cu).
struct GroupSim {
    const double* val;                         // its K_h blocks
    const double* K0inv;                       // its coarse inverse
    double c;                                  // dt sigma / 2
    const double* b;
    double* x;
    double* r[2];
    double* p[2];
    double* q[2];
    double *z, *zl, *w;
    double *r0p, *y0;
    float* yq;                                 // Q^T X of its subdomains (pass 1 -> pass 2)
    PcgScalars* sc;
};

// Arguments of the lockstep group solve: R <= kMaxRhs simulations on one mesh,
// partition and coarse space whose local solves share one eigenbasis per subdomain.
// Structure arrays (matvec chunks, coarse layout, restriction rows) are the first
// simulation's; values and vectors are per simulation.
struct GroupArgs {
    int grid, R, wstages, n0, ld0, nq, redundant, np_;
    int64_t nc;
    size_t slot_bytes, rp_off, x_off, y_off, r0_off, y0_off, pn_off, td_off, ld_max;
    const int32_t* row_ptr;
    const int32_t* cta_chunk;
    const int64_t* chunk_elem;
    const int32_t* need_ptr;
    const int32_t* need;
    const int32_t* need_aggl;
    const int32_t* need_agg_ptr;
    const int32_t* need_agg;
    const int32_t* col_local;
    const int64_t* elem_ptr;
    const GemvBlock* blocks;                   // first simulation's blocks (RESTRICT rows)
    const int32_t* sub_pairs;
    const int32_t* pair_begin;                 // [n_sub] first entry in sub_pairs
    const int32_t* pair_count;                 // [n_sub]
    const double* st64;                        // first simulation's fp64 store (rows of R_0)
    const int64_t* pair_ptr;
    const double* T;
    const int32_t* agg;
    const int32_t* crow_ptr;
    const SharedBlock* sblocks;
    const void* qstore;                        // Q_i^T, Q_i (bf16 or fp32)
    const float* lam;
    const double* linv;                        // per element L_K^{-1}
    const GemvRun* pieces;                     // (subdomain, element-aligned row range) per CTA
    const int32_t* piece_ptr;                  // [grid + 1]
    double chi;
    GroupSim sim[kMaxRhs];
    double* partials;
    GridSync* gs;
    int* err;
};

cudaError_t launch_pcg_persistent(int dtype, int np, const PersistArgs& a, size_t smem,
                                  cudaStream_t s);
// Several independent solves in one cooperative launch of n_cta CTAs: CTA b runs
// as CTA map[b].y of the map[b].x-th solve, whose arguments are args[map[b].x]
// (device arrays; args[i].grid = the CTAs mapped to solve i).
cudaError_t launch_pcg_batched(int dtype, int np, const PersistArgs* args_dev, const int2* map_dev,
                               int n_cta, size_t smem, cudaStream_t s);
cudaError_t persistent_occupancy(int dtype, int np, size_t smem, int* blocks_per_sm, int batched);
// The symmetric pair-row store of the fp32 local inverses (LOCAL blocks 0..n_local-1,
// each at its sym_off).
cudaError_t launch_sym_pack(const GemvBlock* blocks, int n_local, const float* st32, float* sym,
                            cudaStream_t s);
// Lockstep groups (kernels_group.cu): one cooperative launch of n_cta CTAs, CTA b runs
// as CTA map[b].y of group map[b].x (args on the device).  qdtype 1 fp32, 2 bf16 store.
cudaError_t launch_pcg_groups(int qdtype, int np, const GroupArgs* args_dev, const int2* map_dev,
                              int n_cta, size_t smem, cudaStream_t s);
cudaError_t group_occupancy(int qdtype, int np, size_t smem, int* blocks_per_sm);

cudaError_t launch_matvec(int mode, int np, const DeviceMatrix& K, const double* val,
                          const double* x, double* y, const double* v1, const double* v2,
                          double c1, double c2, const SimScalars* ss, double dt,
                          double stim_duration, cudaStream_t s);
cudaError_t launch_permute(const double* src, const double* src_odd, double* dst,
                           const int64_t* to_caller, int64_t nc, int np, int to_internal,
                           const PcgScalars* sc, cudaStream_t s);
cudaError_t launch_copy(const double* src, double* dst, int64_t n, const SimScalars* ss,
                        cudaStream_t s);
cudaError_t launch_extract_local(const DeviceMatrix& K, const int64_t* sub_ptr, int n_sub,
                                 const int64_t* mat_off, const int32_t* ld, double* dense,
                                 int np, cudaStream_t s);
cudaError_t launch_chol_inverse(double* store, const int64_t* mat_off, const int32_t* nrow,
                                const int32_t* ld, double* work, const int64_t* work_off,
                                const int32_t* wld, int* status, int nmat, int max_n,
                                cudaStream_t s);
// Blocked FP64 Cholesky inversion of one SPD matrix (chol_blocked.cu): out = A^{-1} (out
// may be A); work holds chol_blocked_work_doubles(n) doubles; *status = 1 on a
// non-positive pivot.
int64_t chol_blocked_work_doubles(int n);
cudaError_t launch_chol_blocked_inverse(const double* A, int64_t lda, int n, double* out, int64_t ldo,
                                        double* work, int* status, cudaStream_t s);
cudaError_t launch_cast_store(const double* src, float* d32, __nv_bfloat16* d16, int64_t n,
                              cudaStream_t s);

// Learned initial guess (kernels_guess.cu).  Features read K_h's block structure
// (face neighbours), the cell diameters and the scales below.
constexpr int kGuessHidden = 128;
struct GuessFeat {
    const int32_t* row_ptr;
    const int32_t* col;
    const double* diam;        // [nc] internal order
    double u_rest, s_u, s_d, h_ref, dt_ref, dt;
    double inv_s_u, inv_s_d;   // 1 / s_u, 1 / s_d (products instead of divisions on the narrow fp64 pipe)
};
int guess_param_count(int np);
size_t guess_train_smem(int np);
cudaError_t guess_prepare(int np);
// The network's proposal x0 = U^k + s_d o for every element (guess_tc.cu, tcgen05): the
// features into xt (guess_tc_tile_bytes(np) per 128 elements), then the three layers with
// the weight image img (guess_tc_image_bytes(np), from launch_guess_tc_image after every
// change of the FP16 weights); *err is raised if a device-side wait ran out.
cudaError_t launch_guess_propose(int np, const GuessFeat& f, const unsigned char* img, const double* Uk,
                                 const double* Uk1, const double* Uk2, double* xg, int64_t nc,
                                 const SimScalars* ss, unsigned char* xt, int* err, int n_sm, cudaStream_t s);
cudaError_t guess_propose_tc_prepare(int np);
size_t guess_tc_image_bytes(int np);
size_t guess_tc_tile_bytes(int np);
cudaError_t launch_guess_tc_image(int np, const __half* w16, unsigned char* img, cudaStream_t s);
cudaError_t launch_guess_select(int np, const DeviceMatrix& K, const double* b, const double* xg,
                                const double* uk, double* partials, SimScalars* ss, int policy,
                                cudaStream_t s);
cudaError_t launch_select_copy(const double* uk, const double* xg, double* x0, int64_t n,
                               const SimScalars* ss, cudaStream_t s);
// Subspace guess: r0 = b - K U^k into W[0], K (U^k - U^{k-1}) into the increment-product
// ring kuring (same slots as the solution ring), K (xg - U^k) into W[1] (with a model);
// then the dot products V^T r0 and
// V^T K V (gram: kSubMaxPairs * kSubMaxCtas partial sums), the Galerkin coefficients (last
// CTA), and x0.  xg == nullptr leaves the learned proposal out.
cudaError_t launch_guess_subspace(int np, const DeviceMatrix& K, const double* b, const double* U,
                                  const double* xg, const double* ring, double* kuring, double* W,
                                  double* gram, int64_t n, SimScalars* ss, cudaStream_t s);
cudaError_t launch_subspace_copy(const double* U, const double* xg, const double* ring,
                                 const double* kuring, const double* W, double* x0, int64_t n,
                                 const SimScalars* ss, cudaStream_t s);
// Ring maintenance: slot(k) <- U and slot(k-1) <- Uprev (new potentials), or `count`
// caller-order solutions [count][n] (U^k first) into the ring, U, Uprev, Uprev2; either way
// the products of the restored increments into the increment-product ring.
cudaError_t launch_history_reset(int np, const DeviceMatrix& K, double* ring, double* kuring,
                                 const double* U, const double* Uprev, int64_t n, SimScalars* ss,
                                 cudaStream_t s);
cudaError_t launch_history_set(const DeviceMatrix& K, const double* hist, int count, double* ring,
                               double* kuring, double* U, double* Uprev, double* Uprev2,
                               const int64_t* to_caller, int64_t nc, int np, SimScalars* ss,
                               cudaStream_t s);
cudaError_t launch_guess_train(int np, const GuessFeat& f, const float* w32, const double* traj,
                               int64_t n_dofs, const int64_t* samples, int64_t n_samples,
                               const int64_t* to_internal, const int64_t* to_caller, float* part,
                               double* lpart, int grid, cudaStream_t s);
cudaError_t launch_guess_adam(const float* part, int ncta, int P, float* w32, float* m, float* v,
                              __half* w16, float lr, float b1, float b2, float eps, float c1, float c2,
                              const double* lpart, double inv_count, double* loss, cudaStream_t s);
cudaError_t launch_to_half(const float* w32, __half* w16, int P, cudaStream_t s);

// Ionic update + ion-current load (Eq. fully-discrete-1), lpc lanes per cell (8, 16 or
// 32, from ionic_lanes_per_cell on the host copy of node_ptr).
cudaError_t launch_ionic(int np, const double* U, const double* Uprev, const int64_t* node_ptr,
                         const double* node_w, const double* node_phi, double* y, double* yc, int64_t nn,
                         int64_t nc, double dt, double* I, const SimScalars* ss, int lpc, cudaStream_t s);
int ionic_lanes_per_cell(const int64_t* node_ptr, int64_t nc);
// Modal ionic state (the second line of Eq. fully-discrete-1 in the DG basis): Ym is
// [5][nc n_p], Minv the per-cell inverse mass blocks [nc][n_p][n_p] (row-major).
cudaError_t launch_ionic_modal(int np, const double* U, const double* Uprev, const int64_t* node_ptr,
                               const double* node_w, const double* node_phi, const double* Minv,
                               double* Ym, double* y, int64_t nn, int64_t nc, double dt, double* I,
                               const SimScalars* ss, cudaStream_t s);
cudaError_t launch_init_modal(double* Ym, int64_t nc, int np, const double* y0, cudaStream_t s);
cudaError_t launch_node_gather(const double* y_int, double* y_caller,
                               const int64_t* node_to_caller_pos, int64_t nn, cudaStream_t s, int ns = 5);
cudaError_t launch_step_finish(double* U, double* Uprev, double* Uprev2, const double* x0,
                               const double* x1, int64_t n, const PcgScalars* sc, SimScalars* ss,
                               double* ring, cudaStream_t s);
cudaError_t launch_step_begin(PcgScalars* sc, SimScalars* ss, cudaStream_t s);
cudaError_t launch_init_y(double* y, int64_t nn, const double* y0, cudaStream_t s);
cudaError_t launch_node_scatter(const double* y_caller, double* y_int,
                                const int64_t* node_to_caller_pos, int64_t nn, cudaStream_t s, int ns = 5);
// The nodal update's carried functions: all of them match (ok = 3: restored with the
// state), or those of u^{k-1} no longer do (ok < 0: the potentials were set from outside).
cudaError_t launch_ionic_aux_valid(SimScalars* ss, cudaStream_t s, int ok = 3);
// Step index k of a simulation (and its failed flag cleared), for a restored state.
cudaError_t launch_set_step(SimScalars* ss, int64_t k, cudaStream_t s);

}  // namespace polydg
