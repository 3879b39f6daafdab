/*
 * polydg.h -- C ABI of the GB300 PolyDG monodomain solver library (libpolydg.so).
 *
 * The library computes, on one NVIDIA GB300 (sm_103a), the time step of the
 * PolyDG-discretised monodomain + Barreto-Cressman model of arXiv 2512.19536:
 *
 *   polydg_setup     Sec. 3 (Eq. eta, Eq. coer): SIP-DG assembly of M_h, A_h and
 *                    K_h = chi_m C_m M_h + dt/2 A_h on a polygonal mesh, plus the
 *                    subdomain partition T_S of Sec. 4 (polydg_setup3d: the same on
 *                    a polyhedral mesh).
 *   asm_setup        Sec. 4: local matrices K_i = R_i K_h R_i^T, the coarse space
 *                    V_0 = P^q on the agglomerates of T_H with R_0^T the L2
 *                    projection, K_0 = R_0 K_h R_0^T, and their factorisations.
 *   asm_apply        Eq. prec: z = B_ad^{-1} r = sum_{i=0}^{N} R_i^T K_i^{-1} R_i r.
 *   pcg_solve        Sec. 4/5: PCG on K_h x = b with B_ad^{-1}, stopping when
 *                    |r|_2 <= rtol |b|_2 (Euclidean norm of the relative residual).
 *   monodomain_step  Eq. fully-discrete-1: explicit ionic update at the element
 *                    quadrature nodes, right-hand side, PCG solve, per time step.
 *
 * Conventions shared by every call:
 *   - All integer arguments and host arrays are read during the call only; the
 *     library copies what it keeps.  Contexts are owned by the library and are
 *     released only by the matching *_destroy call.
 *   - Vectors passed as `*_dev` are caller-owned DEVICE pointers (e.g. from
 *     torch.Tensor.data_ptr()) to contiguous float64 arrays of n_dofs entries,
 *     laid out element-major in the CALLER's cell order: entry c * n_p + j is
 *     the coefficient of basis function j on cell c.  They must not alias
 *     each other unless stated.
 *   - Basis (the paper fixes none): on cell c with axis-aligned bounding box
 *     [x0,x1]x[y0,y1], phi_(a,b) = L_a(xi) L_b(eta), a + b <= p, L_n the Legendre
 *     polynomials, xi = (2x-x0-x1)/(x1-x0), eta likewise; ordered by total
 *     degree, then by increasing b.  n_p = (p+1)(p+2)/2.  In 3D (box
 *     [x0,x1]x[y0,y1]x[z0,z1]) phi_(a,b,c) = L_a(xi) L_b(eta) L_c(zeta),
 *     a + b + c <= p, ordered by total degree, then by increasing c, then by
 *     increasing b; n_p = (p+1)(p+2)(p+3)/6.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *     Work is enqueued on it; calls that return statistics synchronise it.
 *   - Every function returns POLYDG_OK (0) or a negative status; the text of
 *     the last error of the calling thread is available from polydg_last_error.
 *   - A context is not thread-safe: do not call into one context concurrently.
 */
#ifndef POLYDG_H
#define POLYDG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------------- */
#define POLYDG_OK           0
#define POLYDG_EINVAL      -1   /* bad argument (null pointer, size, degree, mesh) */
#define POLYDG_ENOMEM      -2   /* device or host allocation failed */
#define POLYDG_ECUDA       -3   /* a CUDA runtime call failed */
#define POLYDG_ENOTSPD     -4   /* non-positive pivot in a Cholesky factorisation */
#define POLYDG_ENOTCONV    -5   /* maxit reached; outputs hold the last iterate */
#define POLYDG_EBREAKDOWN  -6   /* p^T K p <= 0 or a non-finite PCG coefficient */
#define POLYDG_ENONFINITE  -7   /* NaN/Inf in an input vector or the residual */

/* ---- storage precision of the local subdomain inverses (asm_setup) --------- */
#define POLYDG_FP64  0          /* float64 store, float64 arithmetic            */
#define POLYDG_FP32  1          /* float32 store, float32 arithmetic            */
#define POLYDG_BF16  2          /* bfloat16 store, float32 accumulation         */

typedef struct polydg_ctx polydg_ctx;
typedef struct asm_ctx asm_ctx;
typedef struct sim_ctx sim_ctx;
typedef struct batch_ctx batch_ctx;
typedef struct guess_model guess_model;
typedef struct shared_local shared_local;

/* A 2D polygonal mesh (Sec. 3: T_h, disjoint polygons).  Cells are convex
 * polygons given as counter-clockwise vertex loops in CSR form; two cells
 * share an interior face exactly when an edge's two vertex ids appear in both
 * loops.  Edges used by one cell only are boundary faces (homogeneous Neumann,
 * Eq. monodomain).  sigma holds the piecewise-constant conductivity tensor
 * Sigma_K (Sec. 2) of each cell, row-major 2x2, symmetric positive definite. */
typedef struct {
    int64_t        n_vertices;
    const double  *vertices;   /* [n_vertices * 2] host, (x, y) pairs        */
    int64_t        n_cells;
    const int64_t *cell_ptr;   /* [n_cells + 1] host, cell_ptr[0] = 0        */
    const int32_t *cell_vtx;   /* [cell_ptr[n_cells]] host, CCW vertex loops */
    const double  *sigma;      /* [n_cells * 4] host                         */
} polydg_mesh;

/* A 3D polyhedral mesh (Sec. 3: T_h, disjoint polyhedra).  Each cell is a
 * closed surface of triangle facets, listed in CSR form: cell c owns facets
 * cell_face_ptr[c] .. cell_face_ptr[c+1]-1, facet f being the vertex ids
 * face_vtx[3f], face_vtx[3f+1], face_vtx[3f+2], ordered so that
 * (b - a) x (c - a) points out of the cell.  Every cell must be star-shaped
 * about the average of its vertices (its element quadrature is the cone of
 * tetrahedra from that point over its facets).  Two cells share an interior
 * face exactly when a facet's three vertex ids appear in both, in opposite
 * orientation; facets of one cell only are boundary faces (homogeneous
 * Neumann).  A planar quadrilateral face is two facets; both neighbours must
 * split it along the same diagonal.  sigma holds Sigma_K of each cell,
 * row-major 3x3, symmetric positive definite. */
typedef struct {
    int64_t        n_vertices;
    const double  *vertices;      /* [n_vertices * 3] host, (x, y, z)           */
    int64_t        n_cells;
    const int64_t *cell_face_ptr; /* [n_cells + 1] host, cell_face_ptr[0] = 0   */
    const int32_t *face_vtx;      /* [cell_face_ptr[n_cells] * 3] host          */
    const double  *sigma;         /* [n_cells * 9] host                         */
} polydg_mesh3d;

typedef struct {
    int64_t n_cells;
    int64_t n_dofs;            /* n_cells * n_p                              */
    int64_t n_faces;           /* interior faces                             */
    int64_t n_blocks;          /* n_p x n_p blocks of K_h (n_cells + 2 n_faces) */
    int64_t n_nodes;           /* element quadrature nodes (ionic state)     */
    int32_t p;
    int32_t n_p;
    int32_t n_subdomains;
    int32_t max_subdomain_dofs;
} polydg_info;

typedef struct {
    int32_t iterations;        /* PCG iterations taken                       */
    int32_t status;            /* POLYDG_OK, ENOTCONV, EBREAKDOWN, ENONFINITE */
    double  relres;            /* |r_k|_2 / |b|_2 at exit (recurrence residual) */
    double  bnorm;             /* |b|_2                                      */
} pcg_stats;

/* Parameters of a coupled simulation (Eq. monodomain, Eq. fully-discrete-1).
 * Initial potential u^0 = u0 (constant), ionic state y^0 = the model's rest
 * state at u0.  External current I_ext(x, t) = stim_amplitude *
 * exp(-|x - (stim_x0, stim_y0)|^2 / (2 stim_width^2)) while t < stim_duration,
 * evaluated at the Crank-Nicolson midpoint t^{k+1/2}.  Each step's PCG starts
 * from U^k and stops at |r|_2 <= rtol |b|_2. */
typedef struct {
    double  u0;
    double  stim_x0, stim_y0, stim_amplitude, stim_width, stim_duration;
    double  rtol;
    int32_t maxit;
    int32_t flexible;          /* 0: standard PCG; 1: flexible PCG (required with FP32/BF16
                                  local inverses); 2: pipelined PCG (as pcg_solve)          */
    double  stim_z0;           /* stimulus centre's z (3D meshes; ignored in 2D) */
} sim_params;

typedef struct {
    int64_t steps_done;        /* steps completed by this call               */
    int64_t total_iterations;  /* PCG iterations summed over those steps     */
    int32_t max_iterations;    /* largest per-step PCG iteration count       */
    int32_t status;            /* first non-OK PCG status, else POLYDG_OK    */
    double  last_relres;       /* relative residual of the last step's solve */
    double  pcg_seconds;       /* device time of the PCG solver kernel over these steps,
                                  measured with CUDA events on the caller's stream */
    int64_t guesses_taken;     /* steps whose PCG started from the learned guess */
} step_stats;

/* Sizes of a preconditioner, for bandwidth accounting. */
typedef struct {
    int64_t local_store_bytes;   /* bytes of K_i^{-1} that one application streams,
                                    all subdomains (the lower triangles when
                                    rows_per_tile is 2)                         */
    int64_t coarse_bytes;        /* bytes of K_0^{-1} (float64)                  */
    int64_t restrict_bytes;      /* bytes of the stored rows of R_0 (float64)   */
    int32_t n_subdomains;
    int32_t n_coarse;            /* coarse DOFs n_0 (0: one-level)              */
    int32_t precision;           /* POLYDG_FP64/FP32/BF16                       */
    int32_t grid;                /* CTAs of the persistent PCG kernel           */
    int32_t rows_per_tile;       /* rows of K_i^{-1} per bulk copy: 1, or 2 when
                                    the PCG kernel streams the lower triangles as
                                    pairs of rows m and n_i - 1 - m (FP32 store and
                                    at least four subdomains per CTA)           */
    int32_t l2_keep_permille;    /* share of the K_i^{-1} cache lines kept in L2 across
                                    iterations (evict-last), per mille (asm_autotune) */
} asm_info;

/* Text of the last error raised on the calling thread ("" if none). */
const char *polydg_last_error(void);

/* Assemble K_h (Sec. 3, Eq. eta with Sigma_K read as lambda_max(Sigma_K), Eq. coer)
 * for degree p (1..6) on `mesh`, with interior-penalty constant eta0 > 0,
 * chi_cm = chi_m C_m > 0 and time step dt > 0, and record the subdomain
 * partition T_S (Sec. 4): subdomain_of_cell[c] in [0, n_subdomains), every id
 * used.  Cells are renumbered internally so each subdomain is contiguous; the
 * caller never sees that order.  Uploads K_h (block-sparse, float64) and the
 * quadrature-node tables to the current CUDA device.  Errors: EINVAL for an
 * invalid mesh (non-matching edges, non-convex or clockwise cell, bad sigma),
 * ENOMEM, ECUDA. */
int polydg_setup(const polydg_mesh *mesh, int p, const int32_t *subdomain_of_cell,
                 double chi_cm, double dt, double eta0, polydg_ctx **out);

/* polydg_setup on a polyhedral mesh (degree p = 2, n_p = 10: the device kernels are
 * instantiated for n_p in {3, 6, 10, 15}, and only P2 maps to one of them in 3D).  Element integrals use
 * the cone of tetrahedra from each cell's vertex average, each with a rule exact for
 * polynomials of degree 2p + 1: for p = 2 the fully symmetric 14-point rule of
 * degree 5, otherwise a collapsed rule of (p + 1)^3 points (Gauss-Jacobi in the
 * two collapsed directions, weights s^2 and t, the Jacobian's factors, and
 * Gauss-Legendre in the third); face integrals use the collapsed rule with
 * (p + 1)^2 points per facet.  The quadrature-node tables (ionic state)
 * follow the same element rule.  Errors as polydg_setup, plus EINVAL for a facet
 * shared by more than two cells or without opposite orientation, and for a cell
 * that is not star-shaped about its vertex average. */
int polydg_setup3d(const polydg_mesh3d *mesh, int p, const int32_t *subdomain_of_cell,
                   double chi_cm, double dt, double eta0, polydg_ctx **out);

int polydg_get_info(const polydg_ctx *ctx, polydg_info *out);

/* Interior faces as (K+, K-) caller cell ids with K+ < K-, sorted
 * lexicographically; plus/minus are host arrays of n_faces entries. */
int polydg_get_faces(const polydg_ctx *ctx, int64_t *plus, int64_t *minus);

/* y = K_h x (float64, caller order).  x_dev and y_dev must not alias. */
int polydg_matvec(polydg_ctx *ctx, const double *x_dev, double *y_dev, void *stream);

/* Build the two-level additive Schwarz preconditioner of Eq. prec on the
 * subdomains given to polydg_setup.  coarse_of_cell (host, [n_cells]) assigns
 * every cell to an agglomerate of T_H (ids 0..N_0-1, all used); NULL builds
 * the one-level operator (no coarse space).  q (1 <= q <= p; at most 4 in 2D and 2
 * in 3D) is the coarse degree.  The local inverses K_i^{-1} are formed in float64 on the device by
 * Cholesky factorisation and stored in `precision` (POLYDG_FP64/FP32/BF16);
 * the coarse inverse K_0^{-1} is always float64.  R_0 is the Euclidean
 * transpose of R_0^T, so B_ad is symmetric.  Errors: EINVAL, ENOTSPD, ENOMEM,
 * ECUDA. */
int asm_setup(polydg_ctx *ctx, const int32_t *coarse_of_cell, int q, int precision,
              asm_ctx **out);

int asm_get_info(const asm_ctx *pc, asm_info *out);

/* Autotune how pcg_solve and monodomain_step with this preconditioner split their work
 * over the CTAs: time `iterations` PCG iterations (a fixed right-hand side on the
 * context's work vectors, default stream) with per-CTA cycle counters, then alternate two
 * moves `rounds` times each -- re-cut the rows of the local inverses with every CTA's
 * tile costs rescaled by its measured / modelled P-phase share, and re-split the elements
 * so that the CTAs' measured CM-phase cycles even out -- keeping a move only if the timed
 * iterations got faster.  Before the moves it times five fractions (0, 1/4, 1/2, 3/4, 1)
 * of the local-inverse cache lines kept in L2 across iterations (evict-last; the rest
 * streams evict-first) and keeps the fastest (always 8 + 4 rounds timed solves).
 * *gain (may be NULL) = time before / time after.  Later solves
 * change only by rounding (the per-CTA partial sums are grouped differently).
 * Synchronises the device.  Errors: EINVAL, ENOMEM, ECUDA. */
int asm_autotune(asm_ctx *pc, int rounds, int iterations, double *gain);

/* z = B_ad^{-1} r (Eq. prec).  r_dev and z_dev are caller-order device vectors
 * and must not alias.  Runs one launch of the persistent PCG kernel in its
 * one-application mode (the local solves, restriction, coarse solve and prolongation
 * of one PCG iteration, with the same work split and arithmetic as pcg_solve), on the
 * context's work vectors (so not concurrently with pcg_solve on the same context).
 * Synchronises `stream`.  Returns POLYDG_OK, POLYDG_ENONFINITE (NaN/Inf in r),
 * POLYDG_ECUDA (a device-side wait timed out, or a CUDA error), POLYDG_EINVAL. */
int asm_apply(asm_ctx *pc, const double *r_dev, double *z_dev, void *stream);

/* Number of polls a grid barrier of the persistent PCG kernels makes before it gives
 * up (default 2^22, about a second); polls < 0 restores the default.  Process-wide; it
 * applies to launches whose arguments are built afterwards (pcg_solve, asm_apply,
 * monodomain_step, and batches created afterwards).  When a barrier gives up, the
 * kernel waits for its own copies in flight (with the default limit), stops, and the
 * call returns POLYDG_ECUDA ("a device-side wait timed out"); the context stays
 * usable.  A small limit is a way to exercise that path without a fault.
 * Returns POLYDG_OK or POLYDG_EINVAL. */
int polydg_set_wait_limit(int64_t polls);

/* Solve K_h x = b by PCG (Saad Alg. 9.1) with B_ad^{-1} (pc != NULL) or without
 * preconditioner (pc == NULL: plain CG).  x_dev holds x0 on entry and the
 * solution on exit.  flexible = 1 takes beta = z_{k+1}.(r_{k+1} - r_k) / (z_k.r_k).
 * flexible = 2 runs pipelined PCG (Ghysels and Vanroose): the same Krylov iterates as the
 * standard form in exact arithmetic, with the auxiliary recurrences u = B r, w = K u, m = B w,
 * n = K m, so that gamma = r.u, delta = w.u and |r|^2 are one reduction per iteration (the
 * other grid barrier of the iteration carries no sums); standard beta, for FP64 local
 * inverses (with FP32/BF16 ones use flexible = 1).  Sims and batches take the same flag
 * through sim_params.flexible (lockstep groups of shared local solves run flexible PCG).
 * The whole iteration runs in one cooperative (persistent) kernel launch with
 * one CTA per SM and grid barriers between its phases; the call synchronises
 * `stream` and fills *stats (may be NULL).
 * Returns POLYDG_OK, ENOTCONV (x holds the last iterate), EBREAKDOWN,
 * ENONFINITE, EINVAL (rtol <= 0, maxit < 1), ECUDA.  b = 0 gives x = 0. */
int pcg_solve(polydg_ctx *ctx, asm_ctx *pc, const double *b_dev, double *x_dev,
              double rtol, int maxit, int flexible, void *stream, pcg_stats *stats);

/* pcg_solve that also records alpha_k (k < capacity) and beta_k (the coefficient that
 * forms p_{k+1}) into host arrays alphas[capacity], betas[capacity] (zeros past the last
 * iteration).  With flexible = 0 they define the Lanczos tridiagonal of B_ad^{-1} K_h
 * (Sec. 5: condition-number estimates; see pcg_lanczos_extremes). */
int pcg_solve_trace(polydg_ctx *ctx, asm_ctx *pc, const double *b_dev, double *x_dev,
                    double rtol, int maxit, int flexible, void *stream, pcg_stats *stats,
                    double *alphas, double *betas, int capacity);

/* Extreme eigenvalues of the Lanczos tridiagonal T of m PCG steps (host): T_kk =
 * 1/alpha_k + beta_{k-1}/alpha_{k-1}, T_{k,k+1} = sqrt(beta_k)/alpha_k (Saad, Iterative
 * Methods, Sec. 6.7.3); estimates of lambda_min, lambda_max of the preconditioned
 * operator, kappa = lmax / lmin, found by bisection on Sturm counts of T (O(m) memory
 * and work per bisection step).  Returns POLYDG_OK or EINVAL. */
int pcg_lanczos_extremes(const double *alphas, const double *betas, int m, double *lmin,
                         double *lmax);

/* Create a coupled simulation on ctx/pc (pc may be NULL for plain CG). */
int sim_create(polydg_ctx *ctx, asm_ctx *pc, const sim_params *params, sim_ctx **out);

/* ---- representation of the ionic state (sim_set_ionic_form) ------------------ */
#define POLYDG_IONIC_NODAL 0    /* per quadrature node, explicit Euler there (default)   */
#define POLYDG_IONIC_MODAL 1    /* in the DG basis: the second line of Eq.
                                   fully-discrete-1, M_h Y^{k+1} = M_h Y^k - dt G^k     */

/* Choose how the simulation's ionic state is represented, before its first step
 * (EINVAL after it).  NODAL keeps the five states at the element quadrature nodes and
 * advances each node by explicit Euler with u^k there.  MODAL keeps, per cell and
 * state l, the n_p coefficients Y_l of the DG basis, starting from the rest state as
 * a constant, and advances them by Eq. fully-discrete-1 (second line): G_l collects
 * sum_q w_q m_l(u^k(x_q), y_h^k(x_q)) phi(x_q) over the cell's quadrature nodes and
 * Y_l^{k+1} = Y_l^k - dt M_K^{-1} G_l (M_h is block diagonal); the ion current I^{k+1}
 * then uses y_h^{k+1} at the nodes.  In both forms sim_get_state returns the states
 * at the nodes (for MODAL, y_h^{k+1}(x_q)).  Allocates 5 n doubles for Y and, once per
 * context, the inverse mass blocks (n_c n_p^2 doubles).  Errors: EINVAL, ENOMEM, ECUDA. */
int sim_set_ionic_form(sim_ctx *sim, int form);

/* Advance nsteps Crank-Nicolson steps (Eq. fully-discrete-1).  Per step:
 * y^{k+1} = y^k - dt m(u^k, y^k) at every quadrature node; I^{k+1} from
 * u~ = 3/2 U^k - 1/2 U^{k-1} (U^0 on the first step) and y^{k+1}; b =
 * (chi_cm M - dt/2 A) U^k - chi_cm dt I^{k+1} + dt F^{k+1/2}; PCG from U^k.
 * Synchronises `stream`; *stats may be NULL.  Stops at the first step whose
 * solve fails and returns that status. */
int monodomain_step(sim_ctx *sim, int nsteps, void *stream, step_stats *stats);

/* Copy the current potential U^k (caller order, [n_dofs]) to u_dev and, if
 * y_dev != NULL, the ionic state ([5][n_nodes], nodes grouped by caller cell
 * in increasing cell id, each cell's nodes in quadrature order) to y_dev. */
int sim_get_state(sim_ctx *sim, double *u_dev, double *y_dev, void *stream);

/* Overwrite U^k and U^{k-1} (caller order device vectors; uprev_dev may be
 * NULL to use u_dev for both).  The history kept for the subspace guess (policy 3 of
 * sim_set_guess) restarts from these two; the nodal ionic update's carried functions of
 * u^{k-1} (sim_get_ionic_aux) are evaluated afresh at the next step. */
int sim_set_potential(sim_ctx *sim, const double *u_dev, const double *uprev_dev,
                      void *stream);

/* Overwrite the last `count` solutions: hist_dev is a caller-order device array
 * [count][n_dofs] holding U^k, U^{k-1}, ..., U^{k-count+1}.  U^k, U^{k-1} and U^{k-2}
 * become the simulation's potentials, and the first min(count, 25, k + 1) solutions the
 * history of the subspace guess (a caller that keeps the state on the host restores
 * all of it this way); the nodal ionic update's carried functions of u^{k-1} are evaluated
 * afresh at the next step unless sim_set_ionic_aux restores them afterwards.  Enqueued on
 * `stream`. */
int sim_set_history(sim_ctx *sim, const double *hist_dev, int count, void *stream);

/* Restore a simulation's ionic state and step index k >= 0 (checkpoint / resume; with
 * sim_set_history for the potentials and then, in the nodal form, sim_set_ionic_aux, a
 * resumed run continues bit for bit).  Nodal form:
 * y_dev is [5][n_nodes] in sim_get_state's node order (required).  Modal form
 * (sim_set_ionic_form, chosen before this call): Y_dev is [5][n_dofs], per state the
 * caller-order DG coefficients as sim_get_ionic_coeffs returns them (required); y_dev, if
 * given, restores the states at the nodes that sim_get_state reports until the next step.
 * The index k sets the time t^k = k dt of the stimulus and the first-step extrapolation
 * (k = 0), and bounds the history sim_set_history keeps (min(count, 25, k + 1)
 * solutions), so call this before sim_set_history.  Clears a failed flag of an earlier
 * step.  Enqueued on `stream`.  Errors: EINVAL, ECUDA. */
int sim_set_state(sim_ctx *sim, const double *y_dev, const double *Y_dev, int64_t k, void *stream);

/* Modal form only: copy the DG coefficients of the five ionic states to Y_dev
 * ([5][n_dofs], per state caller order).  EINVAL for the nodal form. */
int sim_get_ionic_coeffs(sim_ctx *sim, double *Y_dev, void *stream);

/* Nodal form only: the functions of each node's state that the update carries from one
 * step to the next instead of evaluating them ([6][n_nodes] in sim_get_state's node
 * order: E_Na, E_K, exp(-K_o/5), exp((25 - Na_i)/3) of the Sec. 2 model, the potential
 * u^{k-1} at the node and exp(-u^{k-1}/720); each step updates them from the step's small
 * increments, and every 256th step evaluates them afresh).  sim_get_ionic_aux copies them
 * to aux_dev.  sim_set_ionic_aux, called after sim_set_state and sim_set_history, restores
 * them, so that the resumed run continues bit for bit; without it the first resumed step
 * evaluates them from the restored state and potentials, which changes the results by
 * rounding only.  Enqueued on `stream`.  EINVAL for the modal form. */
int sim_get_ionic_aux(sim_ctx *sim, double *aux_dev, void *stream);
int sim_set_ionic_aux(sim_ctx *sim, const double *aux_dev, void *stream);

/* Current step index k. */
int64_t sim_step_index(const sim_ctx *sim);

/* Group n independent simulations (different meshes, conductivities and stimuli;
 * each with its own preconditioner, all with the same degree and local precision,
 * on one device) so that batch_step advances all of them in one cooperative
 * kernel launch per step for all their PCG solves.  Simulation i gets its own
 * group of CTAs (at least one; 1 <= n <= number of SMs), sized so that the bytes
 * each CTA streams per iteration are as even as possible; within the launch every
 * group runs its own PCG (own scalars, barrier and stopping test), so simulations
 * that converge in fewer iterations stop early without affecting the others.
 * The batch refers to the simulations' own buffers (nothing is copied): the sims
 * must outlive the batch, and sim_get_state / sim_set_potential / monodomain_step
 * still work on them between batch_step calls.  Errors: EINVAL (duplicate sim or
 * shared preconditioner, mixed degree/precision/device, n too large, a subdomain
 * plan that does not fit), ENOMEM, ECUDA. */
int batch_create(sim_ctx *const *sims, int n, batch_ctx **out);

/* CTAs of the batched launch given to each simulation (host array [n]). */
int batch_get_groups(const batch_ctx *batch, int32_t *ctas_of_sim);

/* Advance every simulation of the batch nsteps Crank-Nicolson steps (the step of
 * monodomain_step).  The first call records one step -- the per-simulation ionic,
 * right-hand-side and bookkeeping kernels around one batched PCG launch -- into a
 * CUDA graph on an internal stream; each step is then one launch of that graph on
 * `stream`.  Synchronises `stream`.  per_sim (host array [n], may be NULL) gets each
 * simulation's statistics, with pcg_seconds = device time of the whole batched steps
 * (CUDA events around each graph launch); *seconds (may be NULL) gets the same time.
 * A simulation whose solve fails stops stepping (the others continue); the first
 * failing status is returned. */
int batch_step(batch_ctx *batch, int nsteps, void *stream, step_stats *per_sim, double *seconds);

void batch_destroy(batch_ctx *batch);

/* ---- Learned initial guess.  The paper starts each step's PCG from U^k (Sec. 5);
 * this optional network proposes x0 = U^k + s_d o per element instead, o being the
 * output of a two-hidden-layer ReLU network (width 128) applied to features of the
 * element and its face neighbours from the last three solutions:
 *   own a = (U^k_e - u_rest e_0)/s_u, d1 = (U^k_e - U^{k-1}_e)/s_d, d2 = (U^{k-1}_e - U^{k-2}_e)/s_d
 *   (e_0 = the constant mode), then the elementwise mean and the elementwise max of
 *   [a, d1, d2] over the face neighbours, then h_e/h_ref, dt/dt_ref, (neighbours)/10:
 *   9 n_p + 3 inputs.  Parameters, flat: W1 [128][9 n_p + 3] row-major, b1 [128],
 *   W2 [128][128], b2 [128], W3 [n_p][128], b3 [n_p]; scales = {u_rest, s_u, s_d,
 *   h_ref, dt_ref}.  Inference uses fp16 weights with fp32 activations; training keeps
 *   fp32 weights and Adam state (beta1 0.9, beta2 0.999, eps 1e-8). */

/* Number of parameters for n_p coefficients per element (or POLYDG_EINVAL).  The
 * learned guess supports n_p = 3, 6, 10 (p = 1, 2, 3 in 2D). */
int guess_n_params(int n_p);

/* Create a model on the current device from host parameters [guess_n_params(n_p)]
 * (copied; rounded to float32) and scales [5] (NULL: -67, 50, 1, 1, 0.05). */
int guess_create(int n_p, const double *params, const double *scales, guess_model **out);

/* Copy the float32 parameters and Adam moments (each may be NULL) to host arrays of
 * guess_n_params(n_p) doubles, and the number of Adam steps taken to *adam_t. */
int guess_get_params(const guess_model *model, double *params, double *adam_m, double *adam_v,
                     int64_t *adam_t);

int guess_set_scales(guess_model *model, const double *scales);

/* x = U^k + s_d o for caller-order device vectors uk, uk1, uk2 (U^k, U^{k-1}, U^{k-2})
 * on the mesh of ctx (no safeguard: the raw proposal). */
int guess_propose(guess_model *model, polydg_ctx *ctx, const double *uk, const double *uk1,
                  const double *uk2, double *x_dev, void *stream);

/* One Adam step on the mean squared error of o against (U^{k+1}_e - U^k_e)/s_d over
 * n_samples samples.  traj_dev: device array [n_states][n_dofs] of caller-order
 * solutions of one run on ctx's mesh; samples: host array [n_samples][2] of (state k,
 * caller cell id) with 2 <= k <= n_states - 2.  *loss (may be NULL) gets the minibatch
 * loss before the update.  Synchronises `stream`.  Gradients are summed in a fixed
 * order, so a step is deterministic. */
int guess_train_step(guess_model *model, polydg_ctx *ctx, const double *traj_dev, int64_t n_states,
                     const int64_t *samples, int64_t n_samples, double lr, double *loss,
                     void *stream);

/* Use `model` (NULL: none) for the initial guess of the simulation's later steps: from
 * k = 2 on, each step computes the proposal x0 and starts PCG from it --
 *   policy 0: only if |b - K x0|_2 < |b - K U^k|_2 (else from U^k);
 *   policy 1: always;
 *   policy 2: from U^k + theta (x0 - U^k) with theta minimising |b - K x|_2 on that line
 *             (from the same pass over K_h; the residual never exceeds U^k's);
 *   policy 3: from U^k + sum_d theta_d v_d over the directions v: x0 - U^k (when a
 *             model is given, from k = 2 on) and the last min(16, k) solution increments
 *             U^{k-j+1} - U^{k-j}, theta the Galerkin projection V^T K V theta = V^T (b -
 *             K U^k) (the K-norm of the error is smallest; directions with negligible
 *             Schur-complement pivots dropped).  Policy 3 works without a model (the
 *             increments alone) and keeps the last 25 solutions on the device.
 * The FP64 stopping test decides convergence either way, so only iteration counts
 * change.  The model must outlive its use; it may be shared by several simulations. */
int sim_set_guess(sim_ctx *sim, guess_model *model, int policy);

void guess_destroy(guess_model *model);

/* Invert `batch` symmetric positive definite float64 matrices in place, without
 * allocating any device memory.  The paper has no counterpart: this serves callers
 * that cannot call cudaMalloc -- processes whose device memory belongs to another
 * allocator (a framework's caching allocator, or a fixed arena reserved up front by an
 * embedded or real-time runtime, where a stray cudaMalloc would take memory the arena
 * counted on), and code that must not fail on allocation in the middle of a time step.  It runs the same Cholesky-based kernel that asm_setup
 * uses for K_i^{-1} and K_0^{-1}.
 *   mats_dev: device pointer to batch row-major matrices of order n with leading
 *             dimension ld, matrix m starting at mats_dev + m * n * ld; overwritten
 *             with the inverses (caller-owned, read and written during the call).
 *   Limits: n <= 1024, batch <= 256, batch * roundup(n, 32)^2 <= 1048576 (the
 *           workspace is one fixed 8 MiB array per device, held by every GPU that
 *           loads the library until the process exits); larger requests return
 *           POLYDG_EINVAL with a message and launch nothing.
 *   The first call on a device looks up the array's device address
 *   (cudaGetSymbolAddress); make that first call before any stream capture.  All
 *   calls share the array, so calls that overlap on the GPU (two streams, two
 *   threads) race and must be serialised by the caller.  The call synchronises
 *   `stream`.  Returns POLYDG_OK, POLYDG_ENOTSPD (a non-positive pivot; that
 *   matrix's contents are undefined), POLYDG_EINVAL or POLYDG_ECUDA. */
int polydg_spd_inverse_static(double *mats_dev, int n, int ld, int batch, void *stream);

/* ---- Local solves shared by simulations that differ only in a scalar conductivity.
 * With Sigma_K = sigma I on every cell the SIP stiffness is linear in sigma (Eq. eta takes
 * lambda_max(Sigma_K) = sigma, Eq. coer is linear in Sigma), so K_i(sigma) = chi_cm M_i +
 * (dt sigma/2) A_i(1).  With M_i = L_i L_i^T (per element) and the eigendecomposition
 * L_i^{-1} A_i(1) L_i^{-T} = Q_i diag(lam_i) Q_i^T, one factorisation gives
 * K_i(sigma)^{-1} = L_i^{-T} Q_i diag(1/(chi_cm + dt sigma lam_i / 2)) Q_i^T L_i^{-1} for
 * every sigma, and R simulations' right-hand sides take two passes over Q_i together. */

/* Build the shared factors on the mesh and subdomains of ctx, whose conductivity must be
 * the same scalar multiple of I on every cell (EINVAL otherwise).  Q_i is stored in
 * POLYDG_FP32 or POLYDG_BF16; eigendecompositions on the host (polydg_sym_eig), one
 * thread per hardware thread.  Errors: EINVAL, ENOTSPD, ENOTCONV, ENOMEM, ECUDA. */
int shared_local_setup(polydg_ctx *ctx, int precision, shared_local **out);

/* Bytes of the stored Q_i^T and Q_i, and the conductivity of the context it was built on. */
int shared_local_info(const shared_local *sl, int64_t *store_bytes, double *sigma_ref);

/* z_s = sum_i R_i^T K_i(sigmas[s])^{-1} R_i r_s for s < nrhs: r_dev / z_dev are host
 * arrays of caller-order device vectors on the mesh of the context.  BF16 store: 1..16
 * right-hand sides, both passes over Q_i as tcgen05 BF16 GEMMs with FP32 accumulation (one
 * CTA per subdomain; the inputs enter as two BF16 parts each, so the error is that of the
 * BF16 eigenbasis); subdomains of at most 1024 DOFs.  FP32 store: 1..4, SIMT FP32.
 * Synchronises `stream` (BF16).  Errors: EINVAL, ENOMEM, ECUDA (including a device-side wait
 * that timed out). */
int shared_local_apply(shared_local *sl, int nrhs, const double *const *r_dev,
                       double *const *z_dev, const double *sigmas, void *stream);

/* Let batch_step solve this simulation together with the other simulations of the batch
 * that use the same shared_local: up to four of them run their PCG in lockstep in one CTA
 * group, every local solve of every subdomain one two-pass sweep over the shared
 * eigenbasis for all of them (each with its own conductivity, coarse solve, scalars and
 * stopping test).  The simulation's mesh, subdomains, dt and chi_cm must be those of the
 * shared_local's context, its conductivity one scalar multiple of I, and its
 * preconditioner two-level (its coarse part is used; its local inverses are not).  Set it
 * before batch_create (batch_step refuses a batch whose members changed); NULL detaches.
 * monodomain_step is unaffected. */
int sim_set_shared_local(sim_ctx *sim, shared_local *sl);

void shared_local_destroy(shared_local *sl);

/* Eigendecomposition of a symmetric n x n host matrix a (row-major; destroyed): the
 * eigenvalues ascending in w[n], eigenvector k in qt[k*n .. k*n + n) (host arrays).
 * Householder tridiagonalisation and implicit QR steps with Wilkinson shifts, float64,
 * on the calling thread.  Used at setup by the shared local solves.  Returns POLYDG_OK,
 * POLYDG_EINVAL or POLYDG_ENOTCONV. */
int polydg_sym_eig(int n, double *a, double *w, double *qt);

void sim_destroy(sim_ctx *sim);
void asm_destroy(asm_ctx *pc);
void polydg_destroy(polydg_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif /* POLYDG_H */
