// Internal structures of libpolydg shared by its translation units.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "polydg.h"

namespace polydg {

void set_error(const std::string& msg);

// ---------------------------------------------------------------- host setup
// Everything computed on the host once per mesh (Sec. 3 assembly), in the
// library's internal cell order (cells sorted by subdomain, stable).
struct HostSetup {
    int dim = 2;                       // 2: polygons, 3: polyhedra of triangle facets
    int p = 0, n_p = 0;
    int64_t nc = 0;
    double chi_cm = 1.0, dt = 0.0, eta0 = 0.0;
    // caller <-> internal numbering
    std::vector<int64_t> to_caller;    // [nc] internal -> caller id
    std::vector<int64_t> to_internal;  // [nc] caller -> internal id
    // subdomains (contiguous internal ranges)
    int n_sub = 0;
    std::vector<int64_t> sub_ptr;      // [n_sub+1] internal cell ranges
    // geometry, caller order
    std::vector<double> bbox;          // [nc*2*dim] x0 x1 y0 y1 (z0 z1)
    std::vector<double> diam, area;    // area: the cell's area (2D) or volume (3D)
    std::vector<double> sigma;         // [nc*dim*dim]
    // mesh copy (caller numbering), for agglomerate boxes and quadrature.  2D:
    // cell_vtx[cell_ptr[c]..] is the CCW vertex loop; 3D: it lists the cell's
    // outward triangle facets, three vertex ids each.
    std::vector<double> verts;         // [n_vertices*dim]
    std::vector<int64_t> cell_ptr;
    std::vector<int32_t> cell_vtx;
    // interior faces, caller ids, K+ < K-, sorted
    std::vector<int64_t> f_plus, f_minus;
    // block-sparse K_h and (chi_cm M - dt/2 A) in internal order.  Row e holds
    // blocks row_ptr[e]..row_ptr[e+1]-1; the first one is the diagonal block.
    std::vector<int32_t> row_ptr, col;
    std::vector<double> Kval, Kminus_val;   // [n_blocks * n_p * n_p], row-major blocks
    std::vector<double> Mblk;               // [nc * n_p * n_p] internal order
    // element quadrature nodes, internal cell order
    std::vector<int64_t> node_ptr;          // [nc+1]
    std::vector<double> node_w;             // [nn]
    std::vector<double> node_x;             // [nn*dim]
    std::vector<double> node_phi;           // [nn*n_p]
    std::vector<int64_t> node_to_caller_pos;// [nn] position of internal node in caller node order
};

int host_setup(const polydg_mesh* mesh, int p, const int32_t* sub, double chi_cm,
               double dt, double eta0, HostSetup& out);
int host_setup3d(const polydg_mesh3d* mesh, int p, const int32_t* sub, double chi_cm,
                 double dt, double eta0, HostSetup& out);

// Gauss-Legendre nodes/weights on [0,1], ascending.
void gauss_legendre01(int n, std::vector<double>& x, std::vector<double>& w);
// Modal basis values (and gradients [n_p][dim] if grad != nullptr) at x[dim] for a box.
int n_modes(int p, int dim);
void eval_basis(int dim, int p, const double* box, const double* x, double* val, double* grad);
// Element rule: 2D vertex-0 fan, 3D cone from the vertex average over the facets;
// collapsed Gauss rules with n = npts points per direction (npts + 1 along the
// collapsed direction of a tetrahedron).  xs receives dim coordinates per point.
void element_rule(const HostSetup& S, int64_t caller_cell, int npts,
                  std::vector<double>& xs, std::vector<double>& w);

// Symmetric eigendecomposition (host): a (n x n, row-major) is destroyed; w ascending,
// qt[k * n + i] = component i of eigenvector k.  False if the iteration did not converge.
bool sym_eig(int n, double* a, double* w, double* qt);
// Inverse of a dense SPD matrix (n x n row-major) on the host threads; false if a
// Cholesky pivot is not positive.
bool spd_inverse(int64_t n, const double* A, double* Ainv);

// Coarse-space data (Sec. 4) computed on the host for asm_setup.
struct CoarseSetup {
    int q = 0, n_q = 0, n_agg = 0;
    std::vector<int32_t> agg_of_cell;     // [nc] internal order
    std::vector<int64_t> agg_ptr;         // [n_agg+1] CSR of internal cells per agglomerate
    std::vector<int32_t> agg_cells;
    std::vector<double> T;                // [nc * n_p * n_q] internal order, T_K row-major
    std::vector<double> K0;               // [n0 * n0] dense, n0 = n_agg * n_q
};
int coarse_setup(const HostSetup& S, const int32_t* coarse_of_cell, int q, CoarseSetup& out);
int mass_inverse_blocks(const HostSetup& S, std::vector<double>& out);

}  // namespace polydg
