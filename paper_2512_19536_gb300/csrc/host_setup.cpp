// Host-side setup of libpolydg: connectivity, geometry, quadrature, modal basis
// and the symmetric interior-penalty assembly of Sec. 3 (Eq. eta, Eq. coer),
// plus the coarse-space transfer and Galerkin matrix of Sec. 4, for polygonal (2D)
// and polyhedral (3D) meshes.  Runs once per mesh; the per-step work runs in the
// CUDA kernels.  Loops over cells and faces run on all host threads; every cell
// and face writes only its own outputs, so the result does not depend on the
// thread count.
#include <algorithm>
#include <array>
#include <atomic>
#include <cmath>
#include <cstring>
#include <numeric>
#include <thread>
#include <tuple>

#include "internal.h"

namespace polydg {

// Runs body(i0, i1) on contiguous chunks of [0, n) on the host's threads.
template <class F>
static void parallel_chunks(int64_t n, F body) {
    const unsigned hw = std::max(1u, std::thread::hardware_concurrency());
    const int64_t T = std::min<int64_t>(std::min<unsigned>(hw, 64u), std::max<int64_t>(1, n / 64));
    if (T <= 1) { body(int64_t(0), n); return; }
    std::vector<std::thread> th;
    for (int64_t t = 0; t < T; ++t) th.emplace_back([&, t] { body(n * t / T, n * (t + 1) / T); });
    for (auto& x : th) x.join();
}

// --------------------------------------------------------------- quadrature
// Gauss-Legendre: roots of L_n by Newton's method from the Chebyshev-like
// guesses cos(pi (i + 3/4) / (n + 1/2)); weights 2 / ((1 - t^2) L_n'(t)^2).
void gauss_legendre01(int n, std::vector<double>& x, std::vector<double>& w) {
    x.assign(n, 0.0);
    w.assign(n, 0.0);
    for (int i = 0; i < n; ++i) {
        double t = std::cos(M_PI * (i + 0.75) / (n + 0.5));
        double dL = 1.0;
        for (int it = 0; it < 100; ++it) {
            double Lm = 1.0, Ln = t;                 // L_{n-1}, L_n by recurrence
            for (int k = 1; k < n; ++k) {
                const double L2 = ((2.0 * k + 1.0) * t * Ln - k * Lm) / (k + 1.0);
                Lm = Ln;
                Ln = L2;
            }
            dL = n * (t * Ln - Lm) / (t * t - 1.0);
            const double step = Ln / dL;
            t -= step;
            if (std::fabs(step) < 1e-16) break;
        }
        // roots come out in decreasing t; store ascending on [0, 1]
        x[n - 1 - i] = 0.5 * (t + 1.0);
        w[n - 1 - i] = 1.0 / ((1.0 - t * t) * dL * dL);
    }
}

// Gauss-Jacobi on [0, 1] for the weight s^power (power >= 1), by Golub-Welsch: the
// nodes are the eigenvalues of the Jacobi matrix of the monic polynomials orthogonal
// for (1 + x)^power on [-1, 1] (recurrence a_k = b^2 / ((2k+b)(2k+b+2)),
// beta_k = 4k^2(k+b)^2 / ((2k+b)^2 (2k+b+1)(2k+b-1)), b = power), the weights mu_0 times
// the squared first eigenvector components, mu_0 = 2^(b+1)/(b+1); then s = (1 + x)/2.
static void gauss_jacobi01(int n, int power, std::vector<double>& x, std::vector<double>& w) {
    const double b = power;
    std::vector<double> J((size_t)n * n, 0.0), ev(n), vec((size_t)n * n);
    for (int k = 0; k < n; ++k) {
        J[(size_t)k * n + k] = b * b / ((2 * k + b) * (2 * k + b + 2));
        if (k >= 1) {
            const double t = 2 * k + b;
            const double off = std::sqrt(4.0 * k * k * (k + b) * (k + b) / (t * t * (t + 1) * (t - 1)));
            J[(size_t)k * n + k - 1] = J[(size_t)(k - 1) * n + k] = off;
        }
    }
    sym_eig(n, J.data(), ev.data(), vec.data());
    const double mu0 = std::pow(2.0, b + 1) / (b + 1);
    x.assign(n, 0.0);
    w.assign(n, 0.0);
    for (int i = 0; i < n; ++i) {
        x[i] = 0.5 * (ev[i] + 1.0);
        w[i] = mu0 * vec[(size_t)i * n] * vec[(size_t)i * n] / std::pow(2.0, b + 1);
    }
}

int n_modes(int p, int dim) {
    return dim == 3 ? (p + 1) * (p + 2) * (p + 3) / 6 : (p + 1) * (p + 2) / 2;
}

// Legendre values and derivatives L_0..L_p at t.
static void legendre(int p, double t, double* L, double* D) {
    L[0] = 1.0;
    D[0] = 0.0;
    if (p >= 1) { L[1] = t; D[1] = 1.0; }
    for (int n = 1; n < p; ++n) {
        L[n + 1] = ((2.0 * n + 1.0) * t * L[n] - n * L[n - 1]) / (n + 1.0);
        D[n + 1] = D[n - 1] + (2.0 * n + 1.0) * L[n];
    }
}

// 2D: phi_(a,b) = L_a(xi) L_b(eta), order: total degree d, then b = 0..d.
// 3D: phi_(a,b,c) = L_a(xi) L_b(eta) L_c(zeta), order: total degree d, then c = 0..d,
// then b = 0..d-c.  box = {x0, x1, y0, y1[, z0, z1]}; grad (optional) is [n_p][dim].
void eval_basis(int dim, int p, const double* box, const double* x, double* val, double* grad) {
    double L[3][16], D[3][16], s[3];
    for (int d = 0; d < dim; ++d) {
        const double lo = box[2 * d], hi = box[2 * d + 1];
        s[d] = 2.0 / (hi - lo);
        legendre(p, s[d] * x[d] - (lo + hi) / (hi - lo), L[d], D[d]);
    }
    int j = 0;
    if (dim == 2) {
        for (int d = 0; d <= p; ++d)
            for (int b = 0; b <= d; ++b, ++j) {
                const int a = d - b;
                val[j] = L[0][a] * L[1][b];
                if (grad) {
                    grad[2 * j] = s[0] * D[0][a] * L[1][b];
                    grad[2 * j + 1] = s[1] * L[0][a] * D[1][b];
                }
            }
        return;
    }
    for (int d = 0; d <= p; ++d)
        for (int c = 0; c <= d; ++c)
            for (int b = 0; b <= d - c; ++b, ++j) {
                const int a = d - b - c;
                val[j] = L[0][a] * L[1][b] * L[2][c];
                if (grad) {
                    grad[3 * j] = s[0] * D[0][a] * L[1][b] * L[2][c];
                    grad[3 * j + 1] = s[1] * L[0][a] * D[1][b] * L[2][c];
                    grad[3 * j + 2] = s[2] * L[0][a] * L[1][b] * D[2][c];
                }
            }
}

// Apex of a polyhedron's cone rule: the average of its distinct vertices.
static void cell_apex3d(const HostSetup& S, int64_t c, double* apex) {
    std::vector<int32_t> ids(S.cell_vtx.begin() + S.cell_ptr[c], S.cell_vtx.begin() + S.cell_ptr[c + 1]);
    std::sort(ids.begin(), ids.end());
    ids.erase(std::unique(ids.begin(), ids.end()), ids.end());
    apex[0] = apex[1] = apex[2] = 0.0;
    for (int32_t v : ids)
        for (int d = 0; d < 3; ++d) apex[d] += S.verts[3 * v + d];
    for (int d = 0; d < 3; ++d) apex[d] /= (double)ids.size();
}

// Fully symmetric 14-point rule on a tetrahedron, exact to degree 5 -- the degree of the
// 3 x 3 x 3 collapsed rule with about half its points (the element quadrature nodes carry
// the ionic state, so their number sets the cost of the ionic update).  Barycentric
// orbits, in this order: (a, a, a, 1 - 3a) and (b, b, b, 1 - 3b) with the odd coordinate
// at vertex 0..3, then (c, c, 1/2 - c, 1/2 - c) with the c's at the vertex pairs (0,1),
// (0,2), (0,3), (1,2), (1,3), (2,3).  A rule invariant under the vertex permutations is
// exact for a polynomial when it is exact for its average over the permutations, so
// degree 5 needs only the invariant polynomials: with P_k = sum_i l_i^k and
// l_1 + .. + l_4 = 1 these are spanned by 1, P_2, P_3, P_4, P_2^2 and P_2 P_3, whose
// means over the tetrahedron are 1, 2/5, 1/5, 4/35, 6/35, 13/140 (the mean of l^alpha is
// 3! alpha! / (|alpha| + 3)!).  The six equations in (a, b, c, w_a, w_b, w_c) are solved
// once by Newton's method with a central-difference Jacobian from a nearby start.
struct SymTet5 { double lam[14][4]; double w[14]; };

static void sym_tet5_points(const double* v, SymTet5& r) {
    int k = 0;
    for (int o = 0; o < 2; ++o)
        for (int i = 0; i < 4; ++i, ++k) {
            for (int j = 0; j < 4; ++j) r.lam[k][j] = v[o];
            r.lam[k][i] = 1.0 - 3.0 * v[o];
            r.w[k] = v[3 + o];
        }
    for (int i = 0; i < 4; ++i)
        for (int j = i + 1; j < 4; ++j, ++k) {
            for (int l = 0; l < 4; ++l) r.lam[k][l] = 0.5 - v[2];
            r.lam[k][i] = r.lam[k][j] = v[2];
            r.w[k] = v[5];
        }
}

static void sym_tet5_residual(const double* v, double* F) {
    static const double mean[6] = {1.0, 2.0 / 5.0, 1.0 / 5.0, 4.0 / 35.0, 6.0 / 35.0, 13.0 / 140.0};
    SymTet5 r;
    sym_tet5_points(v, r);
    for (int e = 0; e < 6; ++e) F[e] = -mean[e];
    for (int k = 0; k < 14; ++k) {
        double P2 = 0.0, P3 = 0.0, P4 = 0.0;
        for (int i = 0; i < 4; ++i) {
            const double l = r.lam[k][i], l2 = l * l;
            P2 += l2; P3 += l2 * l; P4 += l2 * l2;
        }
        const double g[6] = {1.0, P2, P3, P4, P2 * P2, P2 * P3};
        for (int e = 0; e < 6; ++e) F[e] += r.w[k] * g[e];
    }
}

static const SymTet5& sym_tet5() {
    static const SymTet5 rule = [] {
        double v[6] = {0.09, 0.31, 0.045, 0.07, 0.11, 0.04};
        for (int it = 0; it < 40; ++it) {
            double J[6][7], F[6];
            sym_tet5_residual(v, F);
            for (int c = 0; c < 6; ++c) {
                const double h = 1e-6;
                double vp[6], vm[6], Fp[6], Fm[6];
                for (int i = 0; i < 6; ++i) vp[i] = vm[i] = v[i];
                vp[c] += h;
                vm[c] -= h;
                sym_tet5_residual(vp, Fp);
                sym_tet5_residual(vm, Fm);
                for (int r = 0; r < 6; ++r) J[r][c] = (Fp[r] - Fm[r]) / (2.0 * h);
            }
            for (int r = 0; r < 6; ++r) J[r][6] = -F[r];
            for (int c = 0; c < 6; ++c) {              // elimination with partial pivoting
                int piv = c;
                for (int r = c + 1; r < 6; ++r)
                    if (std::fabs(J[r][c]) > std::fabs(J[piv][c])) piv = r;
                for (int k = 0; k < 7; ++k) std::swap(J[c][k], J[piv][k]);
                for (int r = c + 1; r < 6; ++r) {
                    const double f = J[r][c] / J[c][c];
                    for (int k = c; k < 7; ++k) J[r][k] -= f * J[c][k];
                }
            }
            double dx[6];
            for (int r = 5; r >= 0; --r) {
                double t = J[r][6];
                for (int k = r + 1; k < 6; ++k) t -= J[r][k] * dx[k];
                dx[r] = t / J[r][r];
            }
            for (int i = 0; i < 6; ++i) v[i] += dx[i];
        }
        SymTet5 r;
        sym_tet5_points(v, r);
        return r;
    }();
    return rule;
}

// 2D: fan of triangles (v0, v_k, v_{k+1}); on each the collapsed rule
// x(s,t) = A + s (B - A) + s t (C - B), weight w_s w_t s |(B-A) x (C-A)|.
// 3D: cone of tetrahedra (apex, a, b, c) over the outward facets; on each
// x(s,t,u) = A + s (B-A) + s t (C-B) + s t u (D-C) with Jacobian 6|T| s^2 t, taken as
// the weights of npts-point Gauss-Jacobi rules in s (s^2) and t (t), Gauss-Legendre in
// u: exact to total degree 2 npts - 1; for npts = 3 the symmetric 14-point rule of the
// same degree instead.
void element_rule(const HostSetup& S, int64_t c, int npts, std::vector<double>& xs,
                  std::vector<double>& w) {
    std::vector<double> g, gw;
    gauss_legendre01(npts, g, gw);
    const double* V = S.verts.data();
    xs.clear();
    w.clear();
    if (S.dim == 2) {
        const int64_t b = S.cell_ptr[c], m = S.cell_ptr[c + 1] - b;
        const double ax = V[2 * S.cell_vtx[b]], ay = V[2 * S.cell_vtx[b] + 1];
        for (int64_t k = 1; k + 1 < m; ++k) {
            const double bx = V[2 * S.cell_vtx[b + k]], by = V[2 * S.cell_vtx[b + k] + 1];
            const double cx = V[2 * S.cell_vtx[b + k + 1]], cy = V[2 * S.cell_vtx[b + k + 1] + 1];
            const double jac = std::fabs((bx - ax) * (cy - ay) - (by - ay) * (cx - ax));
            for (int i = 0; i < npts; ++i)
                for (int j = 0; j < npts; ++j) {
                    const double s = g[i], t = g[j];
                    xs.push_back(ax + s * (bx - ax) + s * t * (cx - bx));
                    xs.push_back(ay + s * (by - ay) + s * t * (cy - by));
                    w.push_back(gw[i] * gw[j] * s * jac);
                }
        }
        return;
    }
    std::vector<double> gs, gsw, gt, gtw;
    gauss_jacobi01(npts, 2, gs, gsw);
    gauss_jacobi01(npts, 1, gt, gtw);
    double A[3];
    cell_apex3d(S, c, A);
    for (int64_t k = S.cell_ptr[c]; k < S.cell_ptr[c + 1]; k += 3) {
        const double* B = V + 3 * S.cell_vtx[k];
        const double* C = V + 3 * S.cell_vtx[k + 1];
        const double* D = V + 3 * S.cell_vtx[k + 2];
        double e1[3], e2[3], e3[3];
        for (int d = 0; d < 3; ++d) { e1[d] = B[d] - A[d]; e2[d] = C[d] - A[d]; e3[d] = D[d] - A[d]; }
        const double six_vol = std::fabs(e1[0] * (e2[1] * e3[2] - e2[2] * e3[1]) -
                                         e1[1] * (e2[0] * e3[2] - e2[2] * e3[0]) +
                                         e1[2] * (e2[0] * e3[1] - e2[1] * e3[0]));
        if (npts == 3) {
            const SymTet5& R = sym_tet5();
            for (int q = 0; q < 14; ++q) {
                for (int d = 0; d < 3; ++d)
                    xs.push_back(R.lam[q][0] * A[d] + R.lam[q][1] * B[d] + R.lam[q][2] * C[d] +
                                 R.lam[q][3] * D[d]);
                w.push_back(R.w[q] * (six_vol / 6.0));
            }
            continue;
        }
        for (int i = 0; i < npts; ++i)
            for (int j = 0; j < npts; ++j)
                for (int l = 0; l < npts; ++l) {
                    const double s = gs[i], t = gt[j], u = g[l];
                    for (int d = 0; d < 3; ++d)
                        xs.push_back(A[d] + s * (B[d] - A[d]) + s * t * (C[d] - B[d]) + s * t * u * (D[d] - C[d]));
                    w.push_back(gsw[i] * gtw[j] * gw[l] * six_vol);
                }
    }
}

static int64_t element_rule_size(const HostSetup& S, int64_t c, int npts) {
    const int64_t m = S.cell_ptr[c + 1] - S.cell_ptr[c];
    return S.dim == 2 ? (m - 2) * npts * npts : (m / 3) * (npts == 3 ? 14 : npts * npts * npts);
}

// ---------------------------------------------------------------- geometry
static void cross3(const double* a, const double* b, double* out) {
    out[0] = a[1] * b[2] - a[2] * b[1];
    out[1] = a[2] * b[0] - a[0] * b[2];
    out[2] = a[0] * b[1] - a[1] * b[0];
}

// Checks each cell, fills bbox, diameter and area/volume (caller order).
static int cell_geometry(HostSetup& S) {
    const int64_t nc = S.nc;
    const int dim = S.dim;
    const double* V = S.verts.data();
    S.bbox.assign(2 * dim * nc, 0.0);
    S.diam.assign(nc, 0.0);
    S.area.assign(nc, 0.0);
    if (dim == 2) {
        for (int64_t c = 0; c < nc; ++c) {
            const int64_t b = S.cell_ptr[c], n = S.cell_ptr[c + 1] - b;
            double x0 = 1e300, x1 = -1e300, y0 = 1e300, y1 = -1e300, a2 = 0.0, d2 = 0.0;
            for (int64_t k = 0; k < n; ++k) {
                const int32_t i = S.cell_vtx[b + k];
                x0 = std::min(x0, V[2 * i]); x1 = std::max(x1, V[2 * i]);
                y0 = std::min(y0, V[2 * i + 1]); y1 = std::max(y1, V[2 * i + 1]);
            }
            const double ext = (x1 - x0) + (y1 - y0);
            for (int64_t k = 0; k < n; ++k) {
                const int32_t i = S.cell_vtx[b + k], j = S.cell_vtx[b + (k + 1) % n],
                              l = S.cell_vtx[b + (k + 2) % n];
                const double xi = V[2 * i], yi = V[2 * i + 1];
                a2 += xi * V[2 * j + 1] - V[2 * j] * yi;
                const double cr = (V[2 * j] - xi) * (V[2 * l + 1] - V[2 * j + 1]) -
                                  (V[2 * j + 1] - yi) * (V[2 * l] - V[2 * j]);
                if (cr < -1e-14 * ext * ext) {
                    set_error("polydg_setup: cell is not convex with counter-clockwise vertices");
                    return POLYDG_EINVAL;
                }
                for (int64_t k2 = k + 1; k2 < n; ++k2) {
                    const int32_t o = S.cell_vtx[b + k2];
                    const double dx = V[2 * o] - xi, dy = V[2 * o + 1] - yi;
                    d2 = std::max(d2, dx * dx + dy * dy);
                }
            }
            if (!(a2 > 0)) { set_error("polydg_setup: cell with non-positive area (clockwise?)"); return POLYDG_EINVAL; }
            S.area[c] = 0.5 * a2;
            S.diam[c] = std::sqrt(d2);
            double* bb = &S.bbox[4 * c];
            bb[0] = x0; bb[1] = x1; bb[2] = y0; bb[3] = y1;
        }
        return POLYDG_OK;
    }
    std::atomic<int> bad{0};
    parallel_chunks(nc, [&](int64_t c0, int64_t c1) {
        for (int64_t c = c0; c < c1; ++c) {
            const int64_t b = S.cell_ptr[c], e = S.cell_ptr[c + 1];
            double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300}, d2 = 0.0;
            for (int64_t k = b; k < e; ++k)
                for (int d = 0; d < 3; ++d) {
                    lo[d] = std::min(lo[d], V[3 * S.cell_vtx[k] + d]);
                    hi[d] = std::max(hi[d], V[3 * S.cell_vtx[k] + d]);
                }
            for (int64_t k = b; k < e; ++k)
                for (int64_t k2 = k + 1; k2 < e; ++k2) {
                    double s = 0.0;
                    for (int d = 0; d < 3; ++d) {
                        const double t = V[3 * S.cell_vtx[k] + d] - V[3 * S.cell_vtx[k2] + d];
                        s += t * t;
                    }
                    d2 = std::max(d2, s);
                }
            const double ext = (hi[0] - lo[0]) + (hi[1] - lo[1]) + (hi[2] - lo[2]);
            double apex[3], vol6 = 0.0;
            cell_apex3d(S, c, apex);
            for (int64_t k = b; k < e; k += 3) {
                double a[3], bb[3], cc[3], cr[3];
                for (int d = 0; d < 3; ++d) {
                    a[d] = V[3 * S.cell_vtx[k] + d] - apex[d];
                    bb[d] = V[3 * S.cell_vtx[k + 1] + d] - apex[d];
                    cc[d] = V[3 * S.cell_vtx[k + 2] + d] - apex[d];
                }
                cross3(bb, cc, cr);
                const double det = a[0] * cr[0] + a[1] * cr[1] + a[2] * cr[2];   // 6 vol of the cone tet
                if (det < -1e-13 * ext * ext * ext) bad = 1;
                vol6 += det;
            }
            if (!(vol6 > 0)) bad = 1;
            S.area[c] = vol6 / 6.0;
            S.diam[c] = std::sqrt(d2);
            double* bx = &S.bbox[6 * c];
            for (int d = 0; d < 3; ++d) { bx[2 * d] = lo[d]; bx[2 * d + 1] = hi[d]; }
        }
    });
    if (bad) {
        set_error("polydg_setup3d: a cell is not star-shaped about its vertex average, or has inward facets");
        return POLYDG_EINVAL;
    }
    return POLYDG_OK;
}

// Interior faces: (K+, K-, vertices in K+'s orientation), sorted by (K+, K-, vertices).
struct Face { int64_t kp, km; std::array<int32_t, 3> v; };

static int match_faces(const HostSetup& S, std::vector<Face>& faces) {
    faces.clear();
    if (S.dim == 2) {
        struct Edge { uint64_t key; int64_t cell; int32_t a, b; };
        std::vector<Edge> edges;
        edges.reserve(S.cell_vtx.size());
        for (int64_t c = 0; c < S.nc; ++c) {
            const int64_t b = S.cell_ptr[c], n = S.cell_ptr[c + 1] - b;
            for (int64_t k = 0; k < n; ++k) {
                const int32_t va = S.cell_vtx[b + k], vb = S.cell_vtx[b + (k + 1) % n];
                const uint64_t lo = (uint64_t)std::min(va, vb), hi = (uint64_t)std::max(va, vb);
                edges.push_back({(lo << 32) | hi, c, va, vb});
            }
        }
        std::sort(edges.begin(), edges.end(), [](const Edge& x, const Edge& y) {
            return std::tie(x.key, x.cell) < std::tie(y.key, y.cell);
        });
        for (size_t i = 0; i < edges.size();) {
            size_t j = i + 1;
            while (j < edges.size() && edges[j].key == edges[i].key) ++j;
            if (j - i > 2) { set_error("polydg_setup: an edge is shared by more than two cells"); return POLYDG_EINVAL; }
            if (j - i == 2) {
                const Edge& e0 = edges[i];   // lower cell id (sorted by cell)
                const Edge& e1 = edges[i + 1];
                if (e0.cell == e1.cell || e0.a != e1.b || e0.b != e1.a) {
                    set_error("polydg_setup: shared edge without opposite orientation");
                    return POLYDG_EINVAL;
                }
                faces.push_back({e0.cell, e1.cell, {e0.a, e0.b, -1}});
            }
            i = j;
        }
    } else {
        struct Tri { std::array<int32_t, 3> key; int64_t cell; std::array<int32_t, 3> v; };
        std::vector<Tri> tris;
        tris.reserve(S.cell_vtx.size() / 3);
        for (int64_t c = 0; c < S.nc; ++c)
            for (int64_t k = S.cell_ptr[c]; k < S.cell_ptr[c + 1]; k += 3) {
                Tri t;
                t.v = {S.cell_vtx[k], S.cell_vtx[k + 1], S.cell_vtx[k + 2]};
                t.key = t.v;
                std::sort(t.key.begin(), t.key.end());
                t.cell = c;
                tris.push_back(t);
            }
        std::sort(tris.begin(), tris.end(), [](const Tri& x, const Tri& y) {
            return std::tie(x.key, x.cell) < std::tie(y.key, y.cell);
        });
        for (size_t i = 0; i < tris.size();) {
            size_t j = i + 1;
            while (j < tris.size() && tris[j].key == tris[i].key) ++j;
            if (j - i > 2) { set_error("polydg_setup3d: a facet is shared by more than two cells"); return POLYDG_EINVAL; }
            if (j - i == 2) {
                const Tri& t0 = tris[i];
                const Tri& t1 = tris[i + 1];
                // t1 must run through the same vertices in the opposite cyclic order
                const std::array<int32_t, 3> r = {t0.v[0], t0.v[2], t0.v[1]};
                const bool opp = t1.v == r || t1.v == std::array<int32_t, 3>{r[1], r[2], r[0]} ||
                                 t1.v == std::array<int32_t, 3>{r[2], r[0], r[1]};
                if (t0.cell == t1.cell || !opp) {
                    set_error("polydg_setup3d: shared facet without opposite orientation");
                    return POLYDG_EINVAL;
                }
                faces.push_back({t0.cell, t1.cell, t0.v});
            }
            i = j;
        }
    }
    std::sort(faces.begin(), faces.end(), [](const Face& x, const Face& y) {
        return std::tie(x.kp, x.km, x.v) < std::tie(y.kp, y.km, y.v);
    });
    return POLYDG_OK;
}

// Quadrature of an interior face: points [n * dim], weights, unit normal out of K+.
static void face_rule(const HostSetup& S, const Face& F, const std::vector<double>& g,
                      const std::vector<double>& gw, std::vector<double>& xs, std::vector<double>& w,
                      double* normal) {
    const double* V = S.verts.data();
    const int nq = (int)g.size();
    xs.clear();
    w.clear();
    if (S.dim == 2) {
        const double ax = V[2 * F.v[0]], ay = V[2 * F.v[0] + 1], bx = V[2 * F.v[1]], by = V[2 * F.v[1] + 1];
        const double len = std::sqrt((bx - ax) * (bx - ax) + (by - ay) * (by - ay));
        normal[0] = (by - ay) / len;
        normal[1] = -(bx - ax) / len;
        for (int k = 0; k < nq; ++k) {
            xs.push_back(ax + g[k] * (bx - ax));
            xs.push_back(ay + g[k] * (by - ay));
            w.push_back(gw[k] * len);
        }
        return;
    }
    const double* A = V + 3 * F.v[0];
    const double* B = V + 3 * F.v[1];
    const double* C = V + 3 * F.v[2];
    double e1[3], e2[3], cr[3];
    for (int d = 0; d < 3; ++d) { e1[d] = B[d] - A[d]; e2[d] = C[d] - A[d]; }
    cross3(e1, e2, cr);
    const double twice_area = std::sqrt(cr[0] * cr[0] + cr[1] * cr[1] + cr[2] * cr[2]);
    for (int d = 0; d < 3; ++d) normal[d] = cr[d] / twice_area;
    for (int i = 0; i < nq; ++i)
        for (int j = 0; j < nq; ++j) {
            const double s = g[i], t = g[j];
            for (int d = 0; d < 3; ++d) xs.push_back(A[d] + s * (B[d] - A[d]) + s * t * (C[d] - B[d]));
            w.push_back(gw[i] * gw[j] * s * twice_area);
        }
}

// --------------------------------------------------------------- validation
static int validate_sigma(int dim, const double* sigma, int64_t nc) {
    for (int64_t c = 0; c < nc; ++c) {
        const double* s = sigma + dim * dim * c;
        double scale = 0.0;
        for (int i = 0; i < dim * dim; ++i) scale += std::fabs(s[i]);
        bool ok = scale > 0 && std::isfinite(scale);
        for (int i = 0; i < dim && ok; ++i)
            for (int j = i + 1; j < dim; ++j)
                if (std::fabs(s[i * dim + j] - s[j * dim + i]) > 1e-13 * scale) ok = false;
        // positive definite: the Cholesky pivots of the (symmetric part) are positive
        double L[9] = {0};
        for (int j = 0; j < dim && ok; ++j) {
            double d = s[j * dim + j];
            for (int k = 0; k < j; ++k) d -= L[j * 3 + k] * L[j * 3 + k];
            if (!(d > 0)) { ok = false; break; }
            L[j * 3 + j] = std::sqrt(d);
            for (int i = j + 1; i < dim; ++i) {
                double t = s[i * dim + j];
                for (int k = 0; k < j; ++k) t -= L[i * 3 + k] * L[j * 3 + k];
                L[i * 3 + j] = t / L[j * 3 + j];
            }
        }
        if (!ok) {
            set_error("polydg_setup: sigma of a cell is not symmetric positive definite");
            return POLYDG_EINVAL;
        }
    }
    return POLYDG_OK;
}

static int validate2d(const polydg_mesh* m, int p, const int32_t* sub) {
    if (!m || !m->vertices || !m->cell_ptr || !m->cell_vtx || !m->sigma || !sub) {
        set_error("polydg_setup: null mesh array");
        return POLYDG_EINVAL;
    }
    if (p < 1 || p > 6) { set_error("polydg_setup: degree p must be in 1..6"); return POLYDG_EINVAL; }
    if (m->n_cells < 1 || m->n_vertices < 3 || m->cell_ptr[0] != 0) {
        set_error("polydg_setup: empty mesh or cell_ptr[0] != 0");
        return POLYDG_EINVAL;
    }
    for (int64_t c = 0; c < m->n_cells; ++c) {
        const int64_t b = m->cell_ptr[c], e = m->cell_ptr[c + 1];
        if (e - b < 3) { set_error("polydg_setup: cell with fewer than 3 vertices"); return POLYDG_EINVAL; }
        for (int64_t k = b; k < e; ++k)
            if (m->cell_vtx[k] < 0 || m->cell_vtx[k] >= m->n_vertices) {
                set_error("polydg_setup: vertex id out of range");
                return POLYDG_EINVAL;
            }
    }
    return validate_sigma(2, m->sigma, m->n_cells);
}

static int validate3d(const polydg_mesh3d* m, int p, const int32_t* sub) {
    if (!m || !m->vertices || !m->cell_face_ptr || !m->face_vtx || !m->sigma || !sub) {
        set_error("polydg_setup3d: null mesh array");
        return POLYDG_EINVAL;
    }
    // the device kernels are instantiated for n_p in {3, 6, 10, 15}; in 3D only p = 2 (n_p = 10) maps
    if (p != 2) { set_error("polydg_setup3d: degree p must be 2 (n_p = 10)"); return POLYDG_EINVAL; }
    if (m->n_cells < 1 || m->n_vertices < 4 || m->cell_face_ptr[0] != 0) {
        set_error("polydg_setup3d: empty mesh or cell_face_ptr[0] != 0");
        return POLYDG_EINVAL;
    }
    for (int64_t c = 0; c < m->n_cells; ++c) {
        const int64_t b = m->cell_face_ptr[c], e = m->cell_face_ptr[c + 1];
        if (e - b < 4) { set_error("polydg_setup3d: cell with fewer than 4 facets"); return POLYDG_EINVAL; }
        for (int64_t k = 3 * b; k < 3 * e; ++k)
            if (m->face_vtx[k] < 0 || m->face_vtx[k] >= m->n_vertices) {
                set_error("polydg_setup3d: vertex id out of range");
                return POLYDG_EINVAL;
            }
    }
    return validate_sigma(3, m->sigma, m->n_cells);
}

// --------------------------------------------------------------- assembly
// Everything after the mesh copy: subdomain renumbering, geometry, faces,
// element and face blocks (Eq. coer, Eq. eta), K_h and the quadrature-node tables.
static int assemble(HostSetup& S, const int32_t* sub) {
    const int64_t nc = S.nc;
    const int dim = S.dim, p = S.p, np = S.n_p;

    // subdomains: ids dense in [0, n_sub)
    int32_t smax = -1;
    for (int64_t c = 0; c < nc; ++c) {
        if (sub[c] < 0) { set_error("polydg_setup: negative subdomain id"); return POLYDG_EINVAL; }
        smax = std::max(smax, sub[c]);
    }
    S.n_sub = smax + 1;
    std::vector<int64_t> count(S.n_sub, 0);
    for (int64_t c = 0; c < nc; ++c) count[sub[c]]++;
    for (int i = 0; i < S.n_sub; ++i)
        if (!count[i]) { set_error("polydg_setup: unused subdomain id"); return POLYDG_EINVAL; }
    S.sub_ptr.assign(S.n_sub + 1, 0);
    for (int i = 0; i < S.n_sub; ++i) S.sub_ptr[i + 1] = S.sub_ptr[i] + count[i];
    S.to_caller.resize(nc);
    S.to_internal.resize(nc);
    {
        std::vector<int64_t> fill(S.sub_ptr.begin(), S.sub_ptr.end() - 1);
        for (int64_t c = 0; c < nc; ++c) {
            const int64_t e = fill[sub[c]]++;
            S.to_caller[e] = c;
            S.to_internal[c] = e;
        }
    }
    if (int st = cell_geometry(S)) return st;
    std::vector<Face> faces;
    if (int st = match_faces(S, faces)) return st;
    const int64_t nf = (int64_t)faces.size();
    S.f_plus.resize(nf);
    S.f_minus.resize(nf);
    for (int64_t f = 0; f < nf; ++f) { S.f_plus[f] = faces[f].kp; S.f_minus[f] = faces[f].km; }

    // spectral norm of each Sigma_K
    std::vector<double> lam(nc);
    for (int64_t c = 0; c < nc; ++c) {
        const double* s = &S.sigma[dim * dim * c];
        if (dim == 2) {      // 2x2 symmetric: (a+c)/2 + sqrt(((a-c)/2)^2 + b^2)
            const double h = 0.5 * (s[0] - s[3]);
            lam[c] = 0.5 * (s[0] + s[3]) + std::sqrt(h * h + s[1] * s[1]);
        } else {
            double a[9], w[3], qt[9];
            for (int i = 0; i < 9; ++i) a[i] = s[i];
            if (!sym_eig(3, a, w, qt)) { set_error("polydg_setup3d: eigenvalues of sigma did not converge"); return POLYDG_EINVAL; }
            lam[c] = w[2];
        }
    }

    const int nq = p + 1;
    const int nn2 = np * np;
    // element blocks, caller order
    std::vector<double> Mc(nc * nn2, 0.0), Ac(nc * nn2, 0.0);
    parallel_chunks(nc, [&](int64_t c0, int64_t c1) {
        std::vector<double> xs, w, phis, grads;
        for (int64_t c = c0; c < c1; ++c) {
            element_rule(S, c, nq, xs, w);
            const size_t nqp = w.size();
            phis.resize(nqp * np);
            grads.resize(nqp * dim * np);
            for (size_t k = 0; k < nqp; ++k)
                eval_basis(dim, p, &S.bbox[2 * dim * c], &xs[dim * k], &phis[k * np], &grads[k * dim * np]);
            const double* s = &S.sigma[dim * dim * c];
            double* M = &Mc[c * nn2];
            double* A = &Ac[c * nn2];
            for (int i = 0; i < np; ++i)
                for (int j = i; j < np; ++j) {
                    double mij = 0.0, aij = 0.0;
                    for (size_t k = 0; k < nqp; ++k) {
                        const double* gi = &grads[(k * np + i) * dim];
                        const double* gj = &grads[(k * np + j) * dim];
                        mij += w[k] * phis[k * np + i] * phis[k * np + j];
                        double e = 0.0;
                        for (int r = 0; r < dim; ++r) {
                            double sg = 0.0;
                            for (int t = 0; t < dim; ++t) sg += s[r * dim + t] * gj[t];
                            e += gi[r] * sg;
                        }
                        aij += w[k] * e;
                    }
                    M[i * np + j] = M[j * np + i] = mij;
                    A[i * np + j] = A[j * np + i] = aij;
                }
        }
    });

    // interior face terms of Eq. coer; sides: 0 = K+, 1 = K-.  Faces are computed in
    // parallel chunks; their self blocks are then added to the element blocks in face
    // order, so the sums do not depend on the thread count.
    std::vector<double> gx, gw;
    gauss_legendre01(nq, gx, gw);
    std::vector<double> Aoff(nf * nn2, 0.0);
    const int64_t fchunk = 1 << 15;
    std::vector<double> self((size_t)std::min<int64_t>(fchunk, std::max<int64_t>(nf, 1)) * 2 * nn2);
    for (int64_t f0 = 0; f0 < nf; f0 += fchunk) {
        const int64_t f1 = std::min(nf, f0 + fchunk);
        parallel_chunks(f1 - f0, [&](int64_t i0, int64_t i1) {
            std::vector<double> xs, w, val(np), grad(dim * np), Vs[2], Fs[2];
            for (int64_t f = f0 + i0; f < f0 + i1; ++f) {
                const Face& F = faces[f];
                double nrm[3];
                face_rule(S, F, gx, gw, xs, w, nrm);
                const int nfq = (int)w.size();
                const double h = 2.0 * S.diam[F.kp] * S.diam[F.km] / (S.diam[F.kp] + S.diam[F.km]);
                const double eta = S.eta0 * 0.5 * (lam[F.kp] + lam[F.km]) * p * p / h;
                const int64_t cells[2] = {F.kp, F.km};
                for (int sd = 0; sd < 2; ++sd) {
                    Vs[sd].resize(nfq * np);
                    Fs[sd].resize(nfq * np);
                    const double* sg = &S.sigma[dim * dim * cells[sd]];
                    double sn[3];                                     // Sigma n
                    for (int r = 0; r < dim; ++r) {
                        sn[r] = 0.0;
                        for (int t = 0; t < dim; ++t) sn[r] += sg[r * dim + t] * nrm[t];
                    }
                    for (int k = 0; k < nfq; ++k) {
                        eval_basis(dim, p, &S.bbox[2 * dim * cells[sd]], &xs[dim * k], val.data(), grad.data());
                        for (int j = 0; j < np; ++j) {
                            Vs[sd][k * np + j] = val[j];
                            double fl = 0.0;
                            for (int r = 0; r < dim; ++r) fl += grad[j * dim + r] * sn[r];
                            Fs[sd][k * np + j] = fl;
                        }
                    }
                }
                const double sgn[2] = {1.0, -1.0};
                double* sp = &self[(size_t)(f - f0) * 2 * nn2];
                std::fill(sp, sp + 2 * nn2, 0.0);
                for (int a = 0; a < 2; ++a)
                    for (int b = 0; b < 2; ++b) {
                        if (b < a) continue;
                        double* out = (a == b) ? sp + a * nn2 : &Aoff[f * nn2];
                        for (int i = 0; i < np; ++i)
                            for (int j = (a == b ? i : 0); j < np; ++j) {
                                double acc = 0.0;
                                for (int k = 0; k < nfq; ++k)
                                    acc += w[k] * (-0.5 * sgn[a] * Vs[a][k * np + i] * Fs[b][k * np + j]
                                                   - 0.5 * sgn[b] * Fs[a][k * np + i] * Vs[b][k * np + j]
                                                   + eta * sgn[a] * sgn[b] * Vs[a][k * np + i] * Vs[b][k * np + j]);
                                if (a == b) {
                                    out[i * np + j] += acc;
                                    if (j != i) out[j * np + i] += acc;
                                } else {
                                    out[i * np + j] = acc;
                                }
                            }
                    }
            }
        });
        for (int64_t f = f0; f < f1; ++f) {
            const double* sp = &self[(size_t)(f - f0) * 2 * nn2];
            double* Ap = &Ac[faces[f].kp * nn2];
            double* Am = &Ac[faces[f].km * nn2];
            for (int t = 0; t < nn2; ++t) { Ap[t] += sp[t]; Am[t] += sp[nn2 + t]; }
        }
    }

    // block-sparse K_h and (chi_cm M - dt/2 A), internal order, rows: diag first then
    // neighbours by increasing internal id; parallel faces between one pair are summed.
    std::vector<std::vector<std::pair<int64_t, int64_t>>> nb(nc);   // (internal col, face) per row
    for (int64_t f = 0; f < nf; ++f) {
        const int64_t ep = S.to_internal[faces[f].kp], em = S.to_internal[faces[f].km];
        nb[ep].push_back({em, f});
        nb[em].push_back({ep, ~f});       // ~f marks the transposed use
    }
    S.row_ptr.assign(nc + 1, 0);
    S.col.clear();
    std::vector<std::vector<int64_t>> row_faces;   // per block: face ids (signed)
    for (int64_t e = 0; e < nc; ++e) {
        auto& L = nb[e];
        std::sort(L.begin(), L.end());
        S.col.push_back((int32_t)e);
        row_faces.push_back({});
        for (size_t i = 0; i < L.size(); ++i) {
            if (i > 0 && L[i].first == L[i - 1].first) {
                row_faces.back().push_back(L[i].second);
                continue;
            }
            S.col.push_back((int32_t)L[i].first);
            row_faces.push_back({L[i].second});
        }
        S.row_ptr[e + 1] = (int32_t)S.col.size();
    }
    const int64_t nblk = (int64_t)S.col.size();
    S.Kval.assign(nblk * nn2, 0.0);
    S.Kminus_val.assign(nblk * nn2, 0.0);
    S.Mblk.assign(nc * nn2, 0.0);
    const double chi_cm = S.chi_cm, dt = S.dt;
    for (int64_t e = 0; e < nc; ++e) {
        const int64_t c = S.to_caller[e];
        for (int32_t bi = S.row_ptr[e]; bi < S.row_ptr[e + 1]; ++bi) {
            double* Kb = &S.Kval[(int64_t)bi * nn2];
            double* Kmb = &S.Kminus_val[(int64_t)bi * nn2];
            if (bi == S.row_ptr[e]) {
                for (int t = 0; t < nn2; ++t) {
                    Kb[t] = chi_cm * Mc[c * nn2 + t] + 0.5 * dt * Ac[c * nn2 + t];
                    Kmb[t] = chi_cm * Mc[c * nn2 + t] - 0.5 * dt * Ac[c * nn2 + t];
                    S.Mblk[e * nn2 + t] = Mc[c * nn2 + t];
                }
                continue;
            }
            std::vector<double> acc(nn2, 0.0);
            for (int64_t fs : row_faces[bi]) {
                const bool tr = fs < 0;
                const int64_t f = tr ? ~fs : fs;
                for (int i = 0; i < np; ++i)
                    for (int j = 0; j < np; ++j)
                        acc[i * np + j] += tr ? Aoff[f * nn2 + j * np + i] : Aoff[f * nn2 + i * np + j];
            }
            for (int t = 0; t < nn2; ++t) {
                Kb[t] = 0.5 * dt * acc[t];
                Kmb[t] = -0.5 * dt * acc[t];
            }
        }
    }

    // element quadrature nodes (ionic state and load vectors), internal cell order
    std::vector<int64_t> caller_node_ptr(nc + 1, 0);
    for (int64_t c = 0; c < nc; ++c) caller_node_ptr[c + 1] = caller_node_ptr[c] + element_rule_size(S, c, nq);
    S.node_ptr.assign(nc + 1, 0);
    for (int64_t e = 0; e < nc; ++e) S.node_ptr[e + 1] = S.node_ptr[e] + element_rule_size(S, S.to_caller[e], nq);
    const int64_t nn = S.node_ptr[nc];
    S.node_w.assign(nn, 0.0);
    S.node_x.assign(nn * dim, 0.0);
    S.node_phi.assign(nn * np, 0.0);
    S.node_to_caller_pos.assign(nn, 0);
    parallel_chunks(nc, [&](int64_t e0, int64_t e1) {
        std::vector<double> xs, w;
        for (int64_t e = e0; e < e1; ++e) {
            const int64_t c = S.to_caller[e];
            element_rule(S, c, nq, xs, w);
            const int64_t q0 = S.node_ptr[e];
            for (size_t k = 0; k < w.size(); ++k) {
                const int64_t qn = q0 + (int64_t)k;
                eval_basis(dim, p, &S.bbox[2 * dim * c], &xs[dim * k], &S.node_phi[qn * np], nullptr);
                S.node_w[qn] = w[k];
                for (int d = 0; d < dim; ++d) S.node_x[qn * dim + d] = xs[dim * k + d];
                S.node_to_caller_pos[qn] = caller_node_ptr[c] + (int64_t)k;
            }
        }
    });
    return POLYDG_OK;
}

static int check_scalars(double chi_cm, double dt, double eta0) {
    if (!(chi_cm > 0) || !(dt > 0) || !(eta0 > 0)) {
        set_error("polydg_setup: chi_cm, dt and eta0 must be positive");
        return POLYDG_EINVAL;
    }
    return POLYDG_OK;
}

int host_setup(const polydg_mesh* m, int p, const int32_t* sub, double chi_cm, double dt,
               double eta0, HostSetup& S) {
    if (int st = validate2d(m, p, sub)) return st;
    if (int st = check_scalars(chi_cm, dt, eta0)) return st;
    const int64_t nc = m->n_cells;
    S.dim = 2;
    S.p = p; S.n_p = n_modes(p, 2); S.nc = nc; S.chi_cm = chi_cm; S.dt = dt; S.eta0 = eta0;
    S.verts.assign(m->vertices, m->vertices + 2 * m->n_vertices);
    S.cell_ptr.assign(m->cell_ptr, m->cell_ptr + nc + 1);
    S.cell_vtx.assign(m->cell_vtx, m->cell_vtx + m->cell_ptr[nc]);
    S.sigma.assign(m->sigma, m->sigma + 4 * nc);
    return assemble(S, sub);
}

int host_setup3d(const polydg_mesh3d* m, int p, const int32_t* sub, double chi_cm, double dt,
                 double eta0, HostSetup& S) {
    if (int st = validate3d(m, p, sub)) return st;
    if (int st = check_scalars(chi_cm, dt, eta0)) return st;
    const int64_t nc = m->n_cells;
    S.dim = 3;
    S.p = p; S.n_p = n_modes(p, 3); S.nc = nc; S.chi_cm = chi_cm; S.dt = dt; S.eta0 = eta0;
    S.verts.assign(m->vertices, m->vertices + 3 * m->n_vertices);
    S.cell_ptr.resize(nc + 1);
    for (int64_t c = 0; c <= nc; ++c) S.cell_ptr[c] = 3 * m->cell_face_ptr[c];
    S.cell_vtx.assign(m->face_vtx, m->face_vtx + S.cell_ptr[nc]);
    S.sigma.assign(m->sigma, m->sigma + 9 * nc);
    return assemble(S, sub);
}

// ------------------------------------------------------------ coarse space
// V_0 = P^q on each agglomerate J (modal basis on J's bounding box).  R_0^T is
// the L2 projection: on fine cell K in J, T_K = M_K^{-1} int_K phi_K psi_J^T
// (exact, V_0 in V_h).  K_0 = R_0 K_h R_0^T with R_0 = (R_0^T)^T.
static bool cholesky_solve_small(int n, const double* A, double* B, int nrhs) {
    std::vector<double> L(n * n, 0.0);
    for (int j = 0; j < n; ++j) {
        double d = A[j * n + j];
        for (int k = 0; k < j; ++k) d -= L[j * n + k] * L[j * n + k];
        if (!(d > 0)) return false;
        L[j * n + j] = std::sqrt(d);
        for (int i = j + 1; i < n; ++i) {
            double s = A[i * n + j];
            for (int k = 0; k < j; ++k) s -= L[i * n + k] * L[j * n + k];
            L[i * n + j] = s / L[j * n + j];
        }
    }
    for (int r = 0; r < nrhs; ++r) {
        for (int i = 0; i < n; ++i) {          // L y = b
            double s = B[i * nrhs + r];
            for (int k = 0; k < i; ++k) s -= L[i * n + k] * B[k * nrhs + r];
            B[i * nrhs + r] = s / L[i * n + i];
        }
        for (int i = n - 1; i >= 0; --i) {     // L^T x = y
            double s = B[i * nrhs + r];
            for (int k = i + 1; k < n; ++k) s -= L[k * n + i] * B[k * nrhs + r];
            B[i * nrhs + r] = s / L[i * n + i];
        }
    }
    return true;
}

// M_K^{-1} of every cell (row-major, internal order), by the Cholesky solve above with
// the identity as right-hand side.
int mass_inverse_blocks(const HostSetup& S, std::vector<double>& out) {
    const int np = S.n_p;
    out.assign((size_t)S.nc * np * np, 0.0);
    int bad = 0;
    for (int64_t e = 0; e < S.nc; ++e) {
        double* B = &out[(size_t)e * np * np];
        for (int i = 0; i < np; ++i) B[i * np + i] = 1.0;
        if (!cholesky_solve_small(np, &S.Mblk[(size_t)e * np * np], B, np)) bad = 1;
    }
    if (bad) { set_error("mass matrix of a cell is not positive definite"); return POLYDG_ENOTSPD; }
    return POLYDG_OK;
}

int coarse_setup(const HostSetup& S, const int32_t* coarse, int q, CoarseSetup& C) {
    if (!coarse) { set_error("asm_setup: null coarse partition"); return POLYDG_EINVAL; }
    if (q < 1 || q > S.p) { set_error("asm_setup: coarse degree q must be in 1..p"); return POLYDG_EINVAL; }
    const int64_t nc = S.nc;
    const int dim = S.dim, np = S.n_p, nqm = n_modes(q, dim);
    int32_t amax = -1;
    for (int64_t c = 0; c < nc; ++c) {
        if (coarse[c] < 0) { set_error("asm_setup: negative agglomerate id"); return POLYDG_EINVAL; }
        amax = std::max(amax, coarse[c]);
    }
    C.q = q; C.n_q = nqm; C.n_agg = amax + 1;
    std::vector<double> abox(2 * dim * (size_t)C.n_agg);
    for (int J = 0; J < C.n_agg; ++J)
        for (int d = 0; d < dim; ++d) { abox[2 * dim * J + 2 * d] = 1e300; abox[2 * dim * J + 2 * d + 1] = -1e300; }
    std::vector<int64_t> cnt(C.n_agg, 0);
    for (int64_t c = 0; c < nc; ++c) {
        const int J = coarse[c];
        cnt[J]++;
        double* bx = &abox[2 * dim * J];
        for (int64_t k = S.cell_ptr[c]; k < S.cell_ptr[c + 1]; ++k)
            for (int d = 0; d < dim; ++d) {
                const double x = S.verts[dim * S.cell_vtx[k] + d];
                bx[2 * d] = std::min(bx[2 * d], x);
                bx[2 * d + 1] = std::max(bx[2 * d + 1], x);
            }
    }
    for (int J = 0; J < C.n_agg; ++J)
        if (!cnt[J]) { set_error("asm_setup: unused agglomerate id"); return POLYDG_EINVAL; }
    C.agg_of_cell.resize(nc);
    C.agg_ptr.assign(C.n_agg + 1, 0);
    for (int J = 0; J < C.n_agg; ++J) C.agg_ptr[J + 1] = C.agg_ptr[J] + cnt[J];
    C.agg_cells.resize(nc);
    std::vector<int64_t> fill(C.agg_ptr.begin(), C.agg_ptr.end() - 1);
    for (int64_t e = 0; e < nc; ++e) {
        const int J = coarse[S.to_caller[e]];
        C.agg_of_cell[e] = J;
        C.agg_cells[fill[J]++] = (int32_t)e;
    }
    // T_K per internal cell
    C.T.assign(nc * np * nqm, 0.0);
    std::atomic<int> bad{0};
    parallel_chunks(nc, [&](int64_t e0, int64_t e1) {
        std::vector<double> xs, w, v(np), psi(nqm);
        for (int64_t e = e0; e < e1; ++e) {
            const int64_t c = S.to_caller[e];
            const int J = C.agg_of_cell[e];
            element_rule(S, c, S.p + 1, xs, w);
            double* T = &C.T[e * np * nqm];
            for (size_t k = 0; k < w.size(); ++k) {
                eval_basis(dim, S.p, &S.bbox[2 * dim * c], &xs[dim * k], v.data(), nullptr);
                eval_basis(dim, q, &abox[2 * dim * J], &xs[dim * k], psi.data(), nullptr);
                for (int i = 0; i < np; ++i)
                    for (int a = 0; a < nqm; ++a) T[i * nqm + a] += w[k] * v[i] * psi[a];
            }
            if (!cholesky_solve_small(np, &S.Mblk[e * np * np], T, nqm)) bad = 1;
        }
    });
    if (bad) {
        set_error("asm_setup: element mass matrix not positive definite");
        return POLYDG_ENOTSPD;
    }
    // K_0 = sum over blocks (e, f): T_e^T K_ef T_f into (J(e), J(f))
    const int64_t n0 = (int64_t)C.n_agg * nqm;
    C.K0.assign(n0 * n0, 0.0);
    std::vector<double> KT(np * nqm);
    for (int64_t e = 0; e < nc; ++e) {
        const int Je = C.agg_of_cell[e];
        const double* Te = &C.T[e * np * nqm];
        for (int32_t bi = S.row_ptr[e]; bi < S.row_ptr[e + 1]; ++bi) {
            const int64_t f = S.col[bi];
            const int Jf = C.agg_of_cell[f];
            const double* Tf = &C.T[f * np * nqm];
            const double* Kb = &S.Kval[(int64_t)bi * np * np];
            for (int i = 0; i < np; ++i)
                for (int b = 0; b < nqm; ++b) {
                    double s = 0.0;
                    for (int j = 0; j < np; ++j) s += Kb[i * np + j] * Tf[j * nqm + b];
                    KT[i * nqm + b] = s;
                }
            for (int a = 0; a < nqm; ++a)
                for (int b = 0; b < nqm; ++b) {
                    double s = 0.0;
                    for (int i = 0; i < np; ++i) s += Te[i * nqm + a] * KT[i * nqm + b];
                    C.K0[(Je * nqm + a) * n0 + (Jf * nqm + b)] += s;
                }
        }
    }
    for (int64_t i = 0; i < n0; ++i)
        for (int64_t j = i + 1; j < n0; ++j) {
            const double s = 0.5 * (C.K0[i * n0 + j] + C.K0[j * n0 + i]);
            C.K0[i * n0 + j] = C.K0[j * n0 + i] = s;
        }
    return POLYDG_OK;
}

}  // namespace polydg
