// Host-side setup of libpolydg: connectivity, geometry, quadrature, modal basis
// and the symmetric interior-penalty assembly of Sec. 3 (Eq. eta, Eq. coer),
// plus the coarse-space transfer and Galerkin matrix of Sec. 4.  Runs once per
// mesh; the per-step work runs in the CUDA kernels.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>
#include <tuple>

#include "internal.h"

namespace polydg {

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

int n_modes(int p) { return (p + 1) * (p + 2) / 2; }

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

// phi_(a,b)(x,y) = L_a(xi) L_b(eta) on box = {x0, x1, y0, y1}; order: total degree d,
// then b = 0..d.  grad (optional) receives [n_p][2].
void eval_basis(int p, const double* box, double x, double y, double* val, double* grad) {
    double Lx[16], Dx[16], Ly[16], Dy[16];
    const double sx = 2.0 / (box[1] - box[0]), sy = 2.0 / (box[3] - box[2]);
    const double xi = sx * x - (box[0] + box[1]) / (box[1] - box[0]);
    const double eta = sy * y - (box[2] + box[3]) / (box[3] - box[2]);
    legendre(p, xi, Lx, Dx);
    legendre(p, eta, Ly, Dy);
    int j = 0;
    for (int d = 0; d <= p; ++d)
        for (int b = 0; b <= d; ++b, ++j) {
            const int a = d - b;
            val[j] = Lx[a] * Ly[b];
            if (grad) {
                grad[2 * j] = sx * Dx[a] * Ly[b];
                grad[2 * j + 1] = sy * Lx[a] * Dy[b];
            }
        }
}

// Fan of triangles (v0, v_k, v_{k+1}); on each the collapsed rule
// x(s,t) = A + s (B - A) + s t (C - B), weight w_s w_t s |(B-A) x (C-A)|.
void element_rule(const HostSetup& S, int64_t c, int npts, std::vector<double>& xy,
                  std::vector<double>& w) {
    std::vector<double> g, gw;
    gauss_legendre01(npts, g, gw);
    const int64_t b = S.cell_ptr[c], m = S.cell_ptr[c + 1] - b;
    const double* V = S.verts.data();
    xy.clear();
    w.clear();
    const double ax = V[2 * S.cell_vtx[b]], ay = V[2 * S.cell_vtx[b] + 1];
    for (int64_t k = 1; k + 1 < m; ++k) {
        const double bx = V[2 * S.cell_vtx[b + k]], by = V[2 * S.cell_vtx[b + k] + 1];
        const double cx = V[2 * S.cell_vtx[b + k + 1]], cy = V[2 * S.cell_vtx[b + k + 1] + 1];
        const double jac = std::fabs((bx - ax) * (cy - ay) - (by - ay) * (cx - ax));
        for (int i = 0; i < npts; ++i)
            for (int j = 0; j < npts; ++j) {
                const double s = g[i], t = g[j];
                xy.push_back(ax + s * (bx - ax) + s * t * (cx - bx));
                xy.push_back(ay + s * (by - ay) + s * t * (cy - by));
                w.push_back(gw[i] * gw[j] * s * jac);
            }
    }
}

// --------------------------------------------------------------- validation
static int validate(const polydg_mesh* m, int p, const int32_t* sub) {
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
        const double* s = m->sigma + 4 * c;
        const double scale = std::fabs(s[0]) + std::fabs(s[1]) + std::fabs(s[2]) + std::fabs(s[3]);
        if (!(s[0] > 0) || !(s[0] * s[3] - s[1] * s[2] > 0) || std::fabs(s[1] - s[2]) > 1e-13 * scale) {
            set_error("polydg_setup: sigma of a cell is not symmetric positive definite");
            return POLYDG_EINVAL;
        }
    }
    return POLYDG_OK;
}

// ---------------------------------------------------------------- assembly
int host_setup(const polydg_mesh* m, int p, const int32_t* sub, double chi_cm, double dt,
               double eta0, HostSetup& S) {
    int st = validate(m, p, sub);
    if (st) return st;
    if (!(chi_cm > 0) || !(dt > 0) || !(eta0 > 0)) {
        set_error("polydg_setup: chi_cm, dt and eta0 must be positive");
        return POLYDG_EINVAL;
    }
    const int64_t nc = m->n_cells;
    const int np = n_modes(p);
    S.p = p; S.n_p = np; S.nc = nc; S.chi_cm = chi_cm; S.dt = dt; S.eta0 = eta0;
    S.verts.assign(m->vertices, m->vertices + 2 * m->n_vertices);
    S.cell_ptr.assign(m->cell_ptr, m->cell_ptr + nc + 1);
    S.cell_vtx.assign(m->cell_vtx, m->cell_vtx + m->cell_ptr[nc]);
    S.sigma.assign(m->sigma, m->sigma + 4 * nc);
    const double* V = S.verts.data();

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

    // geometry (caller order) and convexity / orientation check
    S.bbox.resize(4 * nc);
    S.diam.resize(nc);
    S.area.resize(nc);
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

    // connectivity: sort all edges by their sorted vertex pair
    struct Edge { uint64_t key; int64_t cell; int32_t a, b; };
    std::vector<Edge> edges;
    edges.reserve(S.cell_vtx.size());
    for (int64_t c = 0; c < nc; ++c) {
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
    struct Face { int64_t kp, km; int32_t a, b; };
    std::vector<Face> faces;
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
            faces.push_back({e0.cell, e1.cell, e0.a, e0.b});
        }
        i = j;
    }
    std::sort(faces.begin(), faces.end(), [](const Face& x, const Face& y) {
        return std::tie(x.kp, x.km, x.a) < std::tie(y.kp, y.km, y.a);
    });
    const int64_t nf = (int64_t)faces.size();
    S.f_plus.resize(nf);
    S.f_minus.resize(nf);
    for (int64_t f = 0; f < nf; ++f) { S.f_plus[f] = faces[f].kp; S.f_minus[f] = faces[f].km; }

    // spectral norm of each Sigma_K (2x2 symmetric): (a+c)/2 + sqrt(((a-c)/2)^2 + b^2)
    std::vector<double> lam(nc);
    for (int64_t c = 0; c < nc; ++c) {
        const double* s = &S.sigma[4 * c];
        const double h = 0.5 * (s[0] - s[3]);
        lam[c] = 0.5 * (s[0] + s[3]) + std::sqrt(h * h + s[1] * s[1]);
    }

    const int nq = p + 1;
    const int nn2 = np * np;
    // element blocks, caller order
    std::vector<double> Mc(nc * nn2, 0.0), Ac(nc * nn2, 0.0);
    std::vector<double> xy, w, val(np), grad(2 * np);
    std::vector<double> phis, grads;
    for (int64_t c = 0; c < nc; ++c) {
        element_rule(S, c, nq, xy, w);
        const size_t nqp = w.size();
        phis.resize(nqp * np);
        grads.resize(nqp * 2 * np);
        for (size_t k = 0; k < nqp; ++k)
            eval_basis(p, &S.bbox[4 * c], xy[2 * k], xy[2 * k + 1], &phis[k * np], &grads[k * 2 * np]);
        const double* s = &S.sigma[4 * c];
        double* M = &Mc[c * nn2];
        double* A = &Ac[c * nn2];
        for (int i = 0; i < np; ++i)
            for (int j = i; j < np; ++j) {
                double mij = 0.0, aij = 0.0;
                for (size_t k = 0; k < nqp; ++k) {
                    const double* gi = &grads[k * 2 * np + 2 * i];
                    const double* gj = &grads[k * 2 * np + 2 * j];
                    mij += w[k] * phis[k * np + i] * phis[k * np + j];
                    const double sgx = s[0] * gj[0] + s[1] * gj[1];
                    const double sgy = s[2] * gj[0] + s[3] * gj[1];
                    aij += w[k] * (gi[0] * sgx + gi[1] * sgy);
                }
                M[i * np + j] = M[j * np + i] = mij;
                A[i * np + j] = A[j * np + i] = aij;
            }
    }

    // interior face terms of Eq. coer; sides: 0 = K+, 1 = K-
    std::vector<double> gx, gw;
    gauss_legendre01(nq, gx, gw);
    std::vector<double> Aoff(nf * nn2, 0.0);
    std::vector<double> Vs[2], Fs[2];
    for (int s = 0; s < 2; ++s) { Vs[s].resize(nq * np); Fs[s].resize(nq * np); }
    for (int64_t f = 0; f < nf; ++f) {
        const Face& F = faces[f];
        const double ax = V[2 * F.a], ay = V[2 * F.a + 1], bx = V[2 * F.b], by = V[2 * F.b + 1];
        const double len = std::sqrt((bx - ax) * (bx - ax) + (by - ay) * (by - ay));
        const double nx = (by - ay) / len, ny = -(bx - ax) / len;   // out of K+
        const double h = 2.0 * S.diam[F.kp] * S.diam[F.km] / (S.diam[F.kp] + S.diam[F.km]);
        const double eta = eta0 * 0.5 * (lam[F.kp] + lam[F.km]) * p * p / h;
        const int64_t cells[2] = {F.kp, F.km};
        for (int s = 0; s < 2; ++s) {
            const double* sg = &S.sigma[4 * cells[s]];
            const double snx = sg[0] * nx + sg[1] * ny, sny = sg[2] * nx + sg[3] * ny;  // Sigma n
            for (int k = 0; k < nq; ++k) {
                const double x = ax + gx[k] * (bx - ax), y = ay + gx[k] * (by - ay);
                eval_basis(p, &S.bbox[4 * cells[s]], x, y, val.data(), grad.data());
                for (int j = 0; j < np; ++j) {
                    Vs[s][k * np + j] = val[j];
                    Fs[s][k * np + j] = grad[2 * j] * snx + grad[2 * j + 1] * sny;
                }
            }
        }
        const double sgn[2] = {1.0, -1.0};
        for (int a = 0; a < 2; ++a)
            for (int b = 0; b < 2; ++b) {
                if (b < a) continue;
                double* out = (a == b) ? &Ac[cells[a] * nn2] : &Aoff[f * nn2];
                for (int i = 0; i < np; ++i)
                    for (int j = (a == b ? i : 0); j < np; ++j) {
                        double acc = 0.0;
                        for (int k = 0; k < nq; ++k) {
                            const double wk = gw[k] * len;
                            acc += wk * (-0.5 * sgn[a] * Vs[a][k * np + i] * Fs[b][k * np + j]
                                         - 0.5 * sgn[b] * Fs[a][k * np + i] * Vs[b][k * np + j]
                                         + eta * sgn[a] * sgn[b] * Vs[a][k * np + i] * Vs[b][k * np + j]);
                        }
                        if (a == b) {
                            out[i * np + j] += acc;
                            if (j != i) out[j * np + i] += acc;
                        } else {
                            out[i * np + j] = acc;
                        }
                    }
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
    {
        for (int64_t c = 0; c < nc; ++c) {
            const int64_t ntri = S.cell_ptr[c + 1] - S.cell_ptr[c] - 2;
            caller_node_ptr[c + 1] = caller_node_ptr[c] + ntri * nq * nq;
        }
    }
    S.node_ptr.assign(nc + 1, 0);
    S.node_w.clear(); S.node_xy.clear(); S.node_phi.clear(); S.node_to_caller_pos.clear();
    for (int64_t e = 0; e < nc; ++e) {
        const int64_t c = S.to_caller[e];
        element_rule(S, c, nq, xy, w);
        for (size_t k = 0; k < w.size(); ++k) {
            eval_basis(p, &S.bbox[4 * c], xy[2 * k], xy[2 * k + 1], val.data(), nullptr);
            S.node_w.push_back(w[k]);
            S.node_xy.push_back(xy[2 * k]);
            S.node_xy.push_back(xy[2 * k + 1]);
            S.node_phi.insert(S.node_phi.end(), val.begin(), val.end());
            S.node_to_caller_pos.push_back(caller_node_ptr[c] + (int64_t)k);
        }
        S.node_ptr[e + 1] = (int64_t)S.node_w.size();
    }
    return POLYDG_OK;
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

int coarse_setup(const HostSetup& S, const int32_t* coarse, int q, CoarseSetup& C) {
    if (!coarse) { set_error("asm_setup: null coarse partition"); return POLYDG_EINVAL; }
    if (q < 1 || q > S.p) { set_error("asm_setup: coarse degree q must be in 1..p"); return POLYDG_EINVAL; }
    const int64_t nc = S.nc;
    const int np = S.n_p, nqm = n_modes(q);
    int32_t amax = -1;
    for (int64_t c = 0; c < nc; ++c) {
        if (coarse[c] < 0) { set_error("asm_setup: negative agglomerate id"); return POLYDG_EINVAL; }
        amax = std::max(amax, coarse[c]);
    }
    C.q = q; C.n_q = nqm; C.n_agg = amax + 1;
    std::vector<double> abox(4 * C.n_agg);
    for (int J = 0; J < C.n_agg; ++J) { abox[4*J] = 1e300; abox[4*J+1] = -1e300; abox[4*J+2] = 1e300; abox[4*J+3] = -1e300; }
    std::vector<int64_t> cnt(C.n_agg, 0);
    for (int64_t c = 0; c < nc; ++c) {
        const int J = coarse[c];
        cnt[J]++;
        for (int64_t k = S.cell_ptr[c]; k < S.cell_ptr[c + 1]; ++k) {
            const double x = S.verts[2 * S.cell_vtx[k]], y = S.verts[2 * S.cell_vtx[k] + 1];
            abox[4*J] = std::min(abox[4*J], x); abox[4*J+1] = std::max(abox[4*J+1], x);
            abox[4*J+2] = std::min(abox[4*J+2], y); abox[4*J+3] = std::max(abox[4*J+3], y);
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
    std::vector<double> xy, w, v(np), psi(nqm);
    for (int64_t e = 0; e < nc; ++e) {
        const int64_t c = S.to_caller[e];
        const int J = C.agg_of_cell[e];
        element_rule(S, c, S.p + 1, xy, w);
        double* T = &C.T[e * np * nqm];
        for (size_t k = 0; k < w.size(); ++k) {
            eval_basis(S.p, &S.bbox[4 * c], xy[2 * k], xy[2 * k + 1], v.data(), nullptr);
            eval_basis(q, &abox[4 * J], xy[2 * k], xy[2 * k + 1], psi.data(), nullptr);
            for (int i = 0; i < np; ++i)
                for (int a = 0; a < nqm; ++a) T[i * nqm + a] += w[k] * v[i] * psi[a];
        }
        if (!cholesky_solve_small(np, &S.Mblk[e * np * np], T, nqm)) {
            set_error("asm_setup: element mass matrix not positive definite");
            return POLYDG_ENOTSPD;
        }
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
