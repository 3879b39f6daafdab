// Symmetric eigendecomposition on the host (setup of the shared local solves):
// Householder reduction to tridiagonal form, then implicit symmetric QR steps with
// Wilkinson shifts (Golub & Van Loan, Matrix Computations, Sec. 8.3), accumulating
// the orthogonal factor.  The factor is kept transposed (row k = column k of Q), so
// every update touches contiguous rows.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <numeric>
#include <vector>

#include "internal.h"

namespace polydg {

// a: n x n symmetric, row-major, destroyed.  On return w[k] (ascending) are the
// eigenvalues and qt[k * n + i] = component i of the eigenvector of w[k].
// Returns false if the QR iteration did not converge (30 n sweeps).
bool sym_eig(int n, double* a, double* w, double* qt) {
    if (n <= 0) return true;
    std::vector<double> d(n), e(std::max(n - 1, 1), 0.0), v(n), p(n), wv(n);
    for (int i = 0; i < n * n; ++i) qt[i] = 0.0;
    for (int i = 0; i < n; ++i) qt[i * n + i] = 1.0;
    // ---- tridiagonalisation: A <- P A P with P = I - beta v v^T on rows/cols k+1..n-1
    for (int k = 0; k + 2 < n; ++k) {
        const int m = n - k - 1;                       // length of x = A[k+1.., k]
        const double* x = a + (size_t)k * n + k + 1;   // row k right of the diagonal (symmetric)
        double sig = 0.0;
        for (int i = 0; i < m; ++i) sig += x[i] * x[i];
        const double nx = std::sqrt(sig);
        if (nx == 0.0) { d[k] = a[(size_t)k * n + k]; e[k] = 0.0; continue; }
        const double alpha = x[0] >= 0.0 ? -nx : nx;   // new off-diagonal entry
        for (int i = 0; i < m; ++i) v[i] = x[i];
        v[0] -= alpha;
        double vv = 0.0;
        for (int i = 0; i < m; ++i) vv += v[i] * v[i];
        const double beta = 2.0 / vv;
        // p = beta A22 v, K = beta/2 p.v, w = p - K v, A22 -= v w^T + w v^T
        for (int i = 0; i < m; ++i) {
            const double* row = a + (size_t)(k + 1 + i) * n + k + 1;
            double s = 0.0;
            for (int j = 0; j < m; ++j) s += row[j] * v[j];
            p[i] = beta * s;
        }
        double pv = 0.0;
        for (int i = 0; i < m; ++i) pv += p[i] * v[i];
        const double K = 0.5 * beta * pv;
        for (int i = 0; i < m; ++i) wv[i] = p[i] - K * v[i];
        for (int i = 0; i < m; ++i) {
            double* row = a + (size_t)(k + 1 + i) * n + k + 1;
            const double vi = v[i], wi = wv[i];
            for (int j = 0; j < m; ++j) row[j] -= vi * wv[j] + wi * v[j];
        }
        d[k] = a[(size_t)k * n + k];
        e[k] = alpha;
        // Q <- Q P:  rows k+1.. of Q^T:  Qt[j] -= beta v_j (v^T Qt[k+1..])
        std::fill(p.begin(), p.end(), 0.0);
        for (int i = 0; i < m; ++i) {
            const double* row = qt + (size_t)(k + 1 + i) * n;
            const double vi = v[i];
            for (int c = 0; c < n; ++c) p[c] += vi * row[c];
        }
        for (int i = 0; i < m; ++i) {
            double* row = qt + (size_t)(k + 1 + i) * n;
            const double f = beta * v[i];
            for (int c = 0; c < n; ++c) row[c] -= f * p[c];
        }
    }
    if (n >= 2) {
        d[n - 2] = a[(size_t)(n - 2) * n + n - 2];
        e[n - 2] = a[(size_t)(n - 2) * n + n - 1];
    }
    d[n - 1] = a[(size_t)(n - 1) * n + n - 1];
    // ---- implicit symmetric QR steps with Wilkinson shifts on (d, e)
    const double eps = 2.220446049250313e-16;
    int m = n - 1;
    long sweeps = 0;
    const long max_sweeps = 30L * n;
    while (m > 0) {
        // deflate negligible off-diagonals at the bottom
        if (std::fabs(e[m - 1]) <= eps * (std::fabs(d[m - 1]) + std::fabs(d[m]))) {
            e[m - 1] = 0.0;
            --m;
            continue;
        }
        int l = m - 1;                                 // start of the unreduced block
        while (l > 0 && std::fabs(e[l - 1]) > eps * (std::fabs(d[l - 1]) + std::fabs(d[l]))) --l;
        if (l > 0) e[l - 1] = 0.0;
        if (++sweeps > max_sweeps) return false;
        const double delta = 0.5 * (d[m - 1] - d[m]);
        const double em = e[m - 1];
        const double den = delta + (delta >= 0.0 ? 1.0 : -1.0) * std::hypot(delta, em);
        const double mu = d[m] - em * em / den;
        double x = d[l] - mu, z = e[l];
        for (int k = l; k < m; ++k) {
            const double r = std::hypot(x, z);
            const double c = r == 0.0 ? 1.0 : x / r, s = r == 0.0 ? 0.0 : -z / r;
            if (k > l) e[k - 1] = r;
            const double ak = d[k], bk = e[k], dk = d[k + 1];
            d[k] = c * c * ak - 2.0 * c * s * bk + s * s * dk;
            d[k + 1] = s * s * ak + 2.0 * c * s * bk + c * c * dk;
            e[k] = c * s * (ak - dk) + (c * c - s * s) * bk;
            if (k + 1 < m) {
                z = -s * e[k + 1];
                e[k + 1] = c * e[k + 1];
                x = e[k];
            }
            // Q <- Q G: columns k, k+1 of Q = rows k, k+1 of Q^T
            double* qk = qt + (size_t)k * n;
            double* qk1 = qt + (size_t)(k + 1) * n;
            for (int i = 0; i < n; ++i) {
                const double u0 = qk[i], u1 = qk1[i];
                qk[i] = c * u0 - s * u1;
                qk1[i] = s * u0 + c * u1;
            }
        }
    }
    // ascending order
    std::vector<int> idx(n);
    std::iota(idx.begin(), idx.end(), 0);
    std::sort(idx.begin(), idx.end(), [&](int i, int j) { return d[i] < d[j]; });
    std::vector<double> tmp((size_t)n * n);
    for (int k = 0; k < n; ++k) {
        w[k] = d[idx[k]];
        std::copy(qt + (size_t)idx[k] * n, qt + (size_t)idx[k] * n + n, tmp.begin() + (size_t)k * n);
    }
    std::copy(tmp.begin(), tmp.end(), qt);
    return true;
}

}  // namespace polydg

extern "C" int polydg_sym_eig(int n, double* a, double* w, double* qt) {
    if (n < 1 || !a || !w || !qt) {
        polydg::set_error("polydg_sym_eig: need n >= 1 and three host arrays");
        return POLYDG_EINVAL;
    }
    if (!polydg::sym_eig(n, a, w, qt)) {
        polydg::set_error("polydg_sym_eig: the QR iteration did not converge");
        return POLYDG_ENOTCONV;
    }
    return POLYDG_OK;
}
