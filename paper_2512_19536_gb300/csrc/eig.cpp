// Symmetric eigendecomposition on the host (setup of the shared local solves):
// Householder reduction to tridiagonal form, then implicit symmetric QR steps with
// Wilkinson shifts (Golub & Van Loan, Matrix Computations, Sec. 8.3), accumulating
// the orthogonal factor.  The factor is kept transposed (row k = column k of Q), so
// every update touches contiguous rows.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdint>
#include <numeric>
#include <thread>
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

// ------------------------------------------------ dense SPD inverse on the host
// For coarse matrices too large for one CTA's factorisation: Cholesky A = L L^T by
// column panels (rows below a panel in parallel) inside the envelope of A (row i of L
// starts at row i's first nonzero of A: no fill left of it), W = L^{-1} transposed
// (rows in parallel: row k of W is column k of L^{-1}, zero before k), then
// A^{-1} = W^T-products: A^{-1}_ij = sum_{m >= max(i,j)} W_im W_jm (rows in parallel).
// Every dot product runs in a fixed order, so the result does not depend on the
// thread count.
static double dot4(const double* a, const double* b, int64_t n) {
    double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
    int64_t k = 0;
    for (; k + 4 <= n; k += 4) {
        s0 += a[k] * b[k];
        s1 += a[k + 1] * b[k + 1];
        s2 += a[k + 2] * b[k + 2];
        s3 += a[k + 3] * b[k + 3];
    }
    for (; k < n; ++k) s0 += a[k] * b[k];
    return (s0 + s1) + (s2 + s3);
}

template <class F>
static void host_parallel(int64_t n, F body) {
    const int64_t T = std::max<int64_t>(1, std::min<int64_t>(std::min<unsigned>(std::thread::hardware_concurrency(), 64u), n));
    if (T <= 1) { for (int64_t i = 0; i < n; ++i) body(i); return; }
    std::atomic<int64_t> next{0};
    std::vector<std::thread> th;
    for (int64_t t = 0; t < T; ++t)
        th.emplace_back([&] {
            for (int64_t i; (i = next.fetch_add(1)) < n;) body(i);
        });
    for (auto& x : th) x.join();
}

bool spd_inverse(int64_t n, const double* A, double* Ainv) {
    // envelope: row i of L is zero left of the first nonzero of row i of A
    std::vector<int64_t> first(n);
    for (int64_t i = 0; i < n; ++i) {
        int64_t f = i;
        for (int64_t j = 0; j < i; ++j)
            if (A[(size_t)i * n + j] != 0.0) { f = j; break; }
        first[i] = f;
    }
    std::vector<double> L((size_t)n * n, 0.0);
    auto entry = [&](int64_t i, int64_t j) {        // L[i][j], j < i, j >= first[i]
        const double* Li = &L[(size_t)i * n];
        const double* Lj = &L[(size_t)j * n];
        const int64_t m0 = std::max(first[i], first[j]);
        return (A[(size_t)i * n + j] - dot4(Li + m0, Lj + m0, j - m0)) / Lj[j];
    };
    const int64_t nb = 64;
    for (int64_t j0 = 0; j0 < n; j0 += nb) {
        const int64_t j1 = std::min(n, j0 + nb);
        for (int64_t j = j0; j < j1; ++j) {
            double* Lj = &L[(size_t)j * n];
            for (int64_t jj = std::max(j0, first[j]); jj < j; ++jj) Lj[jj] = entry(j, jj);
            const double d = A[(size_t)j * n + j] - dot4(Lj + first[j], Lj + first[j], j - first[j]);
            if (!(d > 0)) return false;
            Lj[j] = std::sqrt(d);
        }
        host_parallel(n - j1, [&](int64_t r) {
            const int64_t i = j1 + r;
            double* Li = &L[(size_t)i * n];
            for (int64_t j = std::max(j0, first[i]); j < j1; ++j) Li[j] = entry(i, j);
        });
    }
    std::vector<double> W((size_t)n * n, 0.0);           // W[k][i] = (L^{-1})[i][k]
    host_parallel(n, [&](int64_t k) {
        double* Wk = &W[(size_t)k * n];
        Wk[k] = 1.0 / L[(size_t)k * n + k];
        for (int64_t i = k + 1; i < n; ++i) {
            const double* Li = &L[(size_t)i * n];
            const int64_t m0 = std::max(k, first[i]);
            Wk[i] = m0 < i ? -dot4(Li + m0, Wk + m0, i - m0) / Li[i] : 0.0;
        }
    });
    host_parallel(n, [&](int64_t i) {
        const double* Wi = &W[(size_t)i * n];
        for (int64_t j = i; j < n; ++j) {
            const double* Wj = &W[(size_t)j * n];
            Ainv[(size_t)i * n + j] = dot4(Wi + j, Wj + j, n - j);
        }
    });
    for (int64_t i = 0; i < n; ++i)
        for (int64_t j = 0; j < i; ++j) Ainv[(size_t)i * n + j] = Ainv[(size_t)j * n + i];
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
