// Small dense linear algebra on the host, for the m x m matrices of the
// small-space setup (Gram matrices for Cholesky-QR re-orthonormalisation and
// the Rayleigh-Ritz matrices of the eigensolver), and the Chebyshev
// coefficients of the polynomial P(x) ~ x^{-1/2} (Sec. 2).
//
// Matrices are column-major arrays of (re, im) pairs, A(i, j) = A[i + j n].
#include <algorithm>
#include <cmath>
#include <complex>
#include <numeric>
#include <vector>

#include "ovl_internal.h"

namespace ovl {
namespace {
typedef std::complex<double> cd;
inline cd get(const std::vector<HostCplx>& A, int n, int i, int j) {
    const HostCplx& v = A[i + (size_t)j * n];
    return cd(v.re, v.im);
}
inline void put(std::vector<HostCplx>& A, int n, int i, int j, cd v) {
    A[i + (size_t)j * n] = HostCplx{v.real(), v.imag()};
}
}  // namespace

bool host_cholesky(int n, std::vector<HostCplx>& A) {
    for (int j = 0; j < n; ++j) {
        double d = get(A, n, j, j).real();
        for (int k = 0; k < j; ++k) d -= std::norm(get(A, n, j, k));
        if (!(d > 0.0) || !std::isfinite(d)) return false;
        const double ljj = std::sqrt(d);
        put(A, n, j, j, cd(ljj, 0.0));
        for (int i = j + 1; i < n; ++i) {
            cd s = get(A, n, i, j);
            for (int k = 0; k < j; ++k) s -= get(A, n, i, k) * std::conj(get(A, n, j, k));
            put(A, n, i, j, s / ljj);
        }
        for (int i = 0; i < j; ++i) put(A, n, i, j, cd(0.0, 0.0));  // clear the upper triangle
    }
    return true;
}

void host_inv_lower_dag(int n, const std::vector<HostCplx>& L, std::vector<HostCplx>& R) {
    // X = L^{-1} (lower) by forward substitution, column by column; R = X^+.
    std::vector<cd> X((size_t)n * n, cd(0.0, 0.0));
    for (int c = 0; c < n; ++c) {
        for (int i = c; i < n; ++i) {
            cd s = (i == c) ? cd(1.0, 0.0) : cd(0.0, 0.0);
            for (int k = c; k < i; ++k) s -= get(L, n, i, k) * X[k + (size_t)c * n];
            X[i + (size_t)c * n] = s / get(L, n, i, i);
        }
    }
    R.assign((size_t)n * n, HostCplx{0.0, 0.0});
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) put(R, n, i, j, std::conj(X[j + (size_t)i * n]));
}

void host_eigh(int n, std::vector<HostCplx>& Ain, std::vector<double>& w, std::vector<HostCplx>& Zout) {
    // Cyclic Jacobi for a Hermitian matrix.  Each rotation J acts on columns p, q:
    // with a_pq = r e^{i phi}, D = diag(1, e^{-i phi}) makes the (p, q) block real,
    // and the real rotation [[c, s], [-s, c]] with tan(2 theta) = 2 r / (a_qq - a_pp)
    // zeroes it; A <- J^+ A J and Z <- Z J.
    std::vector<cd> A((size_t)n * n), Z((size_t)n * n, cd(0.0, 0.0));
    for (size_t k = 0; k < A.size(); ++k) A[k] = cd(Ain[k].re, Ain[k].im);
    for (int i = 0; i < n; ++i) Z[i + (size_t)i * n] = 1.0;
    auto at = [&](int i, int j) -> cd& { return A[i + (size_t)j * n]; };
    double fro = 0.0;
    for (auto& v : A) fro += std::norm(v);
    fro = std::sqrt(fro);
    for (int sweep = 0; sweep < 100; ++sweep) {
        double off = 0.0;
        for (int j = 0; j < n; ++j)
            for (int i = 0; i < n; ++i)
                if (i != j) off += std::norm(at(i, j));
        if (std::sqrt(off) <= 1e-15 * fro || fro == 0.0) break;
        for (int p = 0; p < n - 1; ++p) {
            for (int q = p + 1; q < n; ++q) {
                const cd apq = at(p, q);
                const double r = std::abs(apq);
                if (r <= 1e-300) continue;
                const cd e = apq / r;  // e^{i phi}
                const double app = at(p, p).real(), aqq = at(q, q).real();
                const double theta = 0.5 * std::atan2(2.0 * r, aqq - app);
                const double c = std::cos(theta), s = std::sin(theta);
                const cd em = std::conj(e);  // e^{-i phi}
                // columns: col_p' = c col_p - s e^{-i phi} col_q ; col_q' = s col_p + c e^{-i phi} col_q
                for (int k = 0; k < n; ++k) {
                    const cd akp = at(k, p), akq = at(k, q);
                    at(k, p) = c * akp - s * em * akq;
                    at(k, q) = s * akp + c * em * akq;
                    const cd zkp = Z[k + (size_t)p * n], zkq = Z[k + (size_t)q * n];
                    Z[k + (size_t)p * n] = c * zkp - s * em * zkq;
                    Z[k + (size_t)q * n] = s * zkp + c * em * zkq;
                }
                // rows: row_p' = c row_p - s e^{i phi} row_q ; row_q' = s row_p + c e^{i phi} row_q
                for (int k = 0; k < n; ++k) {
                    const cd apk = at(p, k), aqk = at(q, k);
                    at(p, k) = c * apk - s * e * aqk;
                    at(q, k) = s * apk + c * e * aqk;
                }
                at(p, q) = 0.0;
                at(q, p) = 0.0;
                at(p, p) = cd(at(p, p).real(), 0.0);
                at(q, q) = cd(at(q, q).real(), 0.0);
            }
        }
    }
    std::vector<int> order(n);
    std::iota(order.begin(), order.end(), 0);
    std::sort(order.begin(), order.end(), [&](int a, int b) { return at(a, a).real() < at(b, b).real(); });
    w.resize(n);
    Zout.assign((size_t)n * n, HostCplx{0.0, 0.0});
    for (int j = 0; j < n; ++j) {
        w[j] = at(order[j], order[j]).real();
        for (int i = 0; i < n; ++i) {
            const cd v = Z[i + (size_t)order[j] * n];
            Zout[i + (size_t)j * n] = HostCplx{v.real(), v.imag()};
        }
    }
    for (size_t k = 0; k < A.size(); ++k) Ain[k] = HostCplx{A[k].real(), A[k].imag()};
}

namespace {
// Interpolation at the Chebyshev-Gauss nodes y_j = cos(theta_j), theta_j = pi (j + 1/2)/(n + 1),
// mapped to x_j = ((1 - eps) y_j + 1 + eps)/2 in [eps, 1].
template <typename F>
void cheb_interp(int n, double eps, F f, double* out) {
    const double pi = std::acos(-1.0);
    std::vector<double> fv(n + 1), th(n + 1);
    for (int j = 0; j <= n; ++j) {
        th[j] = pi * (j + 0.5) / (n + 1);
        fv[j] = f(((1.0 - eps) * std::cos(th[j]) + 1.0 + eps) / 2.0);
    }
    for (int k = 0; k <= n; ++k) {
        double s = 0.0;
        for (int j = 0; j <= n; ++j) s += fv[j] * std::cos(k * th[j]);
        out[k] = 2.0 * s / (n + 1);
    }
    out[0] *= 0.5;
}
}  // namespace

void host_chebyshev_coeffs(int n, double eps, double* out) {
    cheb_interp(n, eps, [](double x) { return 1.0 / std::sqrt(x); }, out);
}

void host_chebyshev_coeffs_shifted_inverse_root(int n, double eps, double a, double* out) {
    cheb_interp(n, eps, [a](double x) { return 1.0 / (a + std::sqrt(x)); }, out);
}

namespace {
// P(y) = sum_k c_k T_k(y) by Clenshaw.
double cheb_sum(const double* c, int n, double y) {
    double b1 = 0.0, b2 = 0.0;
    for (int k = n; k >= 1; --k) {
        const double b0 = c[k] + 2.0 * y * b1 - b2;
        b2 = b1;
        b1 = b0;
    }
    return c[0] + y * b1 - b2;
}

// Solve A z = r in place (A row-major m x m, destroyed; r becomes z); Gaussian elimination
// with partial pivoting.  False if A is singular to working precision.
bool lu_solve(int m, std::vector<double>& A, std::vector<double>& r) {
    for (int k = 0; k < m; ++k) {
        int piv = k;
        for (int i = k + 1; i < m; ++i)
            if (std::fabs(A[(size_t)i * m + k]) > std::fabs(A[(size_t)piv * m + k])) piv = i;
        if (!(std::fabs(A[(size_t)piv * m + k]) > 0.0)) return false;
        if (piv != k) {
            for (int j = 0; j < m; ++j) std::swap(A[(size_t)k * m + j], A[(size_t)piv * m + j]);
            std::swap(r[k], r[piv]);
        }
        const double inv = 1.0 / A[(size_t)k * m + k];
        for (int i = k + 1; i < m; ++i) {
            const double f = A[(size_t)i * m + k] * inv;
            if (f == 0.0) continue;
            double* ri = &A[(size_t)i * m];
            const double* rk = &A[(size_t)k * m];
            for (int j = k; j < m; ++j) ri[j] -= f * rk[j];
            r[i] -= f * r[k];
        }
    }
    for (int k = m - 1; k >= 0; --k) {
        double s = r[k];
        for (int j = k + 1; j < m; ++j) s -= A[(size_t)k * m + j] * r[j];
        r[k] = s / A[(size_t)k * m + k];
    }
    return true;
}
}  // namespace

double host_minimax_coeffs(int n, double eps, double* out) {
    // Remez exchange for min over P of max over [eps, 1] of |1 - sqrt(x) P(x)|, P = sum_k c_k T_k(y),
    // y = (2x - 1 - eps)/(1 - eps) = -cos(theta).  Reference: n + 2 angles; levelled system
    // sqrt(x_i) P(x_i) + s_i E = 1 with alternating s_i; next reference: the alternating extrema of
    // the error on a grid of 64 points per oscillation, each refined by a parabola in theta.
    const double pi = std::acos(-1.0);
    const int m = n + 2;
    std::vector<double> th(m), sg(m), c(n + 1, 0.0);
    for (int i = 0; i < m; ++i) {
        th[i] = pi * i / (n + 1);
        sg[i] = (i % 2 == 0) ? 1.0 : -1.0;
    }
    const int G = 64 * m;
    const double h = pi / G;
    auto err_at = [&](double t) {
        const double y = -std::cos(t);
        const double x = ((1.0 - eps) * y + 1.0 + eps) / 2.0;
        return 1.0 - std::sqrt(x) * cheb_sum(c.data(), n, y);
    };
    double delta = 1.0, last_gap = 1e300;
    std::vector<double> e(G + 1);
    for (int it = 0; it < 80; ++it) {
        std::vector<double> A((size_t)m * m), r(m, 1.0);
        for (int i = 0; i < m; ++i) {
            const double y = -std::cos(th[i]);
            const double sx = std::sqrt(((1.0 - eps) * y + 1.0 + eps) / 2.0);
            double t0 = 1.0, t1 = y;
            for (int k = 0; k <= n; ++k) {
                const double tk = (k == 0) ? 1.0 : (k == 1 ? y : 2.0 * y * t1 - t0);
                if (k >= 2) {
                    t0 = t1;
                    t1 = tk;
                }
                A[(size_t)i * m + k] = sx * tk;
            }
            A[(size_t)i * m + n + 1] = sg[i];
        }
        if (!lu_solve(m, A, r)) break;
        for (int k = 0; k <= n; ++k) c[k] = r[k];
        const double E = std::fabs(r[n + 1]);
        for (int j = 0; j <= G; ++j) e[j] = err_at(h * j);
        // extrema (ends included), refined, then reduced to an alternating sequence
        std::vector<double> at, av;
        for (int j = 0; j <= G; ++j) {
            const bool end = (j == 0 || j == G);
            if (!end && !((e[j] - e[j - 1]) * (e[j + 1] - e[j]) <= 0.0 && e[j] != e[j - 1])) continue;
            double t = h * j;
            if (!end) {
                const double den = e[j - 1] - 2.0 * e[j] + e[j + 1];
                if (den != 0.0) t += 0.5 * h * (e[j - 1] - e[j + 1]) / den;
            }
            const double v = err_at(t);
            if (!av.empty() && ((v > 0.0) == (av.back() > 0.0))) {
                if (std::fabs(v) > std::fabs(av.back())) {
                    at.back() = t;
                    av.back() = v;
                }
            } else {
                at.push_back(t);
                av.push_back(v);
            }
        }
        while ((int)at.size() > m) {
            if (std::fabs(av.front()) < std::fabs(av.back())) {
                at.erase(at.begin());
                av.erase(av.begin());
            } else {
                at.pop_back();
                av.pop_back();
            }
        }
        delta = 0.0;
        for (double v : av) delta = std::max(delta, std::fabs(v));
        if ((int)at.size() < m) break;
        for (int i = 0; i < m; ++i) {
            th[i] = at[i];
            sg[i] = av[i] > 0.0 ? 1.0 : -1.0;
        }
        // levelled: the gap between the largest error and E is at the rounding of the error
        // function (~1e-14 absolute at delta ~ 1e-10), so also stop once it no longer halves
        const double gap = (delta - E) / E;
        if (gap <= 1e-6 || (gap < 1e-3 && gap > 0.5 * last_gap)) break;
        last_gap = gap;
    }
    for (int k = 0; k <= n; ++k) out[k] = c[k];
    return delta;
}

double host_poly_delta(const double* coeffs, int n, double eps) {
    // max |1 - sqrt(x) P(x)| on a grid uniform in the Chebyshev angle (Clenshaw in FP64)
    const int ng = 4096;
    double worst = 0.0;
    for (int q = 0; q <= ng; ++q) {
        const double y = std::cos(3.141592653589793 * q / ng);
        double b1 = 0.0, b2 = 0.0;
        for (int k = n; k >= 1; --k) {
            const double b0 = coeffs[k] + 2.0 * y * b1 - b2;
            b2 = b1;
            b1 = b0;
        }
        const double P = coeffs[0] + y * b1 - b2;
        const double x = ((1.0 - eps) * y + 1.0 + eps) / 2.0;
        worst = std::max(worst, std::fabs(1.0 - std::sqrt(x) * P));
    }
    return worst;
}

}  // namespace ovl
