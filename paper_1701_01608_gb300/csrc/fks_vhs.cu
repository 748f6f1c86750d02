// fks_vhs.cu -- separable expansion of the variable-hard-sphere kernel.
//
// Method: arXiv 1701.01608, Appendix A.  The fast form of the spectral
// operator needs a Carleman kernel B~(|x|, |y|) = a(|x|) b(|y|); Eq.
// Btilde_pl gives B~ = 4C (|x|^2 + |y|^2)^((alpha-1)/2) for the collision
// kernel B = C |g|^alpha, a product only for alpha = 1 (hard spheres).
// For other alpha the direction-p factor of B_F(l, m) is the radial double
// integral
//   H(t, u) = int_0^R int_0^R [2 r cos(r t)] B~(r, r') [2 pi r' J0(r' u)] dr dr'.
// On a radial quadrature (nodes r_i, weights w_i) it is a bilinear form
//   H = sum_ij c_i(t) K_ij d_j(u),  c_i = 2 sqrt(w_i) cos(r_i t),
//   d_j = 2 pi sqrt(w_j) J0(r_j u),  K_ij = sqrt(w_i) r_i B~(r_i, r_j) r_j sqrt(w_j),
// and the eigen-decomposition K = sum_s lambda_s u_s u_s^T (K is symmetric;
// positive semi-definite for alpha <= 1, B~ being completely monotone in
// r^2 + r'^2) turns it into S separable terms
//   H ~ sum_{s<S} phi_s(t) psi_s(u),
//   phi_s(t) = sum_i ca[s][i] cos(r_i t),  ca[s][i] = sgn(l_s) sqrt|l_s| 2 sqrt(w_i) u_s[i]
//   psi_s(u) = sum_j cb[s][j] J0(r_j u),   cb[s][j] = sqrt|l_s| 2 pi sqrt(w_j) u_s[j]
// keeping the S largest |lambda_s|.  Each term is one more pair of tables
// per direction, so the collision kernels run the same code with M S
// directions.  S is the smallest count whose factor differs from the full
// bilinear form by at most tol max|H| on a grid of (t, u) covering the
// frequencies of the n^3 grid.
#include <algorithm>
#include <cmath>
#include <numeric>
#include <string>
#include <vector>

#include "fks_internal.h"

namespace fks {

namespace {

constexpr double kPi = 3.14159265358979323846;

// Gauss-Legendre rule with m nodes on [a, b] (Newton on the Legendre recurrence)
void legendre_rule(int m, double a, double b, double* x, double* w) {
    for (int i = 0; i < m; ++i) {
        double z = std::cos(kPi * (i + 0.75) / (m + 0.5));
        double dp = 0.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= m; ++k) {
                const double p2 = ((2 * k - 1) * z * p1 - (k - 1) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            dp = m * (z * p1 - p0) / (z * z - 1.0);
            const double dz = p1 / dp;
            z -= dz;
            if (std::fabs(dz) < 1e-16) break;
        }
        x[i] = 0.5 * (b - a) * z + 0.5 * (b + a);
        w[i] = (b - a) / ((1.0 - z * z) * dp * dp);
    }
}

// Radial rule on [0, R]: 16 Gauss nodes on [R/3, 2R/3] and [2R/3, R], and
// 10 on each of 12 panels of [0, R/3] halving towards 0 (the last reaching 0)
// for the corner r = r' = 0 where B~ is singular when alpha < 1.
void radial_rule(double R, std::vector<double>& r, std::vector<double>& w) {
    constexpr int kTop = 16, kLow = 10, kLevels = 12;
    r.clear();
    w.clear();
    double x[kTop], wt[kTop];
    for (int j = 1; j <= 2; ++j) {
        legendre_rule(kTop, j * R / 3.0, (j + 1) * R / 3.0, x, wt);
        r.insert(r.end(), x, x + kTop);
        w.insert(w.end(), wt, wt + kTop);
    }
    double b = R / 3.0;
    for (int lev = 0; lev < kLevels; ++lev) {
        const double a = lev < kLevels - 1 ? 0.5 * b : 0.0;
        legendre_rule(kLow, a, b, x, wt);
        r.insert(r.end(), x, x + kLow);
        w.insert(w.end(), wt, wt + kLow);
        b = a;
    }
}

// Cyclic Jacobi eigen-decomposition of the symmetric n x n matrix A (row-major,
// destroyed): eigenvalues in lam, eigenvectors in the columns of V.
void jacobi_eigen(int n, std::vector<double>& A, std::vector<double>& lam, std::vector<double>& V) {
    V.assign((size_t)n * n, 0.0);
    for (int i = 0; i < n; ++i) V[(size_t)i * n + i] = 1.0;
    auto a = [&](int i, int j) -> double& { return A[(size_t)i * n + j]; };
    for (int sweep = 0; sweep < 100; ++sweep) {
        double off = 0.0, diag = 0.0;
        for (int i = 0; i < n; ++i) {
            diag += a(i, i) * a(i, i);
            for (int j = i + 1; j < n; ++j) off += a(i, j) * a(i, j);
        }
        if (off <= 1e-30 * diag) break;
        for (int p = 0; p < n; ++p)
            for (int q = p + 1; q < n; ++q) {
                const double apq = a(p, q);
                if (std::fabs(apq) < 1e-300) continue;
                // rotation that zeroes A[p][q]
                const double theta = (a(q, q) - a(p, p)) / (2.0 * apq);
                const double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
                const double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
                for (int k = 0; k < n; ++k) {
                    const double akp = a(k, p), akq = a(k, q);
                    a(k, p) = c * akp - s * akq;
                    a(k, q) = s * akp + c * akq;
                }
                for (int k = 0; k < n; ++k) {
                    const double apk = a(p, k), aqk = a(q, k);
                    a(p, k) = c * apk - s * aqk;
                    a(q, k) = s * apk + c * aqk;
                }
                for (int k = 0; k < n; ++k) {
                    const double vkp = V[(size_t)k * n + p], vkq = V[(size_t)k * n + q];
                    V[(size_t)k * n + p] = c * vkp - s * vkq;
                    V[(size_t)k * n + q] = s * vkp + c * vkq;
                }
            }
    }
    lam.resize(n);
    for (int i = 0; i < n; ++i) lam[i] = a(i, i);
}

}  // namespace

fks_status vhs_expand(double alpha, double C, double L, int n, double tol, int terms, VhsExpansion* out,
                      std::string* err) {
    if (!(alpha >= -1.0 && alpha <= 1.0) || !(C > 0.0) || !(L > 0.0) || n < 1 || terms < 0 || terms > kVhsMaxTerms) {
        *err = "VHS expansion: alpha must lie in [-1, 1], C > 0, 0 <= terms <= 64";
        return FKS_ERR_INVALID_ARG;
    }
    const double R = 2.0 / (3.0 + std::sqrt(2.0)) * L;
    std::vector<double> r, w;
    radial_rule(R, r, w);
    const int Q = (int)r.size();
    std::vector<double> K((size_t)Q * Q);
    for (int i = 0; i < Q; ++i)
        for (int j = 0; j < Q; ++j)
            K[(size_t)i * Q + j] = std::sqrt(w[i] * w[j]) * r[i] * r[j] * 4.0 * C *
                                   std::pow(r[i] * r[i] + r[j] * r[j], 0.5 * (alpha - 1.0));
    std::vector<double> lam, V;
    jacobi_eigen(Q, K, lam, V);
    std::vector<int> order(Q);
    std::iota(order.begin(), order.end(), 0);
    std::sort(order.begin(), order.end(), [&](int a, int b) { return std::fabs(lam[a]) > std::fabs(lam[b]); });

    // truncation error of S terms on a (t, u) grid up to the largest |xi| of the n^3 grid
    constexpr int kG = 48;
    const double tmax = kPi / L * (0.5 * n) * std::sqrt(3.0);
    std::vector<double> Y((size_t)kG * Q), Z((size_t)kG * Q);   // [grid][s]
    for (int g = 0; g < kG; ++g) {
        const double t = tmax * g / (kG - 1);
        for (int s = 0; s < Q; ++s) {
            const int e = order[s];
            double y = 0.0, z = 0.0;
            for (int i = 0; i < Q; ++i) {
                y += 2.0 * std::sqrt(w[i]) * std::cos(r[i] * t) * V[(size_t)i * Q + e];
                z += 2.0 * kPi * std::sqrt(w[i]) * j0(r[i] * t) * V[(size_t)i * Q + e];
            }
            Y[(size_t)g * Q + s] = y;
            Z[(size_t)g * Q + s] = z;
        }
    }
    std::vector<double> Hfull((size_t)kG * kG, 0.0), Hs((size_t)kG * kG, 0.0);
    for (int s = 0; s < Q; ++s) {
        const double l = lam[order[s]];
        for (int a = 0; a < kG; ++a)
            for (int b = 0; b < kG; ++b) Hfull[(size_t)a * kG + b] += l * Y[(size_t)a * Q + s] * Z[(size_t)b * Q + s];
    }
    double hmax = 0.0;
    for (double v : Hfull) hmax = std::max(hmax, std::fabs(v));
    const int smax = std::min(Q, kVhsMaxTerms);
    int S = 0;
    double e_s = 0.0;
    for (int s = 0; s < smax; ++s) {
        const double l = lam[order[s]];
        for (int a = 0; a < kG; ++a)
            for (int b = 0; b < kG; ++b) Hs[(size_t)a * kG + b] += l * Y[(size_t)a * Q + s] * Z[(size_t)b * Q + s];
        double dmax = 0.0;
        for (size_t k = 0; k < Hs.size(); ++k) dmax = std::max(dmax, std::fabs(Hs[k] - Hfull[k]));
        e_s = dmax / hmax;
        S = s + 1;
        if (terms > 0 ? S == terms : e_s <= tol) break;
    }
    out->S = S;
    out->Q = Q;
    out->err = e_s;
    out->r = r;
    out->ca.assign((size_t)S * Q, 0.0);
    out->cb.assign((size_t)S * Q, 0.0);
    out->lambda.resize(S);
    for (int s = 0; s < S; ++s) {
        const int e = order[s];
        const double l = lam[e], sl = std::sqrt(std::fabs(l)), sg = l < 0 ? -1.0 : 1.0;
        out->lambda[s] = l;
        for (int i = 0; i < Q; ++i) {
            out->ca[(size_t)s * Q + i] = sg * sl * 2.0 * std::sqrt(w[i]) * V[(size_t)i * Q + e];
            out->cb[(size_t)s * Q + i] = sl * 2.0 * kPi * std::sqrt(w[i]) * V[(size_t)i * Q + e];
        }
    }
    return FKS_OK;
}

}  // namespace fks

extern "C" fks_status fks_vhs_factor(double alpha, double C, double L, int n, int precision, int terms, double t,
                                     double u, double* H, int* S, double* trunc_err) {
    if (!H || (precision != FKS_FP64 && precision != FKS_FP32 && precision != FKS_BF16X3)) return FKS_ERR_INVALID_ARG;
    fks::VhsExpansion x;
    std::string err;
    const fks_status st = fks::vhs_expand(alpha, C, L, n, fks::vhs_tolerance(precision), terms, &x, &err);
    if (st != FKS_OK) return st;
    double h = 0.0;
    for (int s = 0; s < x.S; ++s) h += fks::vhs_phi(x.ca.data() + (size_t)s * x.Q, x.r.data(), x.Q, t) *
                                       fks::vhs_psi(x.cb.data() + (size_t)s * x.Q, x.r.data(), x.Q, u);
    *H = h;
    if (S) *S = x.S;
    if (trunc_err) *trunc_err = x.err;
    return FKS_OK;
}
