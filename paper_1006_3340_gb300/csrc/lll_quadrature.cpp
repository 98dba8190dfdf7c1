// lll_quadrature.cpp -- Gauss rule of the weight x^2 nu(x) on [-a, a] (host, FP64).
//
// The drift of Eq. (LIBOR-drift-PT) integrates an O(x^2) function against the
// Levy measure, so it is written against the bounded weight m(x) = x^2 nu(x):
// int g dF ~= sum_j W_j g(x_j) / x_j^2.  For NIG (Section 4 gives kappa;
// the density is Barndorff-Nielsen's)
//     m(x) = (dbar alpha / pi) |x| e^{beta x} K_1(alpha |x|).
// Steps: (1) discretise m with a composite Gauss-Legendre rule on panels
// graded geometrically towards the origin; (2) Stieltjes recurrence for the
// orthonormal polynomials of the discrete measure, with full
// re-orthogonalisation; (3) nodes = eigenvalues of the Jacobi matrix by
// Sturm-sequence bisection; (4) weights = Christoffel numbers
// 1 / sum_k p_k(x_j)^2.
#include <algorithm>
#include <cmath>
#include <vector>

namespace lll {
namespace {

// Gauss-Legendre nodes/weights on [-1, 1] by Newton iteration on P_G.
void gauss_legendre(int G, std::vector<double> &t, std::vector<double> &w)
{
    t.assign(G, 0.0);
    w.assign(G, 0.0);
    for (int i = 0; i < (G + 1) / 2; ++i) {
        double z = std::cos(M_PI * (i + 0.75) / (G + 0.5));
        double dp = 0.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= G; ++k) {
                const double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            dp = G * (z * p1 - p0) / (z * z - 1.0);
            const double dz = p1 / dp;
            z -= dz;
            if (std::fabs(dz) < 1e-16) break;
        }
        t[i] = -z;
        t[G - 1 - i] = z;
        w[i] = w[G - 1 - i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
}

double x2nu(double x, double alpha, double beta, double dbar)
{
    const double ax = std::fabs(x);
    if (ax == 0.0) return dbar / M_PI;
    return dbar * alpha / M_PI * ax * std::exp(beta * x) * std::cyl_bessel_k(1.0, alpha * ax);
}

}  // namespace

// Returns 0 on success.
int build_nig_rule(double alpha, double beta, double dbar, double a, int Q, double *nodes,
                   double *weights)
{
    const int G = 32;
    std::vector<double> gt, gw;
    gauss_legendre(G, gt, gw);
    std::vector<double> edges;
    edges.push_back(0.0);
    const int outer = 24;
    for (double e = 1e-14 * a; e < a / outer; e /= 0.35) edges.push_back(e);
    for (int i = 1; i <= outer; ++i) edges.push_back(a * i / outer);
    std::vector<double> y, v;
    for (int side = -1; side <= 1; side += 2)
        for (size_t p = 0; p + 1 < edges.size(); ++p) {
            const double lo = edges[p], hi = edges[p + 1];
            const double mid = 0.5 * (lo + hi), half = 0.5 * (hi - lo);
            for (int g = 0; g < G; ++g) {
                const double xx = side * (mid + half * gt[g]);
                y.push_back(xx);
                v.push_back(half * gw[g] * x2nu(xx, alpha, beta, dbar));
            }
        }
    const size_t M = y.size();
    // Stieltjes with orthonormal vectors q_k(y_i) sqrt(v_i).
    std::vector<double> al(Q, 0.0), bt(Q + 1, 0.0);
    double mu0 = 0.0;
    for (size_t i = 0; i < M; ++i) mu0 += v[i];
    if (!(mu0 > 0.0)) return -1;
    std::vector<std::vector<double>> qs;
    std::vector<double> q(M), r(M);
    for (size_t i = 0; i < M; ++i) q[i] = std::sqrt(v[i] / mu0);
    qs.push_back(q);
    for (int k = 0; k < Q; ++k) {
        const std::vector<double> &qk = qs[k];
        double a_k = 0.0;
        for (size_t i = 0; i < M; ++i) a_k += y[i] * qk[i] * qk[i];
        al[k] = a_k;
        if (k + 1 == Q) break;
        for (size_t i = 0; i < M; ++i)
            r[i] = (y[i] - a_k) * qk[i] - (k > 0 ? bt[k] * qs[k - 1][i] : 0.0);
        for (int pass = 0; pass < 2; ++pass)
            for (const auto &qq : qs) {
                double d = 0.0;
                for (size_t i = 0; i < M; ++i) d += qq[i] * r[i];
                for (size_t i = 0; i < M; ++i) r[i] -= d * qq[i];
            }
        double nr = 0.0;
        for (size_t i = 0; i < M; ++i) nr += r[i] * r[i];
        nr = std::sqrt(nr);
        if (!(nr > 0.0)) return -2;
        bt[k + 1] = nr;
        for (size_t i = 0; i < M; ++i) r[i] /= nr;
        qs.push_back(r);
    }
    // Eigenvalues of the Jacobi matrix by bisection on Sturm counts.
    double lo = al[0], hi = al[0];
    for (int k = 0; k < Q; ++k) {
        const double rad = (k > 0 ? bt[k] : 0.0) + (k + 1 < Q ? bt[k + 1] : 0.0);
        lo = std::min(lo, al[k] - rad);
        hi = std::max(hi, al[k] + rad);
    }
    auto count_below = [&](double lam) {
        int cnt = 0;
        double d = 1.0;
        for (int k = 0; k < Q; ++k) {
            const double off = k > 0 ? bt[k] * bt[k] : 0.0;
            d = al[k] - lam - (k > 0 ? off / d : 0.0);
            if (d == 0.0) d = -1e-300;
            if (d < 0.0) ++cnt;
        }
        return cnt;
    };
    for (int j = 0; j < Q; ++j) {
        double a0 = lo, b0 = hi;
        for (int it = 0; it < 200 && b0 - a0 > 0.0; ++it) {
            const double mid = 0.5 * (a0 + b0);
            if (mid <= a0 || mid >= b0) break;
            if (count_below(mid) > j) b0 = mid;
            else a0 = mid;
        }
        nodes[j] = 0.5 * (a0 + b0);
    }
    // Christoffel numbers from the orthonormal recurrence.
    for (int j = 0; j < Q; ++j) {
        const double xx = nodes[j];
        double pm = 0.0, pc = 1.0 / std::sqrt(mu0), s = pc * pc;
        for (int k = 0; k + 1 < Q; ++k) {
            const double pn = ((xx - al[k]) * pc - (k > 0 ? bt[k] * pm : 0.0)) / bt[k + 1];
            pm = pc;
            pc = pn;
            s += pc * pc;
        }
        weights[j] = 1.0 / s;
    }
    return 0;
}

}  // namespace lll
