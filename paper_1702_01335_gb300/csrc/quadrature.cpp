// Host-side velocity quadratures and Hermite bases of the solver (FP64).
//
// Sec. III builds the velocity set from Gauss-Hermite rules for the weight
// omega(p) = exp(-p^2/2)/sqrt(2 pi) of Eq. (H_omega): a full-range rule on the
// axes parallel to the walls (sum w = 1) and a half-range rule on each
// semi-axis of the wall-normal axis (nodes on (0, inf), sum w = 1/2).
//
// Algorithms:
//   * recurrence coefficients: full range is closed form (alpha = 0,
//     beta_k = k); half range uses the discretised Stieltjes procedure on a
//     composite Gauss-Legendre discretisation of omega on (0, 38), with the
//     polynomials kept orthonormal so nothing overflows at degree 64+;
//   * nodes: eigenvalues of the Jacobi matrix by Sturm-sequence bisection,
//     polished by Newton steps on the degree-Q orthonormal polynomial;
//   * weights: Christoffel numbers w_j = 1 / sum_k phat_k(x_j)^2, which keep
//     full relative precision even for weights near 1e-70.
#include "lbs_internal.h"

#include <algorithm>
#include <cmath>
#include <vector>

namespace lbs {

static const double kSqrt2Pi = 2.5066282746310002;

// n-point Gauss-Legendre rule on [-1, 1] (Newton on the Legendre recurrence).
static void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w)
{
    x.assign(n, 0.0);
    w.assign(n, 0.0);
    for (int i = 0; i < n; ++i) {
        double z = std::cos(M_PI * (i + 0.75) / (n + 0.5));
        double dp = 0.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= n; ++k) {
                double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            dp = n * (z * p1 - p0) / (z * z - 1.0);
            double dz = p1 / dp;
            z -= dz;
            if (std::fabs(dz) < 1e-16) break;
        }
        double p0 = 1.0, p1 = z;
        for (int k = 2; k <= n; ++k) {
            double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
            p0 = p1;
            p1 = p2;
        }
        dp = n * (z * p1 - p0) / (z * z - 1.0);
        x[i] = z;
        w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
}

void recurrence(int kind, int n, std::vector<double>& alpha, std::vector<double>& beta)
{
    alpha.assign(n, 0.0);
    beta.assign(n, 0.0);
    if (kind == QUAD_FULL) {
        beta[0] = 1.0;
        for (int k = 1; k < n; ++k) beta[k] = k;
        return;
    }
    // discretised measure: 64 panels of 32-point Gauss-Legendre on [0, 38]
    const int panels = 64, pts = 32;
    const double pmax = 38.0, hw = 0.5 * pmax / panels;
    std::vector<double> gx, gw;
    gauss_legendre(pts, gx, gw);
    std::vector<double> x, w;
    for (int p = 0; p < panels; ++p)
        for (int i = 0; i < pts; ++i) {
            double xx = (2 * p + 1) * hw + hw * gx[i];
            x.push_back(xx);
            w.push_back(hw * gw[i] * std::exp(-0.5 * xx * xx) / kSqrt2Pi);
        }
    const size_t M = x.size();
    // orthonormal Stieltjes: q_{-1} = 0, q_0 = 1/sqrt(beta0)
    std::vector<double> qm(M, 0.0), q(M), qn(M);
    double b0 = 0.0;
    for (size_t d = 0; d < M; ++d) b0 += w[d];
    beta[0] = b0;
    for (size_t d = 0; d < M; ++d) q[d] = 1.0 / std::sqrt(b0);
    double sb = 0.0;  // sqrt(beta_k)
    for (int k = 0; k < n; ++k) {
        double a = 0.0;
        for (size_t d = 0; d < M; ++d) a += w[d] * x[d] * q[d] * q[d];
        alpha[k] = a;
        double nrm = 0.0;
        for (size_t d = 0; d < M; ++d) {
            qn[d] = (x[d] - a) * q[d] - sb * qm[d];
            nrm += w[d] * qn[d] * qn[d];
        }
        if (k + 1 < n) beta[k + 1] = nrm;
        sb = std::sqrt(nrm);
        for (size_t d = 0; d < M; ++d) {
            qm[d] = q[d];
            q[d] = qn[d] / sb;
        }
    }
}

// orthonormal phat_0..phat_{n-1} at x (and derivative of phat_{n-1} if dlast).
static void orthonormal_at(double x, const std::vector<double>& a, const std::vector<double>& b,
                           int n, std::vector<double>& P, double* dlast)
{
    P.assign(n, 0.0);
    std::vector<double> D(n, 0.0);
    P[0] = 1.0 / std::sqrt(b[0]);
    if (n > 1) {
        P[1] = (x - a[0]) * P[0] / std::sqrt(b[1]);
        D[1] = P[0] / std::sqrt(b[1]);
    }
    for (int k = 1; k + 1 < n; ++k) {
        double sk = std::sqrt(b[k]), sk1 = std::sqrt(b[k + 1]);
        P[k + 1] = ((x - a[k]) * P[k] - sk * P[k - 1]) / sk1;
        D[k + 1] = (P[k] + (x - a[k]) * D[k] - sk * D[k - 1]) / sk1;
    }
    if (dlast) *dlast = D[n - 1];
}

// number of eigenvalues of the Jacobi matrix (first Q rows) below x
static int sturm_count(double x, const std::vector<double>& a, const std::vector<double>& b, int Q)
{
    int cnt = 0;
    double d = 1.0;
    for (int i = 0; i < Q; ++i) {
        double off = (i == 0) ? 0.0 : b[i] / d;  // b[i] = (sqrt beta_i)^2
        d = a[i] - x - off;
        if (d == 0.0) d = -1e-300;
        if (d < 0.0) ++cnt;
    }
    return cnt;
}

int gauss_rule(int kind, int Q, double* nodes, double* weights)
{
    if (Q < 1 || Q > kMaxQ1D) return -1;
    std::vector<double> a, b;
    recurrence(kind, Q + 1, a, b);
    double lo = 1e300, hi = -1e300;
    for (int i = 0; i < Q; ++i) {
        double r = (i > 0 ? std::sqrt(b[i]) : 0.0) + (i + 1 < Q ? std::sqrt(b[i + 1]) : 0.0);
        lo = std::min(lo, a[i] - r);
        hi = std::max(hi, a[i] + r);
    }
    std::vector<double> P;
    for (int j = 0; j < Q; ++j) {
        double l = lo, h = hi;  // eigenvalue j: count(<x) passes from j to j+1
        for (int it = 0; it < 200 && h - l > 1e-16 * std::max(1.0, std::fabs(h)); ++it) {
            double m = 0.5 * (l + h);
            if (sturm_count(m, a, b, Q) > j) h = m; else l = m;
        }
        double x = 0.5 * (l + h);
        for (int it = 0; it < 3; ++it) {
            double d;
            orthonormal_at(x, a, b, Q + 1, P, &d);
            if (d != 0.0) x -= P[Q] / d;
        }
        orthonormal_at(x, a, b, Q, P, nullptr);
        double s = 0.0;
        for (int k = 0; k < Q; ++k) s += P[k] * P[k];
        nodes[j] = x;
        weights[j] = 1.0 / s;
    }
    return 0;
}

// He_l(p)/l! for l = 0..N (probabilists' Hermite, Eq. H_ortho normalisation):
// with h_l = He_l / l!, He_{l+1} = p He_l - l He_{l-1} gives
// h_{l+1} = (p h_l - h_{l-1}) / (l + 1).
void hermite_basis(const double* p, int Q, int N, double* out)
{
    for (int i = 0; i < Q; ++i) {
        double hm = 0.0, h = 1.0;
        out[i * (N + 1)] = 1.0;
        for (int l = 0; l < N; ++l) {
            double hn = (p[i] * h - hm) / (l + 1.0);
            hm = h;
            h = hn;
            out[i * (N + 1) + l + 1] = h;
        }
    }
}

// pi_l(xi)/h_l for the monic half-range polynomials, h_l = beta_0 ... beta_l
void half_basis(const double* xi, int Q, int N, const std::vector<double>& a,
                const std::vector<double>& b, double* out)
{
    for (int m = 0; m < Q; ++m) {
        double pm = 0.0, p = 1.0, h = b[0];
        out[m * (N + 1)] = p / h;
        for (int l = 0; l < N; ++l) {
            double pn = (xi[m] - a[l]) * p - (l > 0 ? b[l] * pm : 0.0);
            pm = p;
            p = pn;
            h *= b[l + 1];
            out[m * (N + 1) + l + 1] = p / h;
        }
    }
}

}  // namespace lbs
