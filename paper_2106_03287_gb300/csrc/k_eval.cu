// Distribution quality measures of the experiments: the paper scores an
// estimated pose distribution against a Monte Carlo reference (many SGD-ICP
// runs from spread initial poses) by the Kullback-Leibler divergence, which it
// computes from the samples' covariances, and by the overlapping coefficient
// (OVL, the integral of min(p, q); 0: disjoint, 1: identical).  Both act on
// the Gaussians given by the two sample means and covariances.  Host code in
// float64: a d x d Cholesky factor per Gaussian and, for the OVL, one density
// ratio per Monte Carlo draw.
#include <math.h>
#include <stdint.h>

#include <vector>

#include "../../include/steinicp.h"

namespace {

constexpr int kMaxDim = 64;

// Lower Cholesky factor of the symmetric positive definite S (d x d, row-major); false otherwise.
bool cholesky(const double* S, int d, double* L) {
    for (int i = 0; i < d * d; ++i) L[i] = 0.0;
    for (int i = 0; i < d; ++i)
        for (int j = 0; j <= i; ++j) {
            double s = S[i * d + j];
            for (int k = 0; k < j; ++k) s -= L[i * d + k] * L[j * d + k];
            if (i == j) {
                if (!(s > 0.0) || !isfinite(s)) return false;
                L[i * d + i] = sqrt(s);
            } else {
                L[i * d + j] = s / L[j * d + j];
            }
        }
    return true;
}

// y = L^-1 x (forward substitution)
void lsolve(const double* L, int d, const double* x, double* y) {
    for (int i = 0; i < d; ++i) {
        double s = x[i];
        for (int k = 0; k < i; ++k) s -= L[i * d + k] * y[k];
        y[i] = s / L[i * d + i];
    }
}

double logdet(const double* L, int d) {
    double s = 0.0;
    for (int i = 0; i < d; ++i) s += log(L[i * d + i]);
    return 2.0 * s;
}

// log N(x; m, L L^T) up to the common -d/2 log(2 pi)
double log_density(const double* x, const double* m, const double* L, double ld, int d, double* tmp) {
    double diff[kMaxDim];
    for (int i = 0; i < d; ++i) diff[i] = x[i] - m[i];
    lsolve(L, d, diff, tmp);
    double q = 0.0;
    for (int i = 0; i < d; ++i) q += tmp[i] * tmp[i];
    return -0.5 * q - 0.5 * ld;
}

bool finite_all(const double* a, int64_t n) {
    for (int64_t i = 0; i < n; ++i)
        if (!isfinite(a[i])) return false;
    return true;
}

}  // namespace

extern "C" int sicp_gaussian_kl(const double* mean0, const double* cov0, const double* mean1, const double* cov1,
                                int32_t d, double* out) {
    if (!mean0 || !cov0 || !mean1 || !cov1 || !out || d < 1 || d > kMaxDim) return SICP_EINVAL;
    if (!finite_all(mean0, d) || !finite_all(mean1, d) || !finite_all(cov0, (int64_t)d * d) ||
        !finite_all(cov1, (int64_t)d * d))
        return SICP_EINVAL;
    std::vector<double> L0(d * d), L1(d * d), col(d), y(d);
    if (!cholesky(cov0, d, L0.data()) || !cholesky(cov1, d, L1.data())) return SICP_EINVAL;
    // tr(S1^-1 S0) = ||L1^-1 L0||_F^2
    double tr = 0.0;
    for (int j = 0; j < d; ++j) {
        for (int i = 0; i < d; ++i) col[i] = L0[i * d + j];
        lsolve(L1.data(), d, col.data(), y.data());
        for (int i = 0; i < d; ++i) tr += y[i] * y[i];
    }
    // (m1 - m0)^T S1^-1 (m1 - m0) = ||L1^-1 (m1 - m0)||^2
    for (int i = 0; i < d; ++i) col[i] = mean1[i] - mean0[i];
    lsolve(L1.data(), d, col.data(), y.data());
    double q = 0.0;
    for (int i = 0; i < d; ++i) q += y[i] * y[i];
    *out = 0.5 * (tr + q - (double)d + logdet(L1.data(), d) - logdet(L0.data(), d));
    return SICP_OK;
}

extern "C" int sicp_gaussian_ovl(const double* mean0, const double* cov0, const double* mean1, const double* cov1,
                                 int32_t d, const double* z0, const double* z1, int64_t n, double* out) {
    if (!mean0 || !cov0 || !mean1 || !cov1 || !z0 || !z1 || !out || d < 1 || d > kMaxDim || n < 1)
        return SICP_EINVAL;
    if (!finite_all(mean0, d) || !finite_all(mean1, d) || !finite_all(cov0, (int64_t)d * d) ||
        !finite_all(cov1, (int64_t)d * d) || !finite_all(z0, n * d) || !finite_all(z1, n * d))
        return SICP_EINVAL;
    std::vector<double> L0(d * d), L1(d * d);
    if (!cholesky(cov0, d, L0.data()) || !cholesky(cov1, d, L1.data())) return SICP_EINVAL;
    const double ld0 = logdet(L0.data(), d), ld1 = logdet(L1.data(), d);
    double x[kMaxDim], tmp[kMaxDim];
    double sum[2] = {0.0, 0.0};
    for (int side = 0; side < 2; ++side) {
        const double* m = side ? mean1 : mean0;
        const double* L = side ? L1.data() : L0.data();
        const double* z = side ? z1 : z0;
        for (int64_t s = 0; s < n; ++s) {
            // a draw of this side's Gaussian: m + L z
            for (int i = 0; i < d; ++i) {
                double v = m[i];
                for (int k = 0; k <= i; ++k) v += L[i * d + k] * z[s * d + k];
                x[i] = v;
            }
            const double lp0 = log_density(x, mean0, L0.data(), ld0, d, tmp);
            const double lp1 = log_density(x, mean1, L1.data(), ld1, d, tmp);
            const double r = side ? exp(lp0 - lp1) : exp(lp1 - lp0);   // other / own
            sum[side] += r < 1.0 ? r : 1.0;
        }
    }
    *out = 0.5 * (sum[0] + sum[1]) / (double)n;
    return SICP_OK;
}
