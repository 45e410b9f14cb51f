// Zolotarev coefficients of the rational sign function (Sec. 2.1, Eq. 4) and a
// tridiagonal eigenvalue bound used by the spectrum estimate.  Host code.
//
// R(x) = c0 + sum_{i=1}^{n} c_i / (x + q_i) is the type-(n, n) rational with the
// least maximal relative error for 1/sqrt(x) on [a, b].  Zolotarev's solution
// (as written out for the overlap operator by Chiu et al., PRD 66 (2002) 114502):
// with y = x / a, modulus parameter m = 1 - a/b and K = K(m),
//   e_l = sn^2(u_l | m) / cn^2(u_l | m),  u_l = l K / (2n + 1),  l = 1..2n,
//   R(y) ~ d0 prod_{l=1}^{n} (y + e_{2l}) / (y + e_{2l-1}),
// and d0 makes the relative error equal and opposite at y = 1 and y = b/a
// (both ends are alternation points).  The Jacobi functions are computed with
// the arithmetic-geometric mean and the descending Landen recursion
// (Abramowitz & Stegun 16.4, 17.6).
#include <cmath>
#include <vector>

#include "smpq_internal.cuh"

namespace {

// AGM sequence for parameter m: returns N and fills a[0..N], c[0..N]
int agm(double m, double *a, double *c, int maxn) {
    double an = 1.0, bn = std::sqrt(1.0 - m), cn = std::sqrt(m);
    a[0] = an;
    c[0] = cn;
    int n = 0;
    while (std::fabs(cn) > 1e-17 * an && n + 1 < maxn) {
        double a1 = 0.5 * (an + bn), b1 = std::sqrt(an * bn), c1 = 0.5 * (an - bn);
        an = a1;
        bn = b1;
        cn = c1;
        ++n;
        a[n] = an;
        c[n] = cn;
    }
    return n;
}

// K(m) = pi / (2 AGM(1, sqrt(1 - m)))
double ellip_k(double m) {
    double a[64], c[64];
    int n = agm(m, a, c, 64);
    return M_PI / (2.0 * a[n]);
}

// sn, cn of u with parameter m (descending Landen / AGM method)
void ellip_sncn(double u, double m, double *sn, double *cn) {
    double a[64], c[64];
    int n = agm(m, a, c, 64);
    double phi = std::ldexp(a[n] * u, n);
    for (int k = n; k >= 1; --k) phi = 0.5 * (phi + std::asin(c[k] * std::sin(phi) / a[k]));
    *sn = std::sin(phi);
    *cn = std::cos(phi);
}

} // namespace

int zolotarev_coeffs(int n, double a, double b, double *c0, double *c, double *q, double *delta) {
    if (n < 1 || n > SMPQ_MAX_POLES || !(a > 0) || !(b > a)) return SMPQ_EINVAL;
    const double m = 1.0 - a / b;
    const double K = ellip_k(m);
    std::vector<double> e(2 * n + 1);
    for (int l = 1; l <= 2 * n; ++l) {
        double sn, cn;
        ellip_sncn(l * K / (2 * n + 1), m, &sn, &cn);
        e[l] = (sn * sn) / (cn * cn);
    }
    auto f = [&](double y) {
        double v = std::sqrt(y);
        for (int l = 1; l <= n; ++l) v *= (y + e[2 * l]) / (y + e[2 * l - 1]);
        return v;
    };
    const double f1 = f(1.0), f2 = f(b / a);
    const double d0 = 2.0 / (f1 + f2);
    if (delta) *delta = std::fabs(f1 - f2) / (f1 + f2);
    // partial fractions in y, then back to x = a y:
    // 1/sqrt(x) = a^{-1/2} R(x/a) = d0/sqrt(a) + sum_l (res_l sqrt(a)) / (x + e_{2l-1} a)
    const double sa = std::sqrt(a);
    *c0 = d0 / sa;
    for (int i = 0; i < n; ++i) {
        double pole = e[2 * i + 1];
        double num = 1.0, den = 1.0;
        for (int l = 1; l <= n; ++l) num *= (e[2 * l] - pole);
        for (int l = 0; l < n; ++l)
            if (l != i) den *= (e[2 * l + 1] - pole);
        double res = d0 * num / den;
        c[i] = res * a / sa;
        q[i] = pole * a;
    }
    return SMPQ_OK;
}

// Smallest and largest eigenvalue of the symmetric tridiagonal matrix
// (diag, off) by Sturm-sequence bisection inside the Gershgorin interval.
void tridiag_extremes(const std::vector<double> &d, const std::vector<double> &e, double *lo, double *hi) {
    const int n = (int)d.size();
    double gl = d[0], gu = d[0];
    for (int i = 0; i < n; ++i) {
        double r = (i > 0 ? std::fabs(e[i - 1]) : 0.0) + (i + 1 < n ? std::fabs(e[i]) : 0.0);
        gl = std::fmin(gl, d[i] - r);
        gu = std::fmax(gu, d[i] + r);
    }
    // number of eigenvalues < x
    auto count = [&](double x) {
        int cnt = 0;
        double qv = d[0] - x;
        if (qv < 0) ++cnt;
        for (int i = 1; i < n; ++i) {
            double den = qv != 0.0 ? qv : 1e-300;
            qv = d[i] - x - e[i - 1] * e[i - 1] / den;
            if (qv < 0) ++cnt;
        }
        return cnt;
    };
    auto kth = [&](int k) { // k-th smallest (0-based)
        double l = gl, u = gu;
        for (int it = 0; it < 200 && u - l > 1e-15 * std::fmax(std::fabs(l), std::fabs(u)); ++it) {
            double mid = 0.5 * (l + u);
            if (count(mid) > k) u = mid;
            else l = mid;
        }
        return 0.5 * (l + u);
    };
    *lo = kth(0);
    *hi = kth(n - 1);
}
