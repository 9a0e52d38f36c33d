// Hybrid cost model (Sec. 4.3): time-to-solution fits per shift s = m^2 of the
// CG solver (Eq. "CGtime2") and of the MG solver (Eq. "MGtime2"), and the cost of
// the hybrid with the n largest shifts by multi-shift CG (Eq. "costwo"):
//   t_CG(s) = a + b / ln(1 - 2 / (sqrt(kappa(s)) + 1)),  kappa(s) = (lmax + s) / (lmin + s)
//   t_MG(s) = A + B / ln(1 - (C + s) / (L + s))
//   c_HY(n) = t_CG(s_n) + sum_{i > n} t_MG(s_i)       (shifts descending, n = 1..N)
// Host code.
#include <math.h>

#include <vector>

#include "tmnd_internal.cuh"

namespace {

double xcg(double s, double lmin, double lmax) {
    return 1.0 / log(1.0 - 2.0 / (sqrt((lmax + s) / (lmin + s)) + 1.0));
}
double xmg(double s, double C, double L) { return 1.0 / log(1.0 - (C + s) / (L + s)); }

// least squares of t ~ p0 + p1 x; returns the residual sum of squares
double line_fit(const std::vector<double> &x, const double *t, double *p0, double *p1) {
    const int n = (int)x.size();
    double sx = 0, sy = 0, sxx = 0, sxy = 0;
    for (int i = 0; i < n; i++) {
        sx += x[i];
        sy += t[i];
        sxx += x[i] * x[i];
        sxy += x[i] * t[i];
    }
    const double den = n * sxx - sx * sx;
    *p1 = den != 0 ? (n * sxy - sx * sy) / den : 0.0;
    *p0 = (sy - *p1 * sx) / n;
    double r = 0;
    for (int i = 0; i < n; i++) {
        const double e = *p0 + *p1 * x[i] - t[i];
        r += e * e;
    }
    return r;
}

}  // namespace

extern "C" tmnd_status tmnd_hybrid_cost(const double *sigma, int N, const double *cg, const double *mg,
                                        double *cost, int *n_opt) {
    TMND_ARG_CHECK(sigma && cg && mg && cost && n_opt && N >= 1, "tmnd_hybrid_cost: bad arguments");
    TMND_ARG_CHECK(cg[2] > 0 && cg[3] > cg[2] && mg[3] > 0, "tmnd_hybrid_cost: need 0 < lmin < lmax and L > 0");
    std::vector<double> tm(N);
    for (int i = 0; i < N; i++) tm[i] = mg[0] + mg[1] * xmg(sigma[i], mg[2], mg[3]);
    int best = 1;
    for (int n = 1; n <= N; n++) {
        double c = cg[0] + cg[1] * xcg(sigma[n - 1], cg[2], cg[3]);
        for (int i = n; i < N; i++) c += tm[i];
        cost[n - 1] = c;
        if (c < cost[best - 1]) best = n;
    }
    *n_opt = best;
    return TMND_OK;
}

extern "C" tmnd_status tmnd_fit_cg_time(const double *sigma, const double *t, int N, double lmin, double lmax,
                                        double *a, double *b) {
    TMND_ARG_CHECK(sigma && t && a && b && N >= 2 && lmin > 0 && lmax > lmin, "tmnd_fit_cg_time: bad arguments");
    std::vector<double> x(N);
    for (int i = 0; i < N; i++) x[i] = xcg(sigma[i], lmin, lmax);
    line_fit(x, t, a, b);
    return TMND_OK;
}

// C on a log grid of `grid` points in (1e-8 L, 0.999 L), (A, B) by least squares for each
extern "C" tmnd_status tmnd_fit_mg_time(const double *sigma, const double *t, int N, double L, int grid, double *A,
                                        double *B, double *C) {
    TMND_ARG_CHECK(sigma && t && A && B && C && N >= 3 && L > 0 && grid >= 2, "tmnd_fit_mg_time: bad arguments");
    std::vector<double> x(N);
    double best = INFINITY;
    const double lo = log(1e-8 * L), hi = log(0.999 * L);
    for (int gi = 0; gi < grid; gi++) {
        const double c = exp(lo + (hi - lo) * gi / (grid - 1));
        for (int i = 0; i < N; i++) x[i] = xmg(sigma[i], c, L);
        double p0, p1;
        const double r = line_fit(x, t, &p0, &p1);
        if (r < best) {
            best = r;
            *A = p0;
            *B = p1;
            *C = c;
        }
    }
    return TMND_OK;
}
