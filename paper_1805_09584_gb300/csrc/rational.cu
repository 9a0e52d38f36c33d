// Rational approximation of the inverse square root (Sec. 4.1): Zolotarev's
// optimal approximation R_{n,eps}(y) = a prod_j (y + c_{2j-1})/(y + c_{2j}) of
// 1/sqrt(y) on eps < y < 1 (Eqs. "rational", "deviation", "zolotarev_shifts")
// and its application x = R(Qhat^2 / lmax) b / sqrt(lmax) ~ (Qhat^2)^{-1/2} b
// through the partial fractions of Eq. "ratapp": one multi-shift solve of the n
// systems (Qhat^2 + lmax c_{2i}) x_i = b and one linear combination.
//
// The Jacobi elliptic functions and the complete elliptic integral come from the
// arithmetic-geometric mean (descending Landen) method: with a_0 = 1,
// b_0 = sqrt(1 - m), c_0 = sqrt(m) (m = k^2) and a_{i+1} = (a_i + b_i)/2,
// b_{i+1} = sqrt(a_i b_i), c_{i+1} = (a_i - b_i)/2 until c_N vanishes,
// K = pi / (2 a_N); phi_N = 2^N a_N u, phi_{i-1} = (phi_i + asin(c_i sin(phi_i) / a_i)) / 2,
// sn = sin(phi_0), cn = cos(phi_0).
#include <math.h>
#include <string.h>

#include <vector>

#include "tmnd_internal.cuh"

namespace {

struct Agm {
    double a[64], c[64];
    int N;
};

Agm agm(double m) {
    Agm g;
    double a = 1.0, b = sqrt(1.0 - m), c = sqrt(m);
    g.a[0] = a;
    g.c[0] = c;
    int i = 0;
    while (fabs(c) > 1e-17 * a && i < 62) {
        const double an = 0.5 * (a + b), bn = sqrt(a * b);
        c = 0.5 * (a - b);
        a = an;
        b = bn;
        i++;
        g.a[i] = a;
        g.c[i] = c;
    }
    g.N = i;
    return g;
}

void ellip_sncn(double u, const Agm &g, double *sn, double *cn) {
    double phi = ldexp(g.a[g.N] * u, g.N);
    for (int i = g.N; i >= 1; i--) phi = 0.5 * (phi + asin(g.c[i] * sin(phi) / g.a[i]));
    *sn = sin(phi);
    *cn = cos(phi);
}

// out[i] = w0 * b + sum_j w[j] * xs[j] over up to 33 FP64 spinors (one RHS block each)
constexpr int MAXR = TMND_MAX_SHIFTS + 1;
struct RatArgs {
    const double2 *x[MAXR];
    double w[MAXR];
    int k;
};

__global__ void k_lincomb_n(long n, RatArgs a, double2 *__restrict__ out) {
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        double2 acc = make_double2(0.0, 0.0);
        for (int j = 0; j < a.k; j++) {
            const double2 v = __ldg(&a.x[j][i]);
            acc.x = fma(a.w[j], v.x, acc.x);
            acc.y = fma(a.w[j], v.y, acc.y);
        }
        out[i] = acc;
    }
}

}  // namespace

extern "C" tmnd_status tmnd_zolotarev(int n, double eps, double *a, double *c, double *q, double *delta) {
    TMND_ARG_CHECK(n >= 1 && n <= TMND_MAX_SHIFTS, "tmnd_zolotarev: n = %d not in [1, %d]", n, TMND_MAX_SHIFTS);
    TMND_ARG_CHECK(eps > 0 && eps < 1, "tmnd_zolotarev: eps = %g not in (0, 1)", eps);
    TMND_ARG_CHECK(a && c && q && delta, "tmnd_zolotarev: NULL argument");
    const double m = 1.0 - eps;  // parameter k^2, k = sqrt(1 - eps)
    const Agm g = agm(m);
    const double v = M_PI / (2.0 * g.a[g.N]) / (2 * n + 1);
    std::vector<double> s(2 * n);
    for (int k = 1; k <= 2 * n; k++) {
        double sn, cn;
        ellip_sncn(k * v, g, &sn, &cn);
        c[k - 1] = (cn / sn) * (cn / sn);
        s[k - 1] = sn * sn;
    }
    double d = pow(1.0 - eps, 0.5 * (2 * n + 1)), ratio = 1.0;
    for (int j = 0; j < n; j++) {
        d *= s[2 * j] * s[2 * j];
        ratio *= s[2 * j] / s[2 * j + 1];
    }
    const double root = sqrt(1.0 - d * d);
    *a = 2.0 / (1.0 + root) * ratio;
    // delta = max |1 - sqrt(y) R(y)| on (eps, 1) (Eq. "deviation")
    *delta = d * d / ((1.0 + root) * (1.0 + root));
    for (int i = 0; i < n; i++) {
        const double den = c[2 * i + 1];
        double p = c[2 * i] - den;
        for (int j = 0; j < n; j++)
            if (j != i) p *= (c[2 * j] - den) / (c[2 * j + 1] - den);
        q[i] = p;
    }
    return TMND_OK;
}

extern "C" tmnd_status tmnd_rational_apply(tmnd_gauge *g, const void *b, int nrhs, int n, double lambda_min,
                                           double lambda_max, const tmnd_solve_params *params, void *out,
                                           double *delta_out, tmnd_solve_info *info, void *stream) {
    TMND_ARG_CHECK(g && b && out && params && b != out, "tmnd_rational_apply: bad arguments");
    TMND_ARG_CHECK(nrhs >= 1 && n >= 1 && n <= TMND_MAX_SHIFTS, "tmnd_rational_apply: n = %d, nrhs = %d", n, nrhs);
    TMND_ARG_CHECK(lambda_min > 0 && lambda_max > lambda_min, "tmnd_rational_apply: need 0 < lambda_min < lambda_max");
    cudaGetLastError();
    double a, delta, c[2 * TMND_MAX_SHIFTS], q[TMND_MAX_SHIFTS];
    tmnd_status st = tmnd_zolotarev(n, lambda_min / lambda_max, &a, c, q, &delta);
    if (st != TMND_OK) return st;
    if (delta_out) *delta_out = delta;
    // shifts lmax c_{2i}, descending like c
    double sigma[TMND_MAX_SHIFTS];
    for (int i = 0; i < n; i++) sigma[i] = lambda_max * c[2 * i + 1];
    const size_t sp = tmnd_spinor_bytes(g);
    char *xs = nullptr;
    TMND_CUDA_TRY(cudaMalloc(&xs, sp * nrhs * n));
    void *xp[TMND_MAX_SHIFTS];
    for (int i = 0; i < n; i++) xp[i] = xs + sp * nrhs * i;
    st = mms_cg_solve(g, b, nrhs, sigma, n, xp, params, info, stream);
    if (st == TMND_OK) {
        // out = (a / sqrt(lmax)) (b + lmax sum_i q_i x_i)   (Eq. "ratapp")
        const double f = a / sqrt(lambda_max);
        const long nel = (long)(sp / sizeof(double2));
        int dev = 0, sms = 152;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        const long want = (nel + 255) / 256, cap = (long)sms * 8;
        for (int k = 0; k < nrhs; k++) {
            RatArgs ra;
            ra.k = n + 1;
            ra.x[0] = (const double2 *)b + (size_t)k * nel;
            ra.w[0] = f;
            for (int i = 0; i < n; i++) {
                ra.x[1 + i] = (const double2 *)xp[i] + (size_t)k * nel;
                ra.w[1 + i] = f * lambda_max * q[i];
            }
            k_lincomb_n<<<(unsigned)(want < cap ? want : cap), 256, 0, (cudaStream_t)stream>>>(
                nel, ra, (double2 *)out + (size_t)k * nel);
        }
        cudaError_t e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaStreamSynchronize((cudaStream_t)stream);
        if (e != cudaSuccess) {
            tmnd_set_error("tmnd_rational_apply: %s", cudaGetErrorString(e));
            st = TMND_ERR_CUDA;
        }
    }
    cudaFree(xs);
    return st;
}
