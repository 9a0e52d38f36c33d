// Lagrange-interpolated initial guess (Sec. 4.2.1; App. B):
//   x~(m) = sum_j l_j(m) x_j,   l_j(m) = prod_{i != j} (m - m_i) / (m_j - m_i)
// The weights are k <= 8 FP64 numbers computed on the host; the combination
// is one bandwidth-bound pass (k reads, one write per element).
#include <math.h>
#include <string.h>

#include "tmnd_internal.cuh"

namespace {

constexpr int MAXK = 8;

struct LinArgs {
    const double2 *x[MAXK];
    double w[MAXK];
    int k;
};

__global__ void k_lincomb(long n, LinArgs a, double2 *__restrict__ out) {
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        double2 acc = make_double2(0.0, 0.0);
#pragma unroll
        for (int j = 0; j < MAXK; j++) {
            if (j < a.k) {
                double2 v = __ldg(&a.x[j][i]);
                acc.x = fma(a.w[j], v.x, acc.x);
                acc.y = fma(a.w[j], v.y, acc.y);
            }
        }
        out[i] = acc;
    }
}

}  // namespace

extern "C" tmnd_status lagrange_guess(const tmnd_gauge *g, const double *nodes, const void *const *xs, int k,
                                      double target, void *out, int nrhs, double *lebesgue_out, void *stream) {
    TMND_ARG_CHECK(g && nodes && xs && out, "lagrange_guess: NULL argument");
    TMND_ARG_CHECK(k >= 1 && k <= MAXK, "lagrange_guess: k = %d not in [1, %d]", k, MAXK);
    TMND_ARG_CHECK(nrhs >= 1, "lagrange_guess: nrhs = %d", nrhs);
    TMND_ARG_CHECK(isfinite(target), "lagrange_guess: target must be finite");
    TMND_ARG_CHECK(((uintptr_t)out & 15) == 0, "lagrange_guess: out misaligned");
    for (int j = 0; j < k; j++) {
        TMND_ARG_CHECK(xs[j] != nullptr && ((uintptr_t)xs[j] & 15) == 0, "lagrange_guess: xs[%d] NULL or misaligned", j);
        TMND_ARG_CHECK(xs[j] != out, "lagrange_guess: out aliases xs[%d]", j);
        TMND_ARG_CHECK(isfinite(nodes[j]), "lagrange_guess: nodes[%d] not finite", j);
        for (int i = 0; i < j; i++)
            TMND_ARG_CHECK(nodes[i] != nodes[j], "lagrange_guess: nodes %d and %d coincide", i, j);
    }
    LinArgs a = {};
    a.k = k;
    double leb = 0.0;
    for (int j = 0; j < k; j++) {
        double l = 1.0;
        for (int i = 0; i < k; i++)
            if (i != j) l *= (target - nodes[i]) / (nodes[j] - nodes[i]);
        a.w[j] = l;
        leb += fabs(l);
    }
    if (lebesgue_out) *lebesgue_out = leb;
    const long n = (long)(tmnd_spinor_bytes(g) / sizeof(double2)) * nrhs;
    for (int j = 0; j < k; j++) a.x[j] = (const double2 *)xs[j];
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    long want = (n + 255) / 256, cap = (long)sms * 8;
    k_lincomb<<<(unsigned)(want < cap ? want : cap), 256, 0, (cudaStream_t)stream>>>(n, a, (double2 *)out);
    TMND_CUDA_TRY(cudaGetLastError());
    return TMND_OK;
}

extern "C" tmnd_status tmnd_lincomb(const tmnd_gauge *g, const double *w, const void *const *xs, int k, void *out,
                                    int nrhs, void *stream) {
    TMND_ARG_CHECK(g && w && xs && out, "tmnd_lincomb: NULL argument");
    TMND_ARG_CHECK(k >= 1 && k <= MAXK && nrhs >= 1, "tmnd_lincomb: k = %d not in [1, %d]", k, MAXK);
    cudaGetLastError();
    LinArgs a = {};
    a.k = k;
    for (int j = 0; j < k; j++) {
        TMND_ARG_CHECK(xs[j] && xs[j] != out && isfinite(w[j]), "tmnd_lincomb: bad xs[%d] or weight", j);
        a.x[j] = (const double2 *)xs[j];
        a.w[j] = w[j];
    }
    const long n = (long)(tmnd_spinor_bytes(g) / sizeof(double2)) * nrhs;
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    long want = (n + 255) / 256, cap = (long)sms * 8;
    k_lincomb<<<(unsigned)(want < cap ? want : cap), 256, 0, (cudaStream_t)stream>>>(n, a, (double2 *)out);
    TMND_CUDA_TRY(cudaGetLastError());
    return TMND_OK;
}

// ------------------------------------------------ complex combinations, site norms
// Used by the study of equivalent solutions (App. A): x_C = i/(2 mu) (x_+ - x_-),
// (Qhat -+ i mu) y = Qhat y -+ i mu y, and the smallest / largest local deviation
// (norm of one site's 24 components) of an error vector.
namespace {

struct CLinArgs {
    const double2 *x[MAXK];
    double2 w[MAXK];
    int k;
};

__global__ void k_lincomb_c(long n, CLinArgs a, double2 *__restrict__ out) {
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        double2 acc = make_double2(0.0, 0.0);
#pragma unroll
        for (int j = 0; j < MAXK; j++) {
            if (j < a.k) {
                const double2 v = a.x[j][i];
                acc.x = fma(a.w[j].x, v.x, fma(-a.w[j].y, v.y, acc.x));
                acc.y = fma(a.w[j].x, v.y, fma(a.w[j].y, v.x, acc.y));
            }
        }
        out[i] = acc;
    }
}

// per-site squared norms folded into a min and a max (non-negative doubles order
// like their bit patterns, so integer atomics give an exact, order-free result)
__global__ void k_site_norm_range(int Vh, int nrhs, const double2 *__restrict__ x, unsigned long long *mm) {
    unsigned long long lo = ~0ull, hi = 0ull;
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < (long)Vh * nrhs; i += (long)gridDim.x * blockDim.x) {
        const long k = i / Vh, h = i % Vh;
        const double2 *xk = x + (size_t)k * 24 * Vh;
        double s = 0.0;
        for (int c = 0; c < 24; c++) {
            const double2 v = xk[(size_t)c * Vh + h];
            s = fma(v.x, v.x, fma(v.y, v.y, s));
        }
        const unsigned long long b = (unsigned long long)__double_as_longlong(s);
        lo = b < lo ? b : lo;
        hi = b > hi ? b : hi;
    }
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long l2 = __shfl_xor_sync(0xffffffffu, lo, o), h2 = __shfl_xor_sync(0xffffffffu, hi, o);
        lo = l2 < lo ? l2 : lo;
        hi = h2 > hi ? h2 : hi;
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMin(&mm[0], lo);
        atomicMax(&mm[1], hi);
    }
}

}  // namespace

extern "C" tmnd_status tmnd_lincomb_c(const tmnd_gauge *g, const double *w, const void *const *xs, int k, void *out,
                                      int nrhs, void *stream) {
    TMND_ARG_CHECK(g && w && xs && out, "tmnd_lincomb_c: NULL argument");
    TMND_ARG_CHECK(k >= 1 && k <= MAXK && nrhs >= 1, "tmnd_lincomb_c: k = %d not in [1, %d]", k, MAXK);
    TMND_ARG_CHECK(((uintptr_t)out & 15) == 0, "tmnd_lincomb_c: out misaligned");
    cudaGetLastError();
    CLinArgs a = {};
    a.k = k;
    for (int j = 0; j < k; j++) {
        TMND_ARG_CHECK(xs[j] && ((uintptr_t)xs[j] & 15) == 0 && isfinite(w[2 * j]) && isfinite(w[2 * j + 1]),
                       "tmnd_lincomb_c: bad xs[%d] or weight", j);
        a.x[j] = (const double2 *)xs[j];
        a.w[j] = make_double2(w[2 * j], w[2 * j + 1]);
    }
    const long n = (long)(tmnd_spinor_bytes(g) / sizeof(double2)) * nrhs;
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    long want = (n + 255) / 256, cap = (long)sms * 8;
    k_lincomb_c<<<(unsigned)(want < cap ? want : cap), 256, 0, (cudaStream_t)stream>>>(n, a, (double2 *)out);
    TMND_CUDA_TRY(cudaGetLastError());
    return TMND_OK;
}

extern "C" tmnd_status tmnd_site_norm_range(const tmnd_gauge *g, const void *x, int nrhs, double *min_max,
                                            void *stream) {
    TMND_ARG_CHECK(g && x && min_max && nrhs >= 1, "tmnd_site_norm_range: bad arguments");
    TMND_ARG_CHECK(((uintptr_t)x & 15) == 0, "tmnd_site_norm_range: x misaligned");
    cudaGetLastError();
    unsigned long long *mm = nullptr;
    TMND_CUDA_TRY(cudaMallocAsync((void **)&mm, 2 * sizeof(unsigned long long), (cudaStream_t)stream));
    const unsigned long long init[2] = {~0ull, 0ull};
    cudaMemcpyAsync(mm, init, sizeof(init), cudaMemcpyHostToDevice, (cudaStream_t)stream);
    const int Vh = g->geom.Vh;
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const long n = (long)Vh * nrhs;
    long want = (n + 255) / 256, cap = (long)sms * 4;
    k_site_norm_range<<<(unsigned)(want < cap ? want : cap), 256, 0, (cudaStream_t)stream>>>(Vh, nrhs,
                                                                                           (const double2 *)x, mm);
    unsigned long long res[2] = {0, 0};
    cudaMemcpyAsync(res, mm, sizeof(res), cudaMemcpyDeviceToHost, (cudaStream_t)stream);
    cudaFreeAsync(mm, (cudaStream_t)stream);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e != cudaSuccess) {
        tmnd_set_error("tmnd_site_norm_range: %s", cudaGetErrorString(e));
        return TMND_ERR_CUDA;
    }
    double lo, hi;
    memcpy(&lo, &res[0], 8);
    memcpy(&hi, &res[1], 8);
    min_max[0] = sqrt(lo);
    min_max[1] = sqrt(hi);
    return TMND_OK;
}

// ------------------------------------------------ host helpers of the guesses
// l_j(target) over nodes[0..k), Sec. 4.2.1; returns gamma_k(target) = sum |l_j| (App. B)
static double lagrange_w(const double *nodes, int k, double target, double *w) {
    double leb = 0.0;
    for (int j = 0; j < k; j++) {
        double l = 1.0;
        for (int i = 0; i < k; i++)
            if (i != j) l *= (target - nodes[i]) / (nodes[j] - nodes[i]);
        if (w) w[j] = l;
        leb += fabs(l);
    }
    return leb;
}

static tmnd_status check_nodes(const char *fn, const double *nodes, int k, double target) {
    TMND_ARG_CHECK(nodes, "%s: NULL nodes", fn);
    TMND_ARG_CHECK(k >= 1 && k <= MAXK, "%s: k = %d not in [1, %d]", fn, k, MAXK);
    TMND_ARG_CHECK(isfinite(target), "%s: target must be finite", fn);
    for (int j = 0; j < k; j++) {
        TMND_ARG_CHECK(isfinite(nodes[j]), "%s: nodes[%d] not finite", fn, j);
        for (int i = 0; i < j; i++) TMND_ARG_CHECK(nodes[i] != nodes[j], "%s: nodes %d and %d coincide", fn, i, j);
    }
    return TMND_OK;
}

extern "C" tmnd_status tmnd_lagrange_weights(const double *nodes, int k, double target, double *w, double *gamma) {
    const tmnd_status st = check_nodes("tmnd_lagrange_weights", nodes, k, target);
    if (st != TMND_OK) return st;
    TMND_ARG_CHECK(w, "tmnd_lagrange_weights: NULL w");
    const double leb = lagrange_w(nodes, k, target, w);
    if (gamma) *gamma = leb;
    return TMND_OK;
}

// App. B: when the Lebesgue function grows, truncate the degree of the interpolation.
// The nodes come in order of preference (nearest first); keep the longest prefix
// whose Lebesgue function at the target stays within gamma_max.
extern "C" tmnd_status tmnd_lagrange_degree(const double *nodes, int k, double target, double gamma_max,
                                            int *k_used, double *gamma) {
    const tmnd_status st = check_nodes("tmnd_lagrange_degree", nodes, k, target);
    if (st != TMND_OK) return st;
    TMND_ARG_CHECK(k_used, "tmnd_lagrange_degree: NULL k_used");
    TMND_ARG_CHECK(gamma_max >= 1.0, "tmnd_lagrange_degree: gamma_max = %g < 1", gamma_max);
    int best = 1;
    double gbest = 1.0;  // gamma_1 = |l_1| = 1
    for (int kk = 2; kk <= k; kk++) {
        const double gk = lagrange_w(nodes, kk, target, nullptr);
        if (gk <= gamma_max) {
            best = kk;
            gbest = gk;
        }
    }
    *k_used = best;
    if (gamma) *gamma = gbest;
    return TMND_OK;
}

// H_jk = Re((t - s_j) G_jk (t - s_k)) / bb: with exact solutions x_j of the shifts s_j and
// weights summing to 1, w^T H w is the squared relative residual of sum_j w_j x_j at the
// target shift t (App. B: the residual is - sum_j w_j (t - s_j) x_j); G interleaved re/im.
extern "C" tmnd_status tmnd_guess_quadratic_form(const double *G, const double *nodes, int k, double target,
                                                 double bb, double *H) {
    const tmnd_status st = check_nodes("tmnd_guess_quadratic_form", nodes, k, target);
    if (st != TMND_OK) return st;
    TMND_ARG_CHECK(G && H, "tmnd_guess_quadratic_form: NULL argument");
    TMND_ARG_CHECK(bb > 0 && isfinite(bb), "tmnd_guess_quadratic_form: bb = %g", bb);
    for (int j = 0; j < k; j++)
        for (int q = 0; q < k; q++)
            H[j * k + q] = (target - nodes[j]) * G[2 * (j * k + q)] * (target - nodes[q]) / bb;
    return TMND_OK;
}
