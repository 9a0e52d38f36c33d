// Lagrange-interpolated initial guess (Sec. 4.2.1; App. B):
//   x~(m) = sum_j l_j(m) x_j,   l_j(m) = prod_{i != j} (m - m_i) / (m_j - m_i)
// The weights are k <= 8 FP64 numbers computed on the host; the combination
// is one bandwidth-bound pass (k reads, one write per element).
#include <math.h>

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
