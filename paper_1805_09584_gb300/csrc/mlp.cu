// Learned initial guesses (not in the paper; it extends the Lagrange guesses of
// Sec. 4.2.1).  A network F -> 64 -> 64 -> 2 (tanh) predicts two log-poles o_k for
// a target shift sigma_t; with p_k = exp(o_k) the weights over the solutions x_j of
// 8 solved shifts are those of Lagrange interpolation of prod_k (p_k + sigma) x(sigma),
// divided back:
//   w_j = l_j(sigma_t) prod_k (p_k + sigma_j) / (p_k + sigma_t),
// which sum to 1 for any poles (the partition of unity of App. B) and tend to the
// Lagrange weights as p_k -> infinity.  With exact x_j the guess residual is
// -sum_j w_j (sigma_t - sigma_j) x_j, so |residual|^2/|b|^2 = w^T H w, H = Re(D G D)
// (G the Gram matrix of the x_j).  Training minimises mean log(w^T H w + floor)
// with the project's own forward/backward kernels (FP32 network, FP64 weights and
// loss: the guess residuals reach ~1e-9 |b|, far below what FP32 weights resolve)
// and Adam; inference uses BF16 weights with FP32 accumulation, FP64 output weights.
// Inputs are standardised by per-feature statistics stored with the parameters.
#include <cuda_bf16.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "tmnd_internal.cuh"

constexpr int MLP_H = 64;
constexpr int MLP_K = 8;   // solved shifts combined by the guess
constexpr int MLP_P = 2;   // network outputs: log-poles
constexpr int MLP_MAXF = 64;

struct tmnd_mlp {
    int F;
    int nparam;
    float *theta;              // FP32 master parameters [mu isd W1 b1 W2 b2 W3 b3]
    float *grad, *m, *v;       // gradient, Adam moments
    __nv_bfloat16 *theta_bf;   // inference copy
    double *loss_part;         // per-sample losses
    int loss_cap;
    int step;
};

namespace {

// parameter offsets: input mean and inverse std (not trained), then the layers
__host__ __device__ inline int off_isd(int F) { return F; }
__host__ __device__ inline int off_W1(int F) { return 2 * F; }
__host__ __device__ inline int off_b1(int F) { return off_W1(F) + MLP_H * F; }
__host__ __device__ inline int off_W2(int F) { return off_b1(F) + MLP_H; }
__host__ __device__ inline int off_b2(int F) { return off_W2(F) + MLP_H * MLP_H; }
__host__ __device__ inline int off_W3(int F) { return off_b2(F) + MLP_H; }
__host__ __device__ inline int off_b3(int F) { return off_W3(F) + MLP_P * MLP_H; }
__host__ __device__ inline int nparams(int F) { return off_b3(F) + MLP_P; }

// Rational weights from the poles (thread j < 8 of the block); S = (sigma_t, sigma_1..8).
__device__ inline double pole_weight(int j, const double *S, const double *p) {
    const double t = S[0], sj = S[1 + j];
    double l = 1.0;
    for (int i = 0; i < MLP_K; i++)
        if (i != j) l *= (t - S[1 + i]) / (sj - S[1 + i]);
    for (int k = 0; k < MLP_P; k++) l *= (p[k] + sj) / (p[k] + t);
    return l;
}

// One block of 64 threads per sample: forward, loss log(w^T H w + floor), backward,
// gradients accumulated with atomics (scaled by 1/N).  mu/isd get no gradient.
__global__ void k_mlp_fwd_bwd(int F, int N, const float *__restrict__ th, const float *__restrict__ X,
                              const double *__restrict__ Sg, const double *__restrict__ Hg, double floor_q,
                              float *__restrict__ grad, double *__restrict__ loss) {
    const int n = blockIdx.x, j = threadIdx.x;
    __shared__ float x[MLP_MAXF], h1[MLP_H], h2[MLP_H], dob[MLP_P], da2[MLP_H];
    __shared__ double S[1 + MLP_K], p[MLP_P], w[MLP_K], hw[MLP_K], q_s;
    const float *mu = th, *isd = th + off_isd(F);
    for (int f = j; f < F; f += blockDim.x) x[f] = (X[(size_t)n * F + f] - mu[f]) * isd[f];
    if (j <= MLP_K) S[j] = Sg[(size_t)n * (1 + MLP_K) + j];
    __syncthreads();
    const float *W1 = th + off_W1(F), *b1 = th + off_b1(F), *W2 = th + off_W2(F), *b2 = th + off_b2(F);
    const float *W3 = th + off_W3(F), *b3 = th + off_b3(F);
    const double *H = Hg + (size_t)n * MLP_K * MLP_K;
    float a = b1[j];
    for (int f = 0; f < F; f++) a = fmaf(W1[j * F + f], x[f], a);
    h1[j] = tanhf(a);
    __syncthreads();
    a = b2[j];
    for (int k = 0; k < MLP_H; k++) a = fmaf(W2[j * MLP_H + k], h1[k], a);
    h2[j] = tanhf(a);
    __syncthreads();
    if (j < MLP_P) {
        float o = b3[j];
        for (int k = 0; k < MLP_H; k++) o = fmaf(W3[j * MLP_H + k], h2[k], o);
        p[j] = exp((double)o);
    }
    __syncthreads();
    if (j < MLP_K) w[j] = pole_weight(j, S, p);
    __syncthreads();
    if (j < MLP_K) {
        double acc = 0.0;
        for (int k = 0; k < MLP_K; k++) acc = fma(H[j * MLP_K + k], w[k], acc);
        hw[j] = acc;
    }
    __syncthreads();
    if (j == 0) {
        double q = floor_q;
        for (int i = 0; i < MLP_K; i++) q = fma(w[i], hw[i], q);
        q_s = q;
        loss[n] = log(q);
    }
    __syncthreads();
    if (j < MLP_P) {
        // dL/do_k = sum_i (2 (Hw)_i / (q N)) w_i p_k (1/(p_k + sigma_i) - 1/(p_k + sigma_t))
        const double pk = p[j], ct = 1.0 / (pk + S[0]);
        double acc = 0.0;
        for (int i = 0; i < MLP_K; i++) acc += hw[i] * w[i] * (1.0 / (pk + S[1 + i]) - ct);
        dob[j] = (float)(2.0 * acc * pk / (q_s * (double)N));
    }
    __syncthreads();
    float *gW1 = grad + off_W1(F), *gb1 = grad + off_b1(F), *gW2 = grad + off_W2(F), *gb2 = grad + off_b2(F);
    float *gW3 = grad + off_W3(F), *gb3 = grad + off_b3(F);
    // layer 3
    for (int i = 0; i < MLP_P; i++) atomicAdd(&gW3[i * MLP_H + j], dob[i] * h2[j]);
    if (j < MLP_P) atomicAdd(&gb3[j], dob[j]);
    float dh2 = 0;
    for (int i = 0; i < MLP_P; i++) dh2 = fmaf(dob[i], W3[i * MLP_H + j], dh2);
    da2[j] = dh2 * (1.0f - h2[j] * h2[j]);
    __syncthreads();
    // layer 2
    for (int k = 0; k < MLP_H; k++) atomicAdd(&gW2[j * MLP_H + k], da2[j] * h1[k]);
    atomicAdd(&gb2[j], da2[j]);
    float dh1 = 0;
    for (int i = 0; i < MLP_H; i++) dh1 = fmaf(da2[i], W2[i * MLP_H + j], dh1);
    const float da1 = dh1 * (1.0f - h1[j] * h1[j]);
    // layer 1
    for (int f = 0; f < F; f++) atomicAdd(&gW1[j * F + f], da1 * x[f]);
    atomicAdd(&gb1[j], da1);
}

__global__ void k_adam(int n, float *__restrict__ th, float *__restrict__ g, float *__restrict__ m,
                       float *__restrict__ v, float lr, float b1, float b2, float eps, float c1, float c2) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1 - b1) * gi;
        const float vi = b2 * v[i] + (1 - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        th[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
        g[i] = 0.0f;
    }
}

// per-feature mean and inverse standard deviation of X [N][F] (one block per feature)
__global__ void k_input_stats(int F, int N, const float *__restrict__ X, float *__restrict__ mu,
                              float *__restrict__ isd) {
    __shared__ double red[80];
    __shared__ double mean_s;
    const int f = blockIdx.x;
    double s = 0.0;
    for (int n = threadIdx.x; n < N; n += blockDim.x) s += X[(size_t)n * F + f];
    s = block_sum(s, red);  // valid in thread 0
    if (threadIdx.x == 0) mean_s = s / N;
    __syncthreads();
    const double mean = mean_s;
    double v = 0.0;
    for (int n = threadIdx.x; n < N; n += blockDim.x) {
        const double d = X[(size_t)n * F + f] - mean;
        v += d * d;
    }
    const double var = block_sum(v, red) / N;
    if (threadIdx.x == 0) {
        mu[f] = (float)mean;
        isd[f] = var > 1e-12 ? (float)(1.0 / sqrt(var)) : 1.0f;
    }
}

__global__ void k_to_bf16(int n, const float *__restrict__ a, __nv_bfloat16 *__restrict__ b) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) b[i] = __float2bfloat16_rn(a[i]);
}

// inference: BF16 layer weights, FP32 input statistics, activations and accumulation;
// FP64 output weights W [N][8]
__global__ void k_mlp_infer(int F, const float *__restrict__ th, const __nv_bfloat16 *__restrict__ thb,
                            const float *__restrict__ X, const double *__restrict__ Sg, double *__restrict__ W) {
    const int n = blockIdx.x, j = threadIdx.x;
    __shared__ float x[MLP_MAXF], h1[MLP_H], h2[MLP_H];
    __shared__ double S[1 + MLP_K], p[MLP_P];
    const float *mu = th, *isd = th + off_isd(F);
    for (int f = j; f < F; f += blockDim.x) x[f] = (X[(size_t)n * F + f] - mu[f]) * isd[f];
    if (j <= MLP_K) S[j] = Sg[(size_t)n * (1 + MLP_K) + j];
    __syncthreads();
    const __nv_bfloat16 *W1 = thb + off_W1(F), *b1 = thb + off_b1(F), *W2 = thb + off_W2(F);
    const __nv_bfloat16 *b2 = thb + off_b2(F), *W3 = thb + off_W3(F), *b3 = thb + off_b3(F);
    float a = __bfloat162float(b1[j]);
    for (int f = 0; f < F; f++) a = fmaf(__bfloat162float(W1[j * F + f]), x[f], a);
    h1[j] = tanhf(a);
    __syncthreads();
    a = __bfloat162float(b2[j]);
    for (int k = 0; k < MLP_H; k++) a = fmaf(__bfloat162float(W2[j * MLP_H + k]), h1[k], a);
    h2[j] = tanhf(a);
    __syncthreads();
    if (j < MLP_P) {
        float o = __bfloat162float(b3[j]);
        for (int k = 0; k < MLP_H; k++) o = fmaf(__bfloat162float(W3[j * MLP_H + k]), h2[k], o);
        p[j] = exp((double)o);
    }
    __syncthreads();
    if (j < MLP_K) W[(size_t)n * MLP_K + j] = pole_weight(j, S, p);
}

// Gram matrix G_jk = <x_j, x_k> over k <= 8 FP64 spinors: block partials [nb][k][k] complex
constexpr int GK = 8;
struct GramArgs {
    const double2 *x[GK];
    int k;
};
__global__ void k_gram(long n, GramArgs a, double *__restrict__ part) {
    __shared__ double red[80];
    double acc[GK][GK][2];
    for (int p = 0; p < GK; p++)
        for (int q = 0; q < GK; q++) acc[p][q][0] = acc[p][q][1] = 0.0;
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        double2 v[GK];
#pragma unroll
        for (int p = 0; p < GK; p++) v[p] = p < a.k ? a.x[p][i] : make_double2(0, 0);
#pragma unroll
        for (int p = 0; p < GK; p++)
#pragma unroll
            for (int q = p; q < GK; q++) {
                acc[p][q][0] += v[p].x * v[q].x + v[p].y * v[q].y;
                acc[p][q][1] += v[p].x * v[q].y - v[p].y * v[q].x;
            }
    }
    for (int p = 0; p < a.k; p++)
        for (int q = p; q < a.k; q++)
            for (int c = 0; c < 2; c++) {
                const double s = block_sum(acc[p][q][c], red);
                __syncthreads();
                if (threadIdx.x == 0) part[((size_t)blockIdx.x * GK * GK + p * GK + q) * 2 + c] = s;
            }
}

// deterministic host normal numbers (splitmix64 + Box-Muller)
struct HostRng {
    uint64_t s;
    uint64_t next() {
        uint64_t z = (s += 0x9E3779B97F4A7C15ull);
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        return z ^ (z >> 31);
    }
    double uniform() { return ((next() >> 11) + 0.5) * (1.0 / 9007199254740992.0); }
    double normal() { return sqrt(-2.0 * log(uniform())) * cos(6.283185307179586 * uniform()); }
};

// smallest / largest eigenvalue of a symmetric tridiagonal matrix by bisection (Sturm counts)
int sturm_count(const std::vector<double> &d, const std::vector<double> &e, double x) {
    int c = 0;
    double q = 1.0;
    for (size_t i = 0; i < d.size(); i++) {
        q = d[i] - x - (i ? e[i - 1] * e[i - 1] / q : 0.0);
        if (q == 0.0) q = 1e-300;
        if (q < 0) c++;
    }
    return c;
}
double tridiag_eig(const std::vector<double> &d, const std::vector<double> &e, int index) {
    double lo = 1e300, hi = -1e300;
    for (size_t i = 0; i < d.size(); i++) {
        const double r = (i ? fabs(e[i - 1]) : 0.0) + (i + 1 < d.size() ? fabs(e[i]) : 0.0);
        lo = std::min(lo, d[i] - r);
        hi = std::max(hi, d[i] + r);
    }
    for (int it = 0; it < 200; it++) {
        const double mid = 0.5 * (lo + hi);
        if (sturm_count(d, e, mid) > index) hi = mid;
        else lo = mid;
    }
    return 0.5 * (lo + hi);
}

}  // namespace

extern "C" int tmnd_mlp_num_params(int F) { return nparams(F); }

extern "C" tmnd_status tmnd_mlp_create(int F, unsigned long long seed, tmnd_mlp **out) {
    TMND_ARG_CHECK(out && F >= 1 && F <= MLP_MAXF, "tmnd_mlp_create: F = %d not in [1, %d]", F, MLP_MAXF);
    cudaGetLastError();
    tmnd_mlp *m = new tmnd_mlp();
    memset(m, 0, sizeof *m);
    m->F = F;
    m->nparam = nparams(F);
    const size_t b = sizeof(float) * m->nparam;
    cudaError_t e = cudaMalloc(&m->theta, b);
    if (e == cudaSuccess) e = cudaMalloc(&m->grad, b);
    if (e == cudaSuccess) e = cudaMalloc(&m->m, b);
    if (e == cudaSuccess) e = cudaMalloc(&m->v, b);
    if (e == cudaSuccess) e = cudaMalloc(&m->theta_bf, sizeof(__nv_bfloat16) * m->nparam);
    std::vector<float> h(m->nparam, 0.0f);
    HostRng r{seed};
    for (int i = 0; i < F; i++) h[off_isd(F) + i] = 1.0f;  // identity standardisation until fitted
    for (int i = 0; i < MLP_H * F; i++) h[off_W1(F) + i] = (float)(r.normal() / sqrt((double)F));
    for (int i = 0; i < MLP_H * MLP_H; i++) h[off_W2(F) + i] = (float)(r.normal() / sqrt((double)MLP_H));
    for (int i = 0; i < MLP_P * MLP_H; i++) h[off_W3(F) + i] = (float)(0.1 * r.normal() / sqrt((double)MLP_H));
    // poles start near e^3 = 20, far above the shifts: the initial weights are close to Lagrange's
    for (int k = 0; k < MLP_P; k++) h[off_b3(F) + k] = 3.0f;
    if (e == cudaSuccess) e = cudaMemcpy(m->theta, h.data(), b, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(m->grad, 0, b);
    if (e == cudaSuccess) e = cudaMemset(m->m, 0, b);
    if (e == cudaSuccess) e = cudaMemset(m->v, 0, b);
    if (e != cudaSuccess) {
        tmnd_set_error("tmnd_mlp_create: %s", cudaGetErrorString(e));
        cudaFree(m->theta); cudaFree(m->grad); cudaFree(m->m); cudaFree(m->v); cudaFree(m->theta_bf);
        delete m;
        return TMND_ERR_CUDA;
    }
    *out = m;
    return TMND_OK;
}

extern "C" void tmnd_mlp_destroy(tmnd_mlp *m) {
    if (!m) return;
    cudaDeviceSynchronize();
    cudaFree(m->theta); cudaFree(m->grad); cudaFree(m->m); cudaFree(m->v); cudaFree(m->theta_bf);
    cudaFree(m->loss_part);
    delete m;
}

extern "C" tmnd_status tmnd_mlp_params(tmnd_mlp *m, float *host_get, const float *host_set) {
    TMND_ARG_CHECK(m, "tmnd_mlp_params: NULL handle");
    cudaGetLastError();
    if (host_set) TMND_CUDA_TRY(cudaMemcpy(m->theta, host_set, sizeof(float) * m->nparam, cudaMemcpyHostToDevice));
    if (host_get) TMND_CUDA_TRY(cudaMemcpy(host_get, m->theta, sizeof(float) * m->nparam, cudaMemcpyDeviceToHost));
    return TMND_OK;
}

extern "C" tmnd_status tmnd_mlp_fit_inputs(tmnd_mlp *m, const void *X, int N, void *stream) {
    TMND_ARG_CHECK(m && X && N >= 1, "tmnd_mlp_fit_inputs: bad arguments");
    cudaGetLastError();
    k_input_stats<<<m->F, 256, 0, (cudaStream_t)stream>>>(m->F, N, (const float *)X, m->theta,
                                                          m->theta + off_isd(m->F));
    TMND_CUDA_TRY(cudaGetLastError());
    return TMND_OK;
}

static tmnd_status mlp_grad(tmnd_mlp *m, const float *X, const double *S, const double *H, int N, double floor_q,
                            double *loss, cudaStream_t s) {
    if (N > m->loss_cap) {
        cudaFree(m->loss_part);
        m->loss_part = nullptr;
        TMND_CUDA_TRY(cudaMalloc(&m->loss_part, sizeof(double) * N));
        m->loss_cap = N;
    }
    k_mlp_fwd_bwd<<<N, MLP_H, 0, s>>>(m->F, N, m->theta, X, S, H, floor_q, m->grad, m->loss_part);
    TMND_CUDA_TRY(cudaGetLastError());
    if (loss) {
        std::vector<double> h(N);
        TMND_CUDA_TRY(cudaMemcpyAsync(h.data(), m->loss_part, sizeof(double) * N, cudaMemcpyDeviceToHost, s));
        TMND_CUDA_TRY(cudaStreamSynchronize(s));
        double acc = 0;
        for (double v : h) acc += v;
        *loss = acc / N;
    }
    return TMND_OK;
}

#define MLP_SAMPLE_CHECK(fn)                                                                          \
    TMND_ARG_CHECK(m && X && S && H && N >= 1 && floor_q >= 0 && isfinite(floor_q), fn ": bad arguments"); \
    TMND_ARG_CHECK(((uintptr_t)S & 7) == 0 && ((uintptr_t)H & 7) == 0, fn ": S or H misaligned")

extern "C" tmnd_status tmnd_mlp_loss_grad(tmnd_mlp *m, const void *X, const void *S, const void *H, int N,
                                          double floor_q, double *loss, float *grad_host, void *stream) {
    MLP_SAMPLE_CHECK("tmnd_mlp_loss_grad");
    cudaGetLastError();
    cudaStream_t s = (cudaStream_t)stream;
    TMND_CUDA_TRY(cudaMemsetAsync(m->grad, 0, sizeof(float) * m->nparam, s));
    tmnd_status st = mlp_grad(m, (const float *)X, (const double *)S, (const double *)H, N, floor_q, loss, s);
    if (st != TMND_OK) return st;
    if (grad_host) {
        TMND_CUDA_TRY(cudaMemcpyAsync(grad_host, m->grad, sizeof(float) * m->nparam, cudaMemcpyDeviceToHost, s));
        TMND_CUDA_TRY(cudaStreamSynchronize(s));
    }
    TMND_CUDA_TRY(cudaMemsetAsync(m->grad, 0, sizeof(float) * m->nparam, s));
    return TMND_OK;
}

extern "C" tmnd_status tmnd_mlp_train_step(tmnd_mlp *m, const void *X, const void *S, const void *H, int N,
                                           double lr, double floor_q, double *loss, void *stream) {
    MLP_SAMPLE_CHECK("tmnd_mlp_train_step");
    TMND_ARG_CHECK(lr > 0, "tmnd_mlp_train_step: lr = %g must be > 0", lr);
    cudaGetLastError();
    cudaStream_t s = (cudaStream_t)stream;
    tmnd_status st = mlp_grad(m, (const float *)X, (const double *)S, (const double *)H, N, floor_q, loss, s);
    if (st != TMND_OK) return st;
    m->step++;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.0f - powf(b1, (float)m->step), c2 = 1.0f - powf(b2, (float)m->step);
    // mu/isd have zero gradient, so Adam leaves them unchanged
    k_adam<<<(m->nparam + 255) / 256, 256, 0, s>>>(m->nparam, m->theta, m->grad, m->m, m->v, (float)lr, b1, b2,
                                                   1e-8f, c1, c2);
    TMND_CUDA_TRY(cudaGetLastError());
    return TMND_OK;
}

extern "C" tmnd_status tmnd_mlp_predict(tmnd_mlp *m, const void *X, const void *S, int N, void *W, void *stream) {
    TMND_ARG_CHECK(m && X && S && W && N >= 1, "tmnd_mlp_predict: bad arguments");
    TMND_ARG_CHECK(((uintptr_t)S & 7) == 0 && ((uintptr_t)W & 7) == 0, "tmnd_mlp_predict: S or W misaligned");
    cudaGetLastError();
    cudaStream_t s = (cudaStream_t)stream;
    k_to_bf16<<<(m->nparam + 255) / 256, 256, 0, s>>>(m->nparam, m->theta, m->theta_bf);
    k_mlp_infer<<<N, MLP_H, 0, s>>>(m->F, m->theta, m->theta_bf, (const float *)X, (const double *)S, (double *)W);
    TMND_CUDA_TRY(cudaGetLastError());
    return TMND_OK;
}

extern "C" tmnd_status tmnd_gram(const tmnd_gauge *g, const void *const *xs, int k, double *G_host, void *stream) {
    TMND_ARG_CHECK(g && xs && G_host && k >= 1 && k <= GK, "tmnd_gram: bad arguments");
    cudaGetLastError();
    cudaStream_t s = (cudaStream_t)stream;
    GramArgs a = {};
    a.k = k;
    for (int j = 0; j < k; j++) a.x[j] = (const double2 *)xs[j];
    const long n = 24L * g->geom.Vh;
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int nb = (int)std::min<long>((n + 255) / 256, (long)sms * 2);
    double *part = nullptr;
    TMND_CUDA_TRY(cudaMalloc(&part, sizeof(double) * nb * GK * GK * 2));
    k_gram<<<nb, 256, 0, s>>>(n, a, part);
    std::vector<double> h((size_t)nb * GK * GK * 2);
    cudaError_t e = cudaMemcpyAsync(h.data(), part, sizeof(double) * h.size(), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(part);
    if (e != cudaSuccess) {
        tmnd_set_error("tmnd_gram: %s", cudaGetErrorString(e));
        return TMND_ERR_CUDA;
    }
    for (int p = 0; p < k; p++)
        for (int q = p; q < k; q++) {
            double re = 0, im = 0;
            for (int b = 0; b < nb; b++) {
                re += h[((size_t)b * GK * GK + p * GK + q) * 2];
                im += h[((size_t)b * GK * GK + p * GK + q) * 2 + 1];
            }
            G_host[(p * k + q) * 2] = re;
            G_host[(p * k + q) * 2 + 1] = im;
            G_host[(q * k + p) * 2] = re;
            G_host[(q * k + p) * 2 + 1] = -im;
        }
    return TMND_OK;
}

// Network input for one (target shift, 8 solved shifts) pair, from the shifts and
// the multi-shift CG's scalar history (alpha_k, beta_k of the base system sigma0):
//   [0] log10 sigma_t; [1..8] log10(sigma_j / sigma_t); [9..16] asinh of the Lagrange
//   weights l_j(sigma_t) (Sec. 4.2.1); [17], [18] log10 of the smallest and largest Ritz
//   values of Qhat^2 from the Lanczos tridiagonal of the iteration
//   (T_kk = 1/alpha_k + beta_{k-1}/alpha_{k-1}, T_k,k+1 = sqrt(beta_k)/alpha_k, minus sigma0);
//   [19] log10 of the iteration count.  F = 20.
extern "C" tmnd_status tmnd_mlp_features(const double *nodes, double target, const double *ab_hist, int niter,
                                         double sigma0, float *out) {
    TMND_ARG_CHECK(nodes && out && niter >= 0 && target > 0, "tmnd_mlp_features: bad arguments");
    out[0] = (float)log10(target);
    for (int j = 0; j < 8; j++) {
        TMND_ARG_CHECK(nodes[j] > 0, "tmnd_mlp_features: nodes must be > 0");
        out[1 + j] = (float)log10(nodes[j] / target);
        double l = 1.0;
        for (int i = 0; i < 8; i++)
            if (i != j) l *= (target - nodes[i]) / (nodes[j] - nodes[i]);
        out[9 + j] = (float)asinh(l);
    }
    double lmin = 1e-3, lmax = 1.0;
    const int n = std::min(niter, 256);
    if (ab_hist && n >= 2) {
        std::vector<double> d(n), e(n > 1 ? n - 1 : 0);
        for (int k = 0; k < n; k++) {
            const double a = ab_hist[2 * k], bprev = k ? ab_hist[2 * (k - 1) + 1] : 0.0;
            const double aprev = k ? ab_hist[2 * (k - 1)] : 1.0;
            d[k] = 1.0 / a + (k ? bprev / aprev : 0.0);
            if (k + 1 < n) e[k] = sqrt(fabs(ab_hist[2 * k + 1])) / a;
        }
        lmin = tridiag_eig(d, e, 0) - sigma0;
        lmax = tridiag_eig(d, e, n - 1) - sigma0;
        if (!(lmin > 1e-12)) lmin = 1e-12;
        if (!(lmax > lmin)) lmax = lmin * 10;
    }
    out[17] = (float)log10(lmin);
    out[18] = (float)log10(lmax);
    out[19] = (float)log10((double)std::max(niter, 1));
    return TMND_OK;
}
