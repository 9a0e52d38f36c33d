// Multi-mass-shift CG (Sec. 1 "standard" solver; Sec. 4.2.2) for
// (Qhat^2 + sigma_i) x_i = b on the device, FP64.
//
// One Krylov space, generated by the base system sigma_0 = sigma[nsolve-1]
// (the smallest shift that must converge), serves every shift through
// Jegerlehner's recursion:
//   w = (Qhat^2 + sigma_0) p;  alpha = (r,r)/(p,w)
//   zeta_i' = zeta_i zeta_i^o alpha^o / (alpha beta^o (zeta_i^o - zeta_i) + zeta_i^o alpha^o (1 + alpha d_i))
//   alpha_i = alpha zeta_i'/zeta_i;  x_i += alpha_i p_i
//   r -= alpha w;  beta = (r,r)'/(r,r);  beta_i = beta (zeta_i'/zeta_i)^2
//   p_i = zeta_i' r + beta_i p_i;  p = r + beta p
// and shift i freezes once |zeta_i| |r| <= rho |b| (its residual is zeta_i r).
//
// Per iteration the device runs six kernels and never waits for the host:
//   1 even hop   t = kappa^2 A^-1 H p
//   2 odd hop    y = Mhat p, with block partials |y|^2, |p|^2
//                ((p, w) = |Mhat p|^2 + sigma_0 |p|^2, so w is never formed)
//   3 even hop   t = kappa^2 A(-mu)^-1 H gamma_5 y
//   4 odd hop    w = Mhat^+ y + sigma_0 p is applied directly: r' = r - alpha w
//                into the next slot of a ring of WIN residuals, block partials |r'|^2
//   5 scalars    one thread: deterministic sums of the partials, alpha, beta,
//                zeta_i', alpha_i, beta_i, freezing, done flag, and the window
//                coefficients below (single state in device memory)
//   6 p update   p = r' + beta p
// Windowed shift update: the shifted vectors are touched once per WIN
// iterations.  Within a window starting at iteration k0,
//   p_i^(k0+j) = P_j p_i^(k0) + sum_{l<j} Q_{j,l} r^(k0+l+1)
//   x_i^(k0+j) = x_i^(k0) + a_j p_i^(k0) + sum_l e_{j,l} r^(k0+l+1)
// with P, Q, a, e updated by the scalar kernel from alpha_i, beta_i, zeta_i'
// (P_{j+1} = beta_i P_j, Q_{j+1,l} = beta_i Q_{j,l}, Q_{j+1,j} = zeta_i',
//  a += alpha_i P_j, e_l += alpha_i Q_{j,l}), so that one pass at the end of
// the window applies WIN iterations of the recursion to x_i and p_i (exact
// algebra: the same recursion, regrouped).  This cuts the shifted vectors'
// HBM traffic and arithmetic by ~WIN/2.
// A block of `check_every` iterations (a multiple of WIN) is captured once
// into a CUDA graph and replayed; every kernel returns at once when the done
// flag is set, and the host reads the flag between replays (double-buffered,
// so the GPU never idles).
#include <math.h>
#include <string.h>

#include <chrono>
#include <vector>

#include "tmnd_internal.cuh"

namespace {

constexpr int NS = TMND_MAX_SHIFTS;
constexpr int UPD_THREADS = 256;

struct MMSState {
    double rr;          // (r, r) at the start of the current iteration
    double bb;          // (b, b)
    double alpha_old, beta_old;
    double zeta[NS], zeta_old[NS];
    int active[NS];
    int conv_iter[NS];
    int iter;
    int done;           // set once the base system converged, maxiter was hit, or a NaN appeared
    int status;         // TMND_OK / TMND_ERR_NAN
};

constexpr int WIN = 8;  // iterations per windowed shift update

struct MMSCoef {
    int skip;           // the solve was already done before this iteration
    double beta;
    // window coefficients per shift (see the header comment)
    double P[NS], Q[NS][WIN], a[NS], e[NS][WIN];
    int touched[NS];    // shift was active during this window
};

struct MMSConst {
    int nshift, nsolve, maxiter;
    double sigma0;
    double delta[NS];   // sigma_i - sigma_0
    double rho2;        // rho^2
};

template <typename T>
struct ShiftPtrsT {
    T *x[NS];
    T *p[NS];
};
using ShiftPtrs = ShiftPtrsT<double2>;

__global__ void k_init(long n, const double2 *__restrict__ b, double2 *__restrict__ r, double2 *__restrict__ p,
                       ShiftPtrs sp, int nshift, double *__restrict__ part) {
    __shared__ double red[40];
    double acc = 0.0;
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        double2 v = b[i];
        r[i] = v;
        p[i] = v;
        for (int s = 0; s < nshift; s++) {
            sp.p[s][i] = v;
            sp.x[s][i] = make_double2(0.0, 0.0);
        }
        acc = fma(v.x, v.x, fma(v.y, v.y, acc));
    }
    double s = block_sum(acc, red);
    if (threadIdx.x == 0) part[blockIdx.x] = s;
}

__device__ void init_state(MMSState *st, const double *__restrict__ part, int npart, const MMSConst &c,
                           double *red) {
    double bb = block_reduce_partials(part, npart, red);
    if (threadIdx.x != 0) return;
    st->rr = bb;
    st->bb = bb;
    st->alpha_old = 1.0;
    st->beta_old = 0.0;
    for (int s = 0; s < NS; s++) {
        st->zeta[s] = 1.0;
        st->zeta_old[s] = 1.0;
        st->active[s] = s < c.nshift;
        st->conv_iter[s] = -1;
    }
    st->iter = 0;
    st->done = (bb == 0.0) ? 1 : 0;   // b = 0: x = 0 is exact
    st->status = isfinite(bb) ? TMND_OK : TMND_ERR_NAN;
    if (!isfinite(bb)) st->done = 1;
}

__global__ void k_init_state(MMSState *st, const double *__restrict__ part, int npart, MMSConst c) {
    __shared__ double red[40];
    init_state(st, part, npart, c, red);
}

// Per-right-hand-side base shift and tolerance (batched single-shift solves, nshift = 1)
struct BatchConst {
    int on;
    double sigma0[TMND_MAX_BATCH], rho2[TMND_MAX_BATCH];
};
__device__ __forceinline__ MMSConst const_of(const MMSConst &c, const BatchConst &bc, int k) {
    MMSConst r = c;
    if (bc.on) {
        r.sigma0 = bc.sigma0[k];
        r.rho2 = bc.rho2[k];
    }
    return r;
}

// batched: block k initialises right-hand side k from partials [k][npart]
__global__ void k_init_state_b(MMSState *st, size_t st_stride, const double *__restrict__ part, int npart,
                               MMSConst c, BatchConst bc) {
    __shared__ double red[40];
    const MMSConst ck = const_of(c, bc, blockIdx.x);
    init_state((MMSState *)((char *)st + blockIdx.x * st_stride), part + (size_t)blockIdx.x * npart, npart, ck, red);
}

// Scalar step of the recursion (one block; thread 0 does the arithmetic).
// j = position of this iteration inside its window.
__device__ void scalars_step(MMSState *st, MMSCoef *cf, const double *__restrict__ part_norm, int nb_hop,
                             const double *__restrict__ part_rr, const MMSConst &c, int j, double *hist, int hist_cap,
                             double *red) {
    const int was_done = st->done;
    double yy = 0, pp = 0, rr_new = 0;
    if (!was_done) {
        yy = block_reduce_partials(part_norm, nb_hop, red);
        pp = block_reduce_partials(part_norm + nb_hop, nb_hop, red);
        rr_new = block_reduce_partials(part_rr, nb_hop, red);
    }
    if (threadIdx.x != 0) return;
    if (j == 0) {  // a new window starts: x_i and p_i are up to date
        for (int s = 0; s < c.nshift; s++) {
            cf->P[s] = 1.0;
            cf->a[s] = 0.0;
            cf->touched[s] = 0;
            for (int l = 0; l < WIN; l++) cf->Q[s][l] = cf->e[s][l] = 0.0;
        }
    }
    if (was_done) {
        cf->skip = 1;
        return;
    }
    const double alpha = st->rr / (yy + c.sigma0 * pp);
    const double beta = rr_new / st->rr;
    if (!isfinite(alpha) || !isfinite(rr_new) || !isfinite(beta)) {
        st->status = TMND_ERR_NAN;
        st->done = 1;
        cf->skip = 1;
        return;
    }
    cf->skip = 0;
    cf->beta = beta;
    const int it = st->iter + 1;
    if (hist && it <= hist_cap) {  // scalar history of the base recursion (Lanczos coefficients)
        hist[2 * (it - 1)] = alpha;
        hist[2 * (it - 1) + 1] = beta;
    }
    for (int s = 0; s < c.nshift; s++) {
        if (!st->active[s]) continue;
        const double z = st->zeta[s], zo = st->zeta_old[s];
        const double zn = z * zo * st->alpha_old /
                          (alpha * st->beta_old * (zo - z) + zo * st->alpha_old * (1.0 + alpha * c.delta[s]));
        const double ratio = zn / z;
        const double al = alpha * ratio;        // alpha_i
        const double be = beta * ratio * ratio; // beta_i
        // x_i += alpha_i p_i, with p_i = P p_i(k0) + sum_{l<j} Q_l r_l
        cf->a[s] += al * cf->P[s];
        for (int l = 0; l < j; l++) cf->e[s][l] += al * cf->Q[s][l];
        // p_i <- zeta_i' r' + beta_i p_i, r' in slot j
        cf->P[s] *= be;
        for (int l = 0; l < j; l++) cf->Q[s][l] *= be;
        cf->Q[s][j] = zn;
        cf->touched[s] = 1;
        st->zeta_old[s] = z;
        st->zeta[s] = zn;
        if (s < c.nsolve && zn * zn * rr_new <= c.rho2 * st->bb) {
            st->active[s] = 0;
            st->conv_iter[s] = it;
        }
    }
    st->rr = rr_new;
    st->alpha_old = alpha;
    st->beta_old = beta;
    st->iter = it;
    if (!st->active[c.nsolve - 1] || it >= c.maxiter) st->done = 1;
}

__global__ void k_scalars(MMSState *st, MMSCoef *cf, const double *__restrict__ part_norm, int nb_hop,
                          const double *__restrict__ part_rr, MMSConst c, int j, double *hist, int hist_cap) {
    __shared__ double red[40];
    scalars_step(st, cf, part_norm, nb_hop, part_rr, c, j, hist, hist_cap, red);
}

// Batched: block k runs the scalar step of right-hand side k (state and
// coefficients stride apart; partials [k][2][nb_hop] and [k][nb_hop]); the
// scalar history is kept for k = 0.
__global__ void k_scalars_b(MMSState *st, MMSCoef *cf, size_t st_stride, size_t cf_stride,
                            const double *__restrict__ part_norm, int nb_hop, const double *__restrict__ part_rr,
                            MMSConst c, BatchConst bc, int j, double *hist, int hist_cap) {
    __shared__ double red[40];
    const int k = blockIdx.x;
    const MMSConst ck = const_of(c, bc, k);
    scalars_step((MMSState *)((char *)st + k * st_stride), (MMSCoef *)((char *)cf + k * cf_stride),
                 part_norm + (size_t)2 * k * nb_hop, nb_hop, part_rr + (size_t)k * nb_hop, ck, j,
                 k == 0 ? hist : nullptr, hist_cap, red);
}

// done_all = every right-hand side's solve is done
__global__ void k_all_done(const MMSState *st, size_t st_stride, int nrhs, int *done_all) {
    int d = 1;
    for (int k = 0; k < nrhs; k++) d &= ((const MMSState *)((const char *)st + k * st_stride))->done;
    *done_all = d;
}

// p = r' + beta p (base search direction, every iteration)
__global__ void k_pupdate(long n, const MMSCoef *__restrict__ cf, const double2 *__restrict__ r,
                          double2 *__restrict__ p) {
    if (cf->skip) return;
    const double beta = cf->beta;
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        const double2 rv = r[i], pv = p[i];
        p[i] = make_double2(fma(beta, pv.x, rv.x), fma(beta, pv.y, rv.y));
    }
}

// Windowed multi-shift update (end of each window): for every shift active
// in the window, x_i += a p_i + sum_l e_l r_l and p_i = P p_i + sum_l Q_l r_l
// over the WIN residuals of the window.  The dominant HBM stream of the
// iteration at many shifts, now once per WIN iterations.
template <typename T>
struct RingPtrsT {
    const T *r[WIN];
};
using RingPtrs = RingPtrsT<double2>;

// T = double2 (FP64 path) or float2 (sloppy path; coefficients rounded to FP32)
template <typename T>
__global__ void __launch_bounds__(UPD_THREADS) k_window(long n, const MMSCoef *__restrict__ cf, RingPtrsT<T> ring,
                                                        ShiftPtrsT<T> sp, int nshift) {
    __shared__ double s_P[NS], s_a[NS], s_Q[NS][WIN], s_e[NS][WIN];
    __shared__ int s_idx[NS];
    __shared__ int s_n;
    if (threadIdx.x == 0) {
        int m = 0;
        for (int s = 0; s < nshift; s++)
            if (cf->touched[s]) {
                s_idx[m] = s;
                s_P[m] = cf->P[s];
                s_a[m] = cf->a[s];
                for (int l = 0; l < WIN; l++) {
                    s_Q[m][l] = cf->Q[s][l];
                    s_e[m][l] = cf->e[s][l];
                }
                m++;
            }
        s_n = m;
    }
    __syncthreads();
    const int m = s_n;
    if (m == 0) return;
    using R = decltype(T::x);
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        T rv[WIN];
#pragma unroll
        for (int l = 0; l < WIN; l++) rv[l] = ring.r[l][i];
        for (int k = 0; k < m; k++) {
            const int s = s_idx[k];
            T *xs = sp.x[s];
            T *ps = sp.p[s];
            const T pi = ps[i];
            T xv = xs[i];
            T pn;
            pn.x = (R)s_P[k] * pi.x;
            pn.y = (R)s_P[k] * pi.y;
            xv.x = fma((R)s_a[k], pi.x, xv.x);
            xv.y = fma((R)s_a[k], pi.y, xv.y);
#pragma unroll
            for (int l = 0; l < WIN; l++) {
                xv.x = fma((R)s_e[k][l], rv[l].x, xv.x);
                xv.y = fma((R)s_e[k][l], rv[l].y, xv.y);
                pn.x = fma((R)s_Q[k][l], rv[l].x, pn.x);
                pn.y = fma((R)s_Q[k][l], rv[l].y, pn.y);
            }
            xs[i] = xv;
            ps[i] = pn;
        }
    }
}

// |b - y|^2 partials (true residual)
__global__ void k_diff_norm(long n, const double2 *__restrict__ b, const double2 *__restrict__ y,
                            double *__restrict__ part) {
    __shared__ double red[40];
    double acc = 0.0;
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        double2 u = b[i], v = y[i];
        double dx = u.x - v.x, dy = u.y - v.y;
        acc = fma(dx, dx, fma(dy, dy, acc));
    }
    double s = block_sum(acc, red);
    if (threadIdx.x == 0) part[blockIdx.x] = s;
}


// ------------------------------------------------------------ sloppy path
// Sloppy vectors of R right-hand sides (right-hand side k's block follows k-1's):
//   ring slot l of k: ring0 + (k WIN + l) n;  b of k: b0 + k n;
//   p_s, x_s of k: p0/x0 + (k nshift + s) n;  16-bit p of k: p16 + k sb.
struct SloppyVecs {
    float2 *ring0, *b0, *p0, *x0;
    S16Out p16;
    long n;
    size_t sb;
    int nshift;
};

// One site per thread, right-hand side blockIdx.y: r = b (last ring slot),
// p = quantise(b), p_i = b, x_i = 0, partial |b|^2 into part[k][gridDim.x].
__global__ void k_init_s(int Vh, SloppyVecs v, double *__restrict__ part) {
    __shared__ double red[40];
    const int k = blockIdx.y;
    const float2 *b = v.b0 + k * v.n;
    float2 *r = v.ring0 + ((size_t)k * WIN + WIN - 1) * v.n;
    const S16Out p{(int4 *)((char *)v.p16.q + k * v.sb), (float *)((char *)v.p16.nrm + k * v.sb)};
    double acc = 0.0;
    for (int h = blockIdx.x * blockDim.x + threadIdx.x; h < Vh; h += gridDim.x * blockDim.x) {
        float w[24][2];
        float a = 0.0f;
#pragma unroll
        for (int c = 0; c < 24; c++) {
            const float2 bv = b[(size_t)c * Vh + h];
            w[c][0] = bv.x;
            w[c][1] = bv.y;
            r[(size_t)c * Vh + h] = bv;
            a = fmaf(bv.x, bv.x, fmaf(bv.y, bv.y, a));
            for (int s = 0; s < v.nshift; s++) {
                v.p0[((size_t)k * v.nshift + s) * v.n + (size_t)c * Vh + h] = bv;
                v.x0[((size_t)k * v.nshift + s) * v.n + (size_t)c * Vh + h] = make_float2(0.f, 0.f);
            }
        }
        s16_store_site(p, Vh, h, w);
        acc += a;
    }
    double t = block_sum(acc, red);
    if (threadIdx.x == 0) part[(size_t)k * gridDim.x + blockIdx.x] = t;
}

// p = r' + beta p for right-hand side blockIdx.y (slot j of its ring), p stored in 16 bits
__global__ void k_pupdate_s(int Vh, const MMSCoef *__restrict__ cf0, size_t cf_stride, SloppyVecs v, int j) {
    const int k = blockIdx.y;
    const MMSCoef *cf = (const MMSCoef *)((const char *)cf0 + k * cf_stride);
    if (cf->skip) return;
    const float beta = (float)cf->beta;
    const float2 *r = v.ring0 + ((size_t)k * WIN + j) * v.n;
    const S16Out p{(int4 *)((char *)v.p16.q + k * v.sb), (float *)((char *)v.p16.nrm + k * v.sb)};
    const S16In pin{p.q, p.nrm};
    for (int h = blockIdx.x * blockDim.x + threadIdx.x; h < Vh; h += gridDim.x * blockDim.x) {
        float w[24][2];
        s16_load_site(pin, Vh, h, w);
#pragma unroll
        for (int c = 0; c < 24; c++) {
            const float2 rv = r[(size_t)c * Vh + h];
            w[c][0] = fmaf(beta, w[c][0], rv.x);
            w[c][1] = fmaf(beta, w[c][1], rv.y);
        }
        s16_store_site(p, Vh, h, w);
    }
}

// Windowed multi-shift update of right-hand side blockIdx.y (see k_window), FP32.
__global__ void __launch_bounds__(UPD_THREADS) k_window_s(const MMSCoef *__restrict__ cf0, size_t cf_stride,
                                                          SloppyVecs v) {
    __shared__ float s_P[NS], s_a[NS], s_Q[NS][WIN], s_e[NS][WIN];
    __shared__ int s_idx[NS];
    __shared__ int s_n;
    const int k = blockIdx.y;
    const MMSCoef *cf = (const MMSCoef *)((const char *)cf0 + k * cf_stride);
    if (threadIdx.x == 0) {
        int m = 0;
        for (int s = 0; s < v.nshift; s++)
            if (cf->touched[s]) {
                s_idx[m] = s;
                s_P[m] = (float)cf->P[s];
                s_a[m] = (float)cf->a[s];
                for (int l = 0; l < WIN; l++) {
                    s_Q[m][l] = (float)cf->Q[s][l];
                    s_e[m][l] = (float)cf->e[s][l];
                }
                m++;
            }
        s_n = m;
    }
    __syncthreads();
    const int m = s_n;
    if (m == 0) return;
    const float2 *ring = v.ring0 + (size_t)k * WIN * v.n;
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < v.n; i += (long)gridDim.x * blockDim.x) {
        float2 rv[WIN];
#pragma unroll
        for (int l = 0; l < WIN; l++) rv[l] = ring[l * v.n + i];
        for (int q = 0; q < m; q++) {
            const size_t off = ((size_t)k * v.nshift + s_idx[q]) * v.n + i;
            const float2 pi = v.p0[off];
            float2 xv = v.x0[off];
            float2 pn = make_float2(s_P[q] * pi.x, s_P[q] * pi.y);
            xv.x = fmaf(s_a[q], pi.x, xv.x);
            xv.y = fmaf(s_a[q], pi.y, xv.y);
#pragma unroll
            for (int l = 0; l < WIN; l++) {
                xv.x = fmaf(s_e[q][l], rv[l].x, xv.x);
                xv.y = fmaf(s_e[q][l], rv[l].y, xv.y);
                pn.x = fmaf(s_Q[q][l], rv[l].x, pn.x);
                pn.y = fmaf(s_Q[q][l], rv[l].y, pn.y);
            }
            v.x0[off] = xv;
            v.p0[off] = pn;
        }
    }
}

// x += (double) e  (FP64 accumulation of a sloppy correction)
__global__ void k_add_f32_to_f64(long n, const float2 *__restrict__ e, double2 *__restrict__ x) {
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        const float2 d = e[i];
        double2 v = x[i];
        v.x += (double)d.x;
        v.y += (double)d.y;
        x[i] = v;
    }
}

// r = b - y in FP64 and block partials |r|^2 (true residual of the refinement)
__global__ void k_resid(long n, const double2 *__restrict__ b, const double2 *__restrict__ y,
                        double2 *__restrict__ r, double *__restrict__ part) {
    __shared__ double red[40];
    double acc = 0.0;
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        const double2 u = b[i], v = y[i];
        const double2 d = make_double2(u.x - v.x, u.y - v.y);
        r[i] = d;
        acc = fma(d.x, d.x, fma(d.y, d.y, acc));
    }
    double t = block_sum(acc, red);
    if (threadIdx.x == 0) part[blockIdx.x] = t;
}


// ------------------------------------------------------------- hybrid helpers
// out = in * (ar + i ai) + out (FP64 complex axpy)
__global__ void k_zaxpy64(long n, double ar, double ai, const double2 *__restrict__ in, double2 *__restrict__ out) {
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        const double2 v = in[i];
        double2 o = out[i];
        o.x += ar * v.x - ai * v.y;
        o.y += ar * v.y + ai * v.x;
        out[i] = o;
    }
}
// FP64 -> FP32 with a real scale
__global__ void k_to_f32_scaled(long n, double a, const double2 *__restrict__ in, float2 *__restrict__ out) {
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
        out[i] = make_float2((float)(a * in[i].x), (float)(a * in[i].y));
}
// x = i/(2s) (yp - ym), yp/ym FP32 odd parts, x FP64   (Sec. 3.1, Eq. "lindif")
__global__ void k_casec_combine(long n, double s, const float2 *__restrict__ yp, const float2 *__restrict__ ym,
                                double2 *__restrict__ x) {
    const double c = 1.0 / (2.0 * s);
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        const double dr = (double)yp[i].x - ym[i].x, di = (double)yp[i].y - ym[i].y;
        x[i] = make_double2(-c * di, c * dr);
    }
}

int site_blocks(int Vh) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 152;
    long want = (Vh + 127) / 128, cap = (long)sms * 8;
    return (int)(want < cap ? want : cap);
}

int stream_blocks(long n) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 152;
    long want = (n + UPD_THREADS - 1) / UPD_THREADS;
    long cap = (long)sms * 8;   // 8 resident 256-thread blocks per SM
    return (int)(want < cap ? want : cap);
}


// Capture `check_every` iterations of `body` into a CUDA graph and replay it
// until the device-side done flag is set (or the iteration budget is spent).
// The host reads the flag of replay j-1 while replay j runs.  With profiling,
// body calls mark(0/1/2) to place event-record nodes; two graph instances
// alternate so that one instance's events are read while the other runs.
struct LoopOut {
    long nlaunch = 0;
    std::vector<float> hop_t, upd_t;  // per iteration (profiling only)
};

template <typename Body>
tmnd_status run_graph_loop(cudaStream_t s, const int *done_dev, int maxiter, int check_every, int profile, Body body,
                           LoopOut &out) {
    const int ninst = profile ? 2 : 1;
    cudaGraphExec_t exec[2] = {nullptr, nullptr};
    std::vector<cudaEvent_t> evs;  // [inst][k][3]
    if (profile) {
        evs.resize((size_t)ninst * check_every * 3);
        for (auto &e : evs) cudaEventCreate(&e);
    }
    auto ev = [&](int inst, int k, int j) { return evs[((size_t)inst * check_every + k) * 3 + j]; };
    auto cleanup = [&]() {
        for (int inst = 0; inst < ninst; inst++)
            if (exec[inst]) cudaGraphExecDestroy(exec[inst]);
        for (auto &e : evs) cudaEventDestroy(e);
    };
    for (int inst = 0; inst < ninst; inst++) {
        cudaGraph_t graph = nullptr;
        cudaError_t ce = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
        if (ce == cudaSuccess) {
            for (int k = 0; k < check_every; k++) {
                auto mark = [&](int which) {
                    if (profile) cudaEventRecordWithFlags(ev(inst, k, which), s, cudaEventRecordExternal);
                };
                body(k, mark);
            }
            ce = cudaStreamEndCapture(s, &graph);
        }
        if (ce == cudaSuccess) ce = cudaGraphInstantiate(&exec[inst], graph, 0);
        if (ce != cudaSuccess) {
            // never leave the stream in capture mode, nor the error pending for later calls
            cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
            if (cudaStreamIsCapturing(s, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone) {
                cudaGraph_t g2 = nullptr;
                cudaStreamEndCapture(s, &g2);
                if (g2) cudaGraphDestroy(g2);
            }
            cudaGetLastError();
        }
        if (graph) cudaGraphDestroy(graph);
        if (ce != cudaSuccess) {
            cleanup();
            tmnd_set_error("mms_cg_solve: graph capture failed: %s", cudaGetErrorString(ce));
            return TMND_ERR_CUDA;
        }
    }
    int *flags = nullptr;  // pinned [L + 1]
    const int L = profile ? 1 : 2;  // replays queued ahead of the flag being read
    cudaEvent_t fev[3];
    cudaError_t err = cudaHostAlloc((void **)&flags, (L + 1) * sizeof(int), cudaHostAllocDefault);
    if (err != cudaSuccess) {
        cleanup();
        tmnd_set_error("mms_cg_solve: cudaHostAlloc: %s", cudaGetErrorString(err));
        return TMND_ERR_CUDA;
    }
    for (int i = 0; i <= L; i++) cudaEventCreateWithFlags(&fev[i], cudaEventDisableTiming);
    auto harvest = [&](long j) {  // read the events of replay j (complete)
        int inst = (int)(j % ninst);
        for (int k = 0; k < check_every; k++) {
            float a = 0.f, b2 = 0.f;
            if (cudaEventElapsedTime(&a, ev(inst, k, 0), ev(inst, k, 1)) != cudaSuccess ||
                cudaEventElapsedTime(&b2, ev(inst, k, 1), ev(inst, k, 2)) != cudaSuccess) {
                cudaGetLastError();
                a = b2 = nanf("");
            }
            out.hop_t.push_back(a);
            out.upd_t.push_back(b2);
        }
    };
    const long max_launch = (long)maxiter / check_every + 2 + L;
    for (long j = 0; j < max_launch && err == cudaSuccess; j++) {
        err = cudaGraphLaunch(exec[j % ninst], s);
        if (err != cudaSuccess) break;
        out.nlaunch++;
        cudaMemcpyAsync(&flags[j % (L + 1)], done_dev, sizeof(int), cudaMemcpyDeviceToHost, s);
        cudaEventRecord(fev[j % (L + 1)], s);
        if (j >= L) {
            err = cudaEventSynchronize(fev[(j - L) % (L + 1)]);
            if (err == cudaSuccess && profile) harvest(j - L);
            if (err == cudaSuccess && flags[(j - L) % (L + 1)]) break;
        }
    }
    if (err == cudaSuccess) err = cudaStreamSynchronize(s);
    if (err == cudaSuccess && profile && out.nlaunch > 0) harvest(out.nlaunch - 1);
    for (int i = 0; i <= L; i++) cudaEventDestroy(fev[i]);
    cudaFreeHost(flags);
    cleanup();
    if (err != cudaSuccess) {
        tmnd_set_error("mms_cg_solve: %s", cudaGetErrorString(err));
        return TMND_ERR_CUDA;
    }
    return TMND_OK;
}

}  // namespace

// One right-hand side.  work holds the WIN residual slots, p, y, te, p_i[nshift]
// (spinor-sized each).  Residual r^(k0+j+1) of window position j goes to slot
// j; position 0 reads slot WIN-1 (the last residual of the previous window,
// or b at the start).
static tmnd_status mms_one_rhs(tmnd_gauge *g, const double2 *b, double2 *const *x, const double *sigma, int nshift,
                               int nsolve, double rho, int maxiter, int check_every, int profile,
                               tmnd_solve_info *info, cudaStream_t s, int rhs_index, double *hist, int hist_cap,
                               bool certify = true) {
    const size_t sp = tmnd_spinor_bytes(g);
    const long n = (long)(sp / sizeof(double2));
    char *w = (char *)g->work;
    double2 *slot[WIN];
    RingPtrs ring;
    for (int l = 0; l < WIN; l++) ring.r[l] = slot[l] = (double2 *)(w + l * sp);
    double2 *r = slot[WIN - 1];
    double2 *p = (double2 *)(w + (WIN + 0) * sp);
    double2 *y = (double2 *)(w + (WIN + 1) * sp);
    double2 *te = (double2 *)(w + (WIN + 2) * sp);
    ShiftPtrs ptrs = {};
    for (int i = 0; i < nshift; i++) {
        ptrs.x[i] = x[i] + (size_t)rhs_index * n;
        ptrs.p[i] = (double2 *)(w + (WIN + 3 + i) * sp);
    }
    // small device area after the partials
    const int nb_hop = hop_blocks(g->geom);
    const int nb_str = stream_blocks(n);
    double *part_norm = (double *)g->partials;              // 2 * nb_hop
    double *part_rr = part_norm + 2 * nb_hop;               // nb_hop
    double *part_str = part_rr + nb_hop;                    // nb_str
    char *tail = (char *)(part_str + nb_str);
    tail = (char *)(((uintptr_t)tail + 255) & ~(uintptr_t)255);
    MMSState *st = (MMSState *)tail;
    MMSCoef *cf = (MMSCoef *)(tail + ((sizeof(MMSState) + 255) & ~(size_t)255));

    MMSConst c = {};
    c.nshift = nshift;
    c.nsolve = nsolve;
    c.maxiter = maxiter;
    c.sigma0 = sigma[nsolve - 1];
    for (int i = 0; i < nshift; i++) c.delta[i] = sigma[i] - c.sigma0;
    c.rho2 = rho * rho;

    k_init<<<nb_str, UPD_THREADS, 0, s>>>(n, b, r, p, ptrs, nshift, part_str);
    k_init_state<<<1, 256, 0, s>>>(st, part_str, nb_str, c);
    TMND_CUDA_TRY(cudaGetLastError());

    auto body = [&](int k, auto mark) {
        const int j = k % WIN;  // position inside the window
        mark(0);
        HopEpiArgs e1 = {};
        e1.part_out = part_norm;
        e1.done = &st->done;
        launch_hop_even_f64(g->geom, g->st, g->links, p, te, false, &st->done, s);
        launch_hop_odd_f64(g->geom, g->st, g->links, p, te, y, false, EPI_STORE_NORMS, e1, s);
        launch_hop_even_f64(g->geom, g->st, g->links, y, te, true, &st->done, s);
        HopEpiArgs e2 = {};
        e2.sigma = c.sigma0;
        e2.aux = p;
        e2.r_in = slot[(j + WIN - 1) % WIN];
        e2.r = slot[j];
        e2.part_out = part_rr;
        e2.part_in = part_norm;
        e2.npart_in = nb_hop;
        e2.rr = &st->rr;
        e2.done = &st->done;
        launch_hop_odd_f64(g->geom, g->st, g->links, y, te, nullptr, true, EPI_MMS_R, e2, s);
        mark(1);
        k_scalars<<<1, 256, 0, s>>>(st, cf, part_norm, nb_hop, part_rr, c, j, hist, hist_cap);
        k_pupdate<<<nb_str, UPD_THREADS, 0, s>>>(n, cf, slot[j], p);
        if (j == WIN - 1) k_window<double2><<<nb_str, UPD_THREADS, 0, s>>>(n, cf, ring, ptrs, nshift);
        mark(2);
    };
    LoopOut lo;
    tmnd_status ls = run_graph_loop(s, &st->done, maxiter, check_every, profile, body, lo);
    if (ls != TMND_OK) return ls;
    const long nlaunch = lo.nlaunch;
    std::vector<float> &hop_t = lo.hop_t, &upd_t = lo.upd_t;
    if (info) {
        info->launches += 2 + nlaunch * ((long long)check_every * 6 + check_every / WIN) + 5LL * nshift;
        info->fp64_applies += nshift;
    }

    MMSState hs;
    TMND_CUDA_TRY(cudaMemcpy(&hs, st, sizeof hs, cudaMemcpyDeviceToHost));
    if (!certify) {  // a correction solve: its caller certifies the corrected solution
        if (info) info->iters = hs.iter;
        if (hs.status == TMND_ERR_NAN) {
            tmnd_set_error("mms_cg_solve: NaN/Inf in a reduction of a defect correction at iteration %d", hs.iter);
            return TMND_ERR_NAN;
        }
        return TMND_OK;
    }

    // true residual |b - (Qhat^2 + sigma_i) x_i| / |b| with the operator; leaves the defect
    // b - (Qhat^2 + sigma_i) x_i in r
    std::vector<double> hpart(nb_str);
    auto true_res_of = [&](int i, double *tr) -> tmnd_status {
        HopEpiArgs ea = {};
        launch_hop_even_f64(g->geom, g->st, g->links, ptrs.x[i], te, false, nullptr, s);
        launch_hop_odd_f64(g->geom, g->st, g->links, ptrs.x[i], te, r, false, EPI_STORE, ea, s);
        HopEpiArgs e2 = {};
        e2.sigma = sigma[i];
        e2.aux = ptrs.x[i];
        launch_hop_even_f64(g->geom, g->st, g->links, r, te, true, nullptr, s);
        launch_hop_odd_f64(g->geom, g->st, g->links, r, te, y, true, EPI_SHIFT, e2, s);
        k_resid<<<nb_str, UPD_THREADS, 0, s>>>(n, b, y, r, part_str);
        cudaError_t e3 = cudaMemcpyAsync(hpart.data(), part_str, sizeof(double) * nb_str, cudaMemcpyDeviceToHost, s);
        if (e3 == cudaSuccess) e3 = cudaStreamSynchronize(s);
        if (e3 != cudaSuccess) {
            tmnd_set_error("mms_cg_solve: %s", cudaGetErrorString(e3));
            return TMND_ERR_CUDA;
        }
        double acc = 0;
        for (int k = 0; k < nb_str; k++) acc += hpart[k];
        *tr = hs.bb > 0 ? sqrt(acc / hs.bb) : 0.0;
        return TMND_OK;
    };
    // A required shift whose true residual drifted above rho (the recursively updated residual
    // drifts from the true one by rounding) is finished by FP64 defect correction (Sec. 3.1
    // stopping rule on the true residual): (Qhat^2 + sigma_i) e = d by a single-shift FP64 CG to
    // |d - (Qhat^2 + sigma_i) e| <= rho |b| / 2, x_i += e, the true residual again.
    double2 *corr = nullptr;  // d, e: two spinors, allocated the first time a shift needs them
    tmnd_status cst = TMND_OK;
    for (int i = 0; i < nshift && cst == TMND_OK; i++) {
        double tr = 0;
        cst = true_res_of(i, &tr);
        const bool nan = !isfinite(tr);
        for (int round = 0; cst == TMND_OK && !nan && i < nsolve && hs.status == TMND_OK && tr > rho && round < 4;
             round++) {
            if (!corr && cudaMalloc(&corr, 2 * sizeof(double2) * n) != cudaSuccess) {
                corr = nullptr;
                tmnd_set_error("mms_cg_solve: no device memory for the defect correction");
                cst = TMND_ERR_OOM;
                break;
            }
            double2 *d = corr, *e = corr + n;
            TMND_CUDA_TRY(cudaMemcpyAsync(d, r, sizeof(double2) * n, cudaMemcpyDeviceToDevice, s));
            const double rel = fmin(0.5, 0.5 * rho / tr);  // relative to |d| = tr |b|
            tmnd_solve_info sub = {};
            double2 *ev[1] = {e};
            cst = mms_one_rhs(g, d, ev, sigma + i, 1, 1, rel, maxiter, check_every, 0, &sub, s, 0, nullptr, 0,
                              false);
            if (cst != TMND_OK) break;
            k_zaxpy64<<<nb_str, UPD_THREADS, 0, s>>>(n, 1.0, 0.0, e, ptrs.x[i]);
            cst = true_res_of(i, &tr);
            if (info) {
                info->refine_iters += sub.iters;
                info->fp64_applies += 1;
                info->launches += sub.launches + 6;
                if (round + 1 > info->refine_rounds) info->refine_rounds = round + 1;
            }
        }
        if (info && (rhs_index == 0 || tr > info->true_res[i] || nan)) info->true_res[i] = tr;
    }
    if (corr) cudaFree(corr);
    if (cst != TMND_OK) return cst;
    if (info && profile) {
        // only the iterations that did work (later ones returned at once)
        for (int k = 0; k < hs.iter && k < (int)hop_t.size(); k++) {
            info->hop_ms += hop_t[k];
            info->update_ms += upd_t[k];
        }
    }
    if (info) {
        if (rhs_index == 0 || hs.iter > info->iters) info->iters = hs.iter;
        for (int i = 0; i < nshift; i++) {
            if (rhs_index == 0 || hs.conv_iter[i] > info->conv_iter[i] || hs.conv_iter[i] < 0)
                info->conv_iter[i] = hs.conv_iter[i];
            info->zeta[i] = hs.zeta[i];
        }
    }
    if (hs.status == TMND_ERR_NAN) {
        tmnd_set_error("mms_cg_solve: NaN/Inf in a reduction at iteration %d", hs.iter);
        return TMND_ERR_NAN;
    }
    if (hs.active[nsolve - 1] && hs.bb > 0) {
        tmnd_set_error("mms_cg_solve: base shift not converged after %d iterations", hs.iter);
        return TMND_ERR_NOCONV;
    }
    return TMND_OK;
}


// ---------------------------------------------------------- mixed precision
// Workspace of the mixed solve: FP64 vectors for one right-hand side at a time
// (defect correction), sloppy vectors for nrhs right-hand sides at once.
struct MixedWork {
    double2 *r64, *y64, *te64;          // FP64: defect, (Qhat^2+sigma) x, even temporary
    SloppyVecs v;                       // FP32 ring, b, p_i, x_i and the 16-bit p (nrhs blocks)
    void *y16, *te16;                   // 16-bit stencil temporaries, nrhs blocks of v.sb
    int nrhs;
    float2 *ring(int k, int l) const { return v.ring0 + ((size_t)k * WIN + l) * v.n; }
    float2 *b32(int k) const { return v.b0 + (size_t)k * v.n; }
    float2 *x32(int k, int s) const { return v.x0 + ((size_t)k * v.nshift + s) * v.n; }
    // a view for one right-hand side and one shift on the same memory (right-hand side 0's slots)
    MixedWork single() const {
        MixedWork w = *this;
        w.v.nshift = 1;
        w.nrhs = 1;
        return w;
    }
};

static size_t mixed_work_bytes(int Vh, int nshift, int nrhs = 1) {
    const size_t s64 = spinor_bytes_prec(Vh, TMND_F64), s32 = spinor_bytes_prec(Vh, TMND_F32),
                 s16 = spinor_bytes_prec(Vh, TMND_S16);
    return 3 * s64 + (size_t)nrhs * ((WIN + 1 + 2 * (size_t)nshift) * s32 + 3 * s16);
}

static MixedWork mixed_work(void *base, int Vh, int nshift, int nrhs = 1) {
    const size_t s64 = spinor_bytes_prec(Vh, TMND_F64), s32 = spinor_bytes_prec(Vh, TMND_F32),
                 s16 = spinor_bytes_prec(Vh, TMND_S16);
    char *w = (char *)base;
    MixedWork m;
    m.r64 = (double2 *)w; w += s64;
    m.y64 = (double2 *)w; w += s64;
    m.te64 = (double2 *)w; w += s64;
    m.v.n = 24L * Vh;
    m.v.sb = s16;
    m.v.nshift = nshift;
    m.nrhs = nrhs;
    m.v.ring0 = (float2 *)w; w += (size_t)nrhs * WIN * s32;
    m.v.b0 = (float2 *)w; w += (size_t)nrhs * s32;
    m.v.p0 = (float2 *)w; w += (size_t)nrhs * nshift * s32;
    m.v.x0 = (float2 *)w; w += (size_t)nrhs * nshift * s32;
    m.v.p16 = s16_out(w, Vh); w += (size_t)nrhs * s16;
    m.y16 = w; w += (size_t)nrhs * s16;
    m.te16 = w;
    return m;
}

// Sloppy multi-shift CG on m's right-hand sides b32(k), k < m.nrhs, for shifts
// sigma[0..nshift), solutions into x32(k, i).  Same recursion and kernel sequence
// as the FP64 solver, with the stencil in FP32/16-bit (dslash_s16.cu).  All
// right-hand sides iterate in lockstep: each stencil launch covers all of them,
// each has its own scalars and stops on its own (later launches skip it), and the
// loop ends when all are done.  hs receives the final state of each.
// With sig_k / rho_k (nshift = 1): right-hand side k solves (Qhat^2 + sig_k[k]) e = b_k to rho_k[k].
static tmnd_status mms_sloppy(tmnd_gauge *g, const MixedWork &m, const double *sigma, int nshift, int nsolve,
                              double rho, int maxiter, int check_every, int profile, cudaStream_t s,
                              std::vector<MMSState> &hs, LoopOut &lo, double *hist = nullptr, int hist_cap = 0,
                              const double *sig_k = nullptr, const double *rho_k = nullptr) {
    const int Vh = g->geom.Vh;
    const long n = 24L * Vh;
    const int R = m.nrhs;
    // launch shape of the stencil for R right-hand sides per launch (tuned on first use, before
    // any graph capture); every launch of the solve uses it, so the partial counts agree
    tmnd_status ts = s16_autotune(g, R, s, nullptr, nullptr);
    if (ts != TMND_OK) return ts;
    const int shape = s16_shape_mms(g->geom, R);
    const int nb_hop = hop_blocks_s16(g->geom, shape);
    const int nb_str = stream_blocks(n);
    const int nb_site = site_blocks(Vh);
    double *part_norm = (double *)g->partials;                 // [R][2][nb_hop]
    double *part_rr = part_norm + (size_t)2 * R * nb_hop;      // [R][nb_hop]
    double *part_str = part_rr + (size_t)R * nb_hop;           // [R][nb_site]
    char *tail = (char *)(part_str + (size_t)R * (nb_str > nb_site ? nb_str : nb_site));
    tail = (char *)(((uintptr_t)tail + 255) & ~(uintptr_t)255);
    const size_t st_stride = (sizeof(MMSState) + 255) & ~(size_t)255;
    const size_t cf_stride = (sizeof(MMSCoef) + 255) & ~(size_t)255;
    MMSState *st = (MMSState *)tail;
    MMSCoef *cf = (MMSCoef *)(tail + R * st_stride);
    int *done_all = (int *)(tail + R * (st_stride + cf_stride));

    MMSConst c = {};
    c.nshift = nshift;
    c.nsolve = nsolve;
    c.maxiter = maxiter;
    c.sigma0 = sigma[nsolve - 1];
    for (int i = 0; i < nshift; i++) c.delta[i] = sigma[i] - c.sigma0;
    c.rho2 = rho * rho;
    BatchConst bc = {};
    if (sig_k) {
        bc.on = 1;
        for (int k = 0; k < R; k++) {
            bc.sigma0[k] = sig_k[k];
            bc.rho2[k] = rho_k[k] * rho_k[k];
        }
    }
    SloppyVecs v = m.v;
    v.nshift = nshift;
    const S16Out p16 = v.p16, y16 = s16_out(m.y16, Vh), te16 = s16_out(m.te16, Vh);
    const S16In p16i{p16.q, p16.nrm}, y16i{y16.q, y16.nrm}, te16i{te16.q, te16.nrm};
    S16Batch bt;
    bt.nrhs = R;
    bt.stride = v.sb;
    bt.rdone = &st->done;
    bt.rdone_stride = (int)(st_stride / sizeof(int));
    bt.shape = shape;

    k_init_s<<<dim3(nb_site, R), 128, 0, s>>>(Vh, v, part_str);
    k_init_state_b<<<R, 256, 0, s>>>(st, st_stride, part_str, nb_site, c, bc);
    k_all_done<<<1, 1, 0, s>>>(st, st_stride, R, done_all);
    TMND_CUDA_TRY(cudaGetLastError());

    auto body = [&](int k, auto mark) {
        const int j = k % WIN;
        mark(0);
        S16EpiArgs e1 = {};
        e1.part_out = part_norm;
        e1.done = done_all;
        launch_hop_even_s16(g->geom, g->stf, g->links_s16, p16i, te16, false, done_all, s, bt);
        launch_hop_odd_s16(g->geom, g->stf, g->links_s16, p16i, te16i, y16, false, EPI_STORE_NORMS, e1, s, bt);
        launch_hop_even_s16(g->geom, g->stf, g->links_s16, y16i, te16, true, done_all, s, bt);
        S16EpiArgs e2 = {};
        e2.sigma = c.sigma0;
        e2.aux = p16i;
        e2.r_in = m.ring(0, (j + WIN - 1) % WIN);
        e2.r = m.ring(0, j);
        e2.r_stride = (long)WIN * n;
        e2.part_out = part_rr;
        e2.part_in = part_norm;
        e2.npart_in = nb_hop;
        e2.rr = &st->rr;
        e2.rr_stride = (int)(st_stride / sizeof(double));
        e2.done = done_all;
        e2.per_rhs_sigma = bc.on;
        for (int q = 0; q < R && bc.on; q++) e2.sigma_k[q] = bc.sigma0[q];
        launch_hop_odd_s16(g->geom, g->stf, g->links_s16, y16i, te16i, S16Out{}, true, EPI_MMS_R, e2, s, bt);
        mark(1);
        k_scalars_b<<<R, 256, 0, s>>>(st, cf, st_stride, cf_stride, part_norm, nb_hop, part_rr, c, bc, j, hist,
                                      hist_cap);
        k_all_done<<<1, 1, 0, s>>>(st, st_stride, R, done_all);
        k_pupdate_s<<<dim3(nb_site, R), 128, 0, s>>>(Vh, cf, cf_stride, v, j);
        if (j == WIN - 1) k_window_s<<<dim3(nb_str, R), UPD_THREADS, 0, s>>>(cf, cf_stride, v);
        mark(2);
    };
    tmnd_status ls = run_graph_loop(s, done_all, maxiter, check_every, profile, body, lo);
    if (ls != TMND_OK) return ls;
    hs.resize(R);
    for (int k = 0; k < R; k++)
        TMND_CUDA_TRY(cudaMemcpy(&hs[k], (char *)st + k * st_stride, sizeof(MMSState), cudaMemcpyDeviceToHost));
    for (int k = 0; k < R; k++)
        if (hs[k].status == TMND_ERR_NAN) {
            tmnd_set_error("mms_cg_solve: NaN/Inf in a sloppy reduction at iteration %d (right-hand side %d)",
                           hs[k].iter, k);
            return TMND_ERR_NAN;
        }
    return TMND_OK;
}

// partial-buffer bytes the sloppy solve of nrhs right-hand sides needs
static size_t sloppy_partial_bytes(const Geom &geom, int nrhs) {
    const long n = 24L * geom.Vh;
    const int nb_hop = hop_blocks_s16_max(geom);
    const int nb_str = stream_blocks(n), nb_site = site_blocks(geom.Vh);
    const size_t st_stride = (sizeof(MMSState) + 255) & ~(size_t)255;
    const size_t cf_stride = (sizeof(MMSCoef) + 255) & ~(size_t)255;
    return sizeof(double) * (size_t)nrhs * (3 * (size_t)nb_hop + (nb_str > nb_site ? nb_str : nb_site)) + 256 +
           (size_t)nrhs * (st_stride + cf_stride) + 256;
}

// (Qhat^2 + sigma) x - b in FP64 into m.r64 (as b - (...)), returns |r|^2 on the host.
static tmnd_status fp64_defect(tmnd_gauge *g, const MixedWork &m, const double2 *b, const double2 *x, double sigma,
                               cudaStream_t s, double *rr) {
    const long n = 24L * g->geom.Vh;
    const int nb = stream_blocks(n);
    double *part = (double *)g->partials;
    HopEpiArgs ea = {};
    launch_hop_even_f64(g->geom, g->st, g->links, x, m.te64, false, nullptr, s);
    launch_hop_odd_f64(g->geom, g->st, g->links, x, m.te64, m.r64, false, EPI_STORE, ea, s);
    HopEpiArgs e2 = {};
    e2.sigma = sigma;
    e2.aux = x;
    launch_hop_even_f64(g->geom, g->st, g->links, m.r64, m.te64, true, nullptr, s);
    launch_hop_odd_f64(g->geom, g->st, g->links, m.r64, m.te64, m.y64, true, EPI_SHIFT, e2, s);
    k_resid<<<nb, UPD_THREADS, 0, s>>>(n, b, m.y64, m.r64, part);
    std::vector<double> h(nb);
    TMND_CUDA_TRY(cudaMemcpyAsync(h.data(), part, sizeof(double) * nb, cudaMemcpyDeviceToHost, s));
    TMND_CUDA_TRY(cudaStreamSynchronize(s));
    double acc = 0;
    for (int k = 0; k < nb; k++) acc += h[k];
    *rr = acc;
    return TMND_OK;
}

struct RefineStats {
    int fp64 = 0, rounds = 0, iters = 0, f32 = 0;
    long long launches = 0;
    double hop_ms = 0, upd_ms = 0;
    double fp64_ms = 0;  // wall time of the FP64 defects (each ends with a host read)
};

// wall-clock milliseconds since t0
static double ms_since(std::chrono::steady_clock::time_point t0) {
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
}

// FP64 defect correction (Sec. 3.1 stopping rule on the true residual) of a set of
// (right-hand side, shift) pairs: per round, each pending pair's defect
// r = b - (Qhat^2 + sigma) x in FP64; a pair stops once |r| <= rho |b|; the others
// solve (Qhat^2 + sigma) e = r together in one batched sloppy CG (up to
// TMND_MAX_BATCH pairs per launch, each with its own shift and the tolerance its
// defect needs) and add e in FP64.  *res receives each pair's final FP64 relative
// residual.  The sloppy solve's vectors are laid out over the workspace at base.
struct DCItem {
    const double2 *b;
    double2 *x;
    double sigma, bb;
    double *res;
    double *res0 = nullptr;  // optional: the relative residual of the first round (before any correction)
};

// Inner iterative refinement of one chunk of pairs, in FP32 (between two FP64 defects):
// the defect d (FP32 copy) is solved by batched sloppy CGs on the 16-bit operator, each
// reducing the current inner residual by the factor the pair still needs (at least
// `floor`); after each, the correction accumulated so far is checked with the FP32
// operator, r = d - (Qhat^2 + sigma) e (accurate to ~1e-7 of |d|, where the 16-bit
// operator's own ~4e-5 would stall), and r is the next right-hand side.  A pair stops
// once |r| <= target; the others go on, at most `max_inner` sloppy solves.
tmnd_status apply_f32(tmnd_gauge *g, float2 *out, const float2 *in, int op, double sigma, int nrhs, float2 *te,
                      float2 *yo, cudaStream_t s);

// r = d - y (FP32) and block partials |r|^2 (FP64)
__global__ void k_resid32(long n, const float2 *__restrict__ d, const float2 *__restrict__ y, float2 *__restrict__ r,
                          double *__restrict__ part) {
    __shared__ double red[40];
    double acc = 0.0;
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        const float2 u = d[i], v = y[i];
        const float2 w = make_float2(u.x - v.x, u.y - v.y);
        r[i] = w;
        acc = fma((double)w.x, (double)w.x, fma((double)w.y, (double)w.y, acc));
    }
    const double t = block_sum(acc, red);
    if (threadIdx.x == 0) part[blockIdx.x] = t;
}

// e += c (FP32)
__global__ void k_add32(long n, const float2 *__restrict__ c, float2 *__restrict__ e) {
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        const float2 u = c[i];
        float2 v = e[i];
        v.x += u.x;
        v.y += u.y;
        e[i] = v;
    }
}

// FP32 vectors of the inner refinement after the sloppy workspace: d and e per slot, two temporaries
struct InnerVecs {
    float2 *d0, *e0, *te, *yo;
    long n;
    float2 *d(int c) const { return d0 + (size_t)c * n; }
    float2 *e(int c) const { return e0 + (size_t)c * n; }
};
static size_t dc_work_bytes(int Vh, int R) {
    return mixed_work_bytes(Vh, 1, R) + (2 * (size_t)R + 2) * spinor_bytes_prec(Vh, TMND_F32);
}
static InnerVecs inner_vecs(void *base, int Vh, int R) {
    const size_t s32 = spinor_bytes_prec(Vh, TMND_F32);
    char *w = (char *)base + mixed_work_bytes(Vh, 1, R);
    InnerVecs v;
    v.n = 24L * Vh;
    v.d0 = (float2 *)w;
    v.e0 = (float2 *)(w + (size_t)R * s32);
    v.te = (float2 *)(w + 2 * (size_t)R * s32);
    v.yo = (float2 *)(w + (2 * (size_t)R + 1) * s32);
    return v;
}

static tmnd_status inner_refine(tmnd_gauge *g, const MixedWork &mc, const InnerVecs &iv, const double *sig,
                                const double *target, const double *dnorm, int R, double floor, int max_inner,
                                int maxiter, int check_every, int profile, cudaStream_t s, RefineStats &rs) {
    const int Vh = g->geom.Vh;
    const long n = 24L * Vh;
    const int nb = stream_blocks(n);
    double *part = (double *)g->partials;
    std::vector<double> rn(dnorm, dnorm + R), tl(R);
    std::vector<int> active(R, 1);
    std::vector<double> hpart(nb);
    for (int c = 0; c < R; c++) {
        TMND_CUDA_TRY(cudaMemcpyAsync(iv.d(c), mc.b32(c), sizeof(float2) * n, cudaMemcpyDeviceToDevice, s));
        TMND_CUDA_TRY(cudaMemsetAsync(iv.e(c), 0, sizeof(float2) * n, s));
    }
    for (int j = 0; j < max_inner; j++) {
        int nact = 0;
        for (int c = 0; c < R; c++) {
            if (!active[c]) {  // a zero right-hand side is done at once
                TMND_CUDA_TRY(cudaMemsetAsync(mc.b32(c), 0, sizeof(float2) * n, s));
                tl[c] = 0.5;
                continue;
            }
            nact++;
            const double need = target[c] / rn[c];
            tl[c] = need > floor ? need : floor;
        }
        if (nact == 0) break;
        std::vector<MMSState> hv;
        LoopOut lc;
        tmnd_status st = mms_sloppy(g, mc, sig, 1, 1, floor, maxiter, check_every, profile, s, hv, lc, nullptr, 0,
                                    sig, tl.data());
        if (st != TMND_OK) return st;
        int maxit = 0;
        for (const MMSState &h : hv) {
            rs.iters += h.iter;
            maxit = h.iter > maxit ? h.iter : maxit;
        }
        for (int k = 0; k < maxit && k < (int)lc.hop_t.size(); k++) {
            rs.hop_ms += lc.hop_t[k];
            rs.upd_ms += lc.upd_t[k];
        }
        rs.launches += 3 + lc.nlaunch * ((long long)check_every * 7 + check_every / WIN);
        // accumulate, then the FP32 residual of the accumulated correction as the next right-hand side
        for (int c = 0; c < R; c++) {
            if (!active[c]) continue;
            k_add32<<<nb, UPD_THREADS, 0, s>>>(n, mc.x32(c, 0), iv.e(c));
            st = apply_f32(g, iv.yo + 0, iv.e(c), TMND_OP_QHAT2, sig[c], 1, iv.te, mc.x32(c, 0), s);
            if (st != TMND_OK) return st;
            // apply_f32 left (Qhat^2 + sigma) e in iv.yo (its odd temporary is the slot's x32, free now)
            k_resid32<<<nb, UPD_THREADS, 0, s>>>(n, iv.d(c), iv.yo, mc.b32(c), part);
            TMND_CUDA_TRY(cudaMemcpyAsync(hpart.data(), part, sizeof(double) * nb, cudaMemcpyDeviceToHost, s));
            TMND_CUDA_TRY(cudaStreamSynchronize(s));
            double acc = 0;
            for (int q = 0; q < nb; q++) acc += hpart[q];
            rn[c] = sqrt(acc);
            rs.f32 += 1;
            rs.launches += 5;
            if (!isfinite(rn[c])) {
                tmnd_set_error("solve: NaN/Inf in an FP32 inner residual (shift %g)", sig[c]);
                return TMND_ERR_NAN;
            }
            if (rn[c] <= target[c]) active[c] = 0;
        }
    }
    return TMND_OK;
}

static tmnd_status defect_correct(tmnd_gauge *g, void *base, std::vector<DCItem> todo, double rho,
                                  double rho_inner, int maxiter, int check_every, int profile, cudaStream_t s,
                                  RefineStats &rs, int max_batch) {
    const int Vh = g->geom.Vh;
    const long n = 24L * Vh;
    const int max_rounds = 8;
    tmnd_status st;
    if (max_batch < 1) max_batch = 1;
    if (max_batch > TMND_MAX_BATCH) max_batch = TMND_MAX_BATCH;
    const double floor = rho_inner > 1e-4 ? rho_inner : 1e-4;  // a sloppy correction gains at most ~1/(4e-5)
    for (int round = 0; !todo.empty(); round++) {
        std::vector<DCItem> next;
        size_t q = 0;
        while (q < todo.size()) {
            // defects of up to max_batch pending pairs, each converted into its sloppy slot
            const MixedWork mw = mixed_work(base, Vh, 1, max_batch);
            const InnerVecs iv = inner_vecs(base, Vh, max_batch);
            std::vector<DCItem> chunk;
            std::vector<double> sg, target, dn;
            for (; q < todo.size() && (int)chunk.size() < max_batch; q++) {
                DCItem &it = todo[q];
                double rr = 0;
                TMND_CUDA_TRY(cudaStreamSynchronize(s));
                const auto t_f = std::chrono::steady_clock::now();
                st = fp64_defect(g, mw, it.b, it.x, it.sigma, s, &rr);
                if (st != TMND_OK) return st;
                rs.fp64_ms += ms_since(t_f);  // fp64_defect ends with a host read of its partials
                rs.fp64++;
                rs.launches += 5;
                *it.res = sqrt(rr / it.bb);
                if (round == 0 && it.res0) *it.res0 = *it.res;
                if (!isfinite(*it.res)) {
                    tmnd_set_error("solve: NaN/Inf in an FP64 defect (shift %g)", it.sigma);
                    return TMND_ERR_NAN;
                }
                if (*it.res <= rho) continue;
                if (round >= max_rounds) {
                    tmnd_set_error("solve: shift %g not converged after %d defect-correction rounds (residual %g)",
                                   it.sigma, max_rounds, *it.res);
                    return TMND_ERR_NOCONV;
                }
                st = convert_spinor(Vh, mw.b32((int)chunk.size()), TMND_F32, mw.r64, TMND_F64, 1, s);
                if (st != TMND_OK) return st;
                sg.push_back(it.sigma);
                target.push_back(0.3 * rho * sqrt(it.bb));  // |d - (Qhat^2 + sigma) e| for |b - ... x'| <= rho |b|
                dn.push_back(sqrt(rr));
                chunk.push_back(it);
            }
            if (chunk.empty()) continue;
            MixedWork mc = mw;  // the slots the defects were converted into
            mc.nrhs = (int)chunk.size();
            st = inner_refine(g, mc, iv, sg.data(), target.data(), dn.data(), mc.nrhs, floor, 4, maxiter, check_every,
                              profile, s, rs);
            if (st != TMND_OK) return st;
            for (size_t c = 0; c < chunk.size(); c++) {
                k_add_f32_to_f64<<<stream_blocks(n), UPD_THREADS, 0, s>>>(n, iv.e((int)c), chunk[c].x);
                next.push_back(chunk[c]);
            }
            TMND_CUDA_TRY(cudaGetLastError());
        }
        todo = next;
        if (!todo.empty()) rs.rounds = round + 1;
    }
    return TMND_OK;
}

// (RHS, shift) pairs solved together in one defect-correction round
static int refine_batch(int R, int nsolve) {
    const int p = R * nsolve;
    return p < TMND_MAX_BATCH ? p : TMND_MAX_BATCH;
}

// workspace of the mixed solve of R right-hand sides: the batched multi-shift vectors, then
// (same memory) the single-shift vectors of one batch of defect-correction pairs
static size_t mixed_total_bytes(int Vh, int nshift, int nsolve, int R) {
    const size_t a = mixed_work_bytes(Vh, nshift, R), b = dc_work_bytes(Vh, refine_batch(R, nsolve));
    return a > b ? a : b;
}

// Mixed-precision solve of right-hand sides k0 .. k0+R-1: one batched sloppy
// multi-shift CG for all of them (m holds R sloppy blocks), then per right-hand
// side the FP64 defect correction of the shifts that must converge.
static tmnd_status mixed_batch(tmnd_gauge *g, const double2 *b, double2 *const *x, const double *sigma, int nshift,
                               int nsolve, double rho, double rho_inner, int maxiter, int check_every, int profile,
                               tmnd_solve_info *info, cudaStream_t s, int k0, int R, double *hist, int hist_cap) {
    const int Vh = g->geom.Vh;
    const long n = 24L * Vh;
    MixedWork m = mixed_work(g->work, Vh, nshift, R);
    tmnd_status st;
    // |b_k|^2 in FP64
    std::vector<double> bb(R, 0.0);
    for (int k = 0; k < R; k++) {
        const int nb = stream_blocks(n);
        double *part = (double *)g->partials;
        TMND_CUDA_TRY(cudaMemsetAsync(m.y64, 0, sizeof(double2) * n, s));
        k_diff_norm<<<nb, UPD_THREADS, 0, s>>>(n, b + (size_t)(k0 + k) * n, m.y64, part);
        std::vector<double> h(nb);
        TMND_CUDA_TRY(cudaMemcpyAsync(h.data(), part, sizeof(double) * nb, cudaMemcpyDeviceToHost, s));
        TMND_CUDA_TRY(cudaStreamSynchronize(s));
        for (int q = 0; q < nb; q++) bb[k] += h[q];
        st = convert_spinor(Vh, m.b32(k), TMND_F32, b + (size_t)(k0 + k) * n, TMND_F64, 1, s);
        if (st != TMND_OK) return st;
    }
    // 1. batched sloppy multi-shift CG (a zero right-hand side is done at once)
    std::vector<MMSState> hs;
    LoopOut lo;
    TMND_CUDA_TRY(cudaStreamSynchronize(s));
    const auto t_mms = std::chrono::steady_clock::now();
    st = mms_sloppy(g, m, sigma, nshift, nsolve, rho_inner, maxiter, check_every, profile, s, hs, lo,
                    k0 == 0 ? hist : nullptr, hist_cap);
    if (st != TMND_OK) return st;
    long long launches = 3 + lo.nlaunch * ((long long)check_every * 7 + check_every / WIN);
    double hop_ms = 0, upd_ms = 0;
    int maxit = 0;
    for (int k = 0; k < R; k++) maxit = hs[k].iter > maxit ? hs[k].iter : maxit;
    for (int q = 0; q < maxit && q < (int)lo.hop_t.size(); q++) {
        hop_ms += lo.hop_t[q];
        upd_ms += lo.upd_t[q];
    }
    tmnd_status conv = TMND_OK;
    int fp64 = 0, rounds = 0, riters = 0;
    std::vector<std::vector<double>> res(R, std::vector<double>(nshift, 0.0));
    std::vector<DCItem> items;
    for (int k = 0; k < R; k++) {
        const int rhs = k0 + k;
        double2 *xk[NS];
        for (int i = 0; i < nshift; i++) xk[i] = x[i] + (size_t)rhs * n;
        if (bb[k] == 0.0) {
            for (int i = 0; i < nshift; i++) TMND_CUDA_TRY(cudaMemsetAsync(xk[i], 0, sizeof(double2) * n, s));
            continue;
        }
        for (int i = 0; i < nshift; i++) {
            st = convert_spinor(Vh, xk[i], TMND_F64, m.x32(k, i), TMND_F32, 1, s);
            if (st != TMND_OK) return st;
        }
        launches += nshift + 2;
        if (info) {
            if (rhs == 0 || hs[k].iter > info->iters) info->iters = hs[k].iter;
            for (int i = 0; i < nshift; i++) {
                if (rhs == 0 || hs[k].conv_iter[i] > info->conv_iter[i] || hs[k].conv_iter[i] < 0)
                    info->conv_iter[i] = hs[k].conv_iter[i];
                info->zeta[i] = hs[k].zeta[i];
            }
        }
        for (int i = 0; i < nsolve; i++)
            items.push_back(DCItem{b + (size_t)rhs * n, xk[i], sigma[i], bb[k], &res[k][i]});
    }
    // 2. FP64 defect correction of every (RHS, shift) pair that must converge, batched
    const double mms_ms = ms_since(t_mms);  // the multi-shift solve ends with host reads of its state
    RefineStats rs;
    const auto t_dc = std::chrono::steady_clock::now();
    st = defect_correct(g, g->work, items, rho, rho_inner, maxiter, check_every, profile, s, rs,
                        refine_batch(R, nsolve));
    if (st != TMND_OK && st != TMND_ERR_NOCONV) return st;
    if (st == TMND_ERR_NOCONV) conv = st;
    fp64 += rs.fp64;
    riters += rs.iters;
    rounds = rs.rounds;
    launches += rs.launches;
    hop_ms += rs.hop_ms;
    upd_ms += rs.upd_ms;
    if (info)
        for (int k = 0; k < R; k++)
            for (int i = 0; i < nshift; i++)
                if (k0 + k == 0 || res[k][i] > info->true_res[i]) info->true_res[i] = res[k][i];
    if (info) {
        cudaStreamSynchronize(s);
        info->mms_ms += mms_ms;
        info->fp64_ms += rs.fp64_ms;
        info->refine_ms += ms_since(t_dc) - rs.fp64_ms;
        info->fp64_applies += fp64;
        info->f32_applies += rs.f32;
        info->refine_iters += riters;
        if (rounds > info->refine_rounds) info->refine_rounds = rounds;
        info->launches += launches;
        info->hop_ms += hop_ms;
        info->update_ms += upd_ms;
    }
    return conv;
}

extern "C" tmnd_status mms_cg_solve(tmnd_gauge *g, const void *b, int nrhs, const double *sigma, int nshift,
                                    void *const *x, const tmnd_solve_params *params, tmnd_solve_info *info,
                                    void *stream) {
    TMND_ARG_CHECK(g && b && sigma && x && params, "mms_cg_solve: NULL argument");
    cudaGetLastError();  // clear a stale, non-sticky error left by earlier unrelated calls
    TMND_ARG_CHECK(nshift >= 1 && nshift <= TMND_MAX_SHIFTS, "mms_cg_solve: nshift = %d not in [1, %d]", nshift,
                   TMND_MAX_SHIFTS);
    TMND_ARG_CHECK(nrhs >= 1, "mms_cg_solve: nrhs = %d", nrhs);
    for (int i = 0; i < nshift; i++) {
        TMND_ARG_CHECK(isfinite(sigma[i]) && sigma[i] > 0, "mms_cg_solve: sigma[%d] = %g must be > 0", i, sigma[i]);
        TMND_ARG_CHECK(i == 0 || sigma[i] < sigma[i - 1], "mms_cg_solve: shifts must be strictly descending");
        TMND_ARG_CHECK(x[i] != nullptr && ((uintptr_t)x[i] & 15) == 0, "mms_cg_solve: x[%d] NULL or misaligned", i);
    }
    TMND_ARG_CHECK(((uintptr_t)b & 15) == 0, "mms_cg_solve: b misaligned");
    const int nsolve = params->nsolve > 0 ? params->nsolve : nshift;
    TMND_ARG_CHECK(nsolve <= nshift, "mms_cg_solve: nsolve = %d > nshift", nsolve);
    TMND_ARG_CHECK(params->rho > 0 && params->rho < 1, "mms_cg_solve: rho = %g not in (0, 1)", params->rho);
    TMND_ARG_CHECK(params->maxiter >= 1, "mms_cg_solve: maxiter = %d", params->maxiter);
    int check_every = params->check_every > 0 ? params->check_every : 32;
    TMND_ARG_CHECK(check_every <= 4096, "mms_cg_solve: check_every too large");
    check_every = (check_every + WIN - 1) / WIN * WIN;  // whole windows per graph replay

    const int mixed = params->prec == TMND_S16;
    TMND_ARG_CHECK(params->prec == TMND_F64 || mixed, "mms_cg_solve: prec %d not supported", params->prec);
    const double rho_inner = params->rho_inner > 0 ? params->rho_inner : 1e-5;
    TMND_ARG_CHECK(rho_inner < 1, "mms_cg_solve: rho_inner = %g not in (0, 1)", rho_inner);
    TMND_ARG_CHECK(params->batch >= 0 && params->batch <= TMND_MAX_BATCH, "mms_cg_solve: batch = %d not in [0, %d]",
                   params->batch, TMND_MAX_BATCH);
    // right-hand sides iterated together by the sloppy solver of the mixed path
    int R = params->batch > 0 ? params->batch : TMND_MAX_BATCH;
    if (R > nrhs) R = nrhs;
    const size_t sp = tmnd_spinor_bytes(g);
    tmnd_status st = tmnd_ensure_workspace(
        g, mixed ? mixed_total_bytes(g->geom.Vh, nshift, nsolve, R) : (WIN + 3 + (size_t)nshift) * sp);
    if (st != TMND_OK) return st;
    const long n = (long)(sp / sizeof(double2));
    const int nbh = hop_blocks(g->geom) > hop_blocks_s16_max(g->geom) ? hop_blocks(g->geom)
                                                                       : hop_blocks_s16_max(g->geom);
    const int nbs = stream_blocks(n) > site_blocks(g->geom.Vh) ? stream_blocks(n) : site_blocks(g->geom.Vh);
    size_t pbytes = sizeof(double) * (3 * (size_t)nbh + nbs) + 256 + 2 * 4096 + sizeof(MMSState) + sizeof(MMSCoef);
    if (mixed) {
        const int Rm = R > refine_batch(R, nsolve) ? R : refine_batch(R, nsolve);
        if (sloppy_partial_bytes(g->geom, Rm) > pbytes) pbytes = sloppy_partial_bytes(g->geom, Rm);
    }
    st = tmnd_ensure_partials(g, pbytes);
    if (st != TMND_OK) return st;
    if (info) memset(info, 0, sizeof *info);

    // optional scalar history (alpha_k, beta_k) of the base recursion, first RHS
    double *dhist = nullptr;
    const int hist_cap = params->ab_hist ? params->ab_hist_len / 2 : 0;
    if (hist_cap > 0) TMND_CUDA_TRY(cudaMalloc(&dhist, sizeof(double) * 2 * hist_cap));
    // run on a private stream ordered after the caller's stream (capture needs a non-legacy stream)
    cudaStream_t user = (cudaStream_t)stream;
    cudaStream_t s;
    TMND_CUDA_TRY(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    if (dhist) TMND_CUDA_TRY(cudaMemsetAsync(dhist, 0, sizeof(double) * 2 * hist_cap, s));
    cudaEvent_t e0;
    TMND_CUDA_TRY(cudaEventCreateWithFlags(&e0, cudaEventDisableTiming));
    TMND_CUDA_TRY(cudaEventRecord(e0, user));
    TMND_CUDA_TRY(cudaStreamWaitEvent(s, e0, 0));
    tmnd_status res = TMND_OK;
    if (mixed) {
        for (int k0 = 0; k0 < nrhs && res == TMND_OK; k0 += R) {
            const int r = nrhs - k0 < R ? nrhs - k0 : R;
            tmnd_status rk = mixed_batch(g, (const double2 *)b, (double2 *const *)x, sigma, nshift, nsolve,
                                         params->rho, rho_inner, params->maxiter, check_every,
                                         params->profile ? 1 : 0, info, s, k0, r, dhist, hist_cap);
            if (rk != TMND_OK) res = rk;
        }
    } else {
        for (int k = 0; k < nrhs && res == TMND_OK; k++) {
            const double2 *bk = (const double2 *)b + (size_t)k * (sp / sizeof(double2));
            double *hk = k == 0 ? dhist : nullptr;
            tmnd_status rk = mms_one_rhs(g, bk, (double2 *const *)x, sigma, nshift, nsolve, params->rho,
                                         params->maxiter, check_every, params->profile ? 1 : 0, info, s, k, hk,
                                         hist_cap);
            if (rk != TMND_OK) res = rk;
        }
    }
    cudaEventRecord(e0, s);
    cudaStreamWaitEvent(user, e0, 0);
    cudaStreamSynchronize(s);
    cudaEventDestroy(e0);
    cudaStreamDestroy(s);
    if (dhist) {
        cudaMemcpy(params->ab_hist, dhist, sizeof(double) * 2 * hist_cap, cudaMemcpyDeviceToHost);
        cudaFree(dhist);
    }
    return res;
}

// ------------------------------------------------------------- hybrid solve
// Sec. 4.3 (the paper's combined strategy): multi-shift CG for the n_mms largest
// shifts, iterating the next `n_guess` shifts along as guesses (Sec. 4.2.2);
// every remaining shift, in descending order, starts from a guess (MMS iterate,
// else Lagrange interpolation over the nearest <= 8 solved shifts, Sec. 4.2.1)
// and is solved as case C (Sec. 3.1, Eq. "lindif"):
//   x = i/(2s) [ (Qhat + i s)^-1 b - (Qhat - i s)^-1 b ],  s = sqrt(sigma),
// each single system by the two-level MG (full-lattice D_ND +- i s gamma_5 tau_1
// Pi_odd, right-hand side (0, gamma_5 tau_1 b), initial guess (Qhat -+ i s) x~ with its
// even part eliminated), then the FP64 defect correction to rho.
tmnd_status mg_gcr_solve(tmnd_mg *mg, float2 *x, const float2 *b, double s, double tol, int maxiter, int restart,
                         int nu, cudaStream_t st, int *iters_out, double *res_out, void *scratch);
size_t mg_gcr_scratch_bytes(tmnd_mg *mg, int restart);
tmnd_status tmnd_mg_tc_status(const tmnd_mg *mg);
__global__ void k_g5tau1(int Vh, const double2 *__restrict__ in, double2 *__restrict__ out);

extern "C" tmnd_status tmnd_hybrid_solve(tmnd_gauge *g, tmnd_mg *mg, const void *b, int nrhs, const double *sigma,
                                         int nshift, int n_mms, void *const *x, const tmnd_hybrid_params *hp,
                                         tmnd_hybrid_info *hinfo, void *stream) {
    TMND_ARG_CHECK(g && b && sigma && x && hp, "tmnd_hybrid_solve: NULL argument");
    TMND_ARG_CHECK(hp->guess >= 0 && hp->guess <= 2, "tmnd_hybrid_solve: guess = %d not in {0, 1, 2}", hp->guess);
    TMND_ARG_CHECK(hp->lebesgue_max == 0.0 || hp->lebesgue_max >= 1.0, "tmnd_hybrid_solve: lebesgue_max = %g < 1",
                   hp->lebesgue_max);
    TMND_ARG_CHECK(hp->guess != 2 || (hp->net && n_mms >= 8),
                   "tmnd_hybrid_solve: learned guesses need a network and n_mms >= 8");
    TMND_ARG_CHECK(nshift >= 1 && nshift <= TMND_MAX_SHIFTS && n_mms >= 1 && n_mms <= nshift && nrhs >= 1,
                   "tmnd_hybrid_solve: bad shift counts");
    for (int i = 0; i < nshift; i++)
        TMND_ARG_CHECK(sigma[i] > 0 && (i == 0 || sigma[i] < sigma[i - 1]),
                       "tmnd_hybrid_solve: shifts must be > 0 and strictly descending");
    cudaGetLastError();
    const int Vh = g->geom.Vh;
    const long n = 24L * Vh;
    const size_t sp = tmnd_spinor_bytes(g);
    const int ng = hp->n_guess < 0 ? 0 : (n_mms + hp->n_guess > nshift ? nshift - n_mms : hp->n_guess);
    const int nmms_all = n_mms + ng;
    // 1. multi-shift CG on the largest shifts (+ guess shifts)
    tmnd_solve_params sp1 = {};
    sp1.rho = hp->rho;
    sp1.maxiter = hp->maxiter;
    sp1.nsolve = n_mms;
    sp1.prec = hp->prec;
    sp1.rho_inner = hp->rho_inner;
    // scalar history of the base recursion (first RHS): the network's Lanczos features
    std::vector<double> hist;
    if (hp->guess == 2) {
        hist.assign(2 * (size_t)(hp->maxiter < 4096 ? hp->maxiter : 4096), 0.0);
        sp1.ab_hist = hist.data();
        sp1.ab_hist_len = (int)hist.size();
    }
    tmnd_solve_info si = {};
    const auto t_mms = std::chrono::steady_clock::now();
    tmnd_status st = mms_cg_solve(g, b, nrhs, sigma, nmms_all, x, &sp1, &si, stream);
    if (st != TMND_OK) return st;
    const double mms_ms =
        std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_mms).count();
    if (hinfo) {
        memset(hinfo, 0, sizeof *hinfo);
        hinfo->mms_ms = mms_ms;
        hinfo->launches = si.launches;
        hinfo->mms_iters = si.iters;
        hinfo->fp64_applies = si.fp64_applies;
        hinfo->f32_applies = si.f32_applies;
        hinfo->refine_iters = si.refine_iters;
        for (int i = 0; i < n_mms; i++) hinfo->true_res[i] = si.true_res[i];
    }
    if (n_mms == nshift) return TMND_OK;
    // learned weights (one set for all RHS: the features are the shifts and the first RHS's history)
    std::vector<double> lw;
    const int n_learn = nshift - nmms_all;
    if (hp->guess == 2 && n_learn > 0) {
        // target i: nodes = the 8 shifts just above it (solved before it), features from the
        // history of the multi-shift solve with base shift sigma[n_mms - 1]
        std::vector<float> X((size_t)n_learn * 20);
        std::vector<double> S((size_t)n_learn * 9);
        for (int q = 0; q < n_learn; q++) {
            const int i = nmms_all + q;
            const double *nodes = sigma + (i - 8);
            st = tmnd_mlp_features(nodes, sigma[i], hist.data(), si.iters, sigma[n_mms - 1], &X[(size_t)q * 20]);
            if (st != TMND_OK) return st;
            S[(size_t)q * 9] = sigma[i];
            for (int j = 0; j < 8; j++) S[(size_t)q * 9 + 1 + j] = nodes[j];
        }
        char *dbuf = nullptr;
        const size_t xb = sizeof(float) * X.size(), sb = sizeof(double) * S.size(), wb = sizeof(double) * 8 * n_learn;
        TMND_CUDA_TRY(cudaMalloc(&dbuf, xb + sb + wb + 64));
        double *dS = (double *)(dbuf + ((xb + 15) & ~(size_t)15)), *dW = dS + S.size();
        lw.resize((size_t)8 * n_learn);
        cudaError_t ce = cudaMemcpy(dbuf, X.data(), xb, cudaMemcpyHostToDevice);
        if (ce == cudaSuccess) ce = cudaMemcpy(dS, S.data(), sb, cudaMemcpyHostToDevice);
        tmnd_status ps = ce == cudaSuccess ? tmnd_mlp_predict((tmnd_mlp *)hp->net, dbuf, dS, n_learn, dW, nullptr)
                                           : TMND_ERR_CUDA;
        if (ps == TMND_OK) ce = cudaMemcpy(lw.data(), dW, wb, cudaMemcpyDeviceToHost);
        cudaFree(dbuf);
        if (ps != TMND_OK) return ps;
        if (ce != cudaSuccess) {
            tmnd_set_error("tmnd_hybrid_solve: %s", cudaGetErrorString(ce));
            return TMND_ERR_CUDA;
        }
    }
    // 2. the remaining shifts in descending order; per shift every right-hand side's guess and
    // case-C multigrid solve, then one batched FP64 defect correction of all its (RHS, shift) pairs
    const double rho_inner = hp->rho_inner > 0 ? hp->rho_inner : 1e-5;
    const int dc_batch = nrhs < TMND_MAX_BATCH ? nrhs : TMND_MAX_BATCH;
    st = tmnd_ensure_workspace(g, dc_work_bytes(Vh, dc_batch));
    if (st != TMND_OK) return st;
    const long nfull = 2 * n;  // full-lattice FP32 doublet (complex numbers)
    const size_t f32b = sizeof(float2) * nfull;
    const size_t scratch_b = 3 * sp + 4 * f32b + (mg ? mg_gcr_scratch_bytes(mg, hp->mg_restart > 0 ? hp->mg_restart : 24) : 0);
    char *scr = nullptr;
    TMND_CUDA_TRY(cudaMalloc(&scr, scratch_b));
    double2 *tq = (double2 *)scr, *te = (double2 *)(scr + sp), *gb = (double2 *)(scr + 2 * sp);
    float2 *rhs = (float2 *)(scr + 3 * sp), *yp = (float2 *)(scr + 3 * sp + f32b);
    float2 *ym = (float2 *)(scr + 3 * sp + 2 * f32b);
    void *gcr = scr + 3 * sp + 4 * f32b;
    // private stream ordered after the caller's (the defect correction captures graphs,
    // which the legacy default stream does not allow)
    cudaStream_t user = (cudaStream_t)stream;
    cudaStream_t s;
    cudaEvent_t e0;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
        cudaFree(scr);
        TMND_CUDA_TRY(cudaGetLastError());
    }
    cudaEventCreateWithFlags(&e0, cudaEventDisableTiming);
    cudaEventRecord(e0, user);
    cudaStreamWaitEvent(s, e0, 0);
    const int nbs = stream_blocks(n);
    MixedWork m = mixed_work(g->work, Vh, 1);
    tmnd_status res_status = TMND_OK;
    // |b_k|^2 in FP64
    std::vector<double> bbk(nrhs, 0.0);
    for (int k = 0; k < nrhs && res_status == TMND_OK; k++) {
        double *part = (double *)g->partials;
        cudaMemsetAsync(m.y64, 0, sizeof(double2) * n, s);
        k_diff_norm<<<nbs, UPD_THREADS, 0, s>>>(n, (const double2 *)b + (size_t)k * n, m.y64, part);
        std::vector<double> h(nbs);
        cudaMemcpyAsync(h.data(), part, sizeof(double) * nbs, cudaMemcpyDeviceToHost, s);
        cudaError_t e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) {
            tmnd_set_error("tmnd_hybrid_solve: %s", cudaGetErrorString(e));
            res_status = TMND_ERR_CUDA;
            break;
        }
        for (int q = 0; q < nbs; q++) bbk[k] += h[q];
    }
    for (int i = n_mms; i < nshift && res_status == TMND_OK; i++) {
        const auto t_shift = std::chrono::steady_clock::now();
        const double sq = sqrt(sigma[i]);
        const double mg_tol = hp->mg_tol > 0 ? hp->mg_tol : 1e-4;
        bool mg_shift = mg != nullptr;
        std::vector<double> res(nrhs, 0.0), res0(nrhs, 0.0);
        std::vector<DCItem> items;
        for (int k = 0; k < nrhs && res_status == TMND_OK; k++) {
            const double2 *bk = (const double2 *)b + (size_t)k * n;
            double2 *xk[NS];
            for (int q = 0; q < nshift; q++) xk[q] = (double2 *)x[q] + (size_t)k * n;
            if (bbk[k] == 0.0) {  // b = 0: x = 0 is exact
                cudaMemsetAsync(xk[i], 0, sizeof(double2) * n, s);
                continue;
            }
            // guess (the guess shifts of the multi-shift solve already hold theirs)
            if (i >= nmms_all) {
                if (hp->guess == 2) {
                    const void *xs[8];
                    for (int j = 0; j < 8; j++) xs[j] = xk[i - 8 + j];
                    st = tmnd_lincomb(g, &lw[(size_t)8 * (i - nmms_all)], xs, 8, xk[i], 1, s);
                    if (st != TMND_OK) { res_status = st; break; }
                } else if (hp->guess == 1) {
                    // the nearest solved shifts first, truncated where the Lebesgue function grows (App. B)
                    const int kk = i < 8 ? i : 8;
                    double cand[8];
                    const void *xs[8];
                    for (int j = 0; j < kk; j++) {
                        cand[j] = sigma[i - 1 - j];
                        xs[j] = xk[i - 1 - j];
                    }
                    int ku = kk;
                    double gam = 1.0;
                    st = tmnd_lagrange_degree(cand, kk, sigma[i], hp->lebesgue_max > 0 ? hp->lebesgue_max : 4.0, &ku,
                                              &gam);
                    if (st == TMND_OK) st = lagrange_guess(g, cand, xs, ku, sigma[i], xk[i], 1, nullptr, s);
                    if (st != TMND_OK) { res_status = st; break; }
                    if (hinfo && k == 0) {
                        hinfo->lag_nodes[i] = ku;
                        hinfo->lebesgue[i] = gam;
                    }
                } else {
                    cudaMemsetAsync(xk[i], 0, sizeof(double2) * n, s);
                }
            }
            int mg_it = 0;
            if (mg && k == 0) {  // the guess's FP64 residual (RHS 0), before the multigrid
                double rr0 = 0;
                st = fp64_defect(g, m, bk, xk[i], sigma[i], s, &rr0);
                if (st != TMND_OK) { res_status = st; break; }
                const double gr = bbk[k] > 0 ? sqrt(rr0 / bbk[k]) : 0.0;
                // the multigrid solves a case-C system to mg_tol of |b|; a guess already below that
                // (on RHS 0, taken for every RHS of the shift) leaves it nothing to do: the case-C
                // set-up is skipped and the defect correction starts from the guess
                mg_shift = gr > mg_tol;
                if (hinfo) {
                    hinfo->guess_res[i] = gr;
                    hinfo->fp64_applies += 1;
                }
            }
            if (mg && mg_shift) {
                // case-C right-hand side (0, gamma_5 tau_1 b) in FP32 full layout (parity 0 even, 1 odd)
                k_g5tau1<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(Vh, bk, gb);
                cudaMemsetAsync(rhs, 0, sizeof(float2) * n, s);
                k_to_f32_scaled<<<nbs, 256, 0, s>>>(n, 1.0, gb, rhs + n);
                for (int sgn = 1; sgn >= -1; sgn -= 2) {
                    float2 *y = sgn > 0 ? yp : ym;
                    // odd guess (Qhat - sgn i s) x~ ; Qhat = g5 t1 Mhat
                    HopEpiArgs ea = {};
                    launch_hop_even_f64(g->geom, g->st, g->links, xk[i], te, false, nullptr, s);
                    launch_hop_odd_f64(g->geom, g->st, g->links, xk[i], te, tq, false, EPI_STORE, ea, s);
                    k_g5tau1<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(Vh, tq, gb);
                    k_zaxpy64<<<nbs, 256, 0, s>>>(n, 0.0, -sgn * sq, xk[i], gb);
                    // even part eliminated: x_e = -D_ee^-1 D_eo x_o = kappa A^-1 H x_o = t_e / kappa
                    launch_hop_even_f64(g->geom, g->st, g->links, gb, te, false, nullptr, s);
                    k_to_f32_scaled<<<nbs, 256, 0, s>>>(n, 1.0 / g->act.kappa, te, y);
                    k_to_f32_scaled<<<nbs, 256, 0, s>>>(n, 1.0, gb, y + n);
                    int it = 0;
                    double rres = 0;
                    st = mg_gcr_solve(mg, y, rhs, sgn * sq, mg_tol, hp->mg_maxiter > 0 ? hp->mg_maxiter : 100,
                                      hp->mg_restart > 0 ? hp->mg_restart : 24, hp->mg_nu > 0 ? hp->mg_nu : 4, s, &it,
                                      &rres, gcr);
                    if (st != TMND_OK) { res_status = st; break; }
                    mg_it += it;
                }
                if (res_status != TMND_OK) break;
                k_casec_combine<<<nbs, 256, 0, s>>>(n, sq, yp + n, ym + n, xk[i]);
            }
            if (hinfo && k == 0) hinfo->mg_iters[i] = mg_it;
            items.push_back(DCItem{bk, xk[i], sigma[i], bbk[k], &res[k], &res0[k]});
        }
        if (res_status != TMND_OK) break;
        // FP64 defect correction of this shift's pairs to rho, all right-hand sides together
        RefineStats rs;
        st = defect_correct(g, g->work, items, hp->rho, rho_inner, hp->maxiter, 32, 0, s, rs, dc_batch);
        if (st != TMND_OK) { res_status = st; break; }
        if (hinfo) {
            if (!mg) hinfo->guess_res[i] = res0[0];  // the guess's residual: the first FP64 defect
            cudaStreamSynchronize(s);
            hinfo->shift_ms[i] =
                std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_shift).count();
            hinfo->fp64_applies += rs.fp64;
            hinfo->f32_applies += rs.f32;
            hinfo->refine_iters += rs.iters;
            hinfo->launches += rs.launches;
            for (int k = 0; k < nrhs; k++)
                if (k == 0 || res[k] > hinfo->true_res[i]) hinfo->true_res[i] = res[k];
        }
    }
    cudaEventRecord(e0, s);
    cudaStreamWaitEvent(user, e0, 0);
    cudaError_t fin = cudaStreamSynchronize(s);
    cudaEventDestroy(e0);
    cudaStreamDestroy(s);
    cudaFree(scr);
    if (res_status == TMND_OK && mg) res_status = tmnd_mg_tc_status(mg);
    if (res_status == TMND_OK && fin != cudaSuccess) {
        tmnd_set_error("tmnd_hybrid_solve: %s", cudaGetErrorString(fin));
        return TMND_ERR_CUDA;
    }
    return res_status;
}
