// Two-level multigrid solve (Sec. 3: flexible outer Krylov solver
// preconditioned by the error propagation of Eq. "error_propagation") for the
// full-lattice doublet systems of case C (Sec. 3.1, Eq. "lindif"):
//   D' y = rhs,  D' = D_ND + i s (gamma_5 (x) tau_1) Pi_odd     (s may be negative)
// whose odd-site Schur complement is Mhat + i s gamma_5 tau_1, i.e.
//   (Qhat + i s) y_o = b   <=>   D' (y_e, y_o) = (0, gamma_5 tau_1 b).
// FP32 throughout: outer GCR (flexible, restarted), preconditioner = one
// V-cycle: nu minimal-residual smoothing steps, coarse-grid correction with the
// coarse operator (mg_coarse_apply) solved by coarse GCR, nu post-smoothing steps.
#include <math.h>

#include <vector>

#include "tmnd_internal.cuh"

struct tmnd_mg;  // defined in mg.cu
size_t tmnd_mg_nblock_nv(const tmnd_mg *mg, int *nv);
void tmnd_mg_smoother(const tmnd_mg *mg, int *kind, int *mr, int bd[4]);
tmnd_status launch_sap_color(const tmnd_gauge *g, const int bd[4], int color, double s_odd, const float2 *r,
                             float2 *x, int mr_iters, cudaStream_t s);

namespace {


// Full-lattice doublet operator, output parity P, FP32 (links rounded from FP64):
// y = (1 + i kp g5 t3 - kpp t1 [+ i s g5 t1 on odd sites]) x_P - kappa H x_{1-P}
// nf = 2: doublet (24 components); nf = 1: one flavour, D_TM(+mu) (12 components, kpp and s ignored).
__global__ void k_dnd_full(Geom g, double kappa, float kp, float kpp, float s_odd, const double2 *__restrict__ links,
                           const float2 *__restrict__ in, float2 *__restrict__ out, int nf) {
    const int ncomp = 12 * nf;
    const int Vh = g.Vh;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < 2 * Vh; i += gridDim.x * blockDim.x) {
        const int P = i / Vh, h = i % Vh, Q = 1 - P;
        const int zh = h % g.Zh;
        int r = h / g.Zh;
        const int y0 = r % g.Y;
        r /= g.Y;
        const int x0 = r % g.X;
        const int t0 = r / g.X;
        const int z0 = 2 * zh + ((P + t0 + x0 + y0) & 1);
        float2 acc[2][4][3];
        for (int f = 0; f < 2; f++)
            for (int s = 0; s < 4; s++)
                for (int c = 0; c < 3; c++) acc[f][s][c] = make_float2(0.f, 0.f);
        const int n[4] = {g.T, g.X, g.Y, g.Z};
        for (int d = 0; d < 8; d++) {
            const int mu = d >> 1;
            const bool fwd = (d & 1) == 0;
            int c[4] = {t0, x0, y0, z0};
            float sg = 1.0f;
            if (fwd) {
                if (c[mu] + 1 == n[mu]) { c[mu] = 0; if (mu == 0 && g.apbc) sg = -1.0f; }
                else c[mu]++;
            } else {
                if (c[mu] == 0) { c[mu] = n[mu] - 1; if (mu == 0 && g.apbc) sg = -1.0f; }
                else c[mu]--;
            }
            const int hn = ((c[0] * g.X + c[1]) * g.Y + c[2]) * g.Zh + (c[3] >> 1);
            const double2 *L = fwd ? links + ((size_t)(P * 4 + mu) * 9) * Vh : links + ((size_t)(Q * 4 + mu) * 9) * Vh;
            const int hl = fwd ? h : hn;
            float2 u[3][3];
            for (int a = 0; a < 3; a++)
                for (int b = 0; b < 3; b++) {
                    const double2 w = fwd ? L[(size_t)(a * 3 + b) * Vh + hl] : L[(size_t)(b * 3 + a) * Vh + hl];
                    u[a][b] = fwd ? make_float2((float)w.x, (float)w.y) : make_float2((float)w.x, -(float)w.y);
                }
            const float k = -(float)kappa * sg;
            for (int f = 0; f < nf; f++) {
                float2 ps[4][3];
                for (int s = 0; s < 4; s++)
                    for (int cc = 0; cc < 3; cc++) ps[s][cc] = in[((size_t)Q * ncomp + f * 12 + s * 3 + cc) * Vh + hn];
                for (int cc = 0; cc < 3; cc++) {
                    float2 gp[4];
                    const float2 u0 = ps[0][cc], u1 = ps[1][cc], l0 = ps[2][cc], l1 = ps[3][cc];
                    if (mu == 0) {
                        gp[0] = make_float2(-l0.x, -l0.y); gp[1] = make_float2(-l1.x, -l1.y);
                        gp[2] = make_float2(-u0.x, -u0.y); gp[3] = make_float2(-u1.x, -u1.y);
                    } else if (mu == 1) {
                        gp[0] = make_float2(l1.y, -l1.x); gp[1] = make_float2(l0.y, -l0.x);
                        gp[2] = make_float2(-u1.y, u1.x); gp[3] = make_float2(-u0.y, u0.x);
                    } else if (mu == 2) {
                        gp[0] = make_float2(-l1.x, -l1.y); gp[1] = l0;
                        gp[2] = u1; gp[3] = make_float2(-u0.x, -u0.y);
                    } else {
                        gp[0] = make_float2(l0.y, -l0.x); gp[1] = make_float2(-l1.y, l1.x);
                        gp[2] = make_float2(-u0.y, u0.x); gp[3] = make_float2(u1.y, -u1.x);
                    }
                    const float sgn = fwd ? -1.0f : 1.0f;
                    for (int s = 0; s < 4; s++)
                        ps[s][cc] = make_float2(ps[s][cc].x + sgn * gp[s].x, ps[s][cc].y + sgn * gp[s].y);
                }
                for (int s = 0; s < 4; s++)
                    for (int a = 0; a < 3; a++) {
                        float2 v = make_float2(0.f, 0.f);
                        for (int b = 0; b < 3; b++) v = cfma(u[a][b], ps[s][b], v);
                        acc[f][s][a].x = fmaf(k, v.x, acc[f][s][a].x);
                        acc[f][s][a].y = fmaf(k, v.y, acc[f][s][a].y);
                    }
            }
        }
        const float so = P == 1 ? s_odd : 0.0f;
        if (nf == 1) {
            for (int s = 0; s < 4; s++) {
                const float g5 = s < 2 ? 1.0f : -1.0f;
                for (int c = 0; c < 3; c++) {
                    const float2 x0v = in[((size_t)P * 12 + s * 3 + c) * Vh + h];
                    float2 o0;
                    o0.x = x0v.x - kp * g5 * x0v.y + acc[0][s][c].x;
                    o0.y = x0v.y + kp * g5 * x0v.x + acc[0][s][c].y;
                    out[((size_t)P * 12 + s * 3 + c) * Vh + h] = o0;
                }
            }
            continue;
        }
        for (int s = 0; s < 4; s++) {
            const float g5 = s < 2 ? 1.0f : -1.0f;
            for (int c = 0; c < 3; c++) {
                const float2 x0v = in[((size_t)P * 24 + 0 * 12 + s * 3 + c) * Vh + h];
                const float2 x1v = in[((size_t)P * 24 + 1 * 12 + s * 3 + c) * Vh + h];
                // flavour 0: x0 + i kp g5 x0 - kpp x1 + i so g5 x1 ; flavour 1: x1 - i kp g5 x1 - kpp x0 + i so g5 x0
                float2 o0, o1;
                o0.x = x0v.x - kp * g5 * x0v.y - kpp * x1v.x - so * g5 * x1v.y + acc[0][s][c].x;
                o0.y = x0v.y + kp * g5 * x0v.x - kpp * x1v.y + so * g5 * x1v.x + acc[0][s][c].y;
                o1.x = x1v.x + kp * g5 * x1v.y - kpp * x0v.x - so * g5 * x0v.y + acc[1][s][c].x;
                o1.y = x1v.y - kp * g5 * x1v.x - kpp * x0v.y + so * g5 * x0v.x + acc[1][s][c].y;
                out[((size_t)P * 24 + 0 * 12 + s * 3 + c) * Vh + h] = o0;
                out[((size_t)P * 24 + 1 * 12 + s * 3 + c) * Vh + h] = o1;
            }
        }
    }
}

// complex dot <a, b> partials (double), n complex numbers
__global__ void k_cdot(long n, const float2 *__restrict__ a, const float2 *__restrict__ b, double *part) {
    __shared__ double red[80];
    double re = 0, im = 0;
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        const float2 u = a[i], v = b[i];
        re += (double)u.x * v.x + (double)u.y * v.y;
        im += (double)u.x * v.y - (double)u.y * v.x;
    }
    double sre = block_sum(re, red);
    __syncthreads();
    double sim = block_sum(im, red + 40);
    if (threadIdx.x == 0) {
        part[2 * blockIdx.x] = sre;
        part[2 * blockIdx.x + 1] = sim;
    }
}

// y = y + a x  (a complex)
__global__ void k_caxpy(long n, float ar, float ai, const float2 *__restrict__ x, float2 *__restrict__ y) {
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        const float2 v = x[i];
        float2 w = y[i];
        w.x += ar * v.x - ai * v.y;
        w.y += ar * v.y + ai * v.x;
        y[i] = w;
    }
}

// y = a x (a real)
__global__ void k_cscale(long n, float a, const float2 *__restrict__ x, float2 *__restrict__ y) {
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
        y[i] = make_float2(a * x[i].x, a * x[i].y);
}

// y = b - y
__global__ void k_rsub(long n, const float2 *__restrict__ b, float2 *__restrict__ y) {
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
        y[i] = make_float2(b[i].x - y[i].x, b[i].y - y[i].y);
}

int nblk(long n) {
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    long want = (n + 255) / 256, cap = (long)sms * 4;
    return (int)(want < cap ? want : cap);
}

// Small BLAS-1 context with host-side reductions.
struct Blas {
    cudaStream_t s;
    double *part;      // device partials
    std::vector<double> h;
    int nb_max;
    double2 dot(long n, const float2 *a, const float2 *b) {
        const int nb = nblk(n);
        k_cdot<<<nb, 256, 0, s>>>(n, a, b, part);
        cudaMemcpyAsync(h.data(), part, sizeof(double) * 2 * nb, cudaMemcpyDeviceToHost, s);
        cudaStreamSynchronize(s);
        double re = 0, im = 0;
        for (int k = 0; k < nb; k++) {
            re += h[2 * k];
            im += h[2 * k + 1];
        }
        return make_double2(re, im);
    }
    double norm2(long n, const float2 *a) { return dot(n, a, a).x; }
    void axpy(long n, double2 a, const float2 *x, float2 *y) {
        k_caxpy<<<nblk(n), 256, 0, s>>>(n, (float)a.x, (float)a.y, x, y);
    }
    void scale(long n, double a, const float2 *x, float2 *y) { k_cscale<<<nblk(n), 256, 0, s>>>(n, (float)a, x, y); }
    void copy(long n, const float2 *x, float2 *y) { cudaMemcpyAsync(y, x, sizeof(float2) * n, cudaMemcpyDeviceToDevice, s); }
    void zero(long n, float2 *y) { cudaMemsetAsync(y, 0, sizeof(float2) * n, s); }
};

}  // namespace

// ---------------------------------------------------------------- solver
extern "C" tmnd_status tmnd_mg_coarse_apply_internal(const tmnd_mg *mg, float2 *out, const float2 *in, double s,
                                                     cudaStream_t st);
extern "C" tmnd_status tmnd_mg_restrict(const tmnd_mg *mg, void *out_c, const void *in_fine, int nrhs, void *stream);
extern "C" tmnd_status tmnd_mg_prolong(const tmnd_mg *mg, void *out_fine, const void *in_c, int nrhs, void *stream);
tmnd_gauge *tmnd_mg_gauge(const tmnd_mg *mg);

struct MGSolver {
    tmnd_mg *mg;
    tmnd_gauge *g;
    double s;
    cudaStream_t st;
    Blas blas;
    long n;      // fine complex numbers (2 parities x 24 x Vh)
    long nc;     // coarse complex numbers
    int nu_pre, nu_post, coarse_iters;
    int smoother, sap_mr, bd[4];
    double coarse_tol;
    // fine scratch
    float2 *r1, *t1, *t2, *sm_r, *sm_x;
    // coarse scratch
    float2 *cr, *ce, *cres, *cq[16], *cz[16];

    void apply(const float2 *in, float2 *out) {
        k_dnd_full<<<nblk(n / 24), 256, 0, st>>>(g->geom, g->act.kappa, (float)g->st.kp, (float)g->st.kpp, (float)s,
                                                g->links, in, out, 2);
    }
    // smoothing of D' x = r from x = 0: nu SAP sweeps (each: per colour the residual of the
    // whole lattice, then block-local MR on the blocks of that colour), or nu MR steps
    void smooth(const float2 *r, float2 *x, int nu) {
        blas.zero(n, x);
        if (smoother == 1) {
            for (int k = 0; k < nu; k++)
                for (int color = 0; color < 2; color++) {
                    const float2 *res = r;
                    if (k > 0 || color > 0) {
                        apply(x, sm_r);
                        k_rsub<<<nblk(n), 256, 0, st>>>(n, r, sm_r);  // sm_r = r - D' x
                        res = sm_r;
                    }
                    launch_sap_color(g, bd, color, s, res, x, sap_mr, st);
                }
            return;
        }
        blas.copy(n, r, sm_r);
        for (int k = 0; k < nu; k++) {
            apply(sm_r, t1);
            const double2 num = blas.dot(n, t1, sm_r);
            const double den = blas.norm2(n, t1);
            if (den <= 0) break;
            const double2 om = make_double2(num.x / den, num.y / den);
            blas.axpy(n, om, sm_r, x);
            blas.axpy(n, make_double2(-om.x, -om.y), t1, sm_r);
        }
    }
    // coarse GCR on D'_c e = rc (restarted, no preconditioner)
    void coarse_solve(const float2 *rc, float2 *ec) {
        blas.zero(nc, ec);
        blas.copy(nc, rc, cres);
        const double r0 = sqrt(blas.norm2(nc, rc));
        const int m = 16;
        int it = 0;
        while (it < coarse_iters) {
            for (int k = 0; k < m && it < coarse_iters; k++, it++) {
                blas.copy(nc, cres, cz[k]);
                tmnd_mg_coarse_apply_internal(mg, cq[k], cz[k], s, st);
                for (int j = 0; j < k; j++) {
                    const double2 bj = blas.dot(nc, cq[j], cq[k]);
                    blas.axpy(nc, make_double2(-bj.x, -bj.y), cq[j], cq[k]);
                    blas.axpy(nc, make_double2(-bj.x, -bj.y), cz[j], cz[k]);
                }
                const double qn = sqrt(blas.norm2(nc, cq[k]));
                if (qn == 0) return;
                blas.scale(nc, 1.0 / qn, cq[k], cq[k]);
                blas.scale(nc, 1.0 / qn, cz[k], cz[k]);
                const double2 a = blas.dot(nc, cq[k], cres);
                blas.axpy(nc, a, cz[k], ec);
                blas.axpy(nc, make_double2(-a.x, -a.y), cq[k], cres);
                if (sqrt(blas.norm2(nc, cres)) <= coarse_tol * r0) return;
            }
        }
    }
    // one V-cycle: x = M r
    void vcycle(const float2 *r, float2 *x) {
        smooth(r, x, nu_pre);
        apply(x, r1);
        k_rsub<<<nblk(n), 256, 0, st>>>(n, r, r1);  // r1 = r - D' x
        tmnd_mg_restrict(mg, cr, r1, 1, st);
        coarse_solve(cr, ce);
        tmnd_mg_prolong(mg, t2, ce, 1, st);
        blas.axpy(n, make_double2(1, 0), t2, x);
        if (nu_post > 0) {
            apply(x, r1);
            k_rsub<<<nblk(n), 256, 0, st>>>(n, r, r1);
            smooth(r1, t2, nu_post);
            blas.axpy(n, make_double2(1, 0), t2, x);
        }
    }
};

// exposed for the hybrid driver and tests
tmnd_status mg_gcr_solve(tmnd_mg *mg, float2 *x, const float2 *b, double s, double tol, int maxiter, int restart,
                         int nu, cudaStream_t st, int *iters_out, double *res_out, void *scratch) {
    MGSolver S;
    S.mg = mg;
    S.g = tmnd_mg_gauge(mg);
    S.s = s;
    S.st = st;
    int nv = 0;
    const size_t nblock = tmnd_mg_nblock_nv(mg, &nv);
    S.n = 2L * 24 * S.g->geom.Vh;
    S.nc = (long)nblock * 2 * 2 * nv;
    S.nu_pre = nu;
    S.nu_post = nu;
    tmnd_mg_smoother(mg, &S.smoother, &S.sap_mr, S.bd);
    S.coarse_iters = 64;
    S.coarse_tol = 0.05;
    const int mr = restart > 16 ? 16 : restart;
    // scratch layout: fine: r1 t1 t2 sm_r sm_x r z[mr] q[mr]; coarse: cr ce cres cq[16] cz[16]; partials
    char *w = (char *)scratch;
    auto take = [&](long cnt) { float2 *p = (float2 *)w; w += ((sizeof(float2) * cnt + 255) / 256) * 256; return p; };
    S.r1 = take(S.n); S.t1 = take(S.n); S.t2 = take(S.n); S.sm_r = take(S.n); S.sm_x = take(S.n);
    float2 *r = take(S.n);
    float2 *z[16], *q[16];
    for (int k = 0; k < mr; k++) { z[k] = take(S.n); q[k] = take(S.n); }
    S.cr = take(S.nc); S.ce = take(S.nc); S.cres = take(S.nc);
    for (int k = 0; k < 16; k++) { S.cq[k] = take(S.nc); S.cz[k] = take(S.nc); }
    S.blas.s = st;
    S.blas.part = (double *)w;
    S.blas.nb_max = 1024;
    S.blas.h.resize(2 * 1024);

    // r = b - D' x
    S.apply(x, r);
    k_rsub<<<nblk(S.n), 256, 0, st>>>(S.n, b, r);
    const double bn = sqrt(S.blas.norm2(S.n, b));
    double rn = sqrt(S.blas.norm2(S.n, r));
    int it = 0;
    while (rn > tol * bn && it < maxiter) {
        for (int k = 0; k < mr && it < maxiter; k++, it++) {
            S.vcycle(r, z[k]);
            S.apply(z[k], q[k]);
            for (int j = 0; j < k; j++) {
                const double2 bj = S.blas.dot(S.n, q[j], q[k]);
                S.blas.axpy(S.n, make_double2(-bj.x, -bj.y), q[j], q[k]);
                S.blas.axpy(S.n, make_double2(-bj.x, -bj.y), z[j], z[k]);
            }
            const double qn = sqrt(S.blas.norm2(S.n, q[k]));
            if (qn == 0) break;
            S.blas.scale(S.n, 1.0 / qn, q[k], q[k]);
            S.blas.scale(S.n, 1.0 / qn, z[k], z[k]);
            const double2 a = S.blas.dot(S.n, q[k], r);
            S.blas.axpy(S.n, a, z[k], x);
            S.blas.axpy(S.n, make_double2(-a.x, -a.y), q[k], r);
            rn = sqrt(S.blas.norm2(S.n, r));
            if (rn <= tol * bn) { it++; break; }
        }
        // restart: recompute the true residual
        S.apply(x, r);
        k_rsub<<<nblk(S.n), 256, 0, st>>>(S.n, b, r);
        rn = sqrt(S.blas.norm2(S.n, r));
    }
    TMND_CUDA_TRY(cudaStreamSynchronize(st));
    TMND_CUDA_TRY(cudaGetLastError());
    if (iters_out) *iters_out = it;
    if (res_out) *res_out = bn > 0 ? rn / bn : 0.0;
    return TMND_OK;
}

size_t mg_gcr_scratch_bytes(tmnd_mg *mg, int restart) {
    int nv = 0;
    const size_t nblock = tmnd_mg_nblock_nv(mg, &nv);
    const tmnd_gauge *g = tmnd_mg_gauge(mg);
    const size_t n = 2UL * 24 * g->geom.Vh, nc = nblock * 2 * 2 * nv;
    const int mr = restart > 16 ? 16 : restart;
    auto al = [](size_t c) { return ((sizeof(float2) * c + 255) / 256) * 256; };
    return al(n) * (6 + 2 * mr) + al(nc) * (3 + 32) + sizeof(double) * 2 * 1024;
}

tmnd_status tmnd_mg_tc_status(const tmnd_mg *mg);
extern "C" tmnd_status tmnd_mg_create(tmnd_gauge *g, const tmnd_mg_params *p, const void *test_vectors,
                                      tmnd_mg **out);

extern "C" tmnd_status tmnd_mg_solve(tmnd_mg *mg, void *x, const void *b, double s, double tol, int maxiter,
                                     int restart, int nu, int *iters, double *res, void *stream) {
    TMND_ARG_CHECK(mg && x && b, "tmnd_mg_solve: NULL argument");
    TMND_ARG_CHECK(tol > 0 && tol < 1 && maxiter >= 1 && restart >= 1 && nu >= 0, "tmnd_mg_solve: bad parameters");
    cudaGetLastError();
    void *scratch = nullptr;
    TMND_CUDA_TRY(cudaMalloc(&scratch, mg_gcr_scratch_bytes(mg, restart)));
    tmnd_status st = mg_gcr_solve(mg, (float2 *)x, (const float2 *)b, s, tol, maxiter, restart, nu,
                                  (cudaStream_t)stream, iters, res, scratch);
    cudaFree(scratch);
    const tmnd_status tc = tmnd_mg_tc_status(mg);
    return st != TMND_OK ? st : tc;
}

extern "C" tmnd_status tmnd_dnd_full_apply(tmnd_gauge *g, void *out, const void *in, double s, void *stream) {
    TMND_ARG_CHECK(g && out && in && out != in, "tmnd_dnd_full_apply: bad arguments");
    cudaGetLastError();
    k_dnd_full<<<nblk(2L * g->geom.Vh), 256, 0, (cudaStream_t)stream>>>(
        g->geom, g->act.kappa, (float)g->st.kp, (float)g->st.kpp, (float)s, g->links, (const float2 *)in,
        (float2 *)out, 2);
    TMND_CUDA_TRY(cudaGetLastError());
    return TMND_OK;
}

// Near-null test vectors for the setup (Sec. 3: adaptive setup from O(20) test
// vectors): each vector v (single flavour, fine MG layout) is relaxed by `iters`
// minimal-residual steps on D_TM(mu_bar) x = 0 from x = v, which damps the
// large-eigenvalue components, and normalised.
extern "C" tmnd_status tmnd_mg_smooth_vectors(tmnd_gauge *g, void *vecs, int nvec, int iters, void *stream) {
    TMND_ARG_CHECK(g && vecs && nvec >= 1 && iters >= 0, "tmnd_mg_smooth_vectors: bad arguments");
    cudaGetLastError();
    cudaStream_t st = (cudaStream_t)stream;
    const long n = 2L * 12 * g->geom.Vh;
    float2 *t = nullptr;
    double *part = nullptr;
    TMND_CUDA_TRY(cudaMalloc(&t, sizeof(float2) * n));
    TMND_CUDA_TRY(cudaMalloc(&part, sizeof(double) * 2 * 1024));
    Blas blas;
    blas.s = st;
    blas.part = part;
    blas.nb_max = 1024;
    blas.h.resize(2048);
    for (int v = 0; v < nvec; v++) {
        float2 *x = (float2 *)vecs + (size_t)v * n;
        for (int k = 0; k < iters; k++) {
            k_dnd_full<<<nblk(2L * g->geom.Vh), 256, 0, st>>>(g->geom, g->act.kappa, (float)g->st.kp, 0.f, 0.f,
                                                             g->links, x, t, 1);
            // r = -D x ; minimise |D (x + w r)| -> w = -(Dr... use the residual direction r = -Dx:
            // x <- x - w D x with w = <D x, x-ish>: plain MR on D x = 0: r = -D x, w = <D r, r>/<D r, D r>
            // (here r = -t and D r = -D t; the two signs cancel in w)
            const double2 num = blas.dot(n, t, x);     // <Dx, x>
            const double den = blas.norm2(n, t);       // <Dx, Dx>
            if (den <= 0) break;
            blas.axpy(n, make_double2(-num.x / den, -num.y / den), t, x);
        }
        const double nn = blas.norm2(n, x);
        if (nn > 0) blas.scale(n, 1.0 / sqrt(nn), x, x);
    }
    cudaError_t e = cudaStreamSynchronize(st);
    cudaFree(t);
    cudaFree(part);
    if (e != cudaSuccess) {
        tmnd_set_error("tmnd_mg_smooth_vectors: %s", cudaGetErrorString(e));
        return TMND_ERR_CUDA;
    }
    return TMND_OK;
}

// Adaptive (bootstrap) setup: each test vector v is replaced by the flavour-0 part of
// w ~ D_ND^-1 (v, 0) from `iters` outer iterations of the current two-level method, then
// normalised, and a new hierarchy is built from the improved vectors.
extern "C" tmnd_status tmnd_mg_bootstrap(tmnd_mg *mg, const tmnd_mg_params *p, void *test_vectors, int iters,
                                         tmnd_mg **out, void *stream) {
    TMND_ARG_CHECK(mg && p && test_vectors && out, "tmnd_mg_bootstrap: NULL argument");
    TMND_ARG_CHECK(iters >= 1 && iters <= 1000, "tmnd_mg_bootstrap: iters = %d", iters);
    *out = nullptr;
    cudaGetLastError();
    cudaStream_t st = (cudaStream_t)stream;
    tmnd_gauge *g = tmnd_mg_gauge(mg);
    int nv = 0;
    tmnd_mg_nblock_nv(mg, &nv);
    const long vh = g->geom.Vh, n1 = 2L * 12 * vh, n2 = 2L * 24 * vh;
    const int restart = 16;
    const size_t sb = mg_gcr_scratch_bytes(mg, restart);
    char *buf = nullptr;
    TMND_CUDA_TRY(cudaMalloc(&buf, sb + 2 * sizeof(float2) * n2 + sizeof(double) * 2 * 1024));
    float2 *rhs = (float2 *)(buf + sb), *x = rhs + n2;
    Blas blas;
    blas.s = st;
    blas.part = (double *)(x + n2);
    blas.nb_max = 1024;
    blas.h.resize(2048);
    tmnd_status res = TMND_OK;
    for (int v = 0; v < nv && res == TMND_OK; v++) {
        float2 *tv = (float2 *)test_vectors + (size_t)v * n1;
        // (v, 0) in the doublet layout [parity][flavour][12][V/2]
        cudaMemsetAsync(rhs, 0, sizeof(float2) * n2, st);
        for (int par = 0; par < 2; par++)
            cudaMemcpyAsync(rhs + (size_t)par * 24 * vh, tv + (size_t)par * 12 * vh, sizeof(float2) * 12 * vh,
                            cudaMemcpyDeviceToDevice, st);
        cudaMemsetAsync(x, 0, sizeof(float2) * n2, st);
        int it = 0;
        double rr = 0;
        res = mg_gcr_solve(mg, x, rhs, 0.0, 1e-12, iters, restart, 2, st, &it, &rr, buf);
        if (res != TMND_OK) break;
        for (int par = 0; par < 2; par++)
            cudaMemcpyAsync(tv + (size_t)par * 12 * vh, x + (size_t)par * 24 * vh, sizeof(float2) * 12 * vh,
                            cudaMemcpyDeviceToDevice, st);
        const double nn = blas.norm2(n1, tv);
        if (nn > 0 && isfinite(nn)) blas.scale(n1, 1.0 / sqrt(nn), tv, tv);
    }
    cudaError_t e = cudaStreamSynchronize(st);
    cudaFree(buf);
    if (res != TMND_OK) return res;
    if (e != cudaSuccess) {
        tmnd_set_error("tmnd_mg_bootstrap: %s", cudaGetErrorString(e));
        return TMND_ERR_CUDA;
    }
    const tmnd_status tc = tmnd_mg_tc_status(mg);
    if (tc != TMND_OK) return tc;
    return tmnd_mg_create(g, p, test_vectors, out);
}
