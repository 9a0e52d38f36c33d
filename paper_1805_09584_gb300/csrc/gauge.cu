// Gauge handle, workspace, error reporting, spinor (un)packing, tm_nd_apply.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <complex>
#include <vector>

#include "tmnd_internal.cuh"

// ------------------------------------------------------------------ errors
static thread_local char g_err[512] = "";

void tmnd_set_error(const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof g_err, fmt, ap);
    va_end(ap);
}

extern "C" const char *tmnd_last_error(void) { return g_err; }

// --------------------------------------------------------------- workspace
tmnd_status tmnd_ensure_workspace(tmnd_gauge *g, size_t bytes) {
    if (bytes <= g->work_bytes) return TMND_OK;
    if (g->work) {
        TMND_CUDA_TRY(cudaDeviceSynchronize());
        TMND_CUDA_TRY(cudaFree(g->work));
        g->work = nullptr;
        g->work_bytes = 0;
    }
    TMND_CUDA_TRY(cudaMalloc(&g->work, bytes));
    g->work_bytes = bytes;
    return TMND_OK;
}

tmnd_status tmnd_ensure_partials(tmnd_gauge *g, size_t bytes) {
    if (bytes <= g->partials_bytes) return TMND_OK;
    if (g->partials) {
        TMND_CUDA_TRY(cudaDeviceSynchronize());
        TMND_CUDA_TRY(cudaFree(g->partials));
        g->partials = nullptr;
        g->partials_bytes = 0;
    }
    TMND_CUDA_TRY(cudaMalloc((void **)&g->partials, bytes));
    g->partials_bytes = bytes;
    return TMND_OK;
}

// ------------------------------------------------------------ link packing
// canonical complex128 [4][T][X][Y][Z][3][3] -> [2 parity][4 mu][9][Vh]
__global__ void k_pack_links(Geom g, const double2 *__restrict__ canon, double2 *__restrict__ out) {
    long V = 2L * g.Vh;
    long i = (long)blockIdx.x * blockDim.x + threadIdx.x;  // over 4 * V * 9
    if (i >= 4 * V * 9) return;
    int k = (int)(i % 9);
    long rest = i / 9;
    long lex = rest % V;
    int mu = (int)(rest / V);
    long r = lex;
    int z = (int)(r % g.Z); r /= g.Z;
    int y = (int)(r % g.Y); r /= g.Y;
    int x = (int)(r % g.X);
    int t = (int)(r / g.X);
    int par = (t + x + y + z) & 1;
    long h = lex >> 1;
    out[(((size_t)par * 4 + mu) * 9 + k) * g.Vh + h] = canon[i];
}

static bool su3_ok(const std::complex<double> *u) {
    // |U U^+ - 1|_max and |det U - 1|
    double err = 0;
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) {
            std::complex<double> s = 0;
            for (int k = 0; k < 3; k++) s += u[i * 3 + k] * std::conj(u[j * 3 + k]);
            err = fmax(err, std::abs(s - (i == j ? 1.0 : 0.0)));
        }
    std::complex<double> det = u[0] * (u[4] * u[8] - u[5] * u[7]) - u[1] * (u[3] * u[8] - u[5] * u[6]) +
                               u[2] * (u[3] * u[7] - u[4] * u[6]);
    return err < 1e-10 && std::abs(det - 1.0) < 1e-10;
}

// packed FP64 links -> the same layout in FP32 (the FP32 operator)
__global__ void k_links_to_f32(long n, const double2 *__restrict__ in, float2 *__restrict__ out) {
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
        out[i] = make_float2((float)in[i].x, (float)in[i].y);
}

extern "C" tmnd_status tmnd_gauge_create(const double *host_links, const tmnd_action *act, int prec,
                                         tmnd_gauge **out) {
    TMND_ARG_CHECK(out != nullptr, "tmnd_gauge_create: out is NULL");
    *out = nullptr;
    TMND_ARG_CHECK(host_links != nullptr && act != nullptr, "tmnd_gauge_create: NULL argument");
    TMND_ARG_CHECK(prec == TMND_F64 || prec == TMND_S16, "tmnd_gauge_create: unsupported precision %d", prec);
    for (int d = 0; d < 4; d++)
        TMND_ARG_CHECK(act->dims[d] >= 2 && act->dims[d] % 2 == 0,
                       "tmnd_gauge_create: dims[%d] = %d must be even and >= 2", d, act->dims[d]);
    long V = (long)act->dims[0] * act->dims[1] * act->dims[2] * act->dims[3];
    TMND_ARG_CHECK(V / 2 < (1L << 31) / 24, "tmnd_gauge_create: lattice too large");
    TMND_ARG_CHECK(act->kappa > 0 && isfinite(act->kappa) && isfinite(act->mu_bar) && isfinite(act->eps_bar),
                   "tmnd_gauge_create: kappa must be > 0 and parameters finite");
    const double kp = 2 * act->kappa * act->mu_bar, kpp = 2 * act->kappa * act->eps_bar;
    const double det = 1 + kp * kp - kpp * kpp;
    TMND_ARG_CHECK(fabs(det) > 1e-12, "tmnd_gauge_create: site term A is singular (det = %g)", det);

    const std::complex<double> *u = reinterpret_cast<const std::complex<double> *>(host_links);
    for (long l = 0; l < 4 * V; l++)
        if (!su3_ok(u + 9 * l)) {
            tmnd_set_error("tmnd_gauge_create: link %ld (mu=%ld, site=%ld) is not SU(3)", l, l / V, l % V);
            return TMND_ERR_NOTSU3;
        }

    tmnd_gauge *g = new tmnd_gauge();
    memset(g, 0, sizeof *g);
    g->act = *act;
    g->prec = prec;
    cudaGetDevice(&g->device);
    g->geom.T = act->dims[0];
    g->geom.X = act->dims[1];
    g->geom.Y = act->dims[2];
    g->geom.Z = act->dims[3];
    g->geom.Zh = act->dims[3] / 2;
    g->geom.Vh = (int)(V / 2);
    g->geom.apbc = act->antiperiodic_t ? 1 : 0;
    g->st.kappa2 = act->kappa * act->kappa;
    g->st.kp = kp;
    g->st.kpp = kpp;
    g->st.inv_det = 1.0 / det;
    g->stf.kappa2 = (float)g->st.kappa2;
    g->stf.kp = (float)kp;
    g->stf.kpp = (float)kpp;
    g->stf.inv_det = (float)g->st.inv_det;

    size_t nb = sizeof(double2) * 4 * V * 9;
    double2 *canon = nullptr;
    cudaError_t e = cudaMalloc(&g->links, nb);
    if (e == cudaSuccess) e = cudaMalloc(&g->links_s16, sizeof(int2) * 3 * 4 * (size_t)V);
    if (e == cudaSuccess) e = cudaMalloc(&g->links_f32, sizeof(float2) * 4 * V * 9);
    if (e == cudaSuccess) e = cudaMalloc(&canon, nb);
    if (e == cudaSuccess) e = cudaMemcpy(canon, host_links, nb, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        long n = 4 * V * 9;
        k_pack_links<<<(unsigned)((n + 255) / 256), 256>>>(g->geom, canon, g->links);
        launch_pack_links_s16(g->geom, canon, g->links_s16, 0);
        k_links_to_f32<<<(unsigned)((n + 255) / 256), 256>>>(n, g->links, g->links_f32);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (canon) cudaFree(canon);
    if (e != cudaSuccess) {
        tmnd_set_error("tmnd_gauge_create: %s", cudaGetErrorString(e));
        if (g->links) cudaFree(g->links);
        if (g->links_s16) cudaFree(g->links_s16);
        if (g->links_f32) cudaFree(g->links_f32);
        delete g;
        return e == cudaErrorMemoryAllocation ? TMND_ERR_OOM : TMND_ERR_CUDA;
    }
    *out = g;
    return TMND_OK;
}

extern "C" void tmnd_gauge_destroy(tmnd_gauge *g) {
    if (!g) return;
    cudaDeviceSynchronize();
    if (g->links) cudaFree(g->links);
    if (g->links_s16) cudaFree(g->links_s16);
    if (g->links_f32) cudaFree(g->links_f32);
    if (g->work) cudaFree(g->work);
    if (g->partials) cudaFree(g->partials);
    delete g;
}

extern "C" size_t tmnd_spinor_bytes(const tmnd_gauge *g) {
    return g ? sizeof(double2) * NCOMP * (size_t)g->geom.Vh : 0;
}

// ---------------------------------------------------------- spinor packing
// canonical [nrhs][Vh][24] <-> internal [nrhs][24][Vh], complex128.
// A 32-site x 24-component tile goes through shared memory so that both the
// read and the write are coalesced.
constexpr int PK_SITES = 32;

template <bool PACK>
__global__ void k_spinor_transpose(int Vh, const double2 *__restrict__ src, double2 *__restrict__ dst) {
    __shared__ double2 tile[PK_SITES][NCOMP + 1];
    const size_t rhs_off = (size_t)blockIdx.y * NCOMP * Vh;
    const int h0 = blockIdx.x * PK_SITES;
    const int nsite = min(PK_SITES, Vh - h0);
    // load: PACK reads canonical rows (site-major), UNPACK reads internal planes
    for (int i = threadIdx.x; i < PK_SITES * NCOMP; i += blockDim.x) {
        if (PACK) {
            int s = i / NCOMP, c = i % NCOMP;
            if (s < nsite) tile[s][c] = src[rhs_off + (size_t)(h0 + s) * NCOMP + c];
        } else {
            int c = i / PK_SITES, s = i % PK_SITES;
            if (s < nsite) tile[s][c] = src[rhs_off + (size_t)c * Vh + h0 + s];
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < PK_SITES * NCOMP; i += blockDim.x) {
        if (PACK) {
            int c = i / PK_SITES, s = i % PK_SITES;
            if (s < nsite) dst[rhs_off + (size_t)c * Vh + h0 + s] = tile[s][c];
        } else {
            int s = i / NCOMP, c = i % NCOMP;
            if (s < nsite) dst[rhs_off + (size_t)(h0 + s) * NCOMP + c] = tile[s][c];
        }
    }
}

static tmnd_status spinor_transpose(const tmnd_gauge *g, void *dst, const void *src, int nrhs, void *stream,
                                    bool pack) {
    TMND_ARG_CHECK(g && dst && src, "spinor pack/unpack: NULL argument");
    TMND_ARG_CHECK(nrhs >= 1 && nrhs <= 65535, "spinor pack/unpack: nrhs = %d out of range", nrhs);
    TMND_ARG_CHECK(((uintptr_t)dst & 15) == 0 && ((uintptr_t)src & 15) == 0,
                   "spinor pack/unpack: pointers must be 16-byte aligned");
    dim3 grid((g->geom.Vh + PK_SITES - 1) / PK_SITES, nrhs);
    cudaStream_t s = (cudaStream_t)stream;
    if (pack)
        k_spinor_transpose<true><<<grid, 256, 0, s>>>(g->geom.Vh, (const double2 *)src, (double2 *)dst);
    else
        k_spinor_transpose<false><<<grid, 256, 0, s>>>(g->geom.Vh, (const double2 *)src, (double2 *)dst);
    TMND_CUDA_TRY(cudaGetLastError());
    return TMND_OK;
}

extern "C" tmnd_status tmnd_spinor_pack(const tmnd_gauge *g, void *dev_internal, const void *dev_canonical,
                                        int nrhs, void *stream) {
    return spinor_transpose(g, dev_internal, dev_canonical, nrhs, stream, true);
}

extern "C" tmnd_status tmnd_spinor_unpack(const tmnd_gauge *g, void *dev_canonical, const void *dev_internal,
                                          int nrhs, void *stream) {
    return spinor_transpose(g, dev_canonical, dev_internal, nrhs, stream, false);
}

// --------------------------------------------------------------- operators
// gamma_5 tau_1 on an internal spinor: out_f,s = g5(s) in_{1-f},s
__global__ void k_g5tau1(int Vh, const double2 *__restrict__ in, double2 *__restrict__ out) {
    long n = (long)NCOMP * Vh;
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        int c = (int)(i / Vh);
        int h = (int)(i % Vh);
        int f = c / 12, sc = c % 12;
        double2 v = in[(size_t)((1 - f) * 12 + sc) * Vh + h];
        out[i] = (sc >= 6) ? cneg(v) : v;
    }
}

// Mhat (dag = false) or Mhat^+ applied to one right-hand side; te is an even-site temporary.
static void apply_mhat(const tmnd_gauge *g, const double2 *in, double2 *out, double2 *te, bool dag,
                       HopEpi epi, const HopEpiArgs &ea, cudaStream_t s) {
    launch_hop_even_f64(g->geom, g->st, g->links, in, te, dag, nullptr, s);
    launch_hop_odd_f64(g->geom, g->st, g->links, in, te, out, dag, epi, ea, s);
}

// Sloppy operator on TMND_S16 spinors: all right-hand sides in each stencil launch.
static tmnd_status apply_s16(tmnd_gauge *g, void *out, const void *in, int op, double sigma, int nrhs,
                             cudaStream_t s) {
    const int Vh = g->geom.Vh;
    const size_t sb = spinor_bytes_prec(Vh, TMND_S16);
    tmnd_status st = s16_autotune(g, nrhs, s, nullptr, nullptr);  // first use of (lattice, nrhs)
    if (st != TMND_OK) return st;
    st = tmnd_ensure_workspace(g, 2 * (size_t)nrhs * sb);
    if (st != TMND_OK) return st;
    S16Out te = s16_out(g->work, Vh);
    S16Out yo = s16_out((char *)g->work + (size_t)nrhs * sb, Vh);
    S16In te_in{te.q, te.nrm}, yo_in{yo.q, yo.nrm};
    S16EpiArgs ea = {};
    // the even temporaries of all right-hand sides sit sb apart, like the vectors
    S16Batch bt;
    bt.nrhs = nrhs;
    bt.stride = sb;
    const S16In ik = s16_in(in, Vh);
    const S16Out ok = s16_out(out, Vh);
    switch (op) {
        case TMND_OP_MHAT:
        case TMND_OP_MHAT_DAG: {
            const bool dag = op == TMND_OP_MHAT_DAG;
            launch_hop_even_s16(g->geom, g->stf, g->links_s16, ik, te, dag, nullptr, s, bt);
            launch_hop_odd_s16(g->geom, g->stf, g->links_s16, ik, te_in, ok, dag, EPI_STORE, ea, s, bt);
            break;
        }
        case TMND_OP_QHAT2: {
            launch_hop_even_s16(g->geom, g->stf, g->links_s16, ik, te, false, nullptr, s, bt);
            launch_hop_odd_s16(g->geom, g->stf, g->links_s16, ik, te_in, yo, false, EPI_STORE, ea, s, bt);
            S16EpiArgs e2 = {};
            e2.sigma = sigma;
            e2.aux = ik;
            launch_hop_even_s16(g->geom, g->stf, g->links_s16, yo_in, te, true, nullptr, s, bt);
            launch_hop_odd_s16(g->geom, g->stf, g->links_s16, yo_in, te_in, ok, true, EPI_SHIFT, e2, s, bt);
            break;
        }
        default:
            tmnd_set_error("tm_nd_apply: op %d not available for TMND_S16 spinors", op);
            return TMND_ERR_ARG;
    }
    TMND_CUDA_TRY(cudaGetLastError());
    return TMND_OK;
}

// FP32 operator on TMND_F32 spinors (24 complex64 planes per right-hand side), one
// right-hand side per launch sequence.
tmnd_status apply_f32(tmnd_gauge *g, float2 *out, const float2 *in, int op, double sigma, int nrhs, float2 *te,
                      float2 *yo, cudaStream_t s) {
    const size_t n = (size_t)NCOMP * g->geom.Vh;
    HopEpiArgsF ea = {};
    for (int k = 0; k < nrhs; k++) {
        const float2 *ik = in + k * n;
        float2 *ok = out + k * n;
        switch (op) {
            case TMND_OP_MHAT:
            case TMND_OP_MHAT_DAG: {
                const bool dag = op == TMND_OP_MHAT_DAG;
                launch_hop_even_f32(g->geom, g->st, g->links_f32, ik, te, dag, nullptr, s);
                launch_hop_odd_f32(g->geom, g->st, g->links_f32, ik, te, ok, dag, EPI_STORE, ea, s);
                break;
            }
            case TMND_OP_QHAT2: {
                launch_hop_even_f32(g->geom, g->st, g->links_f32, ik, te, false, nullptr, s);
                launch_hop_odd_f32(g->geom, g->st, g->links_f32, ik, te, yo, false, EPI_STORE, ea, s);
                HopEpiArgsF e2 = {};
                e2.sigma = sigma;
                e2.aux = ik;
                launch_hop_even_f32(g->geom, g->st, g->links_f32, yo, te, true, nullptr, s);
                launch_hop_odd_f32(g->geom, g->st, g->links_f32, yo, te, ok, true, EPI_SHIFT, e2, s);
                break;
            }
            default:
                tmnd_set_error("tm_nd_apply: op %d not available for TMND_F32 spinors", op);
                return TMND_ERR_ARG;
        }
    }
    TMND_CUDA_TRY(cudaGetLastError());
    return TMND_OK;
}

extern "C" tmnd_status tm_nd_apply(tmnd_gauge *g, void *out, const void *in, int op, double sigma, int nrhs,
                                   void *stream) {
    TMND_ARG_CHECK(g && out && in, "tm_nd_apply: NULL argument");
    if (op & TMND_OP_F32) {
        TMND_ARG_CHECK(!(op & TMND_OP_S16), "tm_nd_apply: TMND_OP_F32 and TMND_OP_S16 both set");
        TMND_ARG_CHECK(nrhs >= 1 && out != in && ((uintptr_t)out & 15) == 0 && ((uintptr_t)in & 15) == 0 &&
                           isfinite(sigma),
                       "tm_nd_apply: bad arguments (FP32 spinors)");
        cudaGetLastError();
        const size_t s32 = spinor_bytes_prec(g->geom.Vh, TMND_F32);
        tmnd_status st = tmnd_ensure_workspace(g, 2 * s32);
        if (st != TMND_OK) return st;
        return apply_f32(g, (float2 *)out, (const float2 *)in, op & ~TMND_OP_F32, sigma, nrhs, (float2 *)g->work,
                         (float2 *)((char *)g->work + s32), (cudaStream_t)stream);
    }
    if (op & TMND_OP_S16) {
        TMND_ARG_CHECK(nrhs >= 1 && nrhs <= TMND_MAX_BATCH && out != in && ((uintptr_t)out & 15) == 0 &&
                           ((uintptr_t)in & 15) == 0 && isfinite(sigma),
                       "tm_nd_apply: bad arguments (16-bit spinors: 1 <= nrhs <= %d)", TMND_MAX_BATCH);
        cudaGetLastError();
        return apply_s16(g, out, in, op & ~TMND_OP_S16, sigma, nrhs, (cudaStream_t)stream);
    }
    TMND_ARG_CHECK(op >= TMND_OP_MHAT && op <= TMND_OP_QHAT, "tm_nd_apply: unknown op %d", op);
    TMND_ARG_CHECK(nrhs >= 1, "tm_nd_apply: nrhs = %d", nrhs);
    TMND_ARG_CHECK(out != in, "tm_nd_apply: out and in must not alias");
    TMND_ARG_CHECK(((uintptr_t)out & 15) == 0 && ((uintptr_t)in & 15) == 0,
                   "tm_nd_apply: pointers must be 16-byte aligned");
    TMND_ARG_CHECK(isfinite(sigma), "tm_nd_apply: sigma must be finite");
    cudaGetLastError();  // clear a stale, non-sticky error left by earlier unrelated calls
    const size_t sp = tmnd_spinor_bytes(g);
    tmnd_status st = tmnd_ensure_workspace(g, 2 * sp);
    if (st != TMND_OK) return st;
    double2 *te = (double2 *)g->work;
    double2 *yo = (double2 *)((char *)g->work + sp);
    cudaStream_t s = (cudaStream_t)stream;
    const size_t n = sp / sizeof(double2);
    HopEpiArgs ea = {};
    for (int k = 0; k < nrhs; k++) {
        const double2 *ik = (const double2 *)in + k * n;
        double2 *ok = (double2 *)out + k * n;
        switch (op) {
            case TMND_OP_MHAT: apply_mhat(g, ik, ok, te, false, EPI_STORE, ea, s); break;
            case TMND_OP_MHAT_DAG: apply_mhat(g, ik, ok, te, true, EPI_STORE, ea, s); break;
            case TMND_OP_QHAT2: {
                apply_mhat(g, ik, yo, te, false, EPI_STORE, ea, s);
                HopEpiArgs e2 = {};
                e2.sigma = sigma;
                e2.aux = ik;
                apply_mhat(g, yo, ok, te, true, EPI_SHIFT, e2, s);
                break;
            }
            case TMND_OP_QHAT: {
                apply_mhat(g, ik, yo, te, false, EPI_STORE, ea, s);
                k_g5tau1<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(g->geom.Vh, yo, ok);
                break;
            }
        }
    }
    TMND_CUDA_TRY(cudaGetLastError());
    return TMND_OK;
}
