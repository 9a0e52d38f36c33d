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

struct ShiftPtrs {
    double2 *x[NS];
    double2 *p[NS];
};

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

__global__ void k_init_state(MMSState *st, const double *__restrict__ part, int npart, MMSConst c) {
    __shared__ double red[40];
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

// Scalar step of the recursion (one block; thread 0 does the arithmetic).
// j = position of this iteration inside its window.
__global__ void k_scalars(MMSState *st, MMSCoef *cf, const double *__restrict__ part_norm, int nb_hop,
                          const double *__restrict__ part_rr, MMSConst c, int j) {
    __shared__ double red[40];
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
struct RingPtrs {
    const double2 *r[WIN];
};

__global__ void __launch_bounds__(UPD_THREADS) k_window(long n, const MMSCoef *__restrict__ cf, RingPtrs ring,
                                                        ShiftPtrs sp, int nshift) {
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
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        double2 rv[WIN];
#pragma unroll
        for (int l = 0; l < WIN; l++) rv[l] = ring.r[l][i];
        for (int k = 0; k < m; k++) {
            const int s = s_idx[k];
            double2 *xs = sp.x[s];
            double2 *ps = sp.p[s];
            const double2 pi = ps[i];
            double2 xv = xs[i];
            double2 pn = make_double2(s_P[k] * pi.x, s_P[k] * pi.y);
            xv.x = fma(s_a[k], pi.x, xv.x);
            xv.y = fma(s_a[k], pi.y, xv.y);
#pragma unroll
            for (int l = 0; l < WIN; l++) {
                xv.x = fma(s_e[k][l], rv[l].x, xv.x);
                xv.y = fma(s_e[k][l], rv[l].y, xv.y);
                pn.x = fma(s_Q[k][l], rv[l].x, pn.x);
                pn.y = fma(s_Q[k][l], rv[l].y, pn.y);
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

int stream_blocks(long n) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 152;
    long want = (n + UPD_THREADS - 1) / UPD_THREADS;
    long cap = (long)sms * 8;   // 8 resident 256-thread blocks per SM
    return (int)(want < cap ? want : cap);
}

}  // namespace

// One right-hand side.  work holds the WIN residual slots, p, y, te, p_i[nshift]
// (spinor-sized each).  Residual r^(k0+j+1) of window position j goes to slot
// j; position 0 reads slot WIN-1 (the last residual of the previous window,
// or b at the start).
static tmnd_status mms_one_rhs(tmnd_gauge *g, const double2 *b, double2 *const *x, const double *sigma, int nshift,
                               int nsolve, double rho, int maxiter, int check_every, int profile,
                               tmnd_solve_info *info, cudaStream_t s, int rhs_index) {
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

    // Capture one block of `check_every` iterations into a graph.  With
    // profiling, two instances alternate so that the events of one replay are
    // read on the host while the other replay runs.
    const int ninst = profile ? 2 : 1;
    cudaGraphExec_t exec[2] = {nullptr, nullptr};
    std::vector<cudaEvent_t> evs;  // [inst][k][3]
    if (profile) {
        evs.resize((size_t)ninst * check_every * 3);
        for (auto &e : evs) cudaEventCreate(&e);
    }
    auto ev = [&](int inst, int k, int j) { return evs[((size_t)inst * check_every + k) * 3 + j]; };
    for (int inst = 0; inst < ninst; inst++) {
        cudaGraph_t graph = nullptr;
        TMND_CUDA_TRY(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
        for (int k = 0; k < check_every; k++) {
            const int j = k % WIN;  // position inside the window
            if (profile) cudaEventRecordWithFlags(ev(inst, k, 0), s, cudaEventRecordExternal);
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
            if (profile) cudaEventRecordWithFlags(ev(inst, k, 1), s, cudaEventRecordExternal);
            k_scalars<<<1, 256, 0, s>>>(st, cf, part_norm, nb_hop, part_rr, c, j);
            k_pupdate<<<nb_str, UPD_THREADS, 0, s>>>(n, cf, slot[j], p);
            if (j == WIN - 1) k_window<<<nb_str, UPD_THREADS, 0, s>>>(n, cf, ring, ptrs, nshift);
            if (profile) cudaEventRecordWithFlags(ev(inst, k, 2), s, cudaEventRecordExternal);
        }
        cudaError_t ce = cudaStreamEndCapture(s, &graph);
        if (ce == cudaSuccess) ce = cudaGraphInstantiate(&exec[inst], graph, 0);
        if (graph) cudaGraphDestroy(graph);
        if (ce != cudaSuccess) {
            for (auto &e : evs) cudaEventDestroy(e);
            if (exec[0]) cudaGraphExecDestroy(exec[0]);
            tmnd_set_error("mms_cg_solve: graph capture failed: %s", cudaGetErrorString(ce));
            return TMND_ERR_CUDA;
        }
    }

    // Replay with a double-buffered convergence check: replay j runs while
    // the host waits for replay j-1 and reads its done flag.
    int *flags = nullptr;  // pinned [2]
    cudaEvent_t fev[2];
    TMND_CUDA_TRY(cudaHostAlloc((void **)&flags, 2 * sizeof(int), cudaHostAllocDefault));
    cudaEventCreateWithFlags(&fev[0], cudaEventDisableTiming);
    cudaEventCreateWithFlags(&fev[1], cudaEventDisableTiming);
    std::vector<float> hop_t, upd_t;  // per global iteration
    auto harvest = [&](long j) {       // read the events of replay j (complete)
        int inst = (int)(j % ninst);
        for (int k = 0; k < check_every; k++) {
            float a = 0.f, b2 = 0.f;
            if (cudaEventElapsedTime(&a, ev(inst, k, 0), ev(inst, k, 1)) != cudaSuccess ||
                cudaEventElapsedTime(&b2, ev(inst, k, 1), ev(inst, k, 2)) != cudaSuccess) {
                cudaGetLastError();
                a = b2 = nanf("");
            }
            hop_t.push_back(a);
            upd_t.push_back(b2);
        }
    };
    const long max_launch = (long)maxiter / check_every + 3;
    long nlaunch = 0;
    cudaError_t err = cudaSuccess;
    for (long j = 0; j < max_launch && err == cudaSuccess; j++) {
        err = cudaGraphLaunch(exec[j % ninst], s);
        if (err != cudaSuccess) break;
        nlaunch++;
        cudaMemcpyAsync(&flags[j & 1], &st->done, sizeof(int), cudaMemcpyDeviceToHost, s);
        cudaEventRecord(fev[j & 1], s);
        if (j > 0) {
            err = cudaEventSynchronize(fev[(j - 1) & 1]);
            if (err == cudaSuccess && profile) harvest(j - 1);
            if (err == cudaSuccess && flags[(j - 1) & 1]) break;
        }
    }
    if (err == cudaSuccess) err = cudaStreamSynchronize(s);
    if (err == cudaSuccess && profile && nlaunch > 0) harvest(nlaunch - 1);
    cudaEventDestroy(fev[0]);
    cudaEventDestroy(fev[1]);
    cudaFreeHost(flags);
    for (int inst = 0; inst < ninst; inst++) cudaGraphExecDestroy(exec[inst]);
    for (auto &e : evs) cudaEventDestroy(e);
    if (err != cudaSuccess) {
        tmnd_set_error("mms_cg_solve: %s", cudaGetErrorString(err));
        return TMND_ERR_CUDA;
    }
    if (info) info->launches += 2 + nlaunch * ((long long)check_every * 6 + check_every / WIN) + 5LL * nshift;

    MMSState hs;
    TMND_CUDA_TRY(cudaMemcpy(&hs, st, sizeof hs, cudaMemcpyDeviceToHost));

    // true residuals |b - (Qhat^2 + sigma_i) x_i| / |b| with the operator
    double *hpart = new double[nb_str];
    for (int i = 0; i < nshift; i++) {
        HopEpiArgs ea = {};
        launch_hop_even_f64(g->geom, g->st, g->links, ptrs.x[i], te, false, nullptr, s);
        launch_hop_odd_f64(g->geom, g->st, g->links, ptrs.x[i], te, r, false, EPI_STORE, ea, s);
        HopEpiArgs e2 = {};
        e2.sigma = sigma[i];
        e2.aux = ptrs.x[i];
        launch_hop_even_f64(g->geom, g->st, g->links, r, te, true, nullptr, s);
        launch_hop_odd_f64(g->geom, g->st, g->links, r, te, y, true, EPI_SHIFT, e2, s);
        k_diff_norm<<<nb_str, UPD_THREADS, 0, s>>>(n, b, y, part_str);
        cudaError_t e3 = cudaMemcpyAsync(hpart, part_str, sizeof(double) * nb_str, cudaMemcpyDeviceToHost, s);
        if (e3 == cudaSuccess) e3 = cudaStreamSynchronize(s);
        if (e3 != cudaSuccess) {
            delete[] hpart;
            tmnd_set_error("mms_cg_solve: %s", cudaGetErrorString(e3));
            return TMND_ERR_CUDA;
        }
        double acc = 0;
        for (int k = 0; k < nb_str; k++) acc += hpart[k];
        double tr = hs.bb > 0 ? sqrt(acc / hs.bb) : 0.0;
        if (info && (rhs_index == 0 || tr > info->true_res[i])) info->true_res[i] = tr;
    }
    delete[] hpart;
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

    const size_t sp = tmnd_spinor_bytes(g);
    tmnd_status st = tmnd_ensure_workspace(g, (WIN + 3 + (size_t)nshift) * sp);
    if (st != TMND_OK) return st;
    const long n = (long)(sp / sizeof(double2));
    size_t pbytes = sizeof(double) * (3 * (size_t)hop_blocks(g->geom) + stream_blocks(n)) + 256 + 2 * 4096 +
                    sizeof(MMSState) + sizeof(MMSCoef);
    st = tmnd_ensure_partials(g, pbytes);
    if (st != TMND_OK) return st;
    if (info) memset(info, 0, sizeof *info);

    // run on a private stream ordered after the caller's stream (capture needs a non-legacy stream)
    cudaStream_t user = (cudaStream_t)stream;
    cudaStream_t s;
    TMND_CUDA_TRY(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    cudaEvent_t e0;
    TMND_CUDA_TRY(cudaEventCreateWithFlags(&e0, cudaEventDisableTiming));
    TMND_CUDA_TRY(cudaEventRecord(e0, user));
    TMND_CUDA_TRY(cudaStreamWaitEvent(s, e0, 0));
    tmnd_status res = TMND_OK;
    for (int k = 0; k < nrhs && res == TMND_OK; k++) {
        tmnd_status rk = mms_one_rhs(g, (const double2 *)b + (size_t)k * (sp / sizeof(double2)),
                                     (double2 *const *)x, sigma, nshift, nsolve, params->rho, params->maxiter,
                                     check_every, params->profile ? 1 : 0, info, s, k);
        if (rk != TMND_OK) res = rk;
    }
    cudaEventRecord(e0, s);
    cudaStreamWaitEvent(user, e0, 0);
    cudaStreamSynchronize(s);
    cudaEventDestroy(e0);
    cudaStreamDestroy(s);
    return res;
}
