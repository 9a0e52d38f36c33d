// Sloppy stencil, host side: dispatch over the compiled launch shapes (kernels in
// s16_kernels.cuh, one translation unit per shape: dslash_s16_v*.cu) and the autotuner
// that picks a launch variant per (lattice, right-hand sides per launch).
#include <array>
#include <map>
#include <mutex>

#include "s16_kernels.cuh"

#define TMND_S16_DECL(I, T, B, P)                                                                               \
    int s16_per_sm_##I();                                                                                       \
    void s16_even_##I(const Geom &g, const SiteTermF &st, const int2 *links, S16In in, S16Out out, bool dag,   \
                      const int *done, cudaStream_t s, const S16Batch &bt, int nb);                             \
    void s16_odd_##I(const Geom &g, const SiteTermF &st, const int2 *links, S16In psi, S16In te, S16Out out,    \
                     bool dag, HopEpi epi, const S16EpiArgs &ea, cudaStream_t s, const S16Batch &bt, int nb);
TMND_S16_SHAPE_LIST(TMND_S16_DECL)
#undef TMND_S16_DECL

namespace {

struct ShapeDesc {
    int threads, minb, pf;
};
constexpr ShapeDesc kShapes[] = {
#define TMND_S16_DESC(I, T, B, P) {T, B, P},
    TMND_S16_SHAPE_LIST(TMND_S16_DESC)
#undef TMND_S16_DESC
};
constexpr int NCOMPILED = sizeof(kShapes) / sizeof(kShapes[0]);
// a launch variant = compiled shape (v % NCOMPILED) x loop order (v / NCOMPILED): 0 = every
// block walks its own chunk of sites, all right-hand sides of a site in turn; 1 = the same
// chunk once per right-hand side; 2 = all blocks sweep the lattice together (grid stride),
// all right-hand sides of a site in turn; 3 = grid stride over (32-site group, right-hand
// side) items, one per warp
constexpr int NORDERS = 4;
constexpr int NSHAPES = NORDERS * NCOMPILED;
static_assert(NSHAPES == TMND_S16_SHAPES, "variant count of include/tmnd.h");

// resident blocks per SM of each shape, per device (the smaller of the even and odd kernels')
int g_per_sm[64][NCOMPILED] = {};

int per_sm(int shape) {
    shape %= NCOMPILED;
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) dev = 0;
    if (!g_per_sm[dev][shape]) {
        switch (shape) {
#define TMND_S16_OCC(I, T, B, P) \
    case I: g_per_sm[dev][I] = s16_per_sm_##I(); break;
            TMND_S16_SHAPE_LIST(TMND_S16_OCC)
#undef TMND_S16_OCC
        }
    }
    return g_per_sm[dev][shape];
}

int sm_count() {
    static int cached[64] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) dev = 0;
    if (!cached[dev]) {
        int sms = 0;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cached[dev] = sms > 0 ? sms : 152;
    }
    return cached[dev];
}

// ---------------------------------------------------------------- autotuner state
// (device, T, X, Y, Z, right-hand sides per launch) -> chosen shape
// Two objectives per key: [0] a Qhat^2 + sigma application (tm_nd_apply), [1] the four
// launches of one sloppy multi-shift iteration (the last with the residual-update epilogue).
std::mutex g_tune_mutex;
std::map<std::array<int, 6>, std::array<int, 2>> g_tuned;
std::map<std::array<int, 6>, std::array<std::array<float, NSHAPES>, 2>> g_tune_ms;
int g_forced = -1;

std::array<int, 6> tune_key(const Geom &g, int nrhs) {
    int dev = 0;
    cudaGetDevice(&dev);
    return {dev, g.T, g.X, g.Y, g.Z, nrhs};
}

}  // namespace

// blocks of a stencil launch in this shape: one per resident slot on every SM (persistent
// grid), at most one site per thread
int hop_blocks_s16(const Geom &g, int shape) {
    if (shape < 0 || shape >= NSHAPES) shape = 0;
    const int nt = kShapes[shape % NCOMPILED].threads;
    const int cap = sm_count() * per_sm(shape);
    const int want = (g.Vh + nt - 1) / nt;
    return want < cap ? want : cap;
}

int hop_blocks_s16_max(const Geom &g) {
    int m = 0;
    for (int s = 0; s < NSHAPES; s++) {
        const int b = hop_blocks_s16(g, s);
        m = b > m ? b : m;
    }
    return m;
}

// the shape for this lattice and number of right-hand sides: forced, else tuned, else 0
// (objective 0: operator applications; 1: sloppy multi-shift iterations)
static int shape_for(const Geom &g, int nrhs, int objective) {
    std::lock_guard<std::mutex> lk(g_tune_mutex);
    if (g_forced >= 0) return g_forced;
    auto it = g_tuned.find(tune_key(g, nrhs));
    return it == g_tuned.end() ? 0 : it->second[objective];
}
int s16_shape(const Geom &g, int nrhs) { return shape_for(g, nrhs, 0); }
int s16_shape_mms(const Geom &g, int nrhs) { return shape_for(g, nrhs, 1); }

void launch_hop_even_s16(const Geom &g, const SiteTermF &st, const int2 *links, S16In in, S16Out out, bool dag,
                         const int *done, cudaStream_t s, const S16Batch &bt_in) {
    const int shape = bt_in.shape >= 0 ? bt_in.shape : s16_shape(g, bt_in.nrhs);
    S16Batch bt = bt_in;
    bt.order = shape / NCOMPILED;
    const int nb = hop_blocks_s16(g, shape);
    switch (shape % NCOMPILED) {
#define TMND_S16_EVEN(I, T, B, P) \
    case I: s16_even_##I(g, st, links, in, out, dag, done, s, bt, nb); break;
        TMND_S16_SHAPE_LIST(TMND_S16_EVEN)
#undef TMND_S16_EVEN
        default: break;
    }
}


void launch_hop_odd_s16(const Geom &g, const SiteTermF &st, const int2 *links, S16In psi, S16In te, S16Out out,
                        bool dag, HopEpi epi, const S16EpiArgs &ea, cudaStream_t s, const S16Batch &bt_in) {
    const int shape = bt_in.shape >= 0 ? bt_in.shape : s16_shape(g, bt_in.nrhs);
    S16Batch bt = bt_in;
    bt.order = shape / NCOMPILED;
    const int nb = hop_blocks_s16(g, shape);
    switch (shape % NCOMPILED) {
#define TMND_S16_ODD(I, T, B, P) \
    case I: s16_odd_##I(g, st, links, psi, te, out, dag, epi, ea, s, bt, nb); break;
        TMND_S16_SHAPE_LIST(TMND_S16_ODD)
#undef TMND_S16_ODD
        default: break;
    }
}

// Autotuner: for every launch variant, on scratch data of nrhs right-hand sides (CUDA events,
// best of 3 after one warm-up), time (0) one 16-bit Qhat^2 + sigma as tm_nd_apply launches it,
// and (1) the four launches of a sloppy multi-shift iteration: the same two even and two odd
// launches, the last one with the residual-update epilogue on FP32 residual planes.  Keep the
// fastest variant for each for this (device, lattice, nrhs).  Skipped (shape 0 stays) while the
// stream is being captured; without room for the scratch shape 0 is kept and 0 ms reported.
tmnd_status s16_autotune(tmnd_gauge *g, int nrhs, cudaStream_t s, int *shape_out, float *ms_out, int objective) {
    TMND_ARG_CHECK(nrhs >= 1 && nrhs <= TMND_MAX_BATCH, "tmnd_autotune: nrhs = %d not in [1, %d]", nrhs,
                   TMND_MAX_BATCH);
    TMND_ARG_CHECK(objective == 0 || objective == 1, "tmnd_autotune: objective %d", objective);
    const auto key = tune_key(g->geom, nrhs);
    {
        std::lock_guard<std::mutex> lk(g_tune_mutex);
        auto it = g_tuned.find(key);
        if (it != g_tuned.end()) {
            if (shape_out) *shape_out = it->second[objective];
            if (ms_out) {
                const auto &t = g_tune_ms[key][objective];
                for (int i = 0; i < NSHAPES; i++) ms_out[i] = t[i];
            }
            return TMND_OK;
        }
    }
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cap) != cudaSuccess || cap != cudaStreamCaptureStatusNone) {
        if (shape_out) *shape_out = 0;
        return TMND_OK;
    }
    const int Vh = g->geom.Vh;
    const size_t sb = spinor_bytes_prec(Vh, TMND_S16);
    const int maxgrid = hop_blocks_s16_max(g->geom);
    // scratch: in, t, y (16-bit) | partials [nrhs][2][grid] of the norms launch and [nrhs][grid]
    // of the residual launch | (r, r) per RHS | residual planes in and out (FP32, nrhs each)
    const size_t off_part = 3 * (size_t)nrhs * sb;
    const size_t off_rr = (off_part + sizeof(double) * 3 * (size_t)nrhs * maxgrid + 255) & ~(size_t)255;
    const size_t off_r = (off_rr + sizeof(double) * (size_t)nrhs + 255) & ~(size_t)255;
    const size_t r_elems = 24 * (size_t)Vh * nrhs;  // float2 per residual set
    const size_t total = off_r + 2 * sizeof(float2) * r_elems;
    char *buf = nullptr;
    if (cudaMalloc(&buf, total) != cudaSuccess) {
        // no room for the scratch: keep the default shape for this pair (tuning is an optimisation)
        cudaGetLastError();
        std::lock_guard<std::mutex> lk(g_tune_mutex);
        g_tuned[key] = {0, 0};
        g_tune_ms[key][0].fill(0.0f);
        g_tune_ms[key][1].fill(0.0f);
        if (shape_out) *shape_out = 0;
        if (ms_out)
            for (int i = 0; i < NSHAPES; i++) ms_out[i] = 0.0f;
        return TMND_OK;
    }
    // biased 16-bit words of 0x4000 and unit scales: finite, data-independent timing; partials
    // and residuals zero, (r, r) = the double of bytes 0x3f (a small positive number)
    cudaMemsetAsync(buf, 0x40, off_part, s);
    cudaMemsetAsync(buf + off_part, 0, off_rr - off_part, s);
    cudaMemsetAsync(buf + off_rr, 0x3f, sizeof(double) * (size_t)nrhs, s);
    cudaMemsetAsync(buf + off_r, 0, 2 * sizeof(float2) * r_elems, s);
    const S16In in = s16_in(buf, Vh);
    const S16Out te = s16_out(buf + (size_t)nrhs * sb, Vh), y = s16_out(buf + 2 * (size_t)nrhs * sb, Vh);
    const S16In tei{te.q, te.nrm}, yi{y.q, y.nrm};
    double *part = (double *)(buf + off_part);
    double *part_r = part + 2 * (size_t)nrhs * maxgrid;
    const double *rr = (const double *)(buf + off_rr);
    float2 *r_in = (float2 *)(buf + off_r), *r_out = r_in + r_elems;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    std::array<std::array<float, NSHAPES>, 2> best;
    int choice[2] = {0, 0};
    cudaError_t err = cudaSuccess;
    for (int sh = 0; sh < NSHAPES && err == cudaSuccess; sh++) {
        if (nrhs == 1 && (sh / NCOMPILED == 1 || sh / NCOMPILED == 3)) {
            // one right-hand side: orders 0 and 1 are the same launch, and so are orders 2 and 3
            best[0][sh] = best[0][sh - NCOMPILED];
            best[1][sh] = best[1][sh - NCOMPILED];
            continue;
        }
        S16Batch bt;
        bt.nrhs = nrhs;
        bt.stride = sb;
        bt.shape = sh;
        S16EpiArgs e1a = {};
        e1a.part_out = part;
        S16EpiArgs e2a = {};  // the application's sigma term
        e2a.sigma = 0.01;
        e2a.aux = in;
        S16EpiArgs e3a = {};  // the multi-shift iteration's residual update
        e3a.sigma = 0.01;
        e3a.aux = in;
        e3a.r_in = r_in;
        e3a.r = r_out;
        e3a.r_stride = 24L * Vh;
        e3a.part_out = part_r;
        e3a.part_in = part;
        e3a.npart_in = hop_blocks_s16(g->geom, sh);
        e3a.rr = rr;
        e3a.rr_stride = 1;
        for (int obj = 0; obj < 2; obj++) {
            best[obj][sh] = 1e30f;
            for (int rep = 0; rep < 4 && err == cudaSuccess; rep++) {
                cudaEventRecord(e0, s);
                launch_hop_even_s16(g->geom, g->stf, g->links_s16, in, te, false, nullptr, s, bt);
                launch_hop_odd_s16(g->geom, g->stf, g->links_s16, in, tei, y, false, EPI_STORE_NORMS, e1a, s, bt);
                launch_hop_even_s16(g->geom, g->stf, g->links_s16, yi, te, true, nullptr, s, bt);
                if (obj == 0)
                    launch_hop_odd_s16(g->geom, g->stf, g->links_s16, yi, tei, te, true, EPI_SHIFT, e2a, s, bt);
                else
                    launch_hop_odd_s16(g->geom, g->stf, g->links_s16, yi, tei, S16Out{}, true, EPI_MMS_R, e3a, s,
                                       bt);
                cudaEventRecord(e1, s);
                err = cudaEventSynchronize(e1);
                float ms = 0;
                if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
                if (rep > 0 && ms < best[obj][sh]) best[obj][sh] = ms;
            }
            if (best[obj][sh] < best[obj][choice[obj]]) choice[obj] = sh;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(buf);
    if (err != cudaSuccess) {
        tmnd_set_error("tmnd_autotune: %s", cudaGetErrorString(err));
        return TMND_ERR_CUDA;
    }
    {
        std::lock_guard<std::mutex> lk(g_tune_mutex);
        g_tuned[key] = {choice[0], choice[1]};
        g_tune_ms[key] = best;
    }
    if (shape_out) *shape_out = choice[objective];
    if (ms_out)
        for (int i = 0; i < NSHAPES; i++) ms_out[i] = best[objective][i];
    return TMND_OK;
}

static tmnd_status autotune_entry(tmnd_gauge *g, int nrhs, int *shape_out, double *ms_out, void *stream,
                                  int objective) {
    TMND_ARG_CHECK(g, "tmnd_autotune: NULL handle");
    cudaGetLastError();
    float ms[NSHAPES] = {};
    int sh = 0;
    const tmnd_status st = s16_autotune(g, nrhs, (cudaStream_t)stream, &sh, ms, objective);
    if (st != TMND_OK) return st;
    if (shape_out) *shape_out = sh;
    if (ms_out)
        for (int i = 0; i < NSHAPES; i++) ms_out[i] = ms[i];
    return TMND_OK;
}

extern "C" tmnd_status tmnd_autotune(tmnd_gauge *g, int nrhs, int *shape_out, double *ms_out, void *stream) {
    return autotune_entry(g, nrhs, shape_out, ms_out, stream, 0);
}

extern "C" tmnd_status tmnd_autotune_mms(tmnd_gauge *g, int nrhs, int *shape_out, double *ms_out, void *stream) {
    return autotune_entry(g, nrhs, shape_out, ms_out, stream, 1);
}

extern "C" tmnd_status tmnd_s16_force_shape(int shape) {
    TMND_ARG_CHECK(shape >= -1 && shape < NSHAPES, "tmnd_s16_force_shape: shape %d not in [-1, %d)", shape, NSHAPES);
    std::lock_guard<std::mutex> lk(g_tune_mutex);
    g_forced = shape;
    return TMND_OK;
}

extern "C" tmnd_status tmnd_s16_shape_info(int shape, int *threads, int *blocks_per_sm, int *prefetch,
                                           int *order) {
    TMND_ARG_CHECK(shape >= 0 && shape < NSHAPES, "tmnd_s16_shape_info: shape %d not in [0, %d)", shape, NSHAPES);
    const ShapeDesc &d = kShapes[shape % NCOMPILED];
    if (threads) *threads = d.threads;
    if (blocks_per_sm) *blocks_per_sm = d.minb;
    if (prefetch) *prefetch = d.pf;
    if (order) *order = shape / NCOMPILED;
    return TMND_OK;
}
