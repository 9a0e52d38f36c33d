// tm_nd_apply_noalloc: the operator apply of tm_nd_apply, with its two
// intermediate spinors (one even-site, one odd-site) taken from a fixed
// array in device memory that the library declares, instead of the handle's
// workspace (which tm_nd_apply grows with cudaMalloc on first use).
//
// For callers that cannot allocate device memory at call time: programs whose
// device memory is entirely handed to another allocator (a framework's
// caching allocator, a fixed arena) and leaves no room for a library's own
// cudaMalloc, and latency-critical loops that cannot accept the implicit
// device-wide synchronisation of cudaMalloc/cudaFree.
#include <mutex>

#include "tmnd_internal.cuh"

// Scratch: the even-site temporary followed by the odd-site temporary, each
// 24 complex128 planes of at most TMND_NOALLOC_MAX_VH sites (24 MiB total).
// Every GPU that loads the library holds this array until the process exits.
static __device__ __align__(256) double2 g_noalloc_scratch[2 * NCOMP * TMND_NOALLOC_MAX_VH];

// gamma_5 tau_1 kernel of the allocating path (defined in gauge.cu).
__global__ void k_g5tau1(int Vh, const double2 *__restrict__ in, double2 *__restrict__ out);

namespace {

constexpr int MAX_DEVICES = 64;
std::mutex g_mutex;
double2 *g_scratch_addr[MAX_DEVICES] = {};

// Device address of the scratch array on the current device.  In host code
// `g_noalloc_scratch` names a host-side shadow, not device memory, so the
// address is looked up once per device with that device current.
tmnd_status scratch_address(double2 **out) {
    int dev = 0;
    TMND_CUDA_TRY(cudaGetDevice(&dev));
    TMND_ARG_CHECK(dev >= 0 && dev < MAX_DEVICES, "tm_nd_apply_noalloc: device ordinal %d out of range", dev);
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || p == nullptr) {
            tmnd_set_error("tm_nd_apply_noalloc: cudaGetSymbolAddress of the scratch array failed on device %d: %s",
                           dev, cudaGetErrorString(e));
            return TMND_ERR_CUDA;
        }
        g_scratch_addr[dev] = (double2 *)p;
    }
    *out = g_scratch_addr[dev];
    return TMND_OK;
}

}  // namespace

extern "C" tmnd_status tm_nd_apply_noalloc(const tmnd_gauge *g, void *out, const void *in, int op, double sigma,
                                           int nrhs, void *stream) {
    TMND_ARG_CHECK(g && out && in, "tm_nd_apply_noalloc: NULL argument");
    TMND_ARG_CHECK(op >= TMND_OP_MHAT && op <= TMND_OP_QHAT, "tm_nd_apply_noalloc: unknown op %d", op);
    TMND_ARG_CHECK(nrhs >= 1, "tm_nd_apply_noalloc: nrhs = %d", nrhs);
    TMND_ARG_CHECK(out != in, "tm_nd_apply_noalloc: out and in must not alias");
    TMND_ARG_CHECK(((uintptr_t)out & 15) == 0 && ((uintptr_t)in & 15) == 0,
                   "tm_nd_apply_noalloc: pointers must be 16-byte aligned");
    TMND_ARG_CHECK(isfinite(sigma), "tm_nd_apply_noalloc: sigma must be finite");
    TMND_ARG_CHECK(g->geom.Vh <= TMND_NOALLOC_MAX_VH,
                   "tm_nd_apply_noalloc: lattice has V/2 = %d sites, above the fixed scratch limit of %d "
                   "(use tm_nd_apply)", g->geom.Vh, TMND_NOALLOC_MAX_VH);
    int dev = -1;
    TMND_CUDA_TRY(cudaGetDevice(&dev));
    TMND_ARG_CHECK(dev == g->device, "tm_nd_apply_noalloc: current device %d is not the handle's device %d", dev,
                   g->device);
    double2 *scratch = nullptr;
    tmnd_status st = scratch_address(&scratch);
    if (st != TMND_OK) return st;
    cudaGetLastError();  // clear a stale, non-sticky error left by earlier unrelated calls

    // Both temporaries are fully written before they are read, so nothing
    // needs clearing between calls.
    const size_t n = (size_t)NCOMP * g->geom.Vh;
    double2 *te = scratch;
    double2 *yo = scratch + n;
    cudaStream_t s = (cudaStream_t)stream;
    HopEpiArgs ea = {};
    for (int k = 0; k < nrhs; k++) {
        const double2 *ik = (const double2 *)in + k * n;
        double2 *ok = (double2 *)out + k * n;
        switch (op) {
            case TMND_OP_MHAT:
            case TMND_OP_MHAT_DAG: {
                const bool dag = op == TMND_OP_MHAT_DAG;
                launch_hop_even_f64(g->geom, g->st, g->links, ik, te, dag, nullptr, s);
                launch_hop_odd_f64(g->geom, g->st, g->links, ik, te, ok, dag, EPI_STORE, ea, s);
                break;
            }
            case TMND_OP_QHAT2: {
                launch_hop_even_f64(g->geom, g->st, g->links, ik, te, false, nullptr, s);
                launch_hop_odd_f64(g->geom, g->st, g->links, ik, te, yo, false, EPI_STORE, ea, s);
                HopEpiArgs e2 = {};
                e2.sigma = sigma;
                e2.aux = ik;
                launch_hop_even_f64(g->geom, g->st, g->links, yo, te, true, nullptr, s);
                launch_hop_odd_f64(g->geom, g->st, g->links, yo, te, ok, true, EPI_SHIFT, e2, s);
                break;
            }
            case TMND_OP_QHAT: {
                launch_hop_even_f64(g->geom, g->st, g->links, ik, te, false, nullptr, s);
                launch_hop_odd_f64(g->geom, g->st, g->links, ik, te, yo, false, EPI_STORE, ea, s);
                k_g5tau1<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(g->geom.Vh, yo, ok);
                break;
            }
        }
    }
    TMND_CUDA_TRY(cudaGetLastError());
    return TMND_OK;
}
