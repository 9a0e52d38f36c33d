// Coarse doublet operator on the tensor cores (tcgen05, kind::tf32).
//
// Per coarse site b the operator of Sec. 3.2 (Eq. "non-degenerate_coarse")
//   y[f] = sum_{d<9} D_W,c[b][d] x_nb(b,d)[f] + i s G_odd[b] x_b[1-f]
//          + i mu_c Gamma_5,c tau_3 x_b - eps_c tau_1 x_b
// is, for all right-hand sides and both flavours at once, a chain of complex
// (2 nvec) x (2 nvec) by (2 nvec) x (2 nrhs) products accumulated in FP32 tensor
// memory.  A complex product is one real GEMM: a stored row of D (re, im
// interleaved) is a real row of length K = 4 nvec, and with
//   B = [Xa | Xb],  Xa = (Re x, -Im x) interleaved,  Xb = (Im x, Re x) interleaved,
// the real product D B = [Re(D x) | Im(D x)].
//
// Data: D_W,c and G_odd are kept a second time in the operand-tile layout (the
// no-swizzle K-major core-matrix layout: 8 rows x 16 bytes per core matrix,
// K-adjacent core matrices ceil8(2 nvec) * 16 bytes apart, row groups 128 bytes
// apart), one contiguous tile per (site, direction); each application first
// writes every site's B tile in the same layout (k_coarse_btiles).  Each pipeline
// step is then two 1-D bulk copies (cp.async.bulk, completion counted on an
// mbarrier) of an A tile and a B tile into a shared-memory stage.
//
// Kernel (persistent, up to 3 blocks per SM, 4 warps, warp-specialised; as many
// shared-memory stages as fit in 70 KB, 2 to 8):
//   warp 2 lane 0  producer: waits for a free stage, bulk-copies A and B;
//   warp 3 lane 0  MMA issuer: M = 128 (rows >= 2 nvec ignored), N = 4 nrhs rounded
//                  up to 16, K = 8 per instruction; the 9 directions accumulate in
//                  one N-column region of tensor memory, G_odd x in a second; two
//                  such accumulator pairs alternate between sites;
//   warps 0, 1     epilogue: read rows 0..63 from tensor memory, add the mu_c /
//                  eps_c terms and i s G_odd x with the flavours swapped, store y.
// Every wait gives up after a limit (~2 s by default, or once another warp has given
// up), sets *err, waits (bounded) for the bulk copies and the MMAs still in flight
// and ends the kernel.  For tests of that path, `stall` makes the MMA issuer of
// every block wait, after its first MMAs, on a barrier that nothing completes, so
// that the wait runs out and the error path runs (no fault, no hang).  TF32
// keeps 10 mantissa bits of each operand (relative error ~1e-3 per product),
// ample for the coarse correction of the preconditioner.
#include <stdint.h>

#include "bulk.cuh"
#include "tmnd_internal.cuh"

namespace {

constexpr int TC_THREADS = 128;
constexpr int TC_M = 128;
constexpr int TC_MAX_STAGES = 8;
// Shared memory per block for the pipeline stages (at least 2 stages), and resident
// blocks per SM: measured at 32^3x64, 48x48 blocks: 1 block with 8 stages 0.38 ms
// (nrhs 1), 2 with 4 stages 0.24 ms, 3 with 2 stages 0.25 ms (0.31 vs 0.33 ms at nrhs 8).
constexpr size_t TC_SMEM_BUDGET = 70 * 1024;
constexpr int TC_MAX_CTAS = 3;
constexpr int TC_SLACK = 2048;  // A rows 2nvec..127 read (and ignore) what follows an A tile

struct TCGeom {
    int nblock, n2, nrhs, npad;
    int nbd[4];
    uint32_t lboA, lboB, abytes, bbytes;  // tile strides and sizes
};

__host__ __device__ inline TCGeom tc_geom(int nblock, const int nbd[4], int nv, int nrhs) {
    TCGeom t;
    t.nblock = nblock;
    t.n2 = 2 * nv;
    t.nrhs = nrhs;
    t.npad = (4 * nrhs + 15) / 16 * 16;
    for (int i = 0; i < 4; i++) t.nbd[i] = nbd[i];
    const int nkg = t.n2 / 2;  // K / 4 = 4 nvec / 4
    t.lboA = (uint32_t)((t.n2 + 7) / 8) * 128u;
    t.lboB = (uint32_t)t.npad * 16u;
    t.abytes = (uint32_t)nkg * t.lboA;
    t.bbytes = (uint32_t)nkg * t.lboB;
    return t;
}

struct TCArgs {
    TCGeom g;
    int stages;
    const unsigned char *Dt, *Gt, *Bt;  // operand tiles: [site][9], [site], [site]
    const float2 *x;
    float2 *y;
    float mu_c, eps_c, s_odd;
    int *err;
    uint64_t wait_ns;  // limit of every bounded wait
    int stall;         // test hook: the MMA issuer waits on a barrier nothing completes
};

// shared-memory matrix descriptor, no swizzle, K-major: lbo = byte step between core
// matrices along K, sbo = byte step between 8-row groups along M (or N)
__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)((lbo & 0x3FFFFu) >> 4) << 16) |
           ((uint64_t)((sbo & 0x3FFFFu) >> 4) << 32) | (1ull << 46);
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void mma_tf32(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}" ::"r"(d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}
__device__ __forceinline__ void mma_commit(uint32_t mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
                 : "memory");
}

// 16 consecutive FP32 columns of this thread's TMEM lane; the wait is tied to the registers
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float v[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
                   "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]),
                   "+r"(r[15])::"memory");
#pragma unroll
    for (int i = 0; i < 16; i++) v[i] = __uint_as_float(r[i]);
}

// neighbour coarse site of b in direction t (0 self, 1 + 2 mu + {0 fwd, 1 bwd}, 9 self)
__device__ __forceinline__ int coarse_nbr(const TCGeom &a, int b, int t) {
    if (t == 0 || t == 9) return b;
    int c[4], r = b;
    c[3] = r % a.nbd[3]; r /= a.nbd[3];
    c[2] = r % a.nbd[2]; r /= a.nbd[2];
    c[1] = r % a.nbd[1];
    c[0] = r / a.nbd[1];
    const int d = t - 1, mu = d >> 1;
    c[mu] = (d & 1) == 0 ? (c[mu] + 1) % a.nbd[mu] : (c[mu] + a.nbd[mu] - 1) % a.nbd[mu];
    return ((c[0] * a.nbd[1] + c[1]) * a.nbd[2] + c[2]) * a.nbd[3] + c[3];
}

// complex (2nvec x 2nvec) row-major blocks -> operand tiles (rows past 2 nvec up to
// the next multiple of 8 zero); one block of threads per tile
__global__ void k_coarse_atiles(const float2 *__restrict__ src, unsigned char *__restrict__ dst, int n2,
                                uint32_t lboA, uint32_t abytes) {
    const int nkg = n2 / 2, mrows = (n2 + 7) / 8 * 8;
    const float4 *s = (const float4 *)(src + (size_t)blockIdx.x * n2 * n2);
    unsigned char *d = dst + (size_t)blockIdx.x * abytes;
    for (int i = threadIdx.x; i < mrows * nkg; i += blockDim.x) {
        const int m = i / nkg, kg = i % nkg;
        const float4 v = m < n2 ? s[(size_t)m * nkg + kg] : make_float4(0.f, 0.f, 0.f, 0.f);
        *(float4 *)(d + kg * lboA + (m >> 3) * 128 + (m & 7) * 16) = v;
    }
}

// B tile of every site for this application: element (n', k'), k' = 2k + {0, 1};
// n' < 2 nrhs: (Re x_k, -Im x_k), 2 nrhs <= n' < 4 nrhs: (Im x_k, Re x_k) of column
// c = n' mod 2 nrhs = f nrhs + r; zero beyond
__global__ void k_coarse_btiles(TCGeom g, const float2 *__restrict__ x, unsigned char *__restrict__ bt) {
    const int b = blockIdx.x, nkg = g.n2 / 2, ncol = 2 * g.nrhs;
    unsigned char *d = bt + (size_t)b * g.bbytes;
    for (int i = threadIdx.x; i < g.npad * nkg; i += blockDim.x) {
        const int np = i / nkg, kg = i % nkg;
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (np < 2 * ncol) {
            const int c = np % ncol, f = c / g.nrhs, r = c % g.nrhs;
            const float4 xv = *(const float4 *)(x + (((size_t)r * g.nblock + b) * 2 + f) * g.n2 + 2 * kg);
            v = np < ncol ? make_float4(xv.x, -xv.y, xv.z, -xv.w) : make_float4(xv.y, xv.x, xv.w, xv.z);
        }
        *(float4 *)(d + kg * g.lboB + (np >> 3) * 128 + (np & 7) * 16) = v;
    }
}

__global__ void __launch_bounds__(TC_THREADS, TC_MAX_CTAS) k_coarse_apply_tc(TCArgs a) {
    extern __shared__ __align__(1024) unsigned char sm[];
    const TCGeom &g = a.g;
    const int n2 = g.n2, K = 2 * n2, ncol = 2 * g.nrhs, N = g.npad;
    const bool godd = a.s_odd != 0.0f;
    const int nsteps = godd ? 10 : 9;
    const uint32_t stage = g.abytes + g.bbytes;
    const int S = a.stages;
    uint64_t *bar = (uint64_t *)(sm + S * stage + TC_SLACK);
    uint64_t *full = bar, *empty = bar + TC_MAX_STAGES, *accf = bar + 2 * TC_MAX_STAGES, *acce = accf + 2;
    uint64_t *drain = acce + 2, *never = drain + 1;  // MMA drain on the error path; the stall hook's barrier
    uint32_t *tholder = (uint32_t *)(never + 1);
    volatile int *sflag = (volatile int *)(tholder + 1);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    uint32_t ncols = 32;
    while ((int)ncols < 4 * N) ncols <<= 1;

    if (tid == 0) {
        for (int j = 0; j < S; j++) {
            mbar_init(smem_u32(&full[j]), 1);
            mbar_init(smem_u32(&empty[j]), 1);
        }
        for (int j = 0; j < 2; j++) {
            mbar_init(smem_u32(&accf[j]), 1);
            mbar_init(smem_u32(&acce[j]), 64);
        }
        mbar_init(smem_u32(drain), 1);
        mbar_init(smem_u32(never), 1);
        *sflag = 0;
        mbar_init_fence();
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tholder)),
                     "r"(ncols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t taddr = *tholder;
    const int nsite = g.nblock > (int)blockIdx.x ? (g.nblock - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;

    // warps 2 and 3 run their loops warp-uniformly; lane 0 issues the copies / MMAs
    if (warp == 2) {  // producer
        int issued = 0;
        for (int q = 0; q < nsite * nsteps; q++) {
            const int b = blockIdx.x + (q / nsteps) * gridDim.x, t = q % nsteps, s = q % S, k = q / S;
            bool ok = k < 1 || mbar_wait(smem_u32(&empty[s]), (uint32_t)((k - 1) & 1), sflag, a.wait_ns);
            if (__any_sync(0xffffffffu, !ok || *sflag)) { *sflag = 1; break; }
            issued = q + 1;
            if (lane == 0) {
                const uint32_t fb = smem_u32(&full[s]), dst = smem_u32(sm + s * stage);
                mbar_expect_tx(fb, stage);
                const unsigned char *A = t < 9 ? a.Dt + ((size_t)b * 9 + t) * g.abytes : a.Gt + (size_t)b * g.abytes;
                bulk_g2s(dst, A, g.abytes, fb);
                bulk_g2s(dst + g.abytes, a.Bt + (size_t)coarse_nbr(g, b, t) * g.bbytes, g.bbytes, fb);
            }
            __syncwarp();
        }
        // after an error, wait (bounded) for the copies still in flight before the block ends
        if (*sflag && lane == 0)
            for (int q = issued - S > 0 ? issued - S : 0; q < issued; q++)
                mbar_wait(smem_u32(&full[q % S]), (uint32_t)((q / S) & 1));
    } else if (warp == 3) {  // MMA issuer
        const uint32_t idesc =
            (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(TC_M >> 4) << 24);
        bool stop = false;
        for (int i = 0, q = 0; i < nsite && !stop; i++) {
            const int buf = i & 1, u = i >> 1;
            bool ok = u < 1 || mbar_wait(smem_u32(&acce[buf]), (uint32_t)((u - 1) & 1), sflag, a.wait_ns);
            if (__any_sync(0xffffffffu, !ok || *sflag)) { *sflag = 1; break; }
            tc_fence_after();
            const uint32_t dmain = taddr + (uint32_t)(buf * 2 * N), dg = dmain + (uint32_t)N;
            for (int t = 0; t < nsteps; t++, q++) {
                const int s = q % S, k = q / S;
                if (a.stall && q == 1) {  // test hook: a wait that runs out (MMAs of step 0 are in flight)
                    ok = mbar_wait(smem_u32(never), 0u, sflag, a.wait_ns);
                    if (__any_sync(0xffffffffu, !ok || *sflag)) { *sflag = 1; stop = true; break; }
                }
                ok = mbar_wait(smem_u32(&full[s]), (uint32_t)(k & 1), sflag, a.wait_ns);
                if (__any_sync(0xffffffffu, !ok || *sflag)) { *sflag = 1; stop = true; break; }
                tc_fence_after();
                if (lane == 0) {
                    const uint32_t a0 = smem_u32(sm + s * stage), b0 = a0 + g.abytes;
                    for (int ks = 0; ks < K / 8; ks++)
                        mma_tf32(t < 9 ? dmain : dg, sdesc(a0 + 2 * ks * g.lboA, g.lboA, 128),
                                 sdesc(b0 + 2 * ks * g.lboB, g.lboB, 128), idesc,
                                 ((t > 0 && t < 9) || ks > 0) ? 1u : 0u);
                    mma_commit(smem_u32(&empty[s]));
                }
                __syncwarp();
            }
            if (stop) break;
            if (lane == 0) mma_commit(smem_u32(&accf[buf]));
            __syncwarp();
        }
        // after an error, wait (bounded) until every MMA this thread issued has completed, so that
        // none still reads shared memory or writes tensor memory when the block frees them
        if (*sflag && lane == 0) {
            mma_commit(smem_u32(drain));
            mbar_wait(smem_u32(drain), 0u);
        }
        __syncwarp();
    } else {  // warps 0, 1: epilogue, rows 0..63 (tensor-memory lanes 32 w + lane)
        const int row = warp * 32 + lane;
        float acc[64], gz[64];
        for (int i = 0; i < nsite; i++) {
            const int b = blockIdx.x + i * gridDim.x, buf = i & 1, u = i >> 1;
            const bool ok = mbar_wait(smem_u32(&accf[buf]), (uint32_t)(u & 1), sflag, a.wait_ns);
            if (__any_sync(0xffffffffu, !ok || *sflag)) { *sflag = 1; break; }
            tc_fence_after();
            const uint32_t tl = taddr + ((uint32_t)(warp * 32) << 16) + (uint32_t)(buf * 2 * N);
            for (int c0 = 0; c0 < N; c0 += 16) tmem_ld16(tl + c0, acc + c0);
            if (godd)
                for (int c0 = 0; c0 < N; c0 += 16) tmem_ld16(tl + N + c0, gz + c0);
            tc_fence_before();
            mbar_arrive(smem_u32(&acce[buf]));
            if (row < n2) {
                const float g5 = row < n2 / 2 ? 1.0f : -1.0f;
                for (int c = 0; c < ncol; c++) {
                    const int f = c / g.nrhs, r = c % g.nrhs, co = (1 - f) * g.nrhs + r;
                    const float2 xf = a.x[(((size_t)r * g.nblock + b) * 2 + f) * n2 + row];
                    const float2 xo = a.x[(((size_t)r * g.nblock + b) * 2 + 1 - f) * n2 + row];
                    const float t3 = f == 0 ? 1.0f : -1.0f;
                    float2 y = make_float2(acc[c], acc[ncol + c]);
                    y.x += -a.mu_c * g5 * t3 * xf.y - a.eps_c * xo.x;
                    y.y += a.mu_c * g5 * t3 * xf.x - a.eps_c * xo.y;
                    if (godd) {  // + i s (G_odd x)[other flavour]
                        y.x -= a.s_odd * gz[ncol + co];
                        y.y += a.s_odd * gz[co];
                    }
                    a.y[(((size_t)r * g.nblock + b) * 2 + f) * n2 + row] = y;
                }
            }
        }
    }
    __syncthreads();
    if (*sflag && tid == 0) atomicExch(a.err, 1);
    tc_fence_after();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

}  // namespace

// Pipeline stages and shared-memory bytes of the tensor-core coarse apply (0 if the
// shape is not supported: 2 nvec a multiple of 4 and <= 64, nrhs <= 16).
static int coarse_tc_stages(int n2, int nrhs) {
    const int nbd[4] = {1, 1, 1, 1};
    const TCGeom g = tc_geom(1, nbd, n2 / 2, nrhs);
    int st = (int)((TC_SMEM_BUDGET - TC_SLACK - 256) / (g.abytes + g.bbytes));
    return st > TC_MAX_STAGES ? TC_MAX_STAGES : (st < 2 ? 2 : st);
}
size_t coarse_tc_smem(int n2, int nrhs) {
    if (n2 % 4 || n2 > 64 || nrhs < 1 || nrhs > 16) return 0;
    const int nbd[4] = {1, 1, 1, 1};
    const TCGeom g = tc_geom(1, nbd, n2 / 2, nrhs);
    return coarse_tc_stages(n2, nrhs) * (size_t)(g.abytes + g.bbytes) + TC_SLACK + 256;
}

// bytes of the operand tiles of one coarse operator (9 directions) or G_odd, per site
size_t coarse_tc_atile_bytes(int nv) {
    const int nbd[4] = {1, 1, 1, 1};
    return tc_geom(1, nbd, nv, 1).abytes;
}

// operand tiles of nmat complex (2nvec x 2nvec) blocks
tmnd_status coarse_tc_make_atiles(const float2 *src, void *dst, long nmat, int nv, cudaStream_t s) {
    const int nbd[4] = {1, 1, 1, 1};
    const TCGeom g = tc_geom(1, nbd, nv, 1);
    k_coarse_atiles<<<(unsigned)nmat, 256, 0, s>>>(src, (unsigned char *)dst, 2 * nv, g.lboA, g.abytes);
    TMND_CUDA_TRY(cudaGetLastError());
    return TMND_OK;
}

// bytes of the B tiles of one application (all sites)
size_t coarse_tc_btile_bytes(int nblock, int nv, int nrhs) {
    const int nbd[4] = {1, 1, 1, 1};
    return (size_t)nblock * tc_geom(nblock, nbd, nv, nrhs).bbytes;
}

tmnd_status launch_coarse_apply_tc(const void *Dt, const void *Gt, void *btiles, const float2 *x, float2 *y,
                                   int nblock, const int nbd[4], int nv, int nrhs, float mu_c, float eps_c,
                                   float s_odd, int *err, uint64_t wait_ns, int stall, cudaStream_t s) {
    const size_t smem = coarse_tc_smem(2 * nv, nrhs);
    TMND_ARG_CHECK(smem > 0, "mg_coarse_apply: tensor-core path needs 2 nvec % 4 == 0, <= 64 and nrhs <= 16");
    TCArgs a;
    a.g = tc_geom(nblock, nbd, nv, nrhs);
    a.stages = coarse_tc_stages(2 * nv, nrhs);
    a.Dt = (const unsigned char *)Dt;
    a.Gt = (const unsigned char *)Gt;
    a.Bt = (const unsigned char *)btiles;
    a.x = x; a.y = y;
    a.mu_c = mu_c; a.eps_c = eps_c; a.s_odd = s_odd; a.err = err;
    a.wait_ns = wait_ns;
    a.stall = stall;
    k_coarse_btiles<<<nblock, 256, 0, s>>>(a.g, x, (unsigned char *)btiles);
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    TMND_CUDA_TRY(cudaFuncSetAttribute(k_coarse_apply_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    TMND_CUDA_TRY(cudaFuncSetAttribute(k_coarse_apply_tc, cudaFuncAttributePreferredSharedMemoryCarveout, 100));
    // resident blocks: shared memory (228 KB per SM, 1 KB reserved per block), at most TC_MAX_CTAS,
    // and the tensor-memory columns of all of them within the SM's 512
    int per_sm = (int)((228 * 1024) / (smem + 1024)), ncols = 32;
    while (ncols < 4 * a.g.npad) ncols <<= 1;
    if (per_sm > TC_MAX_CTAS) per_sm = TC_MAX_CTAS;
    if (per_sm > 512 / ncols) per_sm = 512 / ncols;  // tensor-memory columns of the resident blocks
    if (per_sm < 1) per_sm = 1;
    const int grid = nblock < per_sm * sms ? nblock : per_sm * sms;
    k_coarse_apply_tc<<<grid, TC_THREADS, smem, s>>>(a);
    TMND_CUDA_TRY(cudaGetLastError());
    return TMND_OK;
}
