// Kernels of the sloppy stencil: FP32 arithmetic on 16-bit storage (the inner operator of
// the mixed-precision solver).  Same operator as the FP64 kernels
// (Sec. 2: even-odd Schur complement of the ND twisted-mass operator):
//   even:  t_e = kappa^2 A^-1 H_eo psi_o        (dag: kappa^2 A(-mu)^-1 H_eo gamma_5 psi_o)
//   odd :  y_o = A psi_o - H_oe t_e             (dag: A(-mu) psi_o - gamma_5 H_oe t_e)
//
// Storage (16-bit word codec of tmnd_internal.cuh: one complex number per word)
//   spinor (per right-hand side): blocks of 8 sites, each 6 planes of int4,
//     plane j holding complex components 4j..4j+3 (component c = flavour*12 +
//     spin*3 + colour), then the sites' dequantisation scales
//     nrm = max|v| / 32767 (s16_qi / s16_ni of tmnd_internal.cuh).  100 B per site.
//   links: 12-real compression, rows 0 and 1 of U at scale 32767 (|u_ij| <= 1),
//     blocks of 8 sites x 3 planes of int2 per direction and parity (s16_li);
//     row 2 is rebuilt as
//     conj(row0 x row1) (det U = +1, Sec. 2: U in SU(3)).  The antiperiodic
//     sign is applied in the kernel, never folded into links.
//
// The kernels read every neighbour word straight from global memory; the
// arithmetic is in s16_hop.cuh.
//   * PF: the words of the next direction are loaded before the current one is
//     processed (more memory requests in flight per warp).
//   * Links are read once per launch, so their loads bypass L1.
//
// This header holds the kernel templates; each compiled launch shape is instantiated
// in a translation unit of its own (dslash_s16_v*.cu, built in parallel) through
// TMND_S16_DEFINE_SHAPE; dslash_s16.cu dispatches between them and runs the autotuner.
#pragma once

#include "s16_hop.cuh"

namespace {


// Launch shapes the kernels are compiled in: threads per block, resident blocks per
// SM the register budget is cut for, next-direction prefetch.  The autotuner below
// times each on the GPU per (lattice, right-hand sides per launch) and keeps the
// fastest; shape 0 is the default (168 registers, 12 warps per SM; 4 blocks of 128
// at 128 registers spill and ran slower).
#define TMND_S16_SHAPE_LIST(X) X(0, 128, 3, true) X(1, 128, 3, false) X(2, 64, 6, true) X(3, 256, 1, true)

__device__ __forceinline__ int2 ld_link(const int2 *p) {
    int2 r;
    asm("ld.global.nc.L1::no_allocate.v2.s32 {%0, %1}, [%2];" : "=r"(r.x), "=r"(r.y) : "l"(p));
    return r;
}

__device__ __forceinline__ void load_raw(const int4 *__restrict__ q, const float *__restrict__ nrm, int Vh, int hn,
                                         const int2 *__restrict__ L, int hl, Raw &r) {
#pragma unroll
    for (int f = 0; f < 2; f++)
#pragma unroll
        for (int j = 0; j < 3; j++) r.q[f][j] = __ldg(&q[s16_qi(f * 3 + j, hn)]);
#pragma unroll
    for (int j = 0; j < 3; j++) r.l[j] = ld_link(&L[s16_li(j, hl)]);
    r.nrm = __ldg(&nrm[s16_ni(hn)]);
}

// neighbour table of one site: direction d = 2 mu + (0 forward, 1 backward)
struct Nbr {
    int hn[8], hl[8];
    float sg[8];
};

template <int P>
__device__ __forceinline__ void neighbours(const Geom &g, int h, Nbr &n) {
    int zh = h % g.Zh;
    int r = h / g.Zh;
    const int y = r % g.Y;
    r /= g.Y;
    const int x = r % g.X;
    const int t = r / g.X;
    const int z = 2 * zh + ((P + t + x + y) & 1);
    auto idx = [&](int tt, int xx, int yy, int zz) { return ((tt * g.X + xx) * g.Y + yy) * g.Zh + (zz >> 1); };
    const int tf = (t + 1 == g.T) ? 0 : t + 1, tb = (t == 0) ? g.T - 1 : t - 1;
    const int xf = (x + 1 == g.X) ? 0 : x + 1, xb = (x == 0) ? g.X - 1 : x - 1;
    const int yf = (y + 1 == g.Y) ? 0 : y + 1, yb = (y == 0) ? g.Y - 1 : y - 1;
    const int zf = (z + 1 == g.Z) ? 0 : z + 1, zb = (z == 0) ? g.Z - 1 : z - 1;
    n.hn[0] = idx(tf, x, y, z); n.hn[1] = idx(tb, x, y, z);
    n.hn[2] = idx(t, xf, y, z); n.hn[3] = idx(t, xb, y, z);
    n.hn[4] = idx(t, x, yf, z); n.hn[5] = idx(t, x, yb, z);
    n.hn[6] = idx(t, x, y, zf); n.hn[7] = idx(t, x, y, zb);
#pragma unroll
    for (int d = 0; d < 8; d++) {
        n.hl[d] = (d & 1) ? n.hn[d] : h;  // forward: link at x; backward: link at x - mu
        n.sg[d] = 1.0f;
    }
    if (g.apbc && t + 1 == g.T) n.sg[0] = -1.0f;
    if (g.apbc && t == 0) n.sg[1] = -1.0f;
}

// links of direction d: forward from this parity's planes, backward from the other's
template <int P, int D>
__device__ __forceinline__ const int2 *link_base(const int2 *__restrict__ links, int Vh) {
    constexpr int par = (D & 1) ? 1 - P : P;
    return links + ((size_t)par * 4 + D / 2) * 3 * Vh;
}

template <int P, int D, bool G5IN, bool PF>
__device__ __forceinline__ void hop_seq(const int2 *__restrict__ links, const int4 *__restrict__ q,
                                        const float *__restrict__ nrm, int Vh, const Nbr &n, const Raw &cur,
                                        f2 acc[4][3][2]) {
    Raw nxt;
    if constexpr (PF && D < 7) load_raw(q, nrm, Vh, n.hn[D + 1], link_base<P, D + 1>(links, Vh), n.hl[D + 1], nxt);
    hop_dir<D / 2, (D & 1) ? -1 : 1, G5IN, D == 0>(cur, n.sg[D], acc);
    if constexpr (D < 7) {
        if constexpr (!PF) load_raw(q, nrm, Vh, n.hn[D + 1], link_base<P, D + 1>(links, Vh), n.hl[D + 1], nxt);
        hop_seq<P, D + 1, G5IN, PF>(links, q, nrm, Vh, n, nxt, acc);
    }
}

template <int P, bool G5IN, bool PF>
__device__ __forceinline__ void hop_all(const Geom &g, const int2 *__restrict__ links, const int4 *__restrict__ q,
                                        const float *__restrict__ nrm, int h, f2 acc[4][3][2]) {
    Nbr n;
    neighbours<P>(g, h, n);
    Raw r0;
    load_raw(q, nrm, g.Vh, n.hn[0], link_base<P, 0>(links, g.Vh), n.hl[0], r0);
    hop_seq<P, 0, G5IN, PF>(links, q, nrm, g.Vh, n, r0, acc);
}

// Loop order 3: grid stride over (group of 32 consecutive sites, right-hand side) work items,
// one per warp, the right-hand sides of a group on consecutive warps.  All warps move through
// the lattice together as in order 2, but each carries one right-hand side, so the band of
// sites in flight (and the neighbour words it keeps live in L2) is nrhs times narrower; the
// warps of a group read the same links side by side.
template <class F>
__device__ __forceinline__ void grid_stride_rhs_warps(int Vh, const S16Batch &bt, F &&site) {
    const int lane = threadIdx.x & 31;
    const long nwarps = (long)gridDim.x * (blockDim.x >> 5);
    const long items = (long)((Vh + 31) >> 5) * bt.nrhs;
    for (long w = (long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); w < items; w += nwarps) {
        const int k = (int)(w % bt.nrhs);
        const int h = (int)(w / bt.nrhs) * 32 + lane;
        if (h >= Vh || (bt.rdone && bt.rdone[k * bt.rdone_stride])) continue;
        site(h, k);
    }
}

template <bool DAG, bool PF, int NT, int MB>
__global__ void __launch_bounds__(NT, MB) k_hop_even_s16(Geom g, SiteTermF st, const int2 *__restrict__ links,
                                                         S16In in, S16Out out, const int *__restrict__ done,
                                                         int chunk, S16Batch bt) {
    if (done && *done) return;
    const int h_end = min(g.Vh, (int)(blockIdx.x + 1) * chunk);
    auto site = [&](int h, int k) {
        const S16In ik = s16_at(in, k * bt.stride);
        f2 acc[4][3][2];
        hop_all<0, DAG, PF>(g, links, ik.q, ik.nrm, h, acc);
        f2 o[4][3][2];
        even_term<DAG>(st, acc, o);
        const S16Out ok = s16_at(out, k * bt.stride);
        store_site(ok.q, ok.nrm, g.Vh, h, o);
    };
    if (bt.order == 3) {
        grid_stride_rhs_warps(g.Vh, bt, site);
    } else if (bt.order == 2) {  // grid-stride sweep: all blocks move through the lattice together, so
                                 // every right-hand side's neighbours stay in L2 while the band passes
        for (int h = blockIdx.x * blockDim.x + threadIdx.x; h < g.Vh; h += gridDim.x * blockDim.x)
            for (int k = 0; k < bt.nrhs; k++) {
                if (bt.rdone && bt.rdone[k * bt.rdone_stride]) continue;
                site(h, k);
            }
    } else if (bt.order == 1) {  // each right-hand side over the block's chunk, one after another
        for (int k = 0; k < bt.nrhs; k++) {
            if (bt.rdone && bt.rdone[k * bt.rdone_stride]) continue;
            for (int h = blockIdx.x * chunk + threadIdx.x; h < h_end; h += blockDim.x) site(h, k);
        }
    } else {  // every right-hand side of a site before the next site (links hot in cache)
        for (int h = blockIdx.x * chunk + threadIdx.x; h < h_end; h += blockDim.x)
            for (int k = 0; k < bt.nrhs; k++) {
                if (bt.rdone && bt.rdone[k * bt.rdone_stride]) continue;
                site(h, k);
            }
    }
}

// Per-right-hand-side block partials: each thread keeps its running sums in its own
// slots of dynamic shared memory, part[(q * nrhs + k) * blockDim + tid], q = 0, 1.
template <bool DAG, int EPI, bool PF, int NT, int MB>
__global__ void __launch_bounds__(NT, MB) k_hop_odd_s16(Geom g, SiteTermF st, const int2 *__restrict__ links,
                                                        S16In psi_all, S16In te_all, S16Out out_all, S16EpiArgs ea,
                                                        int chunk, S16Batch bt) {
    __shared__ double red[40];
    __shared__ float alpha_s[TMND_MAX_BATCH];
    extern __shared__ double part[];
    if (ea.done && *ea.done) return;
    const int Vh = g.Vh;
    constexpr bool SUMS = EPI == EPI_STORE_NORMS || EPI == EPI_MMS_R;
    if (EPI == EPI_MMS_R) {
        for (int k = 0; k < bt.nrhs; k++) {
            const double yy = block_reduce_partials(ea.part_in + (size_t)(2 * k) * ea.npart_in, ea.npart_in, red);
            const double pp = block_reduce_partials(ea.part_in + (size_t)(2 * k + 1) * ea.npart_in, ea.npart_in, red);
            const double sg = ea.per_rhs_sigma ? ea.sigma_k[k] : ea.sigma;
            if (threadIdx.x == 0) alpha_s[k] = (float)(ea.rr[(size_t)k * ea.rr_stride] / (yy + sg * pp));
        }
    }
    if (SUMS)
        for (int k = 0; k < 2 * bt.nrhs; k++) part[k * blockDim.x + threadIdx.x] = 0.0;
    __syncthreads();
    const int h_end = min(Vh, (int)(blockIdx.x + 1) * chunk);
    auto site = [&](int h, int k) {
        const S16In te = s16_at(te_all, k * bt.stride), psi = s16_at(psi_all, k * bt.stride);
        const S16Out out = s16_at(out_all, k * bt.stride);
        f2 acc[4][3][2];
        hop_all<1, false, PF>(g, links, te.q, te.nrm, h, acc);
        if constexpr (EPI == EPI_MMS_R) {  // w = y + sigma aux; r' = r - alpha w (FP32 planes), plane by plane
            const S16In aux = s16_at(ea.aux, k * bt.stride);
            const float sg = (float)(ea.per_rhs_sigma ? ea.sigma_k[k] : ea.sigma);
            const float s1 = odd_mms_r_fused<DAG>(st, acc, GSite{psi.q, psi.nrm, h}, GSite{aux.q, aux.nrm, h}, sg,
                                                  alpha_s[k], ea.r_in + k * ea.r_stride, ea.r + k * ea.r_stride, Vh,
                                                  h);
            part[k * blockDim.x + threadIdx.x] += s1;
            return;
        }
        f2 p[4][3][2];
        load_site(GSite{psi.q, psi.nrm, h}, p);
        f2 y[4][3][2];
        float s1 = 0.0f, s2 = 0.0f;
        odd_term<DAG, EPI == EPI_STORE_NORMS>(st, acc, p, y, s1, s2);
        if (EPI == EPI_STORE || EPI == EPI_STORE_NORMS) {
            store_site(out.q, out.nrm, Vh, h, y);
            if (EPI == EPI_STORE_NORMS) {
                part[k * blockDim.x + threadIdx.x] += s1;
                part[(bt.nrhs + k) * blockDim.x + threadIdx.x] += s2;
            }
        } else {  // EPI_SHIFT: y + sigma aux
            const S16In aux = s16_at(ea.aux, k * bt.stride);
            add_shift(GSite{aux.q, aux.nrm, h}, (float)ea.sigma, y);
            store_site(out.q, out.nrm, Vh, h, y);
        }
    };
    if (bt.order == 3) {
        grid_stride_rhs_warps(Vh, bt, site);
    } else if (bt.order == 2) {
        for (int h = blockIdx.x * blockDim.x + threadIdx.x; h < Vh; h += gridDim.x * blockDim.x)
            for (int k = 0; k < bt.nrhs; k++) {
                if (bt.rdone && bt.rdone[k * bt.rdone_stride]) continue;
                site(h, k);
            }
    } else if (bt.order == 1) {
        for (int k = 0; k < bt.nrhs; k++) {
            if (bt.rdone && bt.rdone[k * bt.rdone_stride]) continue;
            for (int h = blockIdx.x * chunk + threadIdx.x; h < h_end; h += blockDim.x) site(h, k);
        }
    } else {
        for (int h = blockIdx.x * chunk + threadIdx.x; h < h_end; h += blockDim.x)
            for (int k = 0; k < bt.nrhs; k++) {
                if (bt.rdone && bt.rdone[k * bt.rdone_stride]) continue;
                site(h, k);
            }
    }
    if (SUMS) {
        const int nq = EPI == EPI_STORE_NORMS ? 2 : 1;
        for (int q = 0; q < nq; q++)
            for (int k = 0; k < bt.nrhs; k++) {
                const double t = block_sum(part[(q * bt.nrhs + k) * blockDim.x + threadIdx.x], red);
                if (threadIdx.x == 0) ea.part_out[(size_t)(nq * k + q) * gridDim.x + blockIdx.x] = t;
                __syncthreads();
            }
    }
}

template <bool DAG, int EPI, bool PF, int NT, int MB>
void odd_smem_attr() {
    static bool done = false;  // dynamic shared memory above 48 KB needs an opt-in (256 threads, 16 RHS)
    if (!done) {
        cudaFuncSetAttribute(k_hop_odd_s16<DAG, EPI, PF, NT, MB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(sizeof(double) * 2 * TMND_MAX_BATCH * NT));
        done = true;
    }
}

template <bool PF, int NT, int MB>
int per_sm_of(int dev) {
    int a = 0, b = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_hop_odd_s16<true, EPI_MMS_R, PF, NT, MB>, NT,
                                                  sizeof(double) * 2 * NT);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_hop_even_s16<true, PF, NT, MB>, NT, 0);
    a = a < b ? a : b;
    (void)dev;
    return a > 0 ? a : 1;
}

template <bool PF, int NT, int MB>
void launch_odd_shape(const Geom &g, const SiteTermF &st, const int2 *links, S16In psi, S16In te, S16Out out,
                      bool dag, HopEpi epi, const S16EpiArgs &ea, cudaStream_t s, const S16Batch &bt, int nb) {
    const int chunk = (g.Vh + nb - 1) / nb;
    const size_t smem = sizeof(double) * 2 * bt.nrhs * NT;
#define TMND_ODD16(D, E)                                                                              \
    do {                                                                                              \
        odd_smem_attr<D, E, PF, NT, MB>();                                                            \
        k_hop_odd_s16<D, E, PF, NT, MB><<<nb, NT, smem, s>>>(g, st, links, psi, te, out, ea, chunk, bt); \
    } while (0)
    if (!dag) {
        switch (epi) {
            case EPI_STORE: TMND_ODD16(false, EPI_STORE); break;
            case EPI_STORE_NORMS: TMND_ODD16(false, EPI_STORE_NORMS); break;
            case EPI_SHIFT: TMND_ODD16(false, EPI_SHIFT); break;
            case EPI_MMS_R: TMND_ODD16(false, EPI_MMS_R); break;
        }
    } else {
        switch (epi) {
            case EPI_STORE: TMND_ODD16(true, EPI_STORE); break;
            case EPI_STORE_NORMS: TMND_ODD16(true, EPI_STORE_NORMS); break;
            case EPI_SHIFT: TMND_ODD16(true, EPI_SHIFT); break;
            case EPI_MMS_R: TMND_ODD16(true, EPI_MMS_R); break;
        }
    }
#undef TMND_ODD16
}

}  // namespace

// the extern entry points of one compiled shape (I, threads T, blocks per SM B, prefetch P)
#define TMND_S16_DEFINE_SHAPE(I, T, B, P)                                                                        \
    int s16_per_sm_##I() { return per_sm_of<P, T, B>(0); }                                                      \
    void s16_even_##I(const Geom &g, const SiteTermF &st, const int2 *links, S16In in, S16Out out, bool dag,    \
                      const int *done, cudaStream_t s, const S16Batch &bt, int nb) {                             \
        const int chunk = (g.Vh + nb - 1) / nb;                                                                  \
        if (dag)                                                                                                 \
            k_hop_even_s16<true, P, T, B><<<nb, T, 0, s>>>(g, st, links, in, out, done, chunk, bt);              \
        else                                                                                                     \
            k_hop_even_s16<false, P, T, B><<<nb, T, 0, s>>>(g, st, links, in, out, done, chunk, bt);             \
    }                                                                                                            \
    void s16_odd_##I(const Geom &g, const SiteTermF &st, const int2 *links, S16In psi, S16In te, S16Out out,     \
                     bool dag, HopEpi epi, const S16EpiArgs &ea, cudaStream_t s, const S16Batch &bt, int nb) {   \
        launch_odd_shape<P, T, B>(g, st, links, psi, te, out, dag, epi, ea, s, bt, nb);                         \
    }
