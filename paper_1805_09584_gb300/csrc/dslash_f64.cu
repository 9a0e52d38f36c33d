// FP64 hopping kernels for the even-odd reduced ND twisted-mass operator.
//
//   even kernel:  t_e = kappa^2 A^-1 H_eo psi_o
//   odd  kernel:  y_o = A psi_o - H_oe t_e                 => y = Mhat psi  (Sec. 2 even-odd reduction)
//   dagger:       Mhat^+ = gamma_5 Mhat(-mu_bar) gamma_5     (A and gamma_5 commute; H is gamma_5-hermitian)
//                 even: kappa^2 A(-mu)^-1 H_eo gamma_5 psi_o
//                 odd : A(-mu) psi_o - gamma_5 H_oe t_e
//
// H psi(x) = sum_mu (1 - gamma_mu) U_mu(x) psi(x+mu) + (1 + gamma_mu) U_mu(x-mu)^+ psi(x-mu)
// (Sec. 2, Eq. "Wilson" in the hopping normalisation).  In the chiral basis
// gamma_mu = [[0, B_mu],[B_mu^+, 0]] with B_0 = -1, B_k = -i sigma_k, so
//   (1 - gamma_mu) psi = (chi, -B^+ chi),  chi = psi_up - B psi_lo
//   (1 + gamma_mu) psi = (chi,  B^+ chi),  chi = psi_up + B psi_lo
// and only the two-spin chi is multiplied by the link (spin projection).
//
// One thread owns one output site and both flavours: the flavours share the
// eight links (the doublet is two right-hand sides of the same hop).  On
// GB300 the FP64 path is bound by the FP64 pipe, not by HBM, so the kernel
// minimises FP64 instructions: links are kept uncompressed (no
// reconstruction arithmetic), boundary signs and gamma_5 are applied as
// sign-bit flips on the integer pipe, multiplications by +-i are swaps, and
// kappa^2 is folded into the A^-1 coefficients.
#include "tmnd_internal.cuh"

namespace {

// (B_mu v) for the lower two spins, v[2][3]
template <int MU, typename C>
__device__ __forceinline__ C Bmul(const C v[2][3], int s, int c) {
    if (MU == 0) return cneg(v[s][c]);
    if (MU == 1) return cmulmi(v[1 - s][c]);                 // -i sigma_1
    if (MU == 2) return s == 0 ? cneg(v[1][c]) : v[0][c];    // -i sigma_2 = [[0,-1],[1,0]]
    return s == 0 ? cmulmi(v[0][c]) : cmuli(v[1][c]);        // -i sigma_3 = diag(-i, i)
}

// (B_mu^+ v)
template <int MU, typename C>
__device__ __forceinline__ C Bdag(const C v[2][3], int s, int c) {
    if (MU == 0) return cneg(v[s][c]);
    if (MU == 1) return cmuli(v[1 - s][c]);                  // i sigma_1
    if (MU == 2) return s == 0 ? v[1][c] : cneg(v[0][c]);    // i sigma_2 = [[0,1],[-1,0]]
    return s == 0 ? cmuli(v[0][c]) : cmulmi(v[1][c]);        // i sigma_3 = diag(i, -i)
}

// Accumulate the hop from neighbour hn in direction MU, DIR (+1 forward
// with U_mu(x), -1 backward with U_mu(x-mu)^+) into acc[flavour][spin][colour].
// G5IN: the input field is gamma_5 psi (lower spins negated).
template <typename C, int MU, int DIR, bool G5IN, bool FIRST = false>
__device__ __forceinline__ void hop_dir(const C *__restrict__ in, int Vh, int hn, const C *__restrict__ U, int hl,
                                        unsigned long long smask, C acc[2][4][3]) {
    C u[3][3];
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++) u[i][j] = __ldg(&U[(i * 3 + j) * Vh + hl]);
    // sign of the B psi_lo term in chi: forward -, backward +; gamma_5 on input flips it
    constexpr bool plus = (DIR < 0) != G5IN;
#pragma unroll
    for (int f = 0; f < 2; f++) {
        C up[2][3], lo[2][3];
#pragma unroll
        for (int s = 0; s < 2; s++)
#pragma unroll
            for (int c = 0; c < 3; c++) {
                up[s][c] = __ldg(&in[(f * 12 + s * 3 + c) * Vh + hn]);
                lo[s][c] = __ldg(&in[(f * 12 + (s + 2) * 3 + c) * Vh + hn]);
            }
        C chi[2][3];
#pragma unroll
        for (int s = 0; s < 2; s++)
#pragma unroll
            for (int c = 0; c < 3; c++) {
                C b = Bmul<MU>(lo, s, c);
                chi[s][c] = cflip(plus ? cadd(up[s][c], b) : csub(up[s][c], b), smask);
            }
        C v[2][3];
#pragma unroll
        for (int s = 0; s < 2; s++)
#pragma unroll
            for (int i = 0; i < 3; i++) {
                if (DIR > 0) {
                    C t = cmul(u[i][0], chi[s][0]);
                    t = cfma(u[i][1], chi[s][1], t);
                    v[s][i] = cfma(u[i][2], chi[s][2], t);
                } else {
                    C t = cmul_conj(u[0][i], chi[s][0]);
                    t = cfma_conj(u[1][i], chi[s][1], t);
                    v[s][i] = cfma_conj(u[2][i], chi[s][2], t);
                }
            }
#pragma unroll
        for (int s = 0; s < 2; s++)
#pragma unroll
            for (int c = 0; c < 3; c++) {
                C b = Bdag<MU>(v, s, c);
                if (FIRST) {  // the first direction initialises the accumulator
                    acc[f][s][c] = v[s][c];
                    acc[f][s + 2][c] = (DIR > 0) ? cneg(b) : b;
                } else {
                    acc[f][s][c] = cadd(acc[f][s][c], v[s][c]);
                    acc[f][s + 2][c] = (DIR > 0) ? csub(acc[f][s + 2][c], b) : cadd(acc[f][s + 2][c], b);
                }
            }
    }
}

// H applied at output site of parity P, half-index h; in = field on parity 1-P.
template <typename C, int P, bool G5IN>
__device__ __forceinline__ void hop_all(const Geom &g, const C *__restrict__ links, const C *__restrict__ in, int h,
                                        C acc[2][4][3]) {
    const int Vh = g.Vh;
    int zh = h % g.Zh;
    int r = h / g.Zh;
    int y = r % g.Y;
    r /= g.Y;
    int x = r % g.X;
    int t = r / g.X;
    int z = 2 * zh + ((P + t + x + y) & 1);
    const C *Lp = links + (size_t)P * 4 * 9 * Vh;         // links based at parity P sites
    const C *Lq = links + (size_t)(1 - P) * 4 * 9 * Vh;   // links based at parity 1-P sites
    const unsigned long long NEG = 0x8000000000000000ull;
    auto idx = [&](int tt, int xx, int yy, int zz) { return ((tt * g.X + xx) * g.Y + yy) * g.Zh + (zz >> 1); };

    // mu = 0 (time), with the antiperiodic sign on boundary-crossing hops
    {
        int tf = (t + 1 == g.T) ? 0 : t + 1;
        int tb = (t == 0) ? g.T - 1 : t - 1;
        unsigned long long mf = (g.apbc && t + 1 == g.T) ? NEG : 0ull;
        unsigned long long mb = (g.apbc && t == 0) ? NEG : 0ull;
        int hf = idx(tf, x, y, z), hb = idx(tb, x, y, z);
        hop_dir<C, 0, +1, G5IN, true>(in, Vh, hf, Lp + 0 * 9 * (size_t)Vh, h, mf, acc);
        hop_dir<C, 0, -1, G5IN>(in, Vh, hb, Lq + 0 * 9 * (size_t)Vh, hb, mb, acc);
    }
    {
        int xf = (x + 1 == g.X) ? 0 : x + 1;
        int xb = (x == 0) ? g.X - 1 : x - 1;
        int hf = idx(t, xf, y, z), hb = idx(t, xb, y, z);
        hop_dir<C, 1, +1, G5IN>(in, Vh, hf, Lp + 1 * 9 * (size_t)Vh, h, 0ull, acc);
        hop_dir<C, 1, -1, G5IN>(in, Vh, hb, Lq + 1 * 9 * (size_t)Vh, hb, 0ull, acc);
    }
    {
        int yf = (y + 1 == g.Y) ? 0 : y + 1;
        int yb = (y == 0) ? g.Y - 1 : y - 1;
        int hf = idx(t, x, yf, z), hb = idx(t, x, yb, z);
        hop_dir<C, 2, +1, G5IN>(in, Vh, hf, Lp + 2 * 9 * (size_t)Vh, h, 0ull, acc);
        hop_dir<C, 2, -1, G5IN>(in, Vh, hb, Lq + 2 * 9 * (size_t)Vh, hb, 0ull, acc);
    }
    {
        int zf = (z + 1 == g.Z) ? 0 : z + 1;
        int zb = (z == 0) ? g.Z - 1 : z - 1;
        int hf = idx(t, x, y, zf), hb = idx(t, x, y, zb);
        hop_dir<C, 3, +1, G5IN>(in, Vh, hf, Lp + 3 * 9 * (size_t)Vh, h, 0ull, acc);
        hop_dir<C, 3, -1, G5IN>(in, Vh, hb, Lq + 3 * 9 * (size_t)Vh, hb, 0ull, acc);
    }
}

// even sites: t_e = kappa^2 A^-1 H psi  (DAG: kappa^2 A(-mu)^-1 H gamma_5 psi)
template <typename C, bool DAG>
__global__ void __launch_bounds__(HOP_THREADS) k_hop_even(Geom g, SiteTerm st, const C *__restrict__ links,
                                                         const C *__restrict__ psi, C *__restrict__ out,
                                                         const int *__restrict__ done, int chunk) {
    using R = decltype(C::x);
    if (done && *done) return;
    const int h_end = min(g.Vh, (blockIdx.x + 1) * chunk);
    for (int h = blockIdx.x * chunk + threadIdx.x; h < h_end; h += blockDim.x) {
    C acc[2][4][3];
    hop_all<C, 0, DAG>(g, links, psi, h, acc);
    const R a = (R)(st.kappa2 * st.inv_det);
    const R e = (R)(st.kappa2 * st.inv_det * st.kpp);
    const int Vh = g.Vh;
#pragma unroll
    for (int s = 0; s < 4; s++) {
        // A^-1 = [[1 - i kp g, kpp],[kpp, 1 + i kp g]] / det, g = gamma_5 eigenvalue
        const R b = a * (R)(DAG ? -st.kp : st.kp) * (s < 2 ? (R)1 : (R)-1);
#pragma unroll
        for (int c = 0; c < 3; c++) {
            C p0 = acc[0][s][c], p1 = acc[1][s][c];
            C o0, o1;
            o0.x = fma(a, p0.x, fma(b, p0.y, e * p1.x));
            o0.y = fma(a, p0.y, fma(-b, p0.x, e * p1.y));
            o1.x = fma(a, p1.x, fma(-b, p1.y, e * p0.x));
            o1.y = fma(a, p1.y, fma(b, p1.x, e * p0.y));
            out[(0 * 12 + s * 3 + c) * Vh + h] = o0;
            out[(1 * 12 + s * 3 + c) * Vh + h] = o1;
        }
    }
    }
}

// odd sites: y = A psi - H t  (DAG: A(-mu) psi - gamma_5 H t), then the epilogue.
template <typename C, bool DAG, int EPI>
__global__ void __launch_bounds__(HOP_THREADS) k_hop_odd(Geom g, SiteTerm st, const C *__restrict__ links,
                                                        const C *__restrict__ psi, const C *__restrict__ te,
                                                        C *__restrict__ out, HopEpiT<C> ea, int chunk) {
    using R = decltype(C::x);
    __shared__ double red[40];
    if (ea.done && *ea.done) return;
    const int Vh = g.Vh;
    double alpha = 0.0;
    if (EPI == EPI_MMS_R) {
        // (p, w) = |Mhat p|^2 + sigma |p|^2 from the previous kernel's partials
        double yy = block_reduce_partials(ea.part_in, ea.npart_in, red);
        double pp = block_reduce_partials(ea.part_in + ea.npart_in, ea.npart_in, red);
        alpha = *ea.rr / (yy + ea.sigma * pp);
    }
    double n1 = 0.0, n2 = 0.0;
    const int h_end = min(Vh, (int)(blockIdx.x + 1) * chunk);
    for (int h = blockIdx.x * chunk + threadIdx.x; h < h_end; h += blockDim.x) {
        C acc[2][4][3];
        hop_all<C, 1, false>(g, links, te, h, acc);
        const R kp = (R)(DAG ? -st.kp : st.kp);
        const R kpp = (R)st.kpp;
        const R al = (R)alpha, sg = (R)ea.sigma;
#pragma unroll
        for (int s = 0; s < 4; s++) {
            const R b = kp * (s < 2 ? (R)1 : (R)-1);
            // DAG: gamma_5 on the hop term flips the sign of the lower spins
            const bool hopneg = DAG && s >= 2;
#pragma unroll
            for (int c = 0; c < 3; c++) {
                C p0 = __ldg(&psi[(0 * 12 + s * 3 + c) * Vh + h]);
                C p1 = __ldg(&psi[(1 * 12 + s * 3 + c) * Vh + h]);
                C h0 = acc[0][s][c], h1 = acc[1][s][c];
                if (hopneg) { h0 = cneg(h0); h1 = cneg(h1); }
                // A = [[1 + i kp g, -kpp],[-kpp, 1 - i kp g]]
                C y0, y1;
                y0.x = fma(-b, p0.y, fma(-kpp, p1.x, p0.x - h0.x));
                y0.y = fma(b, p0.x, fma(-kpp, p1.y, p0.y - h0.y));
                y1.x = fma(b, p1.y, fma(-kpp, p0.x, p1.x - h1.x));
                y1.y = fma(-b, p1.x, fma(-kpp, p0.y, p1.y - h1.y));
                const int i0 = (0 * 12 + s * 3 + c) * Vh + h, i1 = (1 * 12 + s * 3 + c) * Vh + h;
                if (EPI == EPI_STORE || EPI == EPI_STORE_NORMS) {
                    out[i0] = y0;
                    out[i1] = y1;
                    if (EPI == EPI_STORE_NORMS) {
                        n1 = fma((double)y0.x, (double)y0.x, fma((double)y0.y, (double)y0.y,
                                 fma((double)y1.x, (double)y1.x, fma((double)y1.y, (double)y1.y, n1))));
                        n2 = fma((double)p0.x, (double)p0.x, fma((double)p0.y, (double)p0.y,
                                 fma((double)p1.x, (double)p1.x, fma((double)p1.y, (double)p1.y, n2))));
                    }
                } else if (EPI == EPI_SHIFT) {
                    C a0 = __ldg(&ea.aux[i0]), a1 = __ldg(&ea.aux[i1]);
                    C o0, o1;
                    o0.x = fma(sg, a0.x, y0.x); o0.y = fma(sg, a0.y, y0.y);
                    o1.x = fma(sg, a1.x, y1.x); o1.y = fma(sg, a1.y, y1.y);
                    out[i0] = o0;
                    out[i1] = o1;
                } else {  // EPI_MMS_R
                    C a0 = __ldg(&ea.aux[i0]), a1 = __ldg(&ea.aux[i1]);
                    C w0, w1;
                    w0.x = fma(sg, a0.x, y0.x); w0.y = fma(sg, a0.y, y0.y);
                    w1.x = fma(sg, a1.x, y1.x); w1.y = fma(sg, a1.y, y1.y);
                    const C *rin = ea.r_in ? ea.r_in : ea.r;
                    C r0 = rin[i0], r1 = rin[i1];
                    r0.x = fma(-al, w0.x, r0.x); r0.y = fma(-al, w0.y, r0.y);
                    r1.x = fma(-al, w1.x, r1.x); r1.y = fma(-al, w1.y, r1.y);
                    ea.r[i0] = r0;
                    ea.r[i1] = r1;
                    n1 = fma((double)r0.x, (double)r0.x, fma((double)r0.y, (double)r0.y,
                             fma((double)r1.x, (double)r1.x, fma((double)r1.y, (double)r1.y, n1))));
                }
            }
        }
    }
    if (EPI == EPI_STORE_NORMS) {
        double s1 = block_sum(n1, red);
        double s2 = block_sum(n2, red);
        if (threadIdx.x == 0) {
            ea.part_out[blockIdx.x] = s1;
            ea.part_out[gridDim.x + blockIdx.x] = s2;
        }
    } else if (EPI == EPI_MMS_R) {
        double s1 = block_sum(n1, red);
        if (threadIdx.x == 0) ea.part_out[blockIdx.x] = s1;
    }
}

}  // namespace

// Persistent, balanced grid: every SM gets the same number of resident
// blocks and every block a contiguous chunk of about the same number of
// sites, so the FP64 pipe of every SM finishes at the same time (a plain
// one-site-per-thread grid leaves a 1.7-wave tail at 16^3x32).
int hop_blocks(const Geom &g) {
    static int cached[64] = {0};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) dev = 0;
    if (!cached[dev]) {
        int sms = 0, per_sm = 0, per_sm2 = 0;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_hop_odd<double2, true, EPI_MMS_R>, HOP_THREADS, 0);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm2, k_hop_even<double2, true>, HOP_THREADS, 0);
        per_sm = per_sm < per_sm2 ? per_sm : per_sm2;
        if (sms <= 0) sms = 152;
        if (per_sm <= 0) per_sm = 1;
        cached[dev] = sms * per_sm;
    }
    int want = (g.Vh + HOP_THREADS - 1) / HOP_THREADS;
    return want < cached[dev] ? want : cached[dev];
}

static int hop_chunk(const Geom &g) {
    int nb = hop_blocks(g);
    return (g.Vh + nb - 1) / nb;
}

void launch_hop_even_f64(const Geom &g, const SiteTerm &st, const double2 *links, const double2 *psi_o,
                         double2 *t_e, bool dag, const int *done, cudaStream_t s) {
    dim3 grid(hop_blocks(g)), block(HOP_THREADS);
    const int chunk = hop_chunk(g);
    if (dag)
        k_hop_even<double2, true><<<grid, block, 0, s>>>(g, st, links, psi_o, t_e, done, chunk);
    else
        k_hop_even<double2, false><<<grid, block, 0, s>>>(g, st, links, psi_o, t_e, done, chunk);
}

void launch_hop_odd_f64(const Geom &g, const SiteTerm &st, const double2 *links, const double2 *psi_o,
                        const double2 *t_e, double2 *y_o, bool dag, HopEpi epi, const HopEpiArgs &ea,
                        cudaStream_t s) {
    dim3 grid(hop_blocks(g)), block(HOP_THREADS);
    const int chunk = hop_chunk(g);
#define TMND_ODD(D, E) k_hop_odd<double2, D, E><<<grid, block, 0, s>>>(g, st, links, psi_o, t_e, y_o, ea, chunk)
    if (!dag) {
        switch (epi) {
            case EPI_STORE: TMND_ODD(false, EPI_STORE); break;
            case EPI_STORE_NORMS: TMND_ODD(false, EPI_STORE_NORMS); break;
            case EPI_SHIFT: TMND_ODD(false, EPI_SHIFT); break;
            case EPI_MMS_R: TMND_ODD(false, EPI_MMS_R); break;
        }
    } else {
        switch (epi) {
            case EPI_STORE: TMND_ODD(true, EPI_STORE); break;
            case EPI_STORE_NORMS: TMND_ODD(true, EPI_STORE_NORMS); break;
            case EPI_SHIFT: TMND_ODD(true, EPI_SHIFT); break;
            case EPI_MMS_R: TMND_ODD(true, EPI_MMS_R); break;
        }
    }
#undef TMND_ODD
}

// ------------------------------------------------------------- FP32 instantiation
// The same stencil on FP32 planes with 18-real FP32 links: HBM-bound (4416 bytes per odd
// site per Qhat^2), accurate to ~1e-7; the inner residuals of the defect correction.
int hop_blocks_f32(const Geom &g) {
    static int cached[64] = {0};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) dev = 0;
    if (!cached[dev]) {
        int sms = 0, per_sm = 0, per_sm2 = 0;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_hop_odd<float2, true, EPI_MMS_R>, HOP_THREADS, 0);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm2, k_hop_even<float2, true>, HOP_THREADS, 0);
        per_sm = per_sm < per_sm2 ? per_sm : per_sm2;
        if (sms <= 0) sms = 152;
        if (per_sm <= 0) per_sm = 1;
        cached[dev] = sms * per_sm;
    }
    int want = (g.Vh + HOP_THREADS - 1) / HOP_THREADS;
    return want < cached[dev] ? want : cached[dev];
}

void launch_hop_even_f32(const Geom &g, const SiteTerm &st, const float2 *links, const float2 *psi_o, float2 *t_e,
                         bool dag, const int *done, cudaStream_t s) {
    const int nb = hop_blocks_f32(g), chunk = (g.Vh + nb - 1) / nb;
    if (dag)
        k_hop_even<float2, true><<<nb, HOP_THREADS, 0, s>>>(g, st, links, psi_o, t_e, done, chunk);
    else
        k_hop_even<float2, false><<<nb, HOP_THREADS, 0, s>>>(g, st, links, psi_o, t_e, done, chunk);
}

void launch_hop_odd_f32(const Geom &g, const SiteTerm &st, const float2 *links, const float2 *psi_o,
                        const float2 *t_e, float2 *y_o, bool dag, HopEpi epi, const HopEpiArgsF &ea, cudaStream_t s) {
    const int nb = hop_blocks_f32(g), chunk = (g.Vh + nb - 1) / nb;
#define TMND_ODD32(D, E) k_hop_odd<float2, D, E><<<nb, HOP_THREADS, 0, s>>>(g, st, links, psi_o, t_e, y_o, ea, chunk)
    if (!dag) {
        switch (epi) {
            case EPI_STORE: TMND_ODD32(false, EPI_STORE); break;
            case EPI_STORE_NORMS: TMND_ODD32(false, EPI_STORE_NORMS); break;
            case EPI_SHIFT: TMND_ODD32(false, EPI_SHIFT); break;
            case EPI_MMS_R: TMND_ODD32(false, EPI_MMS_R); break;
        }
    } else {
        switch (epi) {
            case EPI_STORE: TMND_ODD32(true, EPI_STORE); break;
            case EPI_STORE_NORMS: TMND_ODD32(true, EPI_STORE_NORMS); break;
            case EPI_SHIFT: TMND_ODD32(true, EPI_SHIFT); break;
            case EPI_MMS_R: TMND_ODD32(true, EPI_MMS_R); break;
        }
    }
#undef TMND_ODD32
}
