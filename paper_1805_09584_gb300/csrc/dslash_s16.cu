// Sloppy stencil: FP32 arithmetic on 16-bit storage (the inner operator of
// the mixed-precision solver).  Same operator as the FP64 kernels
// (Sec. 2: even-odd Schur complement of the ND twisted-mass operator):
//   even:  t_e = kappa^2 A^-1 H_eo psi_o        (dag: kappa^2 A(-mu)^-1 H_eo gamma_5 psi_o)
//   odd :  y_o = A psi_o - H_oe t_e             (dag: A(-mu) psi_o - gamma_5 H_oe t_e)
//
// Storage (16-bit word codec of tmnd_internal.cuh: one complex number per word)
//   spinor (per right-hand side): 6 planes of int4 over V/2 sites, plane j
//     holding complex components 4j..4j+3 (component c = flavour*12 + spin*3 +
//     colour), then one float per site, the dequantisation scale
//     nrm = max|v| / 32767 of that site.  100 B per site.
//   links: 12-real compression, rows 0 and 1 of U at scale 32767 (|u_ij| <= 1),
//     3 planes of int2 per direction and parity; row 2 is rebuilt as
//     conj(row0 x row1) (det U = +1, Sec. 2: U in SU(3)).  The antiperiodic
//     sign is applied in the kernel, never folded into links.
//
// Arithmetic
//   * One thread per site, both flavours: the two flavours share every link, so
//     each flavour pair of a spinor component lives in one float2 and all link
//     products, projections and accumulations are packed f32x2 instructions
//     (one instruction for both flavours).
//   * Decoding is one byte permute per value (the float 2^23 + 32768 + n); the
//     spin projection u -+ B l is formed from two decoded floats exactly
//     (their difference, or u + (l - 2 * bias)), so the projected half spinor
//     is exact before the link is applied.
//   * The neighbour's scale nrm/32767 and the boundary sign enter as one factor
//     of the accumulation.
//   * PF: the words of the next direction are loaded before the current one is
//     processed (more memory requests in flight per warp).
//   * Links are read once per launch, so their loads bypass L1.
#include "tmnd_internal.cuh"

namespace {

constexpr int S16_THREADS = 128;
// resident blocks per SM the register budget is cut for (168 registers; 4 blocks
// at 128 registers spill and ran slower)
constexpr int S16_MINB = 3;
constexpr float INV_QMAX = 1.0f / S16_QMAX;

__device__ __forceinline__ int2 ld_link(const int2 *p) {
    int2 r;
    asm("ld.global.nc.L1::no_allocate.v2.s32 {%0, %1}, [%2];" : "=r"(r.x), "=r"(r.y) : "l"(p));
    return r;
}

using f2 = float2;  // (flavour 0, flavour 1)

__device__ __forceinline__ f2 dup(float a) { return make_float2(a, a); }
__device__ __forceinline__ f2 add2(f2 a, f2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ f2 mul2(f2 a, f2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ f2 fma2(f2 a, f2 b, f2 c) { return __ffma2_rn(a, b, c); }

__device__ __forceinline__ S16In s16_at(S16In a, size_t off) {
    return S16In{(const int4 *)((const char *)a.q + off), (const float *)((const char *)a.nrm + off)};
}
__device__ __forceinline__ S16Out s16_at(S16Out a, size_t off) {
    return S16Out{(int4 *)((char *)a.q + off), (float *)((char *)a.nrm + off)};
}

// the words one direction needs: neighbour spinor (both flavours), link, scale
struct Raw {
    int4 q[2][3];
    int2 l[3];
    float nrm;
};

__device__ __forceinline__ void load_raw(const int4 *__restrict__ q, const float *__restrict__ nrm, int Vh, int hn,
                                         const int2 *__restrict__ L, int hl, Raw &r) {
#pragma unroll
    for (int f = 0; f < 2; f++)
#pragma unroll
        for (int j = 0; j < 3; j++) r.q[f][j] = __ldg(&q[(f * 3 + j) * Vh + hn]);
#pragma unroll
    for (int j = 0; j < 3; j++) r.l[j] = ld_link(&L[j * Vh + hl]);
    r.nrm = __ldg(&nrm[hn]);
}

__device__ __forceinline__ int word(const int4 &v, int k) { return k == 0 ? v.x : k == 1 ? v.y : k == 2 ? v.z : v.w; }

// flavour pair of the biased floats of component k (= spin*3 + colour): re, im
__device__ __forceinline__ void comp(const Raw &r, int k, f2 &re, f2 &im) {
    const int w0 = word(r.q[0][k / 4], k % 4), w1 = word(r.q[1][k / 4], k % 4);
    re = make_float2(s16_flo(w0), s16_flo(w1));
    im = make_float2(s16_fhi(w0), s16_fhi(w1));
}

// u + SG * l for biased floats u, l (exact integer result)
template <int SG>
__device__ __forceinline__ f2 comb(f2 u, f2 l) {
    if (SG < 0) return fma2(l, dup(-1.0f), u);
    return add2(u, add2(l, dup(-2.0f * S16_DEC_BIAS)));
}

template <int MU, int DIR, bool G5IN, bool FIRST>
__device__ __forceinline__ void hop_dir(const Raw &r, float sign, f2 acc[4][3][2]) {
    // link rows 0 and 1 (integer-valued floats, scale 32767) and rebuilt row 2 (same scale)
    float ur[3][3], ui[3][3];
    {
        const int wv[6] = {r.l[0].x, r.l[0].y, r.l[1].x, r.l[1].y, r.l[2].x, r.l[2].y};
#pragma unroll
        for (int k = 0; k < 6; k++) {
            ur[k / 3][k % 3] = s16_lo(wv[k]);
            ui[k / 3][k % 3] = s16_hi(wv[k]);
        }
#pragma unroll
        for (int k = 0; k < 3; k++) {
            const int k1 = (k + 1) % 3, k2 = (k + 2) % 3;
            float re = fmaf(ur[0][k1], ur[1][k2], -ui[0][k1] * ui[1][k2]);
            float im = fmaf(ur[0][k1], ui[1][k2], ui[0][k1] * ur[1][k2]);
            re = fmaf(-ur[0][k2], ur[1][k1], fmaf(ui[0][k2], ui[1][k1], re));
            im = fmaf(-ur[0][k2], ui[1][k1], fmaf(-ui[0][k2], ur[1][k1], im));
            ur[2][k] = re * INV_QMAX;
            ui[2][k] = -im * INV_QMAX;
        }
    }
    // projection chi = u -+ B l (upper spins 0, 1), exact integers.
    // B l, by direction (lower spin index, components):
    //   MU 0: lower 2+s,   (-l.re, -l.im)
    //   MU 1: lower 3-s,   (l.im, -l.re)
    //   MU 2: lower 3-s,   s = 0: (-l.re, -l.im); s = 1: (l.re, l.im)
    //   MU 3: lower 2+s,   s = 0: (l.im, -l.re);  s = 1: (-l.im, l.re)
    constexpr bool plus = (DIR < 0) != G5IN;
    constexpr int P = plus ? 1 : -1;
    f2 chr[2][3], chi[2][3];
#pragma unroll
    for (int s = 0; s < 2; s++)
#pragma unroll
        for (int c = 0; c < 3; c++) {
            const int sl = (MU == 0 || MU == 3) ? 2 + s : 3 - s;
            f2 uR, uI, lR, lI;
            comp(r, s * 3 + c, uR, uI);
            comp(r, sl * 3 + c, lR, lI);
            if (MU == 0 || (MU == 2 && s == 0)) {
                chr[s][c] = comb<-P>(uR, lR);
                chi[s][c] = comb<-P>(uI, lI);
            } else if (MU == 2) {
                chr[s][c] = comb<P>(uR, lR);
                chi[s][c] = comb<P>(uI, lI);
            } else if (MU == 1 || s == 0) {  // (l.im, -l.re)
                chr[s][c] = comb<P>(uR, lI);
                chi[s][c] = comb<-P>(uI, lR);
            } else {  // MU 3, s 1: (-l.im, l.re)
                chr[s][c] = comb<-P>(uR, lI);
                chi[s][c] = comb<P>(uI, lR);
            }
        }
    // v = W chi with W = U (forward) or U^+ (backward); both flavours at once.
    //   forward : re = sum ur chr - sum ui chi,  im = sum ur chi + sum ui chr
    //   backward: re = sum ur' chr + sum ui' chi, im = sum ur' chi - sum ui' chr  (ur' = ur[j][i])
    const float cs = sign * r.nrm * INV_QMAX;
    const f2 cs2 = dup(cs), ncs2 = dup(-cs);
    // lower-spin factor cl = -cs (forward) or cs (backward) and its negative
    const f2 cl2 = DIR > 0 ? ncs2 : cs2, ncl2 = DIR > 0 ? cs2 : ncs2;
    f2 vr[2][3], vi[2][3];
#pragma unroll
    for (int i = 0; i < 3; i++) {
        f2 wr[3], wi[3];
#pragma unroll
        for (int j = 0; j < 3; j++) {
            wr[j] = dup(DIR > 0 ? ur[i][j] : ur[j][i]);
            wi[j] = dup(DIR > 0 ? ui[i][j] : ui[j][i]);
        }
#pragma unroll
        for (int s = 0; s < 2; s++) {
            f2 a = mul2(wr[0], chr[s][0]);
            a = fma2(wr[1], chr[s][1], a);
            a = fma2(wr[2], chr[s][2], a);
            f2 b = mul2(wi[0], chi[s][0]);
            b = fma2(wi[1], chi[s][1], b);
            b = fma2(wi[2], chi[s][2], b);
            f2 c = mul2(wr[0], chi[s][0]);
            c = fma2(wr[1], chi[s][1], c);
            c = fma2(wr[2], chi[s][2], c);
            f2 d = mul2(wi[0], chr[s][0]);
            d = fma2(wi[1], chr[s][1], d);
            d = fma2(wi[2], chr[s][2], d);
            if (DIR > 0) {
                vr[s][i] = fma2(b, dup(-1.0f), a);
                vi[s][i] = add2(c, d);
            } else {
                vr[s][i] = add2(a, b);
                vi[s][i] = fma2(d, dup(-1.0f), c);
            }
        }
    }
    // accumulate: upper spins += cs v; lower spins += cl B^+ v
    //   B^+ v by direction: MU 0: -v[s]; MU 1: i sigma_1 -> (-v[1-s].im, v[1-s].re);
    //   MU 2: s = 0: v[1], s = 1: -v[0]; MU 3: s = 0: (-v[0].im, v[0].re), s = 1: (v[1].im, -v[1].re)
#pragma unroll
    for (int s = 0; s < 2; s++)
#pragma unroll
        for (int c = 0; c < 3; c++) {
            f2 lr, li, fr, fi;  // lower contribution = (fr * lr, fi * li)
            if (MU == 0) { lr = vr[s][c]; li = vi[s][c]; fr = ncl2; fi = ncl2; }
            else if (MU == 1) { lr = vi[1 - s][c]; li = vr[1 - s][c]; fr = ncl2; fi = cl2; }
            else if (MU == 2) {
                if (s == 0) { lr = vr[1][c]; li = vi[1][c]; fr = cl2; fi = cl2; }
                else { lr = vr[0][c]; li = vi[0][c]; fr = ncl2; fi = ncl2; }
            } else {
                if (s == 0) { lr = vi[0][c]; li = vr[0][c]; fr = ncl2; fi = cl2; }
                else { lr = vi[1][c]; li = vr[1][c]; fr = cl2; fi = ncl2; }
            }
            if (FIRST) {
                acc[s][c][0] = mul2(cs2, vr[s][c]);
                acc[s][c][1] = mul2(cs2, vi[s][c]);
                acc[s + 2][c][0] = mul2(fr, lr);
                acc[s + 2][c][1] = mul2(fi, li);
            } else {
                acc[s][c][0] = fma2(cs2, vr[s][c], acc[s][c][0]);
                acc[s][c][1] = fma2(cs2, vi[s][c], acc[s][c][1]);
                acc[s + 2][c][0] = fma2(fr, lr, acc[s + 2][c][0]);
                acc[s + 2][c][1] = fma2(fi, li, acc[s + 2][c][1]);
            }
        }
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

// quantise 48 floats of one site (flavour pairs) into the 16-bit spinor at half-index h
__device__ __forceinline__ void store_site(int4 *__restrict__ q, float *__restrict__ nrm, int Vh, int h,
                                           const f2 v[4][3][2]) {
    float m = 0.0f;
#pragma unroll
    for (int s = 0; s < 4; s++)
#pragma unroll
        for (int c = 0; c < 3; c++)
#pragma unroll
            for (int ri = 0; ri < 2; ri++) m = fmaxf(m, fmaxf(fabsf(v[s][c][ri].x), fabsf(v[s][c][ri].y)));
    const float sc = m > 0.0f ? S16_QMAX / m : 0.0f;
    nrm[h] = m * INV_QMAX;
    const f2 sc2 = dup(sc), mg2 = dup(S16_ENC_MAGIC);
    int w[2][12];
#pragma unroll
    for (int k = 0; k < 12; k++) {
        const f2 re = fma2(v[k / 3][k % 3][0], sc2, mg2), im = fma2(v[k / 3][k % 3][1], sc2, mg2);
        w[0][k] = __byte_perm(__float_as_int(re.x), __float_as_int(im.x), 0x5410);
        w[1][k] = __byte_perm(__float_as_int(re.y), __float_as_int(im.y), 0x5410);
    }
#pragma unroll
    for (int f = 0; f < 2; f++)
#pragma unroll
        for (int j = 0; j < 3; j++)
            q[(f * 3 + j) * Vh + h] = make_int4(w[f][4 * j], w[f][4 * j + 1], w[f][4 * j + 2], w[f][4 * j + 3]);
}

// dequantise one site into flavour pairs
__device__ __forceinline__ void load_site(const int4 *__restrict__ q, const float *__restrict__ nrm, int Vh, int h,
                                          f2 v[4][3][2]) {
    const f2 sc2 = dup(__ldg(&nrm[h])), nb2 = dup(-S16_DEC_BIAS);
    int4 a[2][3];
#pragma unroll
    for (int f = 0; f < 2; f++)
#pragma unroll
        for (int j = 0; j < 3; j++) a[f][j] = __ldg(&q[(f * 3 + j) * Vh + h]);
#pragma unroll
    for (int k = 0; k < 12; k++) {
        const int w0 = word(a[0][k / 4], k % 4), w1 = word(a[1][k / 4], k % 4);
        v[k / 3][k % 3][0] = mul2(add2(make_float2(s16_flo(w0), s16_flo(w1)), nb2), sc2);
        v[k / 3][k % 3][1] = mul2(add2(make_float2(s16_fhi(w0), s16_fhi(w1)), nb2), sc2);
    }
}

template <bool DAG, bool PF>
__global__ void __launch_bounds__(S16_THREADS, S16_MINB) k_hop_even_s16(Geom g, SiteTermF st, const int2 *__restrict__ links,
                                                             S16In in, S16Out out, const int *__restrict__ done,
                                                             int chunk, S16Batch bt) {
    if (done && *done) return;
    const int h_end = min(g.Vh, (int)(blockIdx.x + 1) * chunk);
    for (int h = blockIdx.x * chunk + threadIdx.x; h < h_end; h += blockDim.x) {
        for (int k = 0; k < bt.nrhs; k++) {
            if (bt.rdone && bt.rdone[k * bt.rdone_stride]) continue;
            const S16In ik = s16_at(in, k * bt.stride);
            f2 acc[4][3][2];
            hop_all<0, DAG, PF>(g, links, ik.q, ik.nrm, h, acc);
            // kappa^2 A^-1 per spin sign g: [[a - i kp g, kpp], [kpp, a + i kp g]] / det
            const float a = st.kappa2 * st.inv_det;
            const float e = a * st.kpp;
            f2 o[4][3][2];
#pragma unroll
            for (int s = 0; s < 4; s++) {
                const float b = a * (DAG ? -st.kp : st.kp) * (s < 2 ? 1.0f : -1.0f);
#pragma unroll
                for (int c = 0; c < 3; c++) {
                    const f2 pr = acc[s][c][0], pi = acc[s][c][1];
                    o[s][c][0] = make_float2(fmaf(a, pr.x, fmaf(b, pi.x, e * pr.y)), fmaf(a, pr.y, fmaf(-b, pi.y, e * pr.x)));
                    o[s][c][1] = make_float2(fmaf(a, pi.x, fmaf(-b, pr.x, e * pi.y)), fmaf(a, pi.y, fmaf(b, pr.y, e * pi.x)));
                }
            }
            const S16Out ok = s16_at(out, k * bt.stride);
            store_site(ok.q, ok.nrm, g.Vh, h, o);
        }
    }
}

// Per-right-hand-side block partials: each thread keeps its running sums in its own
// slots of dynamic shared memory, part[(q * nrhs + k) * blockDim + tid], q = 0, 1.
template <bool DAG, int EPI, bool PF>
__global__ void __launch_bounds__(S16_THREADS, S16_MINB) k_hop_odd_s16(Geom g, SiteTermF st, const int2 *__restrict__ links,
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
    for (int h = blockIdx.x * chunk + threadIdx.x; h < h_end; h += blockDim.x)
      for (int k = 0; k < bt.nrhs; k++) {
        if (bt.rdone && bt.rdone[k * bt.rdone_stride]) continue;
        const S16In te = s16_at(te_all, k * bt.stride), psi = s16_at(psi_all, k * bt.stride);
        const S16Out out = s16_at(out_all, k * bt.stride);
        f2 acc[4][3][2];
        hop_all<1, false, PF>(g, links, te.q, te.nrm, h, acc);
        f2 p[4][3][2];
        load_site(psi.q, psi.nrm, Vh, h, p);
        const float kp = DAG ? -st.kp : st.kp;
        f2 y[4][3][2];
        float s1 = 0.0f, s2 = 0.0f;
        // y = A psi - H t (dag: A(-mu) psi - gamma_5 H t)
#pragma unroll
        for (int s = 0; s < 4; s++) {
            const float b = kp * (s < 2 ? 1.0f : -1.0f);
            const bool hopneg = DAG && s >= 2;
#pragma unroll
            for (int c = 0; c < 3; c++) {
                f2 hr = acc[s][c][0], hi = acc[s][c][1];
                if (hopneg) { hr = mul2(hr, dup(-1.0f)); hi = mul2(hi, dup(-1.0f)); }
                const f2 pr = p[s][c][0], pi = p[s][c][1];
                y[s][c][0] = make_float2(fmaf(-b, pi.x, fmaf(-st.kpp, pr.y, pr.x - hr.x)),
                                         fmaf(b, pi.y, fmaf(-st.kpp, pr.x, pr.y - hr.y)));
                y[s][c][1] = make_float2(fmaf(b, pr.x, fmaf(-st.kpp, pi.y, pi.x - hi.x)),
                                         fmaf(-b, pr.y, fmaf(-st.kpp, pi.x, pi.y - hi.y)));
                if (EPI == EPI_STORE_NORMS) {
                    const f2 yy = fma2(y[s][c][0], y[s][c][0], mul2(y[s][c][1], y[s][c][1]));
                    const f2 pp = fma2(pr, pr, mul2(pi, pi));
                    s1 += yy.x + yy.y;
                    s2 += pp.x + pp.y;
                }
            }
        }
        if (EPI == EPI_STORE || EPI == EPI_STORE_NORMS) {
            store_site(out.q, out.nrm, Vh, h, y);
            if (EPI == EPI_STORE_NORMS) {
                part[k * blockDim.x + threadIdx.x] += s1;
                part[(bt.nrhs + k) * blockDim.x + threadIdx.x] += s2;
            }
        } else if (EPI == EPI_SHIFT) {  // y + sigma aux, aux streamed plane by plane
            const S16In aux = s16_at(ea.aux, k * bt.stride);
            const float sa = (float)ea.sigma * __ldg(&aux.nrm[h]);
            const f2 sa2 = dup(sa), nb2 = dup(-S16_DEC_BIAS);
#pragma unroll
            for (int j = 0; j < 3; j++) {
                const int4 a0 = __ldg(&aux.q[(0 * 3 + j) * Vh + h]), a1 = __ldg(&aux.q[(1 * 3 + j) * Vh + h]);
#pragma unroll
                for (int m = 0; m < 4; m++) {
                    const int kk = 4 * j + m, w0 = word(a0, m), w1 = word(a1, m);
                    const f2 ar = add2(make_float2(s16_flo(w0), s16_flo(w1)), nb2);
                    const f2 ai = add2(make_float2(s16_fhi(w0), s16_fhi(w1)), nb2);
                    y[kk / 3][kk % 3][0] = fma2(sa2, ar, y[kk / 3][kk % 3][0]);
                    y[kk / 3][kk % 3][1] = fma2(sa2, ai, y[kk / 3][kk % 3][1]);
                }
            }
            store_site(out.q, out.nrm, Vh, h, y);
        } else {  // EPI_MMS_R: w = y + sigma aux; r' = r - alpha w (FP32 planes); aux streamed
            const S16In aux = s16_at(ea.aux, k * bt.stride);
            const float sa = (float)(ea.per_rhs_sigma ? ea.sigma_k[k] : ea.sigma) * __ldg(&aux.nrm[h]);
            const float alpha = alpha_s[k];
            const float2 *rin = ea.r_in + k * ea.r_stride;
            float2 *rout = ea.r + k * ea.r_stride;
#pragma unroll
            for (int f = 0; f < 2; f++)
#pragma unroll
                for (int j = 0; j < 3; j++) {
                    const int4 aw = __ldg(&aux.q[(f * 3 + j) * Vh + h]);
#pragma unroll
                    for (int m = 0; m < 4; m++) {
                        const int kk = 4 * j + m, s = kk / 3, c = kk % 3;
                        const int i = (f * 12 + kk) * Vh + h;
                        const float2 rv = rin[i];
                        const float yr = f ? y[s][c][0].y : y[s][c][0].x, yi = f ? y[s][c][1].y : y[s][c][1].x;
                        const float wx = fmaf(sa, s16_lo(word(aw, m)), yr);
                        const float wy = fmaf(sa, s16_hi(word(aw, m)), yi);
                        const float2 rn = make_float2(fmaf(-alpha, wx, rv.x), fmaf(-alpha, wy, rv.y));
                        rout[i] = rn;
                        s1 = fmaf(rn.x, rn.x, fmaf(rn.y, rn.y, s1));
                    }
                }
            part[k * blockDim.x + threadIdx.x] += s1;
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

constexpr bool PFD = true;  // prefetch the next direction (0.106 vs 0.113 ms for Mhat at 24^3x48)

int s16_blocks_cached[64] = {0};

}  // namespace

// blocks of the stencil launches: one per resident slot (3 per SM at 168 registers), at most one site per thread
int hop_blocks_s16(const Geom &g) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) dev = 0;
    if (!s16_blocks_cached[dev]) {
        int sms = 0, a = 0, b = 0;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_hop_odd_s16<true, EPI_MMS_R, PFD>, S16_THREADS, 0);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_hop_even_s16<true, PFD>, S16_THREADS, 0);
        a = a < b ? a : b;
        if (sms <= 0) sms = 152;
        if (a <= 0) a = 1;
        s16_blocks_cached[dev] = sms * a;
    }
    int want = (g.Vh + S16_THREADS - 1) / S16_THREADS;
    return want < s16_blocks_cached[dev] ? want : s16_blocks_cached[dev];
}

void launch_hop_even_s16(const Geom &g, const SiteTermF &st, const int2 *links, S16In in, S16Out out, bool dag,
                         const int *done, cudaStream_t s, const S16Batch &bt) {
    const int nb = hop_blocks_s16(g);
    const int chunk = (g.Vh + nb - 1) / nb;
    if (dag)
        k_hop_even_s16<true, PFD><<<nb, S16_THREADS, 0, s>>>(g, st, links, in, out, done, chunk, bt);
    else
        k_hop_even_s16<false, PFD><<<nb, S16_THREADS, 0, s>>>(g, st, links, in, out, done, chunk, bt);
}

void launch_hop_odd_s16(const Geom &g, const SiteTermF &st, const int2 *links, S16In psi, S16In te, S16Out out,
                        bool dag, HopEpi epi, const S16EpiArgs &ea, cudaStream_t s, const S16Batch &bt) {
    const int nb = hop_blocks_s16(g);
    const int chunk = (g.Vh + nb - 1) / nb;
    const size_t smem = sizeof(double) * 2 * bt.nrhs * S16_THREADS;
#define TMND_ODD16(D, E) \
    k_hop_odd_s16<D, E, PFD><<<nb, S16_THREADS, smem, s>>>(g, st, links, psi, te, out, ea, chunk, bt)
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
