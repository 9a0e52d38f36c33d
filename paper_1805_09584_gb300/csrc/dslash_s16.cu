// Sloppy stencil: FP32 arithmetic on 16-bit storage (the inner operator of
// the mixed-precision solver).  Same operator as the FP64 kernels
// (Sec. 2: even-odd Schur complement of the ND twisted-mass operator):
//   even:  t_e = kappa^2 A^-1 H_eo psi_o        (dag: kappa^2 A(-mu)^-1 H_eo gamma_5 psi_o)
//   odd :  y_o = A psi_o - H_oe t_e             (dag: A(-mu) psi_o - gamma_5 H_oe t_e)
//
// Storage
//   spinor (per right-hand side): 6 planes of int4 over V/2 sites, plane j
//     holding complex components 4j..4j+3 (component c = flavour*12 + spin*3 +
//     colour; one 32-bit word per component: real part in the low 16 bits,
//     imaginary part in the high 16 bits), then one float per site, the
//     dequantisation scale nrm = max|v| / 32767 of that site.  100 B per site.
//   links: 12-real compression, rows 0 and 1 of U as int16 (scale 32767;
//     |u_ij| <= 1), 3 planes of int2 per direction and parity; row 2 is
//     rebuilt as conj(row0 x row1) (det U = +1, Sec. 2: U in SU(3)).  The
//     antiperiodic sign is applied in the kernel, never folded into links.
//
// Arithmetic: the spin projection is done on the integers (exact), the sum is
// converted to float with an exponent-bias trick on the integer pipe (I2F runs
// at quarter rate on this GPU), and the link is applied to the integer-valued
// floats; the neighbour's scale nrm/32767 and the boundary sign enter as one
// factor of the accumulation FMA.
#include "tmnd_internal.cuh"

namespace {

constexpr int S16_THREADS = 128;
constexpr float QMAX = 32767.0f;
constexpr float INV_QMAX = 1.0f / 32767.0f;

// exact float of an integer |n| < 2^22: bits of 1.5*2^23 + n, minus 1.5*2^23
__device__ __forceinline__ float i2f_exact(int n) { return __int_as_float(n + 0x4B400000) - 12582912.0f; }
__device__ __forceinline__ int lo16(int w) { return (w << 16) >> 16; }
__device__ __forceinline__ int hi16(int w) { return w >> 16; }

struct cf2 {
    float x, y;
};

// 12 words of one flavour of one site
__device__ __forceinline__ void load_flavour(const int4 *__restrict__ q, int Vh, int f, int h, int w[12]) {
    const int4 a = __ldg(&q[(f * 3 + 0) * Vh + h]);
    const int4 b = __ldg(&q[(f * 3 + 1) * Vh + h]);
    const int4 c = __ldg(&q[(f * 3 + 2) * Vh + h]);
    w[0] = a.x; w[1] = a.y; w[2] = a.z; w[3] = a.w;
    w[4] = b.x; w[5] = b.y; w[6] = b.z; w[7] = b.w;
    w[8] = c.x; w[9] = c.y; w[10] = c.z; w[11] = c.w;
}

// link rows 0, 1 (integer-valued floats, scale 32767) and rebuilt row 2 (same scale)
__device__ __forceinline__ void load_link(const int2 *__restrict__ L, int Vh, int hl, cf2 u[3][3]) {
    const int2 a = __ldg(&L[0 * Vh + hl]);
    const int2 b = __ldg(&L[1 * Vh + hl]);
    const int2 c = __ldg(&L[2 * Vh + hl]);
    const int wv[6] = {a.x, a.y, b.x, b.y, c.x, c.y};
#pragma unroll
    for (int k = 0; k < 6; k++) {
        u[k / 3][k % 3].x = i2f_exact(lo16(wv[k]));
        u[k / 3][k % 3].y = i2f_exact(hi16(wv[k]));
    }
    // row 2 = conj(row0 x row1) / 32767
#pragma unroll
    for (int k = 0; k < 3; k++) {
        const int k1 = (k + 1) % 3, k2 = (k + 2) % 3;
        const cf2 a1 = u[0][k1], a2 = u[0][k2], b1 = u[1][k1], b2 = u[1][k2];
        float re = fmaf(a1.x, b2.x, -a1.y * b2.y);
        float im = fmaf(a1.x, b2.y, a1.y * b2.x);
        re = fmaf(-a2.x, b1.x, fmaf(a2.y, b1.y, re));
        im = fmaf(-a2.x, b1.y, fmaf(-a2.y, b1.x, im));
        u[2][k].x = re * INV_QMAX;
        u[2][k].y = -im * INV_QMAX;
    }
}

// integer projection chi = up -+ B lo for one flavour, as exact floats.
// Word index of component (spin s, colour c) = s*3 + c; lower spins are 2, 3.
template <int MU, bool PLUS>
__device__ __forceinline__ void project(const int w[12], cf2 chi[2][3]) {
#pragma unroll
    for (int s = 0; s < 2; s++)
#pragma unroll
        for (int c = 0; c < 3; c++) {
            const int wu = w[s * 3 + c];
            const int ur = lo16(wu), ui = hi16(wu);
            // B lo: (MU 0) -lo_s ; (1) -i lo_{1-s} ; (2) s==0 ? -lo_1 : lo_0 ; (3) s==0 ? -i lo_0 : i lo_1
            int br, bi;
            if (MU == 0) {
                const int wl = w[(2 + s) * 3 + c];
                br = -lo16(wl); bi = -hi16(wl);
            } else if (MU == 1) {
                const int wl = w[(2 + 1 - s) * 3 + c];
                br = hi16(wl); bi = -lo16(wl);           // -i (a + ib) = b - ia
            } else if (MU == 2) {
                const int wl = w[(2 + 1 - s) * 3 + c];
                if (s == 0) { br = -lo16(wl); bi = -hi16(wl); }
                else { br = lo16(wl); bi = hi16(wl); }
            } else {
                const int wl = w[(2 + s) * 3 + c];
                if (s == 0) { br = hi16(wl); bi = -lo16(wl); }   // -i lo_0
                else { br = -hi16(wl); bi = lo16(wl); }          // +i lo_1
            }
            chi[s][c].x = i2f_exact(PLUS ? ur + br : ur - br);
            chi[s][c].y = i2f_exact(PLUS ? ui + bi : ui - bi);
        }
}

// B^+ v for the reconstruction of the lower spins
template <int MU>
__device__ __forceinline__ cf2 Bdag(const cf2 v[2][3], int s, int c) {
    if (MU == 0) return cf2{-v[s][c].x, -v[s][c].y};
    if (MU == 1) return cf2{-v[1 - s][c].y, v[1 - s][c].x};                      // i sigma_1
    if (MU == 2) return s == 0 ? v[1][c] : cf2{-v[0][c].x, -v[0][c].y};          // i sigma_2
    return s == 0 ? cf2{-v[0][c].y, v[0][c].x} : cf2{v[1][c].y, -v[1][c].x};     // i sigma_3
}

template <int MU, int DIR, bool G5IN, bool FIRST>
__device__ __forceinline__ void hop_dir(const int4 *__restrict__ q, const float *__restrict__ nrm, int Vh, int hn,
                                        const int2 *__restrict__ L, int hl, float sign, float acc[2][4][3][2]) {
    cf2 u[3][3];
    load_link(L, Vh, hl, u);
    const float cscale = sign * __ldg(&nrm[hn]) * INV_QMAX;
    constexpr bool plus = (DIR < 0) != G5IN;
#pragma unroll
    for (int f = 0; f < 2; f++) {
        int w[12];
        load_flavour(q, Vh, f, hn, w);
        cf2 chi[2][3];
        project<MU, plus>(w, chi);
        cf2 v[2][3];
#pragma unroll
        for (int s = 0; s < 2; s++)
#pragma unroll
            for (int i = 0; i < 3; i++) {
                float re, im;
                if (DIR > 0) {  // U chi
                    re = u[i][0].x * chi[s][0].x;
                    im = u[i][0].x * chi[s][0].y;
                    re = fmaf(-u[i][0].y, chi[s][0].y, re);
                    im = fmaf(u[i][0].y, chi[s][0].x, im);
#pragma unroll
                    for (int j = 1; j < 3; j++) {
                        re = fmaf(u[i][j].x, chi[s][j].x, fmaf(-u[i][j].y, chi[s][j].y, re));
                        im = fmaf(u[i][j].x, chi[s][j].y, fmaf(u[i][j].y, chi[s][j].x, im));
                    }
                } else {  // U^+ chi
                    re = u[0][i].x * chi[s][0].x;
                    im = u[0][i].x * chi[s][0].y;
                    re = fmaf(u[0][i].y, chi[s][0].y, re);
                    im = fmaf(-u[0][i].y, chi[s][0].x, im);
#pragma unroll
                    for (int j = 1; j < 3; j++) {
                        re = fmaf(u[j][i].x, chi[s][j].x, fmaf(u[j][i].y, chi[s][j].y, re));
                        im = fmaf(u[j][i].x, chi[s][j].y, fmaf(-u[j][i].y, chi[s][j].x, im));
                    }
                }
                v[s][i] = cf2{re, im};
            }
        const float cl = (DIR > 0) ? -cscale : cscale;
#pragma unroll
        for (int s = 0; s < 2; s++)
#pragma unroll
            for (int c = 0; c < 3; c++) {
                const cf2 b = Bdag<MU>(v, s, c);
                if (FIRST) {
                    acc[f][s][c][0] = cscale * v[s][c].x;
                    acc[f][s][c][1] = cscale * v[s][c].y;
                    acc[f][s + 2][c][0] = cl * b.x;
                    acc[f][s + 2][c][1] = cl * b.y;
                } else {
                    acc[f][s][c][0] = fmaf(cscale, v[s][c].x, acc[f][s][c][0]);
                    acc[f][s][c][1] = fmaf(cscale, v[s][c].y, acc[f][s][c][1]);
                    acc[f][s + 2][c][0] = fmaf(cl, b.x, acc[f][s + 2][c][0]);
                    acc[f][s + 2][c][1] = fmaf(cl, b.y, acc[f][s + 2][c][1]);
                }
            }
    }
}

template <int P, bool G5IN>
__device__ __forceinline__ void hop_all(const Geom &g, const int2 *__restrict__ links, const int4 *__restrict__ q,
                                        const float *__restrict__ nrm, int h, float acc[2][4][3][2]) {
    const int Vh = g.Vh;
    int zh = h % g.Zh;
    int r = h / g.Zh;
    int y = r % g.Y;
    r /= g.Y;
    int x = r % g.X;
    int t = r / g.X;
    int z = 2 * zh + ((P + t + x + y) & 1);
    const int2 *Lp = links + (size_t)P * 4 * 3 * Vh;
    const int2 *Lq = links + (size_t)(1 - P) * 4 * 3 * Vh;
    auto idx = [&](int tt, int xx, int yy, int zz) { return ((tt * g.X + xx) * g.Y + yy) * g.Zh + (zz >> 1); };
    {
        int tf = (t + 1 == g.T) ? 0 : t + 1;
        int tb = (t == 0) ? g.T - 1 : t - 1;
        float sf = (g.apbc && t + 1 == g.T) ? -1.0f : 1.0f;
        float sb = (g.apbc && t == 0) ? -1.0f : 1.0f;
        int hf = idx(tf, x, y, z), hb = idx(tb, x, y, z);
        hop_dir<0, +1, G5IN, true>(q, nrm, Vh, hf, Lp + 0 * 3 * (size_t)Vh, h, sf, acc);
        hop_dir<0, -1, G5IN, false>(q, nrm, Vh, hb, Lq + 0 * 3 * (size_t)Vh, hb, sb, acc);
    }
    {
        int xf = (x + 1 == g.X) ? 0 : x + 1;
        int xb = (x == 0) ? g.X - 1 : x - 1;
        int hf = idx(t, xf, y, z), hb = idx(t, xb, y, z);
        hop_dir<1, +1, G5IN, false>(q, nrm, Vh, hf, Lp + 1 * 3 * (size_t)Vh, h, 1.0f, acc);
        hop_dir<1, -1, G5IN, false>(q, nrm, Vh, hb, Lq + 1 * 3 * (size_t)Vh, hb, 1.0f, acc);
    }
    {
        int yf = (y + 1 == g.Y) ? 0 : y + 1;
        int yb = (y == 0) ? g.Y - 1 : y - 1;
        int hf = idx(t, x, yf, z), hb = idx(t, x, yb, z);
        hop_dir<2, +1, G5IN, false>(q, nrm, Vh, hf, Lp + 2 * 3 * (size_t)Vh, h, 1.0f, acc);
        hop_dir<2, -1, G5IN, false>(q, nrm, Vh, hb, Lq + 2 * 3 * (size_t)Vh, hb, 1.0f, acc);
    }
    {
        int zf = (z + 1 == g.Z) ? 0 : z + 1;
        int zb = (z == 0) ? g.Z - 1 : z - 1;
        int hf = idx(t, x, y, zf), hb = idx(t, x, y, zb);
        hop_dir<3, +1, G5IN, false>(q, nrm, Vh, hf, Lp + 3 * 3 * (size_t)Vh, h, 1.0f, acc);
        hop_dir<3, -1, G5IN, false>(q, nrm, Vh, hb, Lq + 3 * 3 * (size_t)Vh, hb, 1.0f, acc);
    }
}

// quantise 48 floats of one site into the 16-bit spinor at half-index h
__device__ __forceinline__ void store_site(int4 *__restrict__ q, float *__restrict__ nrm, int Vh, int h,
                                           const float v[2][4][3][2]) {
    float m = 0.0f;
#pragma unroll
    for (int f = 0; f < 2; f++)
#pragma unroll
        for (int s = 0; s < 4; s++)
#pragma unroll
            for (int c = 0; c < 3; c++) m = fmaxf(m, fmaxf(fabsf(v[f][s][c][0]), fabsf(v[f][s][c][1])));
    const float sc = m > 0.0f ? QMAX / m : 0.0f;
    nrm[h] = m * INV_QMAX;
#pragma unroll
    for (int f = 0; f < 2; f++) {
        int w[12];
#pragma unroll
        for (int k = 0; k < 12; k++) {
            // round-to-nearest integer in the low bits of 1.5*2^23 + x
            const int re = __float_as_int(fmaf(v[f][k / 3][k % 3][0], sc, 12582912.0f));
            const int im = __float_as_int(fmaf(v[f][k / 3][k % 3][1], sc, 12582912.0f));
            w[k] = __byte_perm(re, im, 0x5410);
        }
        q[(f * 3 + 0) * Vh + h] = make_int4(w[0], w[1], w[2], w[3]);
        q[(f * 3 + 1) * Vh + h] = make_int4(w[4], w[5], w[6], w[7]);
        q[(f * 3 + 2) * Vh + h] = make_int4(w[8], w[9], w[10], w[11]);
    }
}

// dequantise one site
__device__ __forceinline__ void load_site(const int4 *__restrict__ q, const float *__restrict__ nrm, int Vh, int h,
                                          float v[2][4][3][2]) {
    const float sc = __ldg(&nrm[h]);
#pragma unroll
    for (int f = 0; f < 2; f++) {
        int w[12];
        load_flavour(q, Vh, f, h, w);
#pragma unroll
        for (int k = 0; k < 12; k++) {
            v[f][k / 3][k % 3][0] = i2f_exact(lo16(w[k])) * sc;
            v[f][k / 3][k % 3][1] = i2f_exact(hi16(w[k])) * sc;
        }
    }
}

template <bool DAG>
__global__ void __launch_bounds__(S16_THREADS) k_hop_even_s16(Geom g, SiteTermF st, const int2 *__restrict__ links,
                                                             S16In in, S16Out out, const int *__restrict__ done,
                                                             int chunk) {
    if (done && *done) return;
    const int h_end = min(g.Vh, (int)(blockIdx.x + 1) * chunk);
    for (int h = blockIdx.x * chunk + threadIdx.x; h < h_end; h += blockDim.x) {
        float acc[2][4][3][2];
        hop_all<0, DAG>(g, links, in.q, in.nrm, h, acc);
        const float a = st.kappa2 * st.inv_det;
        const float e = a * st.kpp;
        float o[2][4][3][2];
#pragma unroll
        for (int s = 0; s < 4; s++) {
            const float b = a * (DAG ? -st.kp : st.kp) * (s < 2 ? 1.0f : -1.0f);
#pragma unroll
            for (int c = 0; c < 3; c++) {
                const float p0x = acc[0][s][c][0], p0y = acc[0][s][c][1];
                const float p1x = acc[1][s][c][0], p1y = acc[1][s][c][1];
                o[0][s][c][0] = fmaf(a, p0x, fmaf(b, p0y, e * p1x));
                o[0][s][c][1] = fmaf(a, p0y, fmaf(-b, p0x, e * p1y));
                o[1][s][c][0] = fmaf(a, p1x, fmaf(-b, p1y, e * p0x));
                o[1][s][c][1] = fmaf(a, p1y, fmaf(b, p1x, e * p0y));
            }
        }
        store_site(out.q, out.nrm, g.Vh, h, o);
    }
}

template <bool DAG, int EPI>
__global__ void __launch_bounds__(S16_THREADS) k_hop_odd_s16(Geom g, SiteTermF st, const int2 *__restrict__ links,
                                                            S16In psi, S16In te, S16Out out, S16EpiArgs ea,
                                                            int chunk) {
    __shared__ double red[40];
    if (ea.done && *ea.done) return;
    const int Vh = g.Vh;
    float alpha = 0.0f;
    if (EPI == EPI_MMS_R) {
        const double yy = block_reduce_partials(ea.part_in, ea.npart_in, red);
        const double pp = block_reduce_partials(ea.part_in + ea.npart_in, ea.npart_in, red);
        alpha = (float)(*ea.rr / (yy + ea.sigma * pp));
    }
    double n1 = 0.0, n2 = 0.0;
    const int h_end = min(Vh, (int)(blockIdx.x + 1) * chunk);
    for (int h = blockIdx.x * chunk + threadIdx.x; h < h_end; h += blockDim.x) {
        float acc[2][4][3][2];
        hop_all<1, false>(g, links, te.q, te.nrm, h, acc);
        float p[2][4][3][2];
        load_site(psi.q, psi.nrm, Vh, h, p);
        const float kp = DAG ? -st.kp : st.kp;
        float y[2][4][3][2];
        float s1 = 0.0f, s2 = 0.0f;
#pragma unroll
        for (int s = 0; s < 4; s++) {
            const float b = kp * (s < 2 ? 1.0f : -1.0f);
            const bool hopneg = DAG && s >= 2;
#pragma unroll
            for (int c = 0; c < 3; c++) {
                float h0x = acc[0][s][c][0], h0y = acc[0][s][c][1];
                float h1x = acc[1][s][c][0], h1y = acc[1][s][c][1];
                if (hopneg) { h0x = -h0x; h0y = -h0y; h1x = -h1x; h1y = -h1y; }
                const float p0x = p[0][s][c][0], p0y = p[0][s][c][1];
                const float p1x = p[1][s][c][0], p1y = p[1][s][c][1];
                y[0][s][c][0] = fmaf(-b, p0y, fmaf(-st.kpp, p1x, p0x - h0x));
                y[0][s][c][1] = fmaf(b, p0x, fmaf(-st.kpp, p1y, p0y - h0y));
                y[1][s][c][0] = fmaf(b, p1y, fmaf(-st.kpp, p0x, p1x - h1x));
                y[1][s][c][1] = fmaf(-b, p1x, fmaf(-st.kpp, p0y, p1y - h1y));
                if (EPI == EPI_STORE_NORMS) {
#pragma unroll
                    for (int f = 0; f < 2; f++) {
                        s1 = fmaf(y[f][s][c][0], y[f][s][c][0], fmaf(y[f][s][c][1], y[f][s][c][1], s1));
                        s2 = fmaf(p[f][s][c][0], p[f][s][c][0], fmaf(p[f][s][c][1], p[f][s][c][1], s2));
                    }
                }
            }
        }
        if (EPI == EPI_STORE || EPI == EPI_STORE_NORMS) {
            store_site(out.q, out.nrm, Vh, h, y);
            n1 += s1;
            n2 += s2;
        } else if (EPI == EPI_SHIFT) {
            float a[2][4][3][2];
            load_site(ea.aux.q, ea.aux.nrm, Vh, h, a);
#pragma unroll
            for (int f = 0; f < 2; f++)
#pragma unroll
                for (int s = 0; s < 4; s++)
#pragma unroll
                    for (int c = 0; c < 3; c++) {
                        y[f][s][c][0] = fmaf((float)ea.sigma, a[f][s][c][0], y[f][s][c][0]);
                        y[f][s][c][1] = fmaf((float)ea.sigma, a[f][s][c][1], y[f][s][c][1]);
                    }
            store_site(out.q, out.nrm, Vh, h, y);
        } else {  // EPI_MMS_R: w = y + sigma aux; r' = r - alpha w (FP32 planes)
            float a[2][4][3][2];
            load_site(ea.aux.q, ea.aux.nrm, Vh, h, a);
            const float sg = (float)ea.sigma;
#pragma unroll
            for (int f = 0; f < 2; f++)
#pragma unroll
                for (int s = 0; s < 4; s++)
#pragma unroll
                    for (int c = 0; c < 3; c++) {
                        const int i = (f * 12 + s * 3 + c) * Vh + h;
                        const float2 rv = ea.r_in[i];
                        const float wx = fmaf(sg, a[f][s][c][0], y[f][s][c][0]);
                        const float wy = fmaf(sg, a[f][s][c][1], y[f][s][c][1]);
                        const float2 rn = make_float2(fmaf(-alpha, wx, rv.x), fmaf(-alpha, wy, rv.y));
                        ea.r[i] = rn;
                        s1 = fmaf(rn.x, rn.x, fmaf(rn.y, rn.y, s1));
                    }
            n1 += s1;
        }
    }
    if (EPI == EPI_STORE_NORMS) {
        double t1 = block_sum(n1, red);
        double t2 = block_sum(n2, red);
        if (threadIdx.x == 0) {
            ea.part_out[blockIdx.x] = t1;
            ea.part_out[gridDim.x + blockIdx.x] = t2;
        }
    } else if (EPI == EPI_MMS_R) {
        double t1 = block_sum(n1, red);
        if (threadIdx.x == 0) ea.part_out[blockIdx.x] = t1;
    }
}

int s16_blocks_cached[64] = {0};

}  // namespace

int hop_blocks_s16(const Geom &g) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) dev = 0;
    if (!s16_blocks_cached[dev]) {
        int sms = 0, a = 0, b = 0;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_hop_odd_s16<true, EPI_MMS_R>, S16_THREADS, 0);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_hop_even_s16<true>, S16_THREADS, 0);
        a = a < b ? a : b;
        if (sms <= 0) sms = 152;
        if (a <= 0) a = 1;
        s16_blocks_cached[dev] = sms * a;
    }
    int want = (g.Vh + S16_THREADS - 1) / S16_THREADS;
    return want < s16_blocks_cached[dev] ? want : s16_blocks_cached[dev];
}

void launch_hop_even_s16(const Geom &g, const SiteTermF &st, const int2 *links, S16In in, S16Out out, bool dag,
                         const int *done, cudaStream_t s) {
    const int nb = hop_blocks_s16(g);
    const int chunk = (g.Vh + nb - 1) / nb;
    if (dag)
        k_hop_even_s16<true><<<nb, S16_THREADS, 0, s>>>(g, st, links, in, out, done, chunk);
    else
        k_hop_even_s16<false><<<nb, S16_THREADS, 0, s>>>(g, st, links, in, out, done, chunk);
}

void launch_hop_odd_s16(const Geom &g, const SiteTermF &st, const int2 *links, S16In psi, S16In te, S16Out out,
                        bool dag, HopEpi epi, const S16EpiArgs &ea, cudaStream_t s) {
    const int nb = hop_blocks_s16(g);
    const int chunk = (g.Vh + nb - 1) / nb;
#define TMND_ODD16(D, E) k_hop_odd_s16<D, E><<<nb, S16_THREADS, 0, s>>>(g, st, links, psi, te, out, ea, chunk)
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
