// Arithmetic of the sloppy stencil (FP32 on 16-bit storage, kernels in
// dslash_s16.cu): per-direction link products and accumulation, the site terms
// of the even and odd kernels and their fused epilogues.
//
// One thread per site, both flavours: the two flavours share every link, so each
// flavour pair of a spinor component lives in one float2 and all link products,
// projections and accumulations are packed f32x2 instructions.  Decoding is one
// byte permute per value (the float 2^23 + 32768 + n); the spin projection
// u -+ B l is formed from two decoded floats exactly (their difference, or
// u + (l - 2 * bias)), so the projected half spinor is exact before the link is
// applied.  The neighbour's scale nrm/32767 and the boundary sign enter as one
// factor of the accumulation.
#pragma once

#include "tmnd_internal.cuh"

namespace {

constexpr float INV_QMAX = 1.0f / S16_QMAX;

using f2 = float2;  // (flavour 0, flavour 1)

__device__ __forceinline__ f2 dup(float a) { return make_float2(a, a); }
// -a by flipping the sign bit on the integer pipe (keeps the FP32 pipe for products)
__device__ __forceinline__ float fneg(float a) { return __int_as_float(__float_as_int(a) ^ (int)0x80000000); }
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
    // (ni = -ui: each output component below is one fused chain of six products)
    float ur[3][3], ui[3][3], ni[3][3];
    {
        const int wv[6] = {r.l[0].x, r.l[0].y, r.l[1].x, r.l[1].y, r.l[2].x, r.l[2].y};
#pragma unroll
        for (int k = 0; k < 6; k++) {
            ur[k / 3][k % 3] = s16_lo(wv[k]);
            ui[k / 3][k % 3] = s16_hi(wv[k]);
            ni[k / 3][k % 3] = fneg(ui[k / 3][k % 3]);
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
            ni[2][k] = fneg(ui[2][k]);
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
        // re = sum_j wr_j chr_j + wa_j chi_j,  im = sum_j wr_j chi_j + wb_j chr_j
        f2 wr[3], wa[3], wb[3];
#pragma unroll
        for (int j = 0; j < 3; j++) {
            wr[j] = dup(DIR > 0 ? ur[i][j] : ur[j][i]);
            wa[j] = dup(DIR > 0 ? ni[i][j] : ui[j][i]);
            wb[j] = dup(DIR > 0 ? ui[i][j] : ni[j][i]);
        }
#pragma unroll
        for (int s = 0; s < 2; s++) {
            f2 a = mul2(wr[0], chr[s][0]);
            a = fma2(wr[1], chr[s][1], a);
            a = fma2(wr[2], chr[s][2], a);
            a = fma2(wa[0], chi[s][0], a);
            a = fma2(wa[1], chi[s][1], a);
            vr[s][i] = fma2(wa[2], chi[s][2], a);
            f2 b = mul2(wr[0], chi[s][0]);
            b = fma2(wr[1], chi[s][1], b);
            b = fma2(wr[2], chi[s][2], b);
            b = fma2(wb[0], chr[s][0], b);
            b = fma2(wb[1], chr[s][1], b);
            vi[s][i] = fma2(wb[2], chr[s][2], b);
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
    nrm[s16_ni(h)] = m * INV_QMAX;
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
            q[s16_qi(f * 3 + j, h)] = make_int4(w[f][4 * j], w[f][4 * j + 1], w[f][4 * j + 2], w[f][4 * j + 3]);
}

// One site of a 16-bit spinor, read through global memory (read-only path) or
// shared memory: word of plane p (0..5) and the dequantisation scale.
// (i counts sites from the first site of the block-structured region at q / nrm)
struct GSite {
    const int4 *q;
    const float *nrm;
    int i;
    __device__ __forceinline__ int4 w(int p) const { return __ldg(&q[s16_qi(p, i)]); }
    __device__ __forceinline__ float s() const { return __ldg(&nrm[s16_ni(i)]); }
};
struct SSite {
    const int4 *q;
    const float *nrm;
    int i;
    __device__ __forceinline__ int4 w(int p) const { return q[s16_qi(p, i)]; }
    __device__ __forceinline__ float s() const { return nrm[s16_ni(i)]; }
};

// dequantise one site into flavour pairs
template <class Site>
__device__ __forceinline__ void load_site(const Site &a, f2 v[4][3][2]) {
    const f2 sc2 = dup(a.s()), nb2 = dup(-S16_DEC_BIAS);
    int4 w[2][3];
#pragma unroll
    for (int f = 0; f < 2; f++)
#pragma unroll
        for (int j = 0; j < 3; j++) w[f][j] = a.w(f * 3 + j);
#pragma unroll
    for (int k = 0; k < 12; k++) {
        const int w0 = word(w[0][k / 4], k % 4), w1 = word(w[1][k / 4], k % 4);
        v[k / 3][k % 3][0] = mul2(add2(make_float2(s16_flo(w0), s16_flo(w1)), nb2), sc2);
        v[k / 3][k % 3][1] = mul2(add2(make_float2(s16_fhi(w0), s16_fhi(w1)), nb2), sc2);
    }
}

// even sites: o = kappa^2 A^-1 acc, per spin sign g A^-1 = [[a - i kp g, kpp], [kpp, a + i kp g]] / det
template <bool DAG>
__device__ __forceinline__ void even_term(const SiteTermF &st, const f2 acc[4][3][2], f2 o[4][3][2]) {
    const float a = st.kappa2 * st.inv_det;
    const float e = a * st.kpp;
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
}

// odd sites: y = A psi - H t (dag: A(-mu) psi - gamma_5 H t); with NORMS the sums |y|^2, |psi|^2
template <bool DAG, bool NORMS>
__device__ __forceinline__ void odd_term(const SiteTermF &st, const f2 acc[4][3][2], const f2 p[4][3][2],
                                         f2 y[4][3][2], float &s1, float &s2) {
    const float kp = DAG ? -st.kp : st.kp;
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
            if (NORMS) {
                const f2 yy = fma2(y[s][c][0], y[s][c][0], mul2(y[s][c][1], y[s][c][1]));
                const f2 pp = fma2(pr, pr, mul2(pi, pi));
                s1 += yy.x + yy.y;
                s2 += pp.x + pp.y;
            }
        }
    }
}

// y += sigma aux (aux decoded plane by plane)
template <class Site>
__device__ __forceinline__ void add_shift(const Site &aux, float sigma, f2 y[4][3][2]) {
    const f2 sa2 = dup(sigma * aux.s()), nb2 = dup(-S16_DEC_BIAS);
#pragma unroll
    for (int j = 0; j < 3; j++) {
        const int4 a0 = aux.w(j), a1 = aux.w(3 + j);
#pragma unroll
        for (int m = 0; m < 4; m++) {
            const int kk = 4 * j + m, w0 = word(a0, m), w1 = word(a1, m);
            const f2 ar = add2(make_float2(s16_flo(w0), s16_flo(w1)), nb2);
            const f2 ai = add2(make_float2(s16_fhi(w0), s16_fhi(w1)), nb2);
            y[kk / 3][kk % 3][0] = fma2(sa2, ar, y[kk / 3][kk % 3][0]);
            y[kk / 3][kk % 3][1] = fma2(sa2, ai, y[kk / 3][kk % 3][1]);
        }
    }
}

// The odd site term fused with the multi-shift residual update, one 16-byte plane of the
// site at a time (4 components, both flavours): p decoded from psi, y = A p - H t (odd_term's
// arithmetic per component), w = y + sigma aux, r' = r - alpha w; returns the site's |r'|^2.
// Plane by plane, so that p, y and w of the whole site are never live at once.
template <bool DAG, class Site>
__device__ __forceinline__ float odd_mms_r_fused(const SiteTermF &st, const f2 acc[4][3][2], const Site &psi,
                                                 const Site &aux, float sigma, float alpha,
                                                 const float2 *__restrict__ rin, float2 *__restrict__ rout, int Vh,
                                                 int h) {
    const float kp = DAG ? -st.kp : st.kp;
    const f2 sc2 = dup(psi.s()), nb2 = dup(-S16_DEC_BIAS);
    const float sa = sigma * aux.s();
    float s1 = 0.0f;
    // loads one plane ahead: plane j + 1's words and residuals are in flight while plane j is
    // computed and stored (no round trip per component, at most two planes' loads live)
    int4 pw[3][2], aw[3][2];
    float2 rv[3][4][2];
    auto load_plane = [&](int j) {
        pw[j][0] = psi.w(j);
        pw[j][1] = psi.w(3 + j);
        aw[j][0] = aux.w(j);
        aw[j][1] = aux.w(3 + j);
#pragma unroll
        for (int m = 0; m < 4; m++)
#pragma unroll
            for (int f = 0; f < 2; f++) rv[j][m][f] = __ldcs(rin + (size_t)(f * 12 + 4 * j + m) * Vh + h);
    };
    load_plane(0);
#pragma unroll
    for (int j = 0; j < 3; j++) {
        if (j + 1 < 3) load_plane(j + 1);
#pragma unroll
        for (int m = 0; m < 4; m++) {
            const int kk = 4 * j + m, sp = kk / 3, c = kk % 3;
            const int w0 = word(pw[j][0], m), w1 = word(pw[j][1], m);
            const f2 pr = mul2(add2(make_float2(s16_flo(w0), s16_flo(w1)), nb2), sc2);
            const f2 pi = mul2(add2(make_float2(s16_fhi(w0), s16_fhi(w1)), nb2), sc2);
            const float b = kp * (sp < 2 ? 1.0f : -1.0f);
            f2 hr = acc[sp][c][0], hi = acc[sp][c][1];
            if (DAG && sp >= 2) { hr = mul2(hr, dup(-1.0f)); hi = mul2(hi, dup(-1.0f)); }
            const f2 yr = make_float2(fmaf(-b, pi.x, fmaf(-st.kpp, pr.y, pr.x - hr.x)),
                                      fmaf(b, pi.y, fmaf(-st.kpp, pr.x, pr.y - hr.y)));
            const f2 yi = make_float2(fmaf(b, pr.x, fmaf(-st.kpp, pi.y, pi.x - hi.x)),
                                      fmaf(-b, pr.y, fmaf(-st.kpp, pi.x, pi.y - hi.y)));
#pragma unroll
            for (int f = 0; f < 2; f++) {
                const int a = word(aw[j][f], m);
                const float wx = fmaf(sa, s16_lo(a), f ? yr.y : yr.x);
                const float wy = fmaf(sa, s16_hi(a), f ? yi.y : yi.x);
                const float2 rn =
                    make_float2(fmaf(-alpha, wx, rv[j][m][f].x), fmaf(-alpha, wy, rv[j][m][f].y));
                __stcs(rout + (size_t)(f * 12 + kk) * Vh + h, rn);  // touched once per launch: evict first
                s1 = fmaf(rn.x, rn.x, fmaf(rn.y, rn.y, s1));
            }
        }
    }
    return s1;
}

}  // namespace
