// Schwarz alternating procedure (SAP) smoother of the multigrid (Sec. 3: DD-alphaAMG
// smooths with SAP on the same blocks it aggregates over), for the full-lattice
// doublet operator of the case-C systems
//   D' = D_ND + i s (gamma_5 (x) tau_1) Pi_odd     (hopping normalisation, FP32).
// The lattice is cut into blocks, coloured red/black by the parity of their block
// coordinates.  One SAP sweep: for each colour, the residual r = b - D' x on the
// whole lattice, then on every block of that colour (independently, in parallel) a
// few minimal-residual steps on the block-local problem D_B e = r_B -- D' restricted
// to the block, hops that leave the block dropped -- and x += e on the block.
//
// Kernel: one CTA per block, one thread per block site; the block residual lives in
// shared memory (every MR step's block operator reads the neighbours from there),
// the thread keeps its site's correction and D_B r in registers; the MR coefficients
// come from CTA-wide reductions (FP64 sums).
#include <math.h>

#include "tmnd_internal.cuh"

namespace {

constexpr int SAP_MAX_SITES = 256;  // 4^4 blocks

struct SapGeom {
    Geom g;
    int bd[4];    // block extents {t, x, y, z}
    int nbd[4];   // blocks per direction
    int nsb;      // sites per block
};

__device__ __forceinline__ float2 c_fma(float2 a, float2 b, float2 c) {
    return make_float2(fmaf(a.x, b.x, fmaf(-a.y, b.y, c.x)), fmaf(a.x, b.y, fmaf(a.y, b.x, c.y)));
}

// D_B v at the thread's site (block-local hops only): v in shared memory as [site][24].
// (1 - gamma_mu) / (1 + gamma_mu) projections as in the full-lattice operator, chiral basis.
__device__ void block_apply(const SapGeom &sg, const float2 *__restrict__ links, double kappa, float kp, float kpp,
                            float so, const float2 (*v)[24], int li, const int lc[4], int P, int h,
                            const int gc[4], float2 out[24]) {
    const Geom &g = sg.g;
    const int Vh = g.Vh, Q = 1 - P;
    float2 acc[2][4][3];
#pragma unroll
    for (int f = 0; f < 2; f++)
#pragma unroll
        for (int s = 0; s < 4; s++)
#pragma unroll
            for (int c = 0; c < 3; c++) acc[f][s][c] = make_float2(0.f, 0.f);
    int lstride[4];
    lstride[3] = 1;
    lstride[2] = sg.bd[3];
    lstride[1] = sg.bd[3] * sg.bd[2];
    lstride[0] = sg.bd[3] * sg.bd[2] * sg.bd[1];
    for (int d = 0; d < 8; d++) {
        const int mu = d >> 1;
        const bool fwd = (d & 1) == 0;
        if (fwd ? lc[mu] + 1 >= sg.bd[mu] : lc[mu] == 0) continue;  // leaves the block: dropped
        const int ln = li + (fwd ? lstride[mu] : -lstride[mu]);
        int c[4] = {gc[0], gc[1], gc[2], gc[3]};
        c[mu] += fwd ? 1 : -1;  // stays inside the lattice (blocks do not wrap)
        const int hn = ((c[0] * g.X + c[1]) * g.Y + c[2]) * g.Zh + (c[3] >> 1);
        const float2 *L = fwd ? links + ((size_t)(P * 4 + mu) * 9) * Vh : links + ((size_t)(Q * 4 + mu) * 9) * Vh;
        const int hl = fwd ? h : hn;
        float2 u[3][3];
        for (int a = 0; a < 3; a++)
            for (int b = 0; b < 3; b++) {
                const float2 w = fwd ? L[(size_t)(a * 3 + b) * Vh + hl] : L[(size_t)(b * 3 + a) * Vh + hl];
                u[a][b] = fwd ? w : make_float2(w.x, -w.y);
            }
        const float k = -(float)kappa;
        for (int f = 0; f < 2; f++) {
            float2 ps[4][3];
            for (int s = 0; s < 4; s++)
                for (int cc = 0; cc < 3; cc++) ps[s][cc] = v[ln][f * 12 + s * 3 + cc];
            for (int cc = 0; cc < 3; cc++) {
                float2 gp[4];
                const float2 u0 = ps[0][cc], u1 = ps[1][cc], l0 = ps[2][cc], l1 = ps[3][cc];
                if (mu == 0) {
                    gp[0] = make_float2(-l0.x, -l0.y); gp[1] = make_float2(-l1.x, -l1.y);
                    gp[2] = make_float2(-u0.x, -u0.y); gp[3] = make_float2(-u1.x, -u1.y);
                } else if (mu == 1) {
                    gp[0] = make_float2(l1.y, -l1.x); gp[1] = make_float2(l0.y, -l0.x);
                    gp[2] = make_float2(-u1.y, u1.x); gp[3] = make_float2(-u0.y, u0.x);
                } else if (mu == 2) {
                    gp[0] = make_float2(-l1.x, -l1.y); gp[1] = l0;
                    gp[2] = u1; gp[3] = make_float2(-u0.x, -u0.y);
                } else {
                    gp[0] = make_float2(l0.y, -l0.x); gp[1] = make_float2(-l1.y, l1.x);
                    gp[2] = make_float2(-u0.y, u0.x); gp[3] = make_float2(u1.y, -u1.x);
                }
                const float sgn = fwd ? -1.0f : 1.0f;
                for (int s = 0; s < 4; s++)
                    ps[s][cc] = make_float2(ps[s][cc].x + sgn * gp[s].x, ps[s][cc].y + sgn * gp[s].y);
            }
            for (int s = 0; s < 4; s++)
                for (int a = 0; a < 3; a++) {
                    float2 w = make_float2(0.f, 0.f);
                    for (int b = 0; b < 3; b++) w = c_fma(u[a][b], ps[s][b], w);
                    acc[f][s][a].x = fmaf(k, w.x, acc[f][s][a].x);
                    acc[f][s][a].y = fmaf(k, w.y, acc[f][s][a].y);
                }
        }
    }
    const float sod = P == 1 ? so : 0.0f;
    for (int s = 0; s < 4; s++) {
        const float g5 = s < 2 ? 1.0f : -1.0f;
        for (int c = 0; c < 3; c++) {
            const float2 x0 = v[li][s * 3 + c], x1 = v[li][12 + s * 3 + c];
            float2 o0, o1;
            o0.x = x0.x - kp * g5 * x0.y - kpp * x1.x - sod * g5 * x1.y + acc[0][s][c].x;
            o0.y = x0.y + kp * g5 * x0.x - kpp * x1.y + sod * g5 * x1.x + acc[0][s][c].y;
            o1.x = x1.x + kp * g5 * x1.y - kpp * x0.x - sod * g5 * x0.y + acc[1][s][c].x;
            o1.y = x1.y - kp * g5 * x1.x - kpp * x0.y + sod * g5 * x0.x + acc[1][s][c].y;
            out[s * 3 + c] = o0;
            out[12 + s * 3 + c] = o1;
        }
    }
}

// CTA-wide sum of three doubles (blockDim a multiple of 32); every thread gets the result.
__device__ void cta_sum3(double a, double b, double c, double *red, double out[3]) {
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, o);
        b += __shfl_xor_sync(0xffffffffu, b, o);
        c += __shfl_xor_sync(0xffffffffu, c, o);
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    __syncthreads();
    if (lane == 0) {
        red[3 * wid] = a;
        red[3 * wid + 1] = b;
        red[3 * wid + 2] = c;
    }
    __syncthreads();
    out[0] = out[1] = out[2] = 0.0;
    for (int w = 0; w < nw; w++) {
        out[0] += red[3 * w];
        out[1] += red[3 * w + 1];
        out[2] += red[3 * w + 2];
    }
}

// One colour of a SAP sweep: r is the residual b - D' x of the whole lattice (fine MG
// layout [parity][24][V/2]), x is updated on the blocks of this colour.
__global__ void __launch_bounds__(SAP_MAX_SITES) k_sap_color(SapGeom sg, const float2 *__restrict__ links,
                                                             double kappa, float kp, float kpp, float so, int color,
                                                             const float2 *__restrict__ r, float2 *__restrict__ x,
                                                             int mr_iters) {
    extern __shared__ float2 sm_r[][24];
    __shared__ double red[3 * (SAP_MAX_SITES / 32)];
    const int b = blockIdx.x;
    int bc[4], rem = b;
    bc[3] = rem % sg.nbd[3]; rem /= sg.nbd[3];
    bc[2] = rem % sg.nbd[2]; rem /= sg.nbd[2];
    bc[1] = rem % sg.nbd[1];
    bc[0] = rem / sg.nbd[1];
    if (((bc[0] + bc[1] + bc[2] + bc[3]) & 1) != color) return;  // whole CTA leaves together
    const Geom &g = sg.g;
    const int li = threadIdx.x;
    const bool active = li < sg.nsb;
    int lc[4] = {0, 0, 0, 0}, gc[4] = {0, 0, 0, 0}, P = 0, h = 0;
    if (active) {
        int q = li;
        lc[3] = q % sg.bd[3]; q /= sg.bd[3];
        lc[2] = q % sg.bd[2]; q /= sg.bd[2];
        lc[1] = q % sg.bd[1];
        lc[0] = q / sg.bd[1];
        for (int m = 0; m < 4; m++) gc[m] = bc[m] * sg.bd[m] + lc[m];
        P = (gc[0] + gc[1] + gc[2] + gc[3]) & 1;
        h = (((gc[0] * g.X + gc[1]) * g.Y + gc[2]) * g.Z + gc[3]) >> 1;
        for (int c = 0; c < 24; c++) sm_r[li][c] = r[((size_t)P * 24 + c) * g.Vh + h];
    }
    float2 e[24];
#pragma unroll
    for (int c = 0; c < 24; c++) e[c] = make_float2(0.f, 0.f);
    __syncthreads();
    for (int it = 0; it < mr_iters; it++) {
        float2 t[24];
        double tr = 0, ti = 0, tt = 0;
        if (active) {
            block_apply(sg, links, kappa, kp, kpp, so, sm_r, li, lc, P, h, gc, t);
            for (int c = 0; c < 24; c++) {
                const float2 rv = sm_r[li][c];
                tr += (double)t[c].x * rv.x + (double)t[c].y * rv.y;   // <t, r>
                ti += (double)t[c].x * rv.y - (double)t[c].y * rv.x;
                tt += (double)t[c].x * t[c].x + (double)t[c].y * t[c].y;
            }
        }
        double sums[3];
        cta_sum3(tr, ti, tt, red, sums);  // ends with the block's reads of sm_r done
        if (!(sums[2] > 0.0)) break;
        const float wr = (float)(sums[0] / sums[2]), wi = (float)(sums[1] / sums[2]);
        __syncthreads();
        if (active)
            for (int c = 0; c < 24; c++) {
                const float2 rv = sm_r[li][c];
                e[c].x += wr * rv.x - wi * rv.y;
                e[c].y += wr * rv.y + wi * rv.x;
                sm_r[li][c] = make_float2(rv.x - (wr * t[c].x - wi * t[c].y), rv.y - (wr * t[c].y + wi * t[c].x));
            }
        __syncthreads();
    }
    if (active)
        for (int c = 0; c < 24; c++) {
            float2 &xv = x[((size_t)P * 24 + c) * g.Vh + h];
            xv = make_float2(xv.x + e[c].x, xv.y + e[c].y);
        }
}

}  // namespace

// One colour of a SAP sweep (see above).  bd: block extents (their product <= 256, each
// dividing the lattice); r: the current residual b - D' x on the whole lattice; x updated
// on the blocks of colour `color`.
tmnd_status launch_sap_color(const tmnd_gauge *g, const int bd[4], int color, double s_odd, const float2 *r,
                             float2 *x, int mr_iters, cudaStream_t s) {
    SapGeom sg;
    sg.g = g->geom;
    const int dims[4] = {g->geom.T, g->geom.X, g->geom.Y, g->geom.Z};
    sg.nsb = 1;
    int nblock = 1;
    for (int m = 0; m < 4; m++) {
        TMND_ARG_CHECK(bd[m] >= 1 && dims[m] % bd[m] == 0, "SAP: block extent %d does not divide %d", bd[m], dims[m]);
        sg.bd[m] = bd[m];
        sg.nbd[m] = dims[m] / bd[m];
        sg.nsb *= bd[m];
        nblock *= sg.nbd[m];
    }
    TMND_ARG_CHECK(sg.nsb <= SAP_MAX_SITES, "SAP: blocks of %d sites (at most %d)", sg.nsb, SAP_MAX_SITES);
    const int threads = (sg.nsb + 31) / 32 * 32;
    const size_t smem = sizeof(float2) * 24 * (size_t)sg.nsb;
    static bool attr = false;
    if (!attr) {
        TMND_CUDA_TRY(cudaFuncSetAttribute(k_sap_color, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)(sizeof(float2) * 24 * SAP_MAX_SITES)));
        attr = true;
    }
    k_sap_color<<<nblock, threads, smem, s>>>(sg, g->links_f32, g->act.kappa, (float)g->st.kp, (float)g->st.kpp,
                                              (float)s_odd, color, r, x, mr_iters);
    TMND_CUDA_TRY(cudaGetLastError());
    return TMND_OK;
}
