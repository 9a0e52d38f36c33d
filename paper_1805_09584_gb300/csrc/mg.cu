// Aggregation-based two-level multigrid (Sec. 3, DD-alphaAMG structure; Sec. 3.2
// for the doublet), FP32 on the device.
//
//   fine vectors   : full lattice, [parity][ncomp][V/2] complex64 (ncomp = 12 for
//                    one flavour, 24 for the doublet, component = flavour*12 + spin*3 + colour)
//   aggregates     : blocks of bt x bx x by x bz sites; block-local site index
//                    s = ((it*bx + ix)*by + iy)*bz + iz; blocks in lexicographic order
//   prolongator P  : [block][chirality][nvec][s][6] complex64 (chirality 0 = spins 0,1,
//                    chirality 1 = spins 2,3; 6 = 2 spins x 3 colours) -- Gamma_5-compatible
//                    (Sec. 3: Gamma_5 P = P Gamma_5,c) and orthonormal per block and chirality
//   coarse Wilson  : D_W,c = P^+ D_W P as [block][9][2 nvec][2 nvec] complex64, direction
//                    0 = self, 1 + 2 mu + (0 forward, 1 backward)
//   coarse vectors : [rhs][block][flavour][2 nvec] complex64
// The doublet coarse operator is applied as (Eq. "non-degenerate_coarse")
//   D_ND,c = D_W,c (x) 1 + i mu_c (Gamma_5,c (x) tau_3) - eps_c (1 (x) tau_1)
// plus, for the shifted systems of case C, + i s (tau_1 (x) G_odd) with
// G_odd = P^+ gamma_5 Pi_odd P (the shift acts on odd sites only).
#include <math.h>

#include <vector>

#include "tmnd_internal.cuh"

struct tmnd_mg {
    tmnd_gauge *g;
    int bd[4];          // block size
    int nbd[4];         // blocks per direction
    int nblock, nsb;    // number of blocks, sites per block
    int nv;             // vectors per chirality
    double mu_c, eps_c; // coarse doublet terms (hopping normalisation)
    float2 *P;          // prolongator
    float2 *Dc;         // coarse Wilson operator
    float2 *Godd;       // [block][2nv][2nv] P^+ gamma_5 Pi_odd P
    void *work;         // fine-vector scratch for the assembly
    size_t work_bytes;
    int tc;             // coarse apply on the tensor cores where the shape allows
    int *tc_err;        // device flag: a tensor-core kernel gave up waiting
    uint64_t wait_ns;   // limit of the tensor-core kernel's bounded waits
    int smoother;       // 0: minimal residual on the whole lattice, 1: SAP on the aggregation blocks
    int sap_mr;         // SAP: minimal-residual steps per block solve
    mutable int stall_next;  // test hook: tensor-core launches still to run with the stall barrier
    void *Dt, *Gt;      // D_W,c and G_odd again, in the tensor-core operand-tile layout
    void *Bt;           // B operand tiles of one application (up to 16 right-hand sides)
};

size_t coarse_tc_smem(int n2, int nrhs);
size_t coarse_tc_atile_bytes(int nv);
size_t coarse_tc_btile_bytes(int nblock, int nv, int nrhs);
tmnd_status coarse_tc_make_atiles(const float2 *src, void *dst, long nmat, int nv, cudaStream_t s);
tmnd_status launch_coarse_apply_tc(const void *Dt, const void *Gt, void *btiles, const float2 *x, float2 *y,
                                   int nblock, const int nbd[4], int nv, int nrhs, float mu_c, float eps_c,
                                   float s_odd, int *err, uint64_t wait_ns, int stall, cudaStream_t s);

namespace {

constexpr int MG_MAXV = 32;

__device__ __forceinline__ float2 cfmaf2(float2 a, float2 b, float2 c) {
    return make_float2(fmaf(a.x, b.x, fmaf(-a.y, b.y, c.x)), fmaf(a.x, b.y, fmaf(a.y, b.x, c.y)));
}
// conj(a) * b + c
__device__ __forceinline__ float2 cfmacf2(float2 a, float2 b, float2 c) {
    return make_float2(fmaf(a.x, b.x, fmaf(a.y, b.y, c.x)), fmaf(a.x, b.y, fmaf(-a.y, b.x, c.y)));
}

struct MGGeom {
    Geom g;
    int bd[4], nbd[4], nsb, nblock, nv;
};

// fine (parity, h) of block b, local site s
__device__ __forceinline__ void block_site(const MGGeom &m, int b, int s, int &par, int &h) {
    int iz = s % m.bd[3], r = s / m.bd[3];
    int iy = r % m.bd[2]; r /= m.bd[2];
    int ix = r % m.bd[1];
    int it = r / m.bd[1];
    int bz = b % m.nbd[3], rb = b / m.nbd[3];
    int by = rb % m.nbd[2]; rb /= m.nbd[2];
    int bx = rb % m.nbd[1];
    int bt = rb / m.nbd[1];
    const int t = bt * m.bd[0] + it, x = bx * m.bd[1] + ix, y = by * m.bd[2] + iy, z = bz * m.bd[3] + iz;
    par = (t + x + y + z) & 1;
    h = (((t * m.g.X + x) * m.g.Y + y) * m.g.Z + z) >> 1;
}

__device__ __forceinline__ int local_coord(const MGGeom &m, int s, int mu) {
    int c[4];
    c[3] = s % m.bd[3];
    int r = s / m.bd[3];
    c[2] = r % m.bd[2];
    r /= m.bd[2];
    c[1] = r % m.bd[1];
    c[0] = r / m.bd[1];
    return c[mu];
}

// Gather the test vectors into P and orthonormalise each (block, chirality)
// set by modified Gram-Schmidt in the given order (FP64 dot products).
// One block of threads per (block, chirality).
__global__ void k_mg_ortho(MGGeom m, const float2 *__restrict__ vecs, float2 *__restrict__ P) {
    const int b = blockIdx.x >> 1, chi = blockIdx.x & 1;
    const int len = m.nsb * 6;
    const size_t Vh = m.g.Vh;
    float2 *Pb = P + ((size_t)(b * 2 + chi) * m.nv) * len;
    for (int k = 0; k < m.nv; k++)
        for (int i = threadIdx.x; i < len; i += blockDim.x) {
            const int s = i / 6, c = i % 6;
            int par, h;
            block_site(m, b, s, par, h);
            Pb[(size_t)k * len + i] = vecs[(((size_t)k * 2 + par) * 12 + chi * 6 + c) * Vh + h];
        }
    __syncthreads();
    __shared__ double red[64];
    for (int k = 0; k < m.nv; k++) {
        float2 *vk = Pb + (size_t)k * len;
        for (int j = 0; j < k; j++) {
            const float2 *vj = Pb + (size_t)j * len;
            double re = 0, im = 0;
            for (int i = threadIdx.x; i < len; i += blockDim.x) {
                const float2 a = vj[i], v = vk[i];
                re += (double)a.x * v.x + (double)a.y * v.y;
                im += (double)a.x * v.y - (double)a.y * v.x;
            }
            double sre = block_sum(re, red);
            __syncthreads();
            double sim = block_sum(im, red + 33);
            __syncthreads();
            if (threadIdx.x == 0) {
                red[62] = sre;
                red[63] = sim;
            }
            __syncthreads();
            const float cr = (float)red[62], ci = (float)red[63];
            for (int i = threadIdx.x; i < len; i += blockDim.x) {
                const float2 a = vj[i];
                float2 v = vk[i];
                v.x -= cr * a.x - ci * a.y;
                v.y -= cr * a.y + ci * a.x;
                vk[i] = v;
            }
            __syncthreads();
        }
        double nn = 0;
        for (int i = threadIdx.x; i < len; i += blockDim.x) nn += (double)vk[i].x * vk[i].x + (double)vk[i].y * vk[i].y;
        double snn = block_sum(nn, red);
        __syncthreads();
        if (threadIdx.x == 0) red[62] = snn;
        __syncthreads();
        const float inv = (float)(1.0 / sqrt(red[62]));
        for (int i = threadIdx.x; i < len; i += blockDim.x) {
            vk[i].x *= inv;
            vk[i].y *= inv;
        }
        __syncthreads();
    }
}

// Restriction  out[rhs][b][f][chi*nv + k] = sum_{s, c} conj(P[b][chi][k][s][c]) v[f][site(b,s)][chi*6 + c]
// ncomp = 12 (one flavour) or 24 (doublet).  mode: 0 all sites; 1 + d: only the sites of the
// block's face in direction d (0 t+, 1 t-, 2 x+, ...); 9: odd sites only, with gamma_5.
// One block of threads per (block, rhs); a warp per output row.
__global__ void k_mg_restrict(MGGeom m, const float2 *__restrict__ P, const float2 *__restrict__ v, int ncomp,
                              float2 *__restrict__ out, int mode, int accumulate) {
    const int b = blockIdx.x, rhs = blockIdx.y;
    const int nf = ncomp / 12;
    const int len = m.nsb * 6;
    const size_t Vh = m.g.Vh;
    const float2 *vr = v + (size_t)rhs * 2 * ncomp * Vh;
    float2 *o = out + ((size_t)rhs * m.nblock + b) * nf * 2 * m.nv;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarp = blockDim.x >> 5;
    for (int row = warp; row < nf * 2 * m.nv; row += nwarp) {
        const int f = row / (2 * m.nv), ck = row % (2 * m.nv), chi = ck / m.nv, k = ck % m.nv;
        const float2 *Pr = P + ((size_t)(b * 2 + chi) * m.nv + k) * len;
        float2 acc = make_float2(0.f, 0.f);
        for (int i = lane; i < len; i += 32) {
            const int s = i / 6, c = i % 6;
            bool use = true;
            float sgn = 1.0f;
            if (mode >= 1 && mode <= 8) {
                const int d = mode - 1, mu = d >> 1;
                const int lc = local_coord(m, s, mu);
                use = (d & 1) == 0 ? (lc == m.bd[mu] - 1) : (lc == 0);
            }
            int par, h;
            block_site(m, b, s, par, h);
            if (mode == 9) {
                use = par == 1;
                sgn = chi == 0 ? 1.0f : -1.0f;
            }
            if (!use) continue;
            const float2 x = vr[(((size_t)par * ncomp) + f * 12 + chi * 6 + c) * Vh + h];
            acc = cfmacf2(Pr[i], make_float2(sgn * x.x, sgn * x.y), acc);
        }
        for (int off = 16; off > 0; off >>= 1) {
            acc.x += __shfl_xor_sync(0xffffffffu, acc.x, off);
            acc.y += __shfl_xor_sync(0xffffffffu, acc.y, off);
        }
        if (lane == 0) {
            if (accumulate) {
                o[row].x += acc.x;
                o[row].y += acc.y;
            } else {
                o[row] = acc;
            }
        }
    }
}

// Prolongation  v[f][site(b,s)][chi*6 + c] (+)= sum_k P[b][chi][k][s][c] in[rhs][b][f][chi*nv + k]
__global__ void k_mg_prolong(MGGeom m, const float2 *__restrict__ P, const float2 *__restrict__ in, int ncomp,
                             float2 *__restrict__ v, int accumulate) {
    const int b = blockIdx.x, rhs = blockIdx.y;
    const int nf = ncomp / 12;
    const int len = m.nsb * 6;
    const size_t Vh = m.g.Vh;
    __shared__ float2 sc[2 * 2 * MG_MAXV];
    const float2 *ir = in + ((size_t)rhs * m.nblock + b) * nf * 2 * m.nv;
    for (int i = threadIdx.x; i < nf * 2 * m.nv; i += blockDim.x) sc[i] = ir[i];
    __syncthreads();
    float2 *vr = v + (size_t)rhs * 2 * ncomp * Vh;
    for (int i = threadIdx.x; i < nf * 2 * len; i += blockDim.x) {
        const int f = i / (2 * len), rem = i % (2 * len), chi = rem / len, sc6 = rem % len;
        const int s = sc6 / 6, c = sc6 % 6;
        float2 acc = make_float2(0.f, 0.f);
        const float2 *Pb = P + ((size_t)(b * 2 + chi) * m.nv) * len + sc6;
        for (int k = 0; k < m.nv; k++) acc = cfmaf2(Pb[(size_t)k * len], sc[f * 2 * m.nv + chi * m.nv + k], acc);
        int par, h;
        block_site(m, b, s, par, h);
        const size_t idx = (((size_t)par * ncomp) + f * 12 + chi * 6 + c) * Vh + h;
        if (accumulate) {
            float2 o = vr[idx];
            vr[idx] = make_float2(o.x + acc.x, o.y + acc.y);
        } else {
            vr[idx] = acc;
        }
    }
}

// Coarse doublet operator: one block of threads per coarse site, thread (row i, column n = f*nrhs + r).
// y = sum_d Dc[b][d] x[nb(b,d)] (per flavour) + i mu_c g5c tau_3 x - eps_c tau_1 x + i s tau_1 Godd x
__global__ void k_coarse_apply(MGGeom m, const float2 *__restrict__ Dc, const float2 *__restrict__ Godd,
                               const float2 *__restrict__ x, float2 *__restrict__ y, int nrhs, float mu_c,
                               float eps_c, float s_odd) {
    extern __shared__ float2 sx[];  // [9][2nv][2*nrhs]
    const int b = blockIdx.x;
    const int n2 = 2 * m.nv, ncol = 2 * nrhs;
    int nbr[9];
    {
        int c[4];
        int r = b;
        c[3] = r % m.nbd[3]; r /= m.nbd[3];
        c[2] = r % m.nbd[2]; r /= m.nbd[2];
        c[1] = r % m.nbd[1];
        c[0] = r / m.nbd[1];
        nbr[0] = b;
        for (int d = 0; d < 8; d++) {
            int cc[4] = {c[0], c[1], c[2], c[3]};
            const int mu = d >> 1;
            cc[mu] = (d & 1) == 0 ? (cc[mu] + 1) % m.nbd[mu] : (cc[mu] + m.nbd[mu] - 1) % m.nbd[mu];
            nbr[1 + d] = ((cc[0] * m.nbd[1] + cc[1]) * m.nbd[2] + cc[2]) * m.nbd[3] + cc[3];
        }
    }
    for (int i = threadIdx.x; i < 9 * n2 * ncol; i += blockDim.x) {
        const int d = i / (n2 * ncol), rem = i % (n2 * ncol), j = rem / ncol, col = rem % ncol;
        const int f = col / nrhs, r = col % nrhs;
        sx[i] = x[(((size_t)r * m.nblock + nbr[d]) * 2 + f) * n2 + j];
    }
    __syncthreads();
    const int row = threadIdx.x / ncol, col = threadIdx.x % ncol;
    if (row >= n2) return;
    const int f = col / nrhs, r = col % nrhs;
    float2 acc = make_float2(0.f, 0.f);
    const float2 *D = Dc + (size_t)b * 9 * n2 * n2;
    for (int d = 0; d < 9; d++) {
        const float2 *Dr = D + ((size_t)d * n2 + row) * n2;
        const float2 *xs = sx + (size_t)d * n2 * ncol + col;
        for (int j = 0; j < n2; j++) acc = cfmaf2(Dr[j], xs[(size_t)j * ncol], acc);
    }
    // flavour structure, self site
    const float2 xs_f = sx[(size_t)row * ncol + col];                         // same flavour
    const float2 xs_o = sx[(size_t)row * ncol + ((1 - f) * nrhs + r)];        // other flavour
    const float g5 = row < m.nv ? 1.0f : -1.0f;
    const float t3 = f == 0 ? 1.0f : -1.0f;
    acc.x += -mu_c * g5 * t3 * xs_f.y - eps_c * xs_o.x;
    acc.y += mu_c * g5 * t3 * xs_f.x - eps_c * xs_o.y;
    if (s_odd != 0.0f) {
        const float2 *G = Godd + ((size_t)b * n2 + row) * n2;
        float2 gx = make_float2(0.f, 0.f);
        for (int j = 0; j < n2; j++) gx = cfmaf2(G[j], sx[(size_t)j * ncol + ((1 - f) * nrhs + r)], gx);
        acc.x += -s_odd * gx.y;
        acc.y += s_odd * gx.x;
    }
    y[(((size_t)r * m.nblock + b) * 2 + f) * n2 + row] = acc;
}

// One direction of the single-flavour hop, w(x) = -kappa (1 -+ gamma_mu) U psi(x +- mu) (with the
// antiperiodic sign), full lattice, FP32 with the FP64 links rounded on the fly.
__global__ void k_hop_dir_f32(Geom g, double kappa, const double2 *__restrict__ links, const float2 *__restrict__ in,
                              float2 *__restrict__ out, int d) {
    const int Vh = g.Vh;
    const int mu = d >> 1;
    const bool fwd = (d & 1) == 0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < 2 * Vh; i += gridDim.x * blockDim.x) {
        const int P = i / Vh, h = i % Vh;
        const int zh = h % g.Zh;
        int r = h / g.Zh;
        int y = r % g.Y;
        r /= g.Y;
        int x = r % g.X;
        int t = r / g.X;
        int z = 2 * zh + ((P + t + x + y) & 1);
        int c[4] = {t, x, y, z}, n[4] = {g.T, g.X, g.Y, g.Z};
        float sg = 1.0f;
        if (fwd) {
            if (c[mu] + 1 == n[mu]) { c[mu] = 0; if (mu == 0 && g.apbc) sg = -1.0f; }
            else c[mu]++;
        } else {
            if (c[mu] == 0) { c[mu] = n[mu] - 1; if (mu == 0 && g.apbc) sg = -1.0f; }
            else c[mu]--;
        }
        const int hn = ((c[0] * g.X + c[1]) * g.Y + c[2]) * g.Zh + (c[3] >> 1);
        const int Q = 1 - P;
        // link U_mu(x) (forward) at (P, h) or U_mu(x - mu) (backward) at (Q, hn)
        const double2 *L = fwd ? links + ((size_t)(P * 4 + mu) * 9) * Vh : links + ((size_t)(Q * 4 + mu) * 9) * Vh;
        const int hl = fwd ? h : hn;
        float2 u[3][3];
        for (int a = 0; a < 3; a++)
            for (int bb = 0; bb < 3; bb++) {
                const double2 w = L[(size_t)(a * 3 + bb) * Vh + hl];
                u[a][bb] = fwd ? make_float2((float)w.x, (float)w.y) : make_float2((float)w.x, -(float)w.y);
            }
        float2 ps[4][3];
        for (int s = 0; s < 4; s++)
            for (int cc = 0; cc < 3; cc++) ps[s][cc] = in[((size_t)Q * 12 + s * 3 + cc) * Vh + hn];
        // (1 -+ gamma_mu) applied to the 4-spinor, then the colour matrix (U or U^+)
        float2 proj[4][3];
        for (int cc = 0; cc < 3; cc++) {
            // gamma_mu psi in the chiral basis: gamma_0 = [[0,-1],[-1,0]], gamma_k = [[0,-i s_k],[i s_k,0]]
            float2 gp[4];
            const float2 u0 = ps[0][cc], u1 = ps[1][cc], l0 = ps[2][cc], l1 = ps[3][cc];
            if (mu == 0) {
                gp[0] = make_float2(-l0.x, -l0.y); gp[1] = make_float2(-l1.x, -l1.y);
                gp[2] = make_float2(-u0.x, -u0.y); gp[3] = make_float2(-u1.x, -u1.y);
            } else if (mu == 1) {  // -i s1: (l0,l1) -> (-i l1, -i l0); i s1: (u0,u1) -> (i u1, i u0)
                gp[0] = make_float2(l1.y, -l1.x); gp[1] = make_float2(l0.y, -l0.x);
                gp[2] = make_float2(-u1.y, u1.x); gp[3] = make_float2(-u0.y, u0.x);
            } else if (mu == 2) {  // -i s2 = [[0,-1],[1,0]]; i s2 = [[0,1],[-1,0]]
                gp[0] = make_float2(-l1.x, -l1.y); gp[1] = l0;
                gp[2] = u1; gp[3] = make_float2(-u0.x, -u0.y);
            } else {  // -i s3 = diag(-i, i); i s3 = diag(i, -i)
                gp[0] = make_float2(l0.y, -l0.x); gp[1] = make_float2(-l1.y, l1.x);
                gp[2] = make_float2(-u0.y, u0.x); gp[3] = make_float2(u1.y, -u1.x);
            }
            const float sgn = fwd ? -1.0f : 1.0f;
            for (int s = 0; s < 4; s++) proj[s][cc] = make_float2(ps[s][cc].x + sgn * gp[s].x, ps[s][cc].y + sgn * gp[s].y);
        }
        const float k = -(float)kappa * sg;
        for (int s = 0; s < 4; s++)
            for (int a = 0; a < 3; a++) {
                float2 acc = make_float2(0.f, 0.f);
                for (int bb = 0; bb < 3; bb++) acc = cfmaf2(fwd ? u[a][bb] : u[bb][a], proj[s][bb], acc);
                out[((size_t)P * 12 + s * 3 + a) * Vh + h] = make_float2(k * acc.x, k * acc.y);
            }
    }
}

}  // namespace

static MGGeom mg_geom(const tmnd_mg *mg) {
    MGGeom m;
    m.g = mg->g->geom;
    for (int i = 0; i < 4; i++) {
        m.bd[i] = mg->bd[i];
        m.nbd[i] = mg->nbd[i];
    }
    m.nsb = mg->nsb;
    m.nblock = mg->nblock;
    m.nv = mg->nv;
    return m;
}

// host: coarse 48x48 block helpers
extern "C" tmnd_status tmnd_mg_create(tmnd_gauge *g, const tmnd_mg_params *p, const void *test_vectors,
                                      tmnd_mg **out) {
    TMND_ARG_CHECK(g && p && test_vectors && out, "tmnd_mg_create: NULL argument");
    *out = nullptr;
    TMND_ARG_CHECK(p->nvec >= 1 && p->nvec <= MG_MAXV, "tmnd_mg_create: nvec = %d not in [1, %d]", p->nvec, MG_MAXV);
    TMND_ARG_CHECK(p->wait_limit_s >= 0 && p->wait_limit_s <= 60 && p->stall_test >= 0,
                   "tmnd_mg_create: wait_limit_s = %g not in [0, 60] or stall_test < 0", p->wait_limit_s);
    TMND_ARG_CHECK(p->smoother == 0 || (p->smoother == 1 && p->block[0] * p->block[1] * p->block[2] * p->block[3] <= 256),
                   "tmnd_mg_create: smoother %d (SAP needs blocks of at most 256 sites)", p->smoother);
    TMND_ARG_CHECK(p->sap_mr >= 0 && p->sap_mr <= 64, "tmnd_mg_create: sap_mr = %d", p->sap_mr);
    for (int i = 0; i < 4; i++)
        TMND_ARG_CHECK(p->block[i] >= 1 && g->act.dims[i] % p->block[i] == 0,
                       "tmnd_mg_create: block[%d] = %d does not divide dims[%d] = %d", i, p->block[i], i,
                       g->act.dims[i]);
    cudaGetLastError();
    tmnd_mg *mg = new tmnd_mg();
    mg->g = g;
    mg->nsb = 1;
    mg->nblock = 1;
    for (int i = 0; i < 4; i++) {
        mg->bd[i] = p->block[i];
        mg->nbd[i] = g->act.dims[i] / p->block[i];
        mg->nsb *= mg->bd[i];
        mg->nblock *= mg->nbd[i];
    }
    mg->nv = p->nvec;
    mg->tc = p->coarse_simt ? 0 : 1;
    mg->wait_ns = p->wait_limit_s > 0 ? (uint64_t)(p->wait_limit_s * 1e9) : 2000000000ull;
    mg->stall_next = p->stall_test;
    mg->smoother = p->smoother;
    mg->sap_mr = p->sap_mr > 0 ? p->sap_mr : 4;
    const double d = p->coarse_mu_factor > 0 ? p->coarse_mu_factor : 1.0;
    mg->mu_c = 2 * g->act.kappa * g->act.mu_bar * d;
    mg->eps_c = 2 * g->act.kappa * g->act.eps_bar;
    const int n2 = 2 * mg->nv;
    const size_t Vh = g->geom.Vh;
    const size_t pbytes = sizeof(float2) * (size_t)mg->nblock * 2 * mg->nv * mg->nsb * 6;
    const size_t dbytes = sizeof(float2) * (size_t)mg->nblock * 9 * n2 * n2;
    const size_t gbytes = sizeof(float2) * (size_t)mg->nblock * n2 * n2;
    mg->work_bytes = 2 * sizeof(float2) * 2 * 12 * Vh;  // two single-flavour full fields
    cudaError_t e = cudaMalloc(&mg->P, pbytes);
    if (e == cudaSuccess) e = cudaMalloc(&mg->Dc, dbytes);
    if (e == cudaSuccess) e = cudaMalloc(&mg->Godd, gbytes);
    if (e == cudaSuccess) e = cudaMalloc(&mg->tc_err, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(mg->tc_err, 0, sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc(&mg->work, mg->work_bytes);
    if (e != cudaSuccess) {
        tmnd_mg_destroy(mg);
        tmnd_set_error("tmnd_mg_create: %s", cudaGetErrorString(e));
        return e == cudaErrorMemoryAllocation ? TMND_ERR_OOM : TMND_ERR_CUDA;
    }
    MGGeom m = mg_geom(mg);
    // 1. prolongator
    k_mg_ortho<<<mg->nblock * 2, 256>>>(m, (const float2 *)test_vectors, mg->P);
    // 2. coarse Wilson operator D_W,c = P^+ (1 - kappa H) P, column by column:
    //    column (chi, k) of every block at once; the hop of one direction d
    //    lands on the block's own face (-> coupling to the neighbour block
    //    in direction d) and on its interior (-> self coupling).
    cudaMemset(mg->Dc, 0, dbytes);
    float2 *col = (float2 *)mg->work;
    float2 *w = col + 2 * 12 * Vh;
    std::vector<float2> hD((size_t)mg->nblock * 9 * n2 * n2);
    float2 *tmpc = nullptr;
    e = cudaMalloc(&tmpc, sizeof(float2) * (size_t)mg->nblock * n2 * 10);
    if (e != cudaSuccess) {
        tmnd_mg_destroy(mg);
        tmnd_set_error("tmnd_mg_create: %s", cudaGetErrorString(e));
        return TMND_ERR_OOM;
    }
    std::vector<float2> htmp((size_t)mg->nblock * n2 * 10);
    std::vector<float2> hG((size_t)mg->nblock * n2 * n2);
    const int gb = (int)((2 * Vh + 255) / 256);
    for (int j = 0; j < n2; j++) {
        // coarse unit vector e_j on every block -> fine column field
        std::vector<float2> unit((size_t)mg->nblock * n2, make_float2(0.f, 0.f));
        for (int b = 0; b < mg->nblock; b++) unit[(size_t)b * n2 + j] = make_float2(1.f, 0.f);
        cudaMemcpy(tmpc, unit.data(), sizeof(float2) * unit.size(), cudaMemcpyHostToDevice);
        k_mg_prolong<<<dim3(mg->nblock, 1), 256>>>(m, mg->P, tmpc, 12, col, 0);
        // identity part (P^+ P = 1) and Godd column
        k_mg_restrict<<<dim3(mg->nblock, 1), 256>>>(m, mg->P, col, 12, tmpc + (size_t)mg->nblock * n2 * 9, 9, 0);
        for (int dd = 0; dd < 8; dd++) {
            k_hop_dir_f32<<<gb, 256>>>(g->geom, g->act.kappa, g->links, col, w, dd);
            // face of the hop direction -> neighbour block column; the rest -> self
            k_mg_restrict<<<dim3(mg->nblock, 1), 256>>>(m, mg->P, w, 12, tmpc + (size_t)mg->nblock * n2 * (1 + dd),
                                                        1 + dd, 0);
            k_mg_restrict<<<dim3(mg->nblock, 1), 256>>>(m, mg->P, w, 12, tmpc, 0, dd > 0);
            // remove the face part from the self accumulation
        }
        e = cudaMemcpy(htmp.data(), tmpc, sizeof(float2) * htmp.size(), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) break;
        // htmp[0]: sum over directions of P_b^+ (hop_d col) over all sites of b;
        // htmp[1+d]: the part of that from b's face in direction d, which hops in from block b+d.
        for (int b = 0; b < mg->nblock; b++) {
            for (int i = 0; i < n2; i++) {
                float2 self = htmp[(size_t)b * n2 + i];
                for (int dd = 0; dd < 8; dd++) {
                    const float2 fc = htmp[(size_t)mg->nblock * n2 * (1 + dd) + (size_t)b * n2 + i];
                    self.x -= fc.x;
                    self.y -= fc.y;
                    hD[(((size_t)b * 9 + 1 + dd) * n2 + i) * n2 + j] = fc;
                }
                if (i == j) self.x += 1.0f;  // the identity of D_W = 1 - kappa H, P^+ P = 1
                hD[(((size_t)b * 9 + 0) * n2 + i) * n2 + j] = self;
                hG[((size_t)b * n2 + i) * n2 + j] = htmp[(size_t)mg->nblock * n2 * 9 + (size_t)b * n2 + i];
            }
        }
    }
    if (e == cudaSuccess) e = cudaMemcpy(mg->Dc, hD.data(), dbytes, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(mg->Godd, hG.data(), gbytes, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e == cudaSuccess && mg->tc && coarse_tc_smem(n2, 1) > 0) {  // operand tiles for the tensor cores
        const size_t at = coarse_tc_atile_bytes(mg->nv);
        e = cudaMalloc(&mg->Dt, at * 9 * mg->nblock);
        if (e == cudaSuccess) e = cudaMalloc(&mg->Gt, at * mg->nblock);
        if (e == cudaSuccess) e = cudaMalloc(&mg->Bt, coarse_tc_btile_bytes(mg->nblock, mg->nv, 16));
        if (e == cudaSuccess &&
            (coarse_tc_make_atiles(mg->Dc, mg->Dt, 9L * mg->nblock, mg->nv, 0) != TMND_OK ||
             coarse_tc_make_atiles(mg->Godd, mg->Gt, mg->nblock, mg->nv, 0) != TMND_OK))
            e = cudaErrorLaunchFailure;
    }
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    cudaFree(tmpc);
    if (e != cudaSuccess) {
        tmnd_mg_destroy(mg);
        tmnd_set_error("tmnd_mg_create: %s", cudaGetErrorString(e));
        return TMND_ERR_CUDA;
    }
    *out = mg;
    return TMND_OK;
}

extern "C" void tmnd_mg_destroy(tmnd_mg *mg) {
    if (!mg) return;
    cudaDeviceSynchronize();
    if (mg->P) cudaFree(mg->P);
    if (mg->Dc) cudaFree(mg->Dc);
    if (mg->tc_err) cudaFree(mg->tc_err);
    if (mg->Dt) cudaFree(mg->Dt);
    if (mg->Gt) cudaFree(mg->Gt);
    if (mg->Bt) cudaFree(mg->Bt);
    if (mg->Godd) cudaFree(mg->Godd);
    if (mg->work) cudaFree(mg->work);
    delete mg;
}

extern "C" size_t tmnd_mg_coarse_bytes(const tmnd_mg *mg) {
    return mg ? sizeof(float2) * (size_t)mg->nblock * 2 * 2 * mg->nv : 0;
}

extern "C" tmnd_status tmnd_mg_restrict(const tmnd_mg *mg, void *out_c, const void *in_fine, int nrhs, void *stream) {
    TMND_ARG_CHECK(mg && out_c && in_fine && nrhs >= 1, "tmnd_mg_restrict: bad arguments");
    cudaGetLastError();
    MGGeom m = mg_geom(mg);
    k_mg_restrict<<<dim3(mg->nblock, nrhs), 256, 0, (cudaStream_t)stream>>>(m, mg->P, (const float2 *)in_fine, 24,
                                                                           (float2 *)out_c, 0, 0);
    TMND_CUDA_TRY(cudaGetLastError());
    return TMND_OK;
}

extern "C" tmnd_status tmnd_mg_prolong(const tmnd_mg *mg, void *out_fine, const void *in_c, int nrhs, void *stream) {
    TMND_ARG_CHECK(mg && out_fine && in_c && nrhs >= 1, "tmnd_mg_prolong: bad arguments");
    cudaGetLastError();
    MGGeom m = mg_geom(mg);
    k_mg_prolong<<<dim3(mg->nblock, nrhs), 256, 0, (cudaStream_t)stream>>>(m, mg->P, (const float2 *)in_c, 24,
                                                                          (float2 *)out_fine, 0);
    TMND_CUDA_TRY(cudaGetLastError());
    return TMND_OK;
}

extern "C" tmnd_status mg_coarse_apply(const tmnd_mg *mg, void *out_c, const void *in_c, int nrhs,
                                       double odd_shift_s, void *stream) {
    TMND_ARG_CHECK(mg && out_c && in_c, "mg_coarse_apply: NULL argument");
    TMND_ARG_CHECK(out_c != in_c, "mg_coarse_apply: out and in must not alias");
    const int n2 = 2 * mg->nv;
    TMND_ARG_CHECK(nrhs >= 1, "mg_coarse_apply: nrhs = %d", nrhs);
    TMND_ARG_CHECK(((uintptr_t)out_c & 15) == 0 && ((uintptr_t)in_c & 15) == 0,
                   "mg_coarse_apply: vectors must be 16-byte aligned");
    cudaGetLastError();
    if (mg->tc && mg->Dt && coarse_tc_smem(n2, nrhs) > 0) {
        const int stall = mg->stall_next > 0;
        if (stall) mg->stall_next--;
        return launch_coarse_apply_tc(mg->Dt, mg->Gt, mg->Bt, (const float2 *)in_c, (float2 *)out_c, mg->nblock,
                                      mg->nbd, mg->nv, nrhs, (float)mg->mu_c, (float)mg->eps_c, (float)odd_shift_s,
                                      mg->tc_err, mg->wait_ns, stall, (cudaStream_t)stream);
    }
    TMND_ARG_CHECK(n2 * 2 * nrhs <= 1024, "mg_coarse_apply: nrhs = %d too large for 2*nvec = %d", nrhs, n2);
    MGGeom m = mg_geom(mg);
    const size_t smem = sizeof(float2) * 9 * n2 * 2 * nrhs;
    TMND_ARG_CHECK(smem <= 96 * 1024, "mg_coarse_apply: nrhs too large");
    if (smem > 48 * 1024)
        TMND_CUDA_TRY(cudaFuncSetAttribute(k_coarse_apply, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_coarse_apply<<<mg->nblock, n2 * 2 * nrhs, smem, (cudaStream_t)stream>>>(
        m, mg->Dc, mg->Godd, (const float2 *)in_c, (float2 *)out_c, nrhs, (float)mg->mu_c, (float)mg->eps_c,
        (float)odd_shift_s);
    TMND_CUDA_TRY(cudaGetLastError());
    return TMND_OK;
}

// reads and clears the tensor-core timeout flag (synchronous)
tmnd_status tmnd_mg_tc_status(const tmnd_mg *mg) {
    TMND_ARG_CHECK(mg, "tmnd_mg_status: NULL handle");
    int h = 0;
    TMND_CUDA_TRY(cudaMemcpy(&h, mg->tc_err, sizeof(int), cudaMemcpyDeviceToHost));
    if (h) {
        cudaMemset(mg->tc_err, 0, sizeof(int));
        tmnd_set_error("mg_coarse_apply: a tensor-core kernel timed out waiting for its MMAs");
        return TMND_ERR_TIMEOUT;
    }
    return TMND_OK;
}

extern "C" tmnd_status tmnd_mg_export(const tmnd_mg *mg, void *P_host, void *Dc_host, void *Godd_host) {
    TMND_ARG_CHECK(mg, "tmnd_mg_export: NULL handle");
    const int n2 = 2 * mg->nv;
    if (P_host)
        TMND_CUDA_TRY(cudaMemcpy(P_host, mg->P, sizeof(float2) * (size_t)mg->nblock * 2 * mg->nv * mg->nsb * 6,
                                 cudaMemcpyDeviceToHost));
    if (Dc_host)
        TMND_CUDA_TRY(cudaMemcpy(Dc_host, mg->Dc, sizeof(float2) * (size_t)mg->nblock * 9 * n2 * n2,
                                 cudaMemcpyDeviceToHost));
    if (Godd_host)
        TMND_CUDA_TRY(cudaMemcpy(Godd_host, mg->Godd, sizeof(float2) * (size_t)mg->nblock * n2 * n2,
                                 cudaMemcpyDeviceToHost));
    return TMND_OK;
}

extern "C" tmnd_status tmnd_mg_status(const tmnd_mg *mg) { return tmnd_mg_tc_status(mg); }

// accessors for the solver translation unit
size_t tmnd_mg_nblock_nv(const tmnd_mg *mg, int *nv) {
    *nv = mg->nv;
    return (size_t)mg->nblock;
}
tmnd_gauge *tmnd_mg_gauge(const tmnd_mg *mg) { return mg->g; }
void tmnd_mg_smoother(const tmnd_mg *mg, int *kind, int *mr, int bd[4]) {
    *kind = mg->smoother;
    *mr = mg->sap_mr;
    for (int i = 0; i < 4; i++) bd[i] = mg->bd[i];
}
extern "C" tmnd_status tmnd_mg_coarse_apply_internal(const tmnd_mg *mg, float2 *out, const float2 *in, double s,
                                                     cudaStream_t st) {
    return mg_coarse_apply(mg, out, in, 1, s, st);
}
