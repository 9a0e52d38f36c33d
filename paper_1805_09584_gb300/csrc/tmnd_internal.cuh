// Internal definitions shared by the libtmnd translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <string>

#include "tmnd.h"

// ------------------------------------------------------------------ errors
void tmnd_set_error(const char *fmt, ...);

#define TMND_CUDA_TRY(call)                                                              \
    do {                                                                                 \
        cudaError_t e_ = (call);                                                         \
        if (e_ != cudaSuccess) {                                                         \
            tmnd_set_error("%s:%d: %s: %s", __FILE__, __LINE__, #call, cudaGetErrorString(e_)); \
            return (e_ == cudaErrorMemoryAllocation) ? TMND_ERR_OOM : TMND_ERR_CUDA;     \
        }                                                                                \
    } while (0)

#define TMND_ARG_CHECK(cond, ...)                  \
    do {                                           \
        if (!(cond)) {                             \
            tmnd_set_error(__VA_ARGS__);           \
            return TMND_ERR_ARG;                   \
        }                                          \
    } while (0)

// ---------------------------------------------------------------- geometry
// Lattice geometry for the even-odd layout.  Half-index h of site (t,x,y,z)
// is lex >> 1 with lex = ((t*X + x)*Y + y)*Z + z; Zh = Z/2.
struct Geom {
    int T, X, Y, Z, Zh;
    int Vh;        // V/2
    int apbc;      // antiperiodic time boundary
};

// Parameters of the site-diagonal term A = 1 + i kp g5 tau3 - kpp tau1 (hopping form):
// kp = 2 kappa mu_bar, kpp = 2 kappa eps_bar; A^-1 = [[1 - i kp g, kpp],[kpp, 1 + i kp g]] / det,
// det = 1 + kp^2 - kpp^2 for gamma_5 eigenvalue g.
struct SiteTerm {
    double kappa2;  // kappa^2, folded into A^-1 in the even-site kernel
    double kp;      // 2 kappa mu_bar
    double kpp;     // 2 kappa eps_bar
    double inv_det; // 1 / (1 + kp^2 - kpp^2)
};

// Site term in FP32 for the sloppy kernels.
struct SiteTermF {
    float kappa2, kp, kpp, inv_det;
};

// Gauge handle.
struct tmnd_gauge {
    tmnd_action act;
    int prec;
    int device;
    Geom geom;
    SiteTerm st;
    double2 *links;        // [2 parity][4 mu][9][Vh] complex, U_mu(x) stored at the parity/half-index of x
    float2 *links_f32;     // the same in FP32 (the FP32 operator)
    int2 *links_s16;       // [2 parity][4 mu][3][Vh]: rows 0, 1 as int16 pairs (scale 32767)
    SiteTermF stf;         // FP32 copy of st for the sloppy kernels
    void *work;            // grow-only workspace
    size_t work_bytes;
    double2 *partials;     // reduction partials (grow-only, separate from work)
    size_t partials_bytes;
};

tmnd_status tmnd_ensure_workspace(tmnd_gauge *g, size_t bytes);
tmnd_status tmnd_ensure_partials(tmnd_gauge *g, size_t bytes);

// Number of complex numbers per site of a doublet spinor.
constexpr int NCOMP = 24;

// --------------------------------------------------------- device helpers
__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
// i * a
__device__ __forceinline__ double2 cmuli(double2 a) { return make_double2(-a.y, a.x); }
// -i * a
__device__ __forceinline__ double2 cmulmi(double2 a) { return make_double2(a.y, -a.x); }
__device__ __forceinline__ double2 cneg(double2 a) { return make_double2(-a.x, -a.y); }
// acc + a*b
__device__ __forceinline__ double2 cfma(double2 a, double2 b, double2 acc) {
    return make_double2(fma(a.x, b.x, fma(-a.y, b.y, acc.x)), fma(a.x, b.y, fma(a.y, b.x, acc.y)));
}
// a*b
__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
    return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
// acc + conj(a)*b
__device__ __forceinline__ double2 cfma_conj(double2 a, double2 b, double2 acc) {
    return make_double2(fma(a.x, b.x, fma(a.y, b.y, acc.x)), fma(a.x, b.y, fma(-a.y, b.x, acc.y)));
}
// conj(a)*b
__device__ __forceinline__ double2 cmul_conj(double2 a, double2 b) {
    return make_double2(fma(a.x, b.x, a.y * b.y), fma(a.x, b.y, -a.y * b.x));
}
// Flip the sign of a double without touching the FP64 pipe (integer XOR of the sign bit).
__device__ __forceinline__ double dflip(double v, unsigned long long mask) {
    return __longlong_as_double(__double_as_longlong(v) ^ (long long)mask);
}
__device__ __forceinline__ double2 cflip(double2 a, unsigned long long mask) {
    return make_double2(dflip(a.x, mask), dflip(a.y, mask));
}

// The same complex helpers in FP32 (the FP32 instantiation of the FP64 stencil).
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmuli(float2 a) { return make_float2(-a.y, a.x); }
__device__ __forceinline__ float2 cmulmi(float2 a) { return make_float2(a.y, -a.x); }
__device__ __forceinline__ float2 cneg(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float2 cfma(float2 a, float2 b, float2 acc) {
    return make_float2(fmaf(a.x, b.x, fmaf(-a.y, b.y, acc.x)), fmaf(a.x, b.y, fmaf(a.y, b.x, acc.y)));
}
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 cfma_conj(float2 a, float2 b, float2 acc) {
    return make_float2(fmaf(a.x, b.x, fmaf(a.y, b.y, acc.x)), fmaf(a.x, b.y, fmaf(-a.y, b.x, acc.y)));
}
__device__ __forceinline__ float2 cmul_conj(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.x, b.y, -a.y * b.x));
}
__device__ __forceinline__ float2 cflip(float2 a, unsigned long long mask) {
    const int m = mask ? (int)0x80000000 : 0;
    return make_float2(__int_as_float(__float_as_int(a.x) ^ m), __int_as_float(__float_as_int(a.y) ^ m));
}

// Block-wide sum of one double (blockDim.x a multiple of 32, <= 1024); result valid in thread 0.
__device__ __forceinline__ double block_sum(double v, double *smem /* >= 32 */) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) smem[wid] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0) {
        int nw = blockDim.x >> 5;
        for (int i = 0; i < nw; i++) s += smem[i];
    }
    return s;
}

// Deterministic sum of n partials, computed by a whole block (fixed order,
// same result in every block); result returned to all threads.
__device__ __forceinline__ double block_reduce_partials(const double *p, int n, double *smem) {
    double v = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) v += p[i];
    double s = block_sum(v, smem);
    __syncthreads();
    if (threadIdx.x == 0) smem[32] = s;
    __syncthreads();
    double r = smem[32];
    __syncthreads();
    return r;
}

// --------------------------------------------------------- launch helpers
// Hop kernels (tm_nd_apply and the solver share these launchers).
enum HopEpi {
    EPI_STORE = 0,        // out = y
    EPI_STORE_NORMS = 1,  // out = y; partials |y|^2, |in|^2
    EPI_SHIFT = 2,        // out = y + sigma * aux
    EPI_MMS_R = 3         // w = y + sigma * aux; r -= alpha w; partial |r|^2  (alpha from partials)
};

constexpr int HOP_THREADS = 128;

template <typename C2>
struct HopEpiT {
    double sigma;
    const C2 *aux;          // EPI_SHIFT / EPI_MMS_R: the vector multiplied by sigma
    C2 *r;                  // EPI_MMS_R: updated residual (written)
    const C2 *r_in;         // EPI_MMS_R: residual before the update (NULL: update r in place)
    double *part_out;       // partial sums written per block (EPI_STORE_NORMS: 2 per block; EPI_MMS_R: 1)
    const double *part_in;  // EPI_MMS_R: partials of |y|^2, |p|^2 from the previous kernel
    int npart_in;           // number of blocks that wrote part_in
    const double *rr;       // EPI_MMS_R: (r,r) before the update (device scalar)
    const int *done;        // if non-null and *done != 0 the kernel returns immediately
};
using HopEpiArgs = HopEpiT<double2>;
using HopEpiArgsF = HopEpiT<float2>;

// even-site kernel: t_e = kappa^2 A^-1 H_eo psi_o   (dag: kappa^2 A(-mu)^-1 H_eo gamma_5 psi_o)
void launch_hop_even_f64(const Geom &g, const SiteTerm &st, const double2 *links, const double2 *psi_o,
                         double2 *t_e, bool dag, const int *done, cudaStream_t s);
// odd-site kernel: y_o = A psi_o - H_oe t_e   (dag: A(-mu) psi_o - gamma_5 H_oe t_e), with epilogue
void launch_hop_odd_f64(const Geom &g, const SiteTerm &st, const double2 *links, const double2 *psi_o,
                        const double2 *t_e, double2 *y_o, bool dag, HopEpi epi, const HopEpiArgs &ea,
                        cudaStream_t s);
// Number of blocks (= reduction partials) of every hop launch for this geometry.
int hop_blocks(const Geom &g);
// The same stencil in FP32 on FP32 planes with 18-real FP32 links (the FP32 operator:
// accurate to ~1e-7, used for inner residuals of the defect correction)
void launch_hop_even_f32(const Geom &g, const SiteTerm &st, const float2 *links, const float2 *psi_o, float2 *t_e,
                         bool dag, const int *done, cudaStream_t s);
void launch_hop_odd_f32(const Geom &g, const SiteTerm &st, const float2 *links, const float2 *psi_o,
                        const float2 *t_e, float2 *y_o, bool dag, HopEpi epi, const HopEpiArgsF &ea, cudaStream_t s);
int hop_blocks_f32(const Geom &g);

// ------------------------------------------------- sloppy (16-bit) path

// 16-bit spinor of one right-hand side, in blocks of 8 consecutive half-lattice
// sites (V/2 is a multiple of 8 for even extents): a block is 800 bytes, 6 planes
// of 8 int4 words (plane j of site h: complex components 4j..4j+3, one 32-bit
// word each), then the 8 sites' float scales.  A run of consecutive sites that
// starts and ends on block boundaries is one contiguous byte range.  q and nrm
// hold the same base address, typed for the two kinds of element.
struct S16In {
    const int4 *q;
    const float *nrm;
};
struct S16Out {
    int4 *q;
    float *nrm;
};
constexpr size_t S16_BYTES_PER_SITE = 6 * 16 + 4;
constexpr int S16_BLOCK_SITES = 8;
// int4 index of plane p of site h, float index of the scale of site h
__host__ __device__ inline size_t s16_qi(int p, size_t h) { return (h >> 3) * 50 + (size_t)p * 8 + (h & 7); }
__host__ __device__ inline size_t s16_ni(size_t h) { return (h >> 3) * 200 + 192 + (h & 7); }
// 16-bit links of one (parity, direction), blocks of 8 sites: int2 index of plane j
// (row-0/row-1 word pair j) of site h; a block is 192 bytes
__host__ __device__ inline size_t s16_li(int j, size_t h) { return (h >> 3) * 24 + (size_t)j * 8 + (h & 7); }
__host__ __device__ inline S16In s16_in(const void *base, int Vh) {
    (void)Vh;
    return S16In{(const int4 *)base, (const float *)base};
}
__host__ __device__ inline S16Out s16_out(void *base, int Vh) {
    (void)Vh;
    return S16Out{(int4 *)base, (float *)base};
}

constexpr int TMND_MAX_BATCH = 16;
struct S16EpiArgs {
    double sigma;
    // EPI_MMS_R with per_rhs_sigma: right-hand side k uses sigma_k[k] instead of sigma
    int per_rhs_sigma;
    double sigma_k[TMND_MAX_BATCH];
    S16In aux;              // EPI_SHIFT / EPI_MMS_R: vector multiplied by sigma
    float2 *r;              // EPI_MMS_R: updated residual (FP32 planes, written)
    const float2 *r_in;     // EPI_MMS_R: residual before the update
    double *part_out;       // block partials: EPI_STORE_NORMS [rhs][2][grid], EPI_MMS_R [rhs][grid]
    const double *part_in;  // EPI_MMS_R: the previous launch's [rhs][2][npart_in]
    int npart_in;
    const double *rr;       // EPI_MMS_R: (r, r) of right-hand side k at rr[k * rr_stride]
    const int *done;
    long r_stride;          // EPI_MMS_R: float2 elements between right-hand sides of r / r_in
    int rr_stride;          // doubles between right-hand sides of rr
};

// Several right-hand sides in one stencil launch (links read once, shared in cache):
// right-hand side k of every 16-bit vector argument starts k * stride bytes after
// the first; k is skipped while rdone[k * rdone_stride] is set (rdone may be NULL).
struct S16Batch {
    int nrhs = 1;
    size_t stride = 0;
    const int *rdone = nullptr;
    int rdone_stride = 0;
    int shape = -1;  // launch variant (dslash_s16.cu); -1: the autotuner's choice for (lattice, nrhs)
    int order = 0;   // set by the launchers from the variant: 0 sites of the block's chunk outside the
                     // right-hand sides, 1 right-hand sides outside the chunk, 2 grid-stride sites outside,
                     // 3 grid stride over (32-site group, right-hand side), one per warp
};

// launch shapes of the 16-bit stencil and their autotuner (dslash_s16.cu)
int hop_blocks_s16(const Geom &g, int shape);
int hop_blocks_s16_max(const Geom &g);
int s16_shape(const Geom &g, int nrhs);      // variant for operator applications
int s16_shape_mms(const Geom &g, int nrhs);  // variant for sloppy multi-shift iterations
// objective 0: operator applications, 1: sloppy multi-shift iterations (both tuned together)
tmnd_status s16_autotune(tmnd_gauge *g, int nrhs, cudaStream_t s, int *shape_out, float *ms_out, int objective = 0);
void launch_hop_even_s16(const Geom &g, const SiteTermF &st, const int2 *links, S16In in, S16Out out, bool dag,
                         const int *done, cudaStream_t s, const S16Batch &bt = S16Batch());
void launch_hop_odd_s16(const Geom &g, const SiteTermF &st, const int2 *links, S16In psi, S16In te, S16Out out,
                        bool dag, HopEpi epi, const S16EpiArgs &ea, cudaStream_t s,
                        const S16Batch &bt = S16Batch());

void launch_pack_links_s16(const Geom &g, const double2 *canon, int2 *out, cudaStream_t s);
size_t spinor_bytes_prec(int Vh, int prec);
tmnd_status convert_spinor(int Vh, void *dst, int dst_prec, const void *src, int src_prec, int nrhs,
                           cudaStream_t s);

// 16-bit word codec shared by every kernel that reads or writes 16-bit data.
// One 32-bit word holds one complex number: the real part in the low 16 bits,
// the imaginary part in the high 16 bits, each an integer n in [-32767, 32767]
// stored biased as n + 32768.  Encoding: fmaf(x, scale, S16_ENC_MAGIC) leaves
// n + 32768 in the low 16 bits of the float's bits (1.5*2^23 + 32768 + n lies in
// [2^23, 2^24), where floats are the integers).  Decoding: one byte permute puts
// the field under the exponent of 2^23, giving the float 2^23 + n + 32768 exactly
// (S16_DEC_BIAS + n); differences of two such floats are exact integers.
constexpr float S16_QMAX = 32767.0f;
constexpr float S16_ENC_MAGIC = 12615680.0f;  // 1.5 * 2^23 + 32768
constexpr float S16_DEC_BIAS = 8421376.0f;    // 2^23 + 32768
__device__ __forceinline__ float s16_flo(int w) { return __int_as_float(__byte_perm(w, 0x4B000000, 0x7410)); }
__device__ __forceinline__ float s16_fhi(int w) { return __int_as_float(__byte_perm(w, 0x4B000000, 0x7432)); }
__device__ __forceinline__ float s16_lo(int w) { return s16_flo(w) - S16_DEC_BIAS; }
__device__ __forceinline__ float s16_hi(int w) { return s16_fhi(w) - S16_DEC_BIAS; }
// pack two values already multiplied by their scale (|x| <= 32767)
__device__ __forceinline__ int s16_pack(float re_scaled, float im_scaled) {
    return __byte_perm(__float_as_int(re_scaled + S16_ENC_MAGIC), __float_as_int(im_scaled + S16_ENC_MAGIC), 0x5410);
}
__device__ __forceinline__ int s16_pack_fma(float re, float im, float sc) {
    return __byte_perm(__float_as_int(fmaf(re, sc, S16_ENC_MAGIC)), __float_as_int(fmaf(im, sc, S16_ENC_MAGIC)), 0x5410);
}
// integer fields, for exact FP64 decoding
__host__ __device__ inline int s16_int_lo(int w) { return (int)((unsigned)w & 0xffffu) - 32768; }
__host__ __device__ inline int s16_int_hi(int w) { return (int)((unsigned)w >> 16) - 32768; }
__host__ __device__ inline int s16_word(int re, int im) {
    return (int)(((unsigned)(re + 32768) & 0xffffu) | ((unsigned)(im + 32768) << 16));
}

// Site-level 16-bit (de)quantisation shared by the sloppy solver kernels.
// v[c][0/1] = real/imaginary part of component c = flavour*12 + spin*3 + colour.
__device__ __forceinline__ void s16_load_site(S16In in, int Vh, int h, float v[24][2]) {
    const float sc = in.nrm[s16_ni(h)];
#pragma unroll
    for (int j = 0; j < 6; j++) {
        const int4 w = in.q[s16_qi(j, h)];
        const int ws[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
        for (int k = 0; k < 4; k++) {
            v[4 * j + k][0] = s16_lo(ws[k]) * sc;
            v[4 * j + k][1] = s16_hi(ws[k]) * sc;
        }
    }
}

__device__ __forceinline__ void s16_store_site(S16Out out, int Vh, int h, const float v[24][2]) {
    float m = 0.0f;
#pragma unroll
    for (int c = 0; c < 24; c++) m = fmaxf(m, fmaxf(fabsf(v[c][0]), fabsf(v[c][1])));
    const float sc = m > 0.0f ? S16_QMAX / m : 0.0f;
    out.nrm[s16_ni(h)] = m * (1.0f / S16_QMAX);
#pragma unroll
    for (int j = 0; j < 6; j++) {
        int w[4];
#pragma unroll
        for (int k = 0; k < 4; k++) w[k] = s16_pack_fma(v[4 * j + k][0], v[4 * j + k][1], sc);
        out.q[s16_qi(j, h)] = make_int4(w[0], w[1], w[2], w[3]);
    }
}
