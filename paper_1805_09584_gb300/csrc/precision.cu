// Precision conversions of internal spinors and the 16-bit link packing.
//   TMND_F64 : 24 planes of complex128 over V/2 sites
//   TMND_F32 : 24 planes of complex64
//   TMND_S16 : blocks of 8 sites, each 6 int4 planes (16-bit fixed point, one
//              word per complex component) + the 8 float scales (tmnd_internal.cuh)
#include <math.h>

#include "tmnd_internal.cuh"

namespace {

constexpr float QMAX = S16_QMAX;

// one site at a time: read 24 complex numbers as floats
template <int SRC>
__device__ __forceinline__ void read_site(const void *src, int Vh, int h, float v[24][2]) {
    if (SRC == TMND_F64) {
        const double2 *s = (const double2 *)src;
#pragma unroll
        for (int c = 0; c < 24; c++) {
            const double2 d = s[(size_t)c * Vh + h];
            v[c][0] = (float)d.x;
            v[c][1] = (float)d.y;
        }
    } else if (SRC == TMND_F32) {
        const float2 *s = (const float2 *)src;
#pragma unroll
        for (int c = 0; c < 24; c++) {
            const float2 d = s[(size_t)c * Vh + h];
            v[c][0] = d.x;
            v[c][1] = d.y;
        }
    } else {
        const S16In s = s16_in(src, Vh);
        const float sc = s.nrm[s16_ni(h)];
#pragma unroll
        for (int j = 0; j < 6; j++) {
            const int4 w = s.q[s16_qi(j, h)];
            const int ws[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
            for (int k = 0; k < 4; k++) {
                v[4 * j + k][0] = s16_lo(ws[k]) * sc;
                v[4 * j + k][1] = s16_hi(ws[k]) * sc;
            }
        }
    }
}

// S16 -> F64 keeps the exact dequantised values (scale applied in FP64)
__global__ void k_s16_to_f64(int Vh, int nrhs, const char *src, char *dst) {
    const size_t sb = S16_BYTES_PER_SITE * (size_t)Vh, db = sizeof(double2) * 24 * (size_t)Vh;
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < (long)Vh * nrhs; i += (long)gridDim.x * blockDim.x) {
        const int k = (int)(i / Vh), h = (int)(i % Vh);
        const S16In s = s16_in(src + k * sb, Vh);
        double2 *d = (double2 *)(dst + k * db);
        const double sc = s.nrm[s16_ni(h)];
        for (int j = 0; j < 6; j++) {
            const int4 w = s.q[s16_qi(j, h)];
            const int ws[4] = {w.x, w.y, w.z, w.w};
            for (int m = 0; m < 4; m++)
                d[(size_t)(4 * j + m) * Vh + h] = make_double2((double)s16_int_lo(ws[m]) * sc, (double)s16_int_hi(ws[m]) * sc);
        }
    }
}

template <int SRC>
__global__ void k_to_s16(int Vh, int nrhs, const char *src, size_t src_rhs_bytes, char *dst) {
    const size_t db = S16_BYTES_PER_SITE * (size_t)Vh;
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < (long)Vh * nrhs; i += (long)gridDim.x * blockDim.x) {
        const int k = (int)(i / Vh), h = (int)(i % Vh);
        float v[24][2];
        read_site<SRC>(src + k * src_rhs_bytes, Vh, h, v);
        float m = 0.0f;
        for (int c = 0; c < 24; c++) m = fmaxf(m, fmaxf(fabsf(v[c][0]), fabsf(v[c][1])));
        const float sc = m > 0.0f ? QMAX / m : 0.0f;
        S16Out o = s16_out(dst + k * db, Vh);
        o.nrm[s16_ni(h)] = m / QMAX;
        for (int j = 0; j < 6; j++) {
            int w[4];
            for (int q = 0; q < 4; q++) w[q] = s16_pack_fma(v[4 * j + q][0], v[4 * j + q][1], sc);
            o.q[s16_qi(j, h)] = make_int4(w[0], w[1], w[2], w[3]);
        }
    }
}

__global__ void k_f64_to_f32(long n, const double2 *src, float2 *dst) {
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
        dst[i] = make_float2((float)src[i].x, (float)src[i].y);
}
__global__ void k_f32_to_f64(long n, const float2 *src, double2 *dst) {
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
        dst[i] = make_double2(src[i].x, src[i].y);
}

// links: canonical complex128 [4][T][X][Y][Z][3][3] -> int2 [2 parity][4 mu][3 Vh]
// (per parity and direction blocks of 8 sites x 3 planes, s16_li), rows 0 and 1
// rounded to integers at scale 32767, stored in the 16-bit word codec
__global__ void k_pack_links_s16(Geom g, const double2 *__restrict__ canon, int2 *__restrict__ out) {
    const long V = 2L * g.Vh;
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;  // over 4 * V links
    if (i >= 4 * V) return;
    const long lex = i % V;
    const int mu = (int)(i / V);
    long r = lex;
    const int z = (int)(r % g.Z); r /= g.Z;
    const int y = (int)(r % g.Y); r /= g.Y;
    const int x = (int)(r % g.X);
    const int t = (int)(r / g.X);
    const int par = (t + x + y + z) & 1;
    const long h = lex >> 1;
    const double2 *u = canon + i * 9;
    int w[6];
    for (int k = 0; k < 6; k++) {
        w[k] = s16_word((int)rint(u[k].x * 32767.0), (int)rint(u[k].y * 32767.0));
    }
    int2 *o = out + ((size_t)par * 4 + mu) * 3 * g.Vh;
    o[s16_li(0, h)] = make_int2(w[0], w[1]);
    o[s16_li(1, h)] = make_int2(w[2], w[3]);
    o[s16_li(2, h)] = make_int2(w[4], w[5]);
}

int grid_for(long n) {
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    long want = (n + 255) / 256, cap = (long)sms * 8;
    return (int)(want < cap ? want : cap);
}

}  // namespace

void launch_pack_links_s16(const Geom &g, const double2 *canon, int2 *out, cudaStream_t s) {
    const long n = 4L * 2 * g.Vh;
    k_pack_links_s16<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(g, canon, out);
}

size_t spinor_bytes_prec(int Vh, int prec) {
    switch (prec) {
        case TMND_F64: return sizeof(double2) * 24 * (size_t)Vh;
        case TMND_F32: return sizeof(float2) * 24 * (size_t)Vh;
        case TMND_S16: return S16_BYTES_PER_SITE * (size_t)Vh;
    }
    return 0;
}

tmnd_status convert_spinor(int Vh, void *dst, int dst_prec, const void *src, int src_prec, int nrhs,
                           cudaStream_t s) {
    const long nsite = (long)Vh * nrhs;
    const long nel = 24L * nsite;
    if (dst_prec == src_prec) {
        TMND_CUDA_TRY(cudaMemcpyAsync(dst, src, spinor_bytes_prec(Vh, src_prec) * nrhs, cudaMemcpyDeviceToDevice, s));
        return TMND_OK;
    }
    if (dst_prec == TMND_S16) {
        const size_t sb = spinor_bytes_prec(Vh, src_prec);
        if (src_prec == TMND_F64)
            k_to_s16<TMND_F64><<<grid_for(nsite), 256, 0, s>>>(Vh, nrhs, (const char *)src, sb, (char *)dst);
        else
            k_to_s16<TMND_F32><<<grid_for(nsite), 256, 0, s>>>(Vh, nrhs, (const char *)src, sb, (char *)dst);
    } else if (src_prec == TMND_S16 && dst_prec == TMND_F64) {
        k_s16_to_f64<<<grid_for(nsite), 256, 0, s>>>(Vh, nrhs, (const char *)src, (char *)dst);
    } else if (src_prec == TMND_F64 && dst_prec == TMND_F32) {
        k_f64_to_f32<<<grid_for(nel), 256, 0, s>>>(nel, (const double2 *)src, (float2 *)dst);
    } else if (src_prec == TMND_F32 && dst_prec == TMND_F64) {
        k_f32_to_f64<<<grid_for(nel), 256, 0, s>>>(nel, (const float2 *)src, (double2 *)dst);
    } else {
        tmnd_set_error("tmnd_spinor_convert: conversion %d -> %d not supported", src_prec, dst_prec);
        return TMND_ERR_ARG;
    }
    TMND_CUDA_TRY(cudaGetLastError());
    return TMND_OK;
}

extern "C" size_t tmnd_spinor_bytes_prec(const tmnd_gauge *g, int prec) {
    return g ? spinor_bytes_prec(g->geom.Vh, prec) : 0;
}

extern "C" tmnd_status tmnd_spinor_convert(const tmnd_gauge *g, void *dst, int dst_prec, const void *src,
                                           int src_prec, int nrhs, void *stream) {
    TMND_ARG_CHECK(g && dst && src, "tmnd_spinor_convert: NULL argument");
    TMND_ARG_CHECK(dst != src, "tmnd_spinor_convert: dst and src must not alias");
    TMND_ARG_CHECK(nrhs >= 1, "tmnd_spinor_convert: nrhs = %d", nrhs);
    TMND_ARG_CHECK(dst_prec >= TMND_F64 && dst_prec <= TMND_S16 && src_prec >= TMND_F64 && src_prec <= TMND_S16,
                   "tmnd_spinor_convert: unknown precision");
    TMND_ARG_CHECK(((uintptr_t)dst & 15) == 0 && ((uintptr_t)src & 15) == 0,
                   "tmnd_spinor_convert: pointers must be 16-byte aligned");
    cudaGetLastError();
    return convert_spinor(g->geom.Vh, dst, dst_prec, src, src_prec, nrhs, (cudaStream_t)stream);
}
