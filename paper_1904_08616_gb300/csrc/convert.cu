// Field re-encoding between precisions, link formats and layouts (the pack/convert
// step: the paper streams links in a reduced form prepared beforehand, Section 2.2).
// One thread per site; formats are the ones documented in include/lq.h.
#include "lq_abi_internal.h"
#include "dslash_kernels.cuh"

namespace lq {

namespace {

constexpr int kConvBS = 256;

// LQ_F64X fields use the LQ_F64 slots with each double replaced by a float pair
__host__ __device__ inline int base_prec(int prec) { return prec == LQ_F64X ? LQ_F64 : prec; }
__host__ __device__ inline int spinor_chunk(int prec) {
    prec = base_prec(prec);
    return prec == LQ_F64 ? 2 : (prec == LQ_F16S ? 8 : 4);
}
__host__ __device__ inline int link_chunk(int prec, int fmt) {
    prec = base_prec(prec);
    return fmt == 18 ? 2 : (prec == LQ_F64 ? 2 : 4);
}

struct FieldDesc {
    void* ptr;
    int prec, layout, fmt;
};

// element index of real j of a spinor site of right-hand side s.rhs among nr (LEX: nr
// stacked complete fields; EO: right-hand sides interleaved per chunk slot).  A stacked
// scaled field is its 24 V elements followed by its V float scales: 26 V halves (F16S)
// or 25 V 4-byte words (I32S) per field.
__device__ inline int64_t sp_elem(const FieldDesc& f, const Geom& g, const Site& s, int j, int nr) {
    if (f.layout == LQ_LAYOUT_LEX) {
        const int64_t field = (f.prec == LQ_F16S ? 26 : (f.prec == LQ_I32S ? 25 : 24)) * (int64_t)g.V;
        return s.rhs * field + (int64_t)s.lex * 24 + j;
    }
    const int w = spinor_chunk(f.prec), K = 24 / w;
    return ((((int64_t)s.p * K + j / w) * g.Vh + s.cb) * nr + s.rhs) * w + (j % w);
}
// index (in floats from the buffer start) of the scale of a site of a scaled field
__device__ inline int64_t sp_scale_idx(const FieldDesc& f, const Geom& g, const Site& s, int nr) {
    if (f.prec == LQ_I32S) {
        if (f.layout == LQ_LAYOUT_LEX) return 25 * (int64_t)g.V * s.rhs + 24 * (int64_t)g.V + s.lex;
        return 24 * (int64_t)g.V * nr + ((int64_t)s.p * g.Vh + s.cb) * nr + s.rhs;
    }
    if (f.layout == LQ_LAYOUT_LEX) return 13 * (int64_t)g.V * s.rhs + 12 * (int64_t)g.V + s.lex;
    return 12 * (int64_t)g.V * nr + ((int64_t)s.p * g.Vh + s.cb) * nr + s.rhs;
}
// element index of real j of link (s, mu)
__device__ inline int64_t lk_elem(const FieldDesc& f, const Geom& g, const Site& s, int mu, int j) {
    if (f.layout == LQ_LAYOUT_LEX) return ((int64_t)s.lex * 4 + mu) * f.fmt + j;
    const int w = link_chunk(f.prec, f.fmt), K = f.fmt / w;
    return ((((int64_t)mu * 2 + s.p) * K + j / w) * g.Vh + s.cb) * w + (j % w);
}

__device__ inline double load_real(const void* base, int prec, int64_t i) {
    if (prec == LQ_F64) return ((const double*)base)[i];
    if (prec == LQ_F64X) return (double)((const float*)base)[2 * i] + (double)((const float*)base)[2 * i + 1];
    if (prec == LQ_F32) return (double)((const float*)base)[i];
    if (prec == LQ_I32S) return (double)((const int*)base)[i];      // the integer; callers scale it
    return (double)__half2float(((const __half*)base)[i]);
}

// F64 or F64X target
__device__ inline void store_wide(void* base, int prec, int64_t i, double v) {
    if (prec == LQ_F64) {
        ((double*)base)[i] = v;
    } else {
        const dd p = dd_from_double(v);
        ((float*)base)[2 * i] = p.hi;
        ((float*)base)[2 * i + 1] = p.lo;
    }
}

__global__ void __launch_bounds__(kConvBS) convert_spinor_kernel(Geom g, FieldDesc src, FieldDesc dst, int nr) {
    const int64_t n = (int64_t)g.V * nr;
    for (int64_t f = blockIdx.x * (int64_t)kConvBS + threadIdx.x; f < n; f += (int64_t)gridDim.x * kConvBS) {
        int c[4];
        const Site s = site_from_lex(g, (int)(f / nr), c, (int)(f % nr));
        double v[24];
        double sc = 1.0;
        if (src.prec == LQ_F16S)
            sc = (double)((const float*)src.ptr)[sp_scale_idx(src, g, s, nr)];
        else if (src.prec == LQ_I32S)
            sc = (double)((const float*)src.ptr)[sp_scale_idx(src, g, s, nr)] * 0x1p-30;
#pragma unroll
        for (int j = 0; j < 24; ++j) v[j] = load_real(src.ptr, src.prec, sp_elem(src, g, s, j, nr)) * sc;
        if (dst.prec == LQ_F64 || dst.prec == LQ_F64X) {
#pragma unroll
            for (int j = 0; j < 24; ++j) store_wide(dst.ptr, dst.prec, sp_elem(dst, g, s, j, nr), v[j]);
        } else if (dst.prec == LQ_F32) {
#pragma unroll
            for (int j = 0; j < 24; ++j) ((float*)dst.ptr)[sp_elem(dst, g, s, j, nr)] = (float)v[j];
        } else if (dst.prec == LQ_I32S) {
            // s = max |fl32(v)|, q = RN(v / s * 2^30) in FP64, ties to even
            float m = 0.f;
#pragma unroll
            for (int j = 0; j < 24; ++j) m = fmaxf(m, fabsf((float)v[j]));
            ((float*)dst.ptr)[sp_scale_idx(dst, g, s, nr)] = m;
            const bool z = !(m > 0.f);
#pragma unroll
            for (int j = 0; j < 24; ++j)
                ((int*)dst.ptr)[sp_elem(dst, g, s, j, nr)] = z ? 0 : __double2int_rn(v[j] / (double)m * 0x1p30);
        } else {
            float fv[24];
            float m = 0.f;
#pragma unroll
            for (int j = 0; j < 24; ++j) { fv[j] = (float)v[j]; m = fmaxf(m, fabsf(fv[j])); }
            ((float*)dst.ptr)[sp_scale_idx(dst, g, s, nr)] = m;
            const bool z = !(m > 0.f);
#pragma unroll
            for (int j = 0; j < 24; ++j)
                ((__half*)dst.ptr)[sp_elem(dst, g, s, j, nr)] = __float2half_rn(z ? 0.f : __fdiv_rn(fv[j], m));
        }
    }
}

__global__ void __launch_bounds__(kConvBS) convert_gauge_kernel(Geom g, FieldDesc src, FieldDesc dst) {
    for (int lex = blockIdx.x * kConvBS + threadIdx.x; lex < g.V; lex += gridDim.x * kConvBS) {
        int c[4];
        const Site s = site_from_lex(g, lex, c);
        for (int mu = 0; mu < 4; ++mu) {
            for (int j = 0; j < dst.fmt; ++j) {
                double v = load_real(src.ptr, src.prec, lk_elem(src, g, s, mu, j));
                if (src.prec == LQ_I32S) v *= 0x1p-30;
                const int64_t i = lk_elem(dst, g, s, mu, j);
                if (dst.prec == LQ_F64 || dst.prec == LQ_F64X) store_wide(dst.ptr, dst.prec, i, v);
                else if (dst.prec == LQ_F32) ((float*)dst.ptr)[i] = (float)v;
                else if (dst.prec == LQ_I32S) ((int*)dst.ptr)[i] = __double2int_rn(v * 0x1p30);   // Q1.30
                else ((__half*)dst.ptr)[i] = __float2half_rn((float)v);
            }
        }
    }
}

int conv_grid(const Geom& g, int nr = 1) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    long long want = ((long long)g.V * nr + kConvBS - 1) / kConvBS;
    long long cap = (long long)sms * 8;
    return (int)(want < cap ? (want > 0 ? want : 1) : cap);
}

}  // namespace

cudaError_t convert_spinor(const Geom& g, int sp, int sl, const void* src, int dp, int dl, void* dst, cudaStream_t st,
                           int nr) {
    convert_spinor_kernel<<<conv_grid(g, nr), kConvBS, 0, st>>>(g, FieldDesc{(void*)src, sp, sl, 0},
                                                                FieldDesc{dst, dp, dl, 0}, nr);
    return cudaGetLastError();
}

cudaError_t convert_gauge(const Geom& g, int sp, int sl, const void* src, int dp, int dfmt, int dl, void* dst,
                          cudaStream_t st) {
    convert_gauge_kernel<<<conv_grid(g), kConvBS, 0, st>>>(g, FieldDesc{(void*)src, sp, sl, 18},
                                                           FieldDesc{dst, dp, dl, dfmt});
    return cudaGetLastError();
}

}  // namespace lq
