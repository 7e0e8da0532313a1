// Field re-encoding between precisions, link formats and layouts (the pack/convert
// step: the paper streams links in a reduced form prepared beforehand, Section 2.2).
// One thread per spinor site or per link; formats are the ones documented in include/lq.h.
#include "lq_abi_internal.h"
#include "dslash_kernels.cuh"

namespace lq {

namespace {

constexpr int kConvBS = 128;

// LQ_F64X fields use the LQ_F64 slots with each double replaced by a float pair
__host__ __device__ inline int base_prec(int prec) { return prec == LQ_F64X ? LQ_F64 : prec; }
__host__ __device__ inline int spinor_chunk(int prec) {
    prec = base_prec(prec);
    return prec == LQ_F64 ? 2 : (prec == LQ_F16S ? 8 : 4);
}
__host__ __device__ inline int link_chunk(int prec, int fmt) {
    prec = base_prec(prec);
    return (fmt == 18 || fmt == 10) ? 2 : (prec == LQ_F64 ? 2 : 4);
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

// x as an FP32 pair, hi = RN32(x) and lo = RN32(x - hi), from integer and FP32 operations:
// the FP64 conversions and subtraction of dd_from_double run on the FP64 units, which are a
// small fraction of the FP32 rate on this GPU and would bound the conversion.  The 53-bit
// significand is cut after 24 bits with round-to-nearest-even (a carry moves into the
// exponent field); the remainder r (|r| <= 2^28) is x - hi in units of 2^(E-52), and is rounded
// once to 24 bits by an FMA of its two exact 16-bit halves.  Values whose pair is not two
// normal floats (zero, |x| < 2^-74, |x| >= 2^127, subnormals, Inf, NaN) take the FP64 route.
__device__ inline dd split_double(double x) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const int E = (int)((b >> 52) & 0x7ffull) - 1023;
    if (E < -74 || E > 126) return dd_from_double(x);
    const unsigned long long M = (b & 0xfffffffffffffull) | (1ull << 52);
    unsigned int keep = (unsigned int)(M >> 29);
    int rem = (int)(M & 0x1fffffffull);
    if (rem > 0x10000000 || (rem == 0x10000000 && (keep & 1u))) {
        keep += 1u;
        rem -= 0x20000000;
    }
    const unsigned int sign = (unsigned int)(b >> 32) & 0x80000000u;
    const float hi = __uint_as_float(sign | (((unsigned int)(E + 127) << 23) + (keep - 0x800000u)));
    float lo = 0.f;
    if (rem != 0) {
        const unsigned int ar = rem < 0 ? (unsigned int)(-rem) : (unsigned int)rem;
        const float a = __fsub_rn(__uint_as_float(0x4B000000u | (ar >> 16)), 8388608.f);
        const float c = __fsub_rn(__uint_as_float(0x4B000000u | (ar & 0xffffu)), 8388608.f);
        const float mag = __fmaf_rn(a, 65536.f, c);
        const float scale = __uint_as_float((unsigned int)(E - 52 + 127) << 23);
        lo = __uint_as_float(__float_as_uint(__fmul_rn(mag, scale)) ^ sign ^ (rem < 0 ? 0x80000000u : 0u));
    }
    return dd{hi, lo};
}

// F64 or F64X target
__device__ inline void store_wide(void* base, int prec, int64_t i, double v) {
    if (prec == LQ_F64) {
        ((double*)base)[i] = v;
    } else {
        const dd p = split_double(v);
        ((float*)base)[2 * i] = p.hi;
        ((float*)base)[2 * i + 1] = p.lo;
    }
}

// FP64 LEX fields are read and written through a per-warp shared-memory tile, so that a
// warp moves contiguous 16-byte words; the other side of the conversion is addressed per
// site.  Stacked LEX fields are contiguous in the field-site index f = rhs V + lex.
__device__ inline bool wide_lex(const FieldDesc& f) { return f.prec == LQ_F64 && f.layout == LQ_LAYOUT_LEX; }

constexpr int kSpStride = 13;   // staged spinor: 12 double2 + 1 pad (conflict-free 16-byte reads)

// the 24 reals of a spinor site from a non-staged source (scale applied)
__device__ inline void load_site(const FieldDesc& src, const Geom& g, const Site& s, int nr, double v[24]) {
    if (src.prec == LQ_F64X && src.layout == LQ_LAYOUT_EO) {
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            const float4 q = ((const float4*)src.ptr)[sp_elem(src, g, s, 2 * k, nr) / 2];
            v[2 * k] = (double)q.x + (double)q.y;
            v[2 * k + 1] = (double)q.z + (double)q.w;
        }
        return;
    }
    double sc = 1.0;
    if (src.prec == LQ_F16S)
        sc = (double)((const float*)src.ptr)[sp_scale_idx(src, g, s, nr)];
    else if (src.prec == LQ_I32S)
        sc = (double)((const float*)src.ptr)[sp_scale_idx(src, g, s, nr)] * 0x1p-30;
#pragma unroll
    for (int j = 0; j < 24; ++j) v[j] = load_real(src.ptr, src.prec, sp_elem(src, g, s, j, nr)) * sc;
}

// the 24 reals of a spinor site to a non-staged destination
__device__ inline void store_site(const FieldDesc& dst, const Geom& g, const Site& s, int nr, const double v[24]) {
    if (dst.prec == LQ_F64X && dst.layout == LQ_LAYOUT_EO) {
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            const dd a = split_double(v[2 * k]), b = split_double(v[2 * k + 1]);
            ((float4*)dst.ptr)[sp_elem(dst, g, s, 2 * k, nr) / 2] = make_float4(a.hi, a.lo, b.hi, b.lo);
        }
    } else if (dst.prec == LQ_F64 || dst.prec == LQ_F64X) {
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

__global__ void __launch_bounds__(kConvBS) convert_spinor_kernel(Geom g, FieldDesc src, FieldDesc dst, int nr) {
    __shared__ double2 stage[kConvBS / 32][32 * kSpStride];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    double2* sw = stage[wib];
    const int64_t n = (int64_t)g.V * nr, tiles = (n + 31) / 32;
    const bool lex_src = wide_lex(src), lex_dst = wide_lex(dst);
    // the loop bound is the same for every lane of a warp, so the warp barriers are uniform
    for (int64_t t = (int64_t)blockIdx.x * (kConvBS / 32) + wib; t < tiles; t += (int64_t)gridDim.x * (kConvBS / 32)) {
        const int64_t f0 = t * 32, f = f0 + lane;
        const int nv = (int)(n - f0 < 32 ? n - f0 : 32);
        const bool ok = lane < nv;
        __syncwarp();
        if (lex_src) {
            const double2* s2 = (const double2*)src.ptr + f0 * 12;
            for (int i = lane; i < nv * 12; i += 32) sw[(i / 12) * kSpStride + i % 12] = __ldg(s2 + i);
            __syncwarp();
        }
        double v[24];
        Site s{};
        if (ok) {
            int c[4];
            s = site_from_lex(g, (int)(f % g.V), c, (int)(f / g.V));
            if (lex_src) {
#pragma unroll
                for (int k = 0; k < 12; ++k) {
                    const double2 q = sw[lane * kSpStride + k];
                    v[2 * k] = q.x;
                    v[2 * k + 1] = q.y;
                }
            } else {
                load_site(src, g, s, nr, v);
            }
        }
        if (lex_dst) {
            __syncwarp();
            if (ok) {
#pragma unroll
                for (int k = 0; k < 12; ++k) sw[lane * kSpStride + k] = make_double2(v[2 * k], v[2 * k + 1]);
            }
            __syncwarp();
            double2* d2 = (double2*)dst.ptr + f0 * 12;
            for (int i = lane; i < nv * 12; i += 32) d2[i] = sw[(i / 12) * kSpStride + i % 12];
        } else if (ok) {
            store_site(dst, g, s, nr, v);
        }
    }
}

// a link real as the destination stores it, read back exactly (Q1.30: the integer)
__device__ inline double stored_link_value(int prec, double x) {
    if (prec == LQ_F32) return (double)(float)x;
    if (prec == LQ_F16S) return (double)__half2float(__float2half_rn((float)x));
    if (prec == LQ_I32S) return (double)__double2int_rn(x * 0x1p30);
    return x;
}

// the reals of link (s, mu) in a destination format: elements j < dst.fmt of the 18-real link;
// the 10-real form keeps row 0 and the two entries of row 1 outside column k, k chosen on
// the stored row 0 (largest max(|Re|, |Im|), lowest on ties)
__device__ inline void store_link(const FieldDesc& dst, const Geom& g, const Site& s, int mu, const double v[18]) {
    if (dst.fmt == 10) {
        double m[3];
#pragma unroll
        for (int j = 0; j < 3; ++j)
            m[j] = abs_max(stored_link_value(dst.prec, v[2 * j]), stored_link_value(dst.prec, v[2 * j + 1]));
        const int k = link10_column(m[0], m[1], m[2]);
        double w[10];
#pragma unroll
        for (int j = 0; j < 6; ++j) w[j] = v[j];
        int at = 6;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            if (c == k) continue;
            w[at] = v[6 + 2 * c];
            w[at + 1] = v[7 + 2 * c];
            at += 2;
        }
#pragma unroll
        for (int j = 0; j < 10; ++j) {
            const int64_t i = lk_elem(dst, g, s, mu, j);
            if (dst.prec == LQ_F64) ((double*)dst.ptr)[i] = w[j];
            else if (dst.prec == LQ_F32) ((float*)dst.ptr)[i] = (float)w[j];
            else if (dst.prec == LQ_I32S) ((int*)dst.ptr)[i] = __double2int_rn(w[j] * 0x1p30);
            else ((__half*)dst.ptr)[i] = __float2half_rn((float)w[j]);
        }
        return;
    }
    if (dst.prec == LQ_F64X && dst.layout == LQ_LAYOUT_EO && dst.fmt == 18) {
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            const dd a = split_double(v[2 * k]), b = split_double(v[2 * k + 1]);
            ((float4*)dst.ptr)[lk_elem(dst, g, s, mu, 2 * k) / 2] = make_float4(a.hi, a.lo, b.hi, b.lo);
        }
        return;
    }
    if (dst.prec == LQ_F16S && dst.layout == LQ_LAYOUT_EO && dst.fmt == 12) {
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const __half2 a = __halves2half2(__float2half_rn((float)v[4 * k]), __float2half_rn((float)v[4 * k + 1]));
            const __half2 b = __halves2half2(__float2half_rn((float)v[4 * k + 2]), __float2half_rn((float)v[4 * k + 3]));
            ((uint2*)dst.ptr)[lk_elem(dst, g, s, mu, 4 * k) / 4] =
                make_uint2(*(const uint32_t*)&a, *(const uint32_t*)&b);
        }
        return;
    }
    if (dst.prec == LQ_F32 && dst.layout == LQ_LAYOUT_EO && dst.fmt == 12) {
#pragma unroll
        for (int k = 0; k < 3; ++k)
            ((float4*)dst.ptr)[lk_elem(dst, g, s, mu, 4 * k) / 4] =
                make_float4((float)v[4 * k], (float)v[4 * k + 1], (float)v[4 * k + 2], (float)v[4 * k + 3]);
        return;
    }
#pragma unroll
    for (int j = 0; j < 18; ++j) {
        if (j >= dst.fmt) break;
        const int64_t i = lk_elem(dst, g, s, mu, j);
        if (dst.prec == LQ_F64 || dst.prec == LQ_F64X) store_wide(dst.ptr, dst.prec, i, v[j]);
        else if (dst.prec == LQ_F32) ((float*)dst.ptr)[i] = (float)v[j];
        else if (dst.prec == LQ_I32S) ((int*)dst.ptr)[i] = __double2int_rn(v[j] * 0x1p30);   // Q1.30
        else ((__half*)dst.ptr)[i] = __float2half_rn((float)v[j]);
    }
}

// one thread per link (site lex, direction mu), link index L = 4 lex + mu; dst2.ptr, if set,
// receives a second encoding of the same links
__global__ void __launch_bounds__(kConvBS) convert_gauge_kernel(Geom g, FieldDesc src, FieldDesc dst, FieldDesc dst2) {
    __shared__ double2 stage[kConvBS / 32][32 * 9];   // lane stride 144 bytes: conflict-free 16-byte reads
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    double2* sw = stage[wib];
    const int64_t n = (int64_t)g.V * 4, tiles = (n + 31) / 32;
    const bool lex_src = wide_lex(src) && src.fmt == 18;
    for (int64_t t = (int64_t)blockIdx.x * (kConvBS / 32) + wib; t < tiles; t += (int64_t)gridDim.x * (kConvBS / 32)) {
        const int64_t L0 = t * 32, L = L0 + lane;
        const int nv = (int)(n - L0 < 32 ? n - L0 : 32);
        __syncwarp();
        if (lex_src) {
            const double2* s2 = (const double2*)src.ptr + L0 * 9;
            for (int i = lane; i < nv * 9; i += 32) sw[i] = __ldg(s2 + i);
            __syncwarp();
        }
        if (lane < nv) {
            int c[4];
            const Site s = site_from_lex(g, (int)(L >> 2), c);
            const int mu = (int)(L & 3);
            double v[18];
            if (lex_src) {
#pragma unroll
                for (int k = 0; k < 9; ++k) {
                    const double2 q = sw[lane * 9 + k];
                    v[2 * k] = q.x;
                    v[2 * k + 1] = q.y;
                }
            } else {
#pragma unroll
                for (int j = 0; j < 18; ++j) {
                    v[j] = load_real(src.ptr, src.prec, lk_elem(src, g, s, mu, j));
                    if (src.prec == LQ_I32S) v[j] *= 0x1p-30;
                }
            }
            store_link(dst, g, s, mu, v);
            if (dst2.ptr) store_link(dst2, g, s, mu, v);
        }
    }
}

int conv_grid(int64_t items) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t per_block = kConvBS;   // one item per thread
    const int64_t want = (items + per_block - 1) / per_block, cap = (int64_t)sms * 16;
    return (int)(want < cap ? (want > 0 ? want : 1) : cap);
}

}  // namespace

cudaError_t convert_spinor(const Geom& g, int sp, int sl, const void* src, int dp, int dl, void* dst, cudaStream_t st,
                           int nr) {
    convert_spinor_kernel<<<conv_grid((int64_t)g.V * nr), kConvBS, 0, st>>>(g, FieldDesc{(void*)src, sp, sl, 0},
                                                                          FieldDesc{dst, dp, dl, 0}, nr);
    return cudaGetLastError();
}

cudaError_t convert_gauge(const Geom& g, int sp, int sl, const void* src, int dp, int dfmt, int dl, void* dst,
                          cudaStream_t st, int dp2, int dfmt2, int dl2, void* dst2) {
    const FieldDesc second = dst2 ? FieldDesc{dst2, dp2, dl2, dfmt2} : FieldDesc{nullptr, 0, 0, 0};
    convert_gauge_kernel<<<conv_grid((int64_t)g.V * 4), kConvBS, 0, st>>>(g, FieldDesc{(void*)src, sp, sl, 18},
                                                                       FieldDesc{dst, dp, dl, dfmt}, second);
    return cudaGetLastError();
}

}  // namespace lq
