// Internal definitions of liblq: complex arithmetic, lattice geometry, field accessors
// for every (precision, layout, link format) the C ABI exposes, and the deterministic
// grid reduction used by the fused solver kernels.
//
// Field formats are the ones documented in include/lq.h.  Nothing here is shared with
// the CPU oracle.
#pragma once

#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <stdint.h>
#include <stddef.h>

#include <type_traits>
#include <utility>

#include "../../include/lq.h"
#include "dd.cuh"

// Helpers are callable from host code as well, so the index arithmetic and the stencil
// algebra can be exercised off the GPU; the library itself only runs them on the device.
#define LQ_HD __host__ __device__ __forceinline__

namespace lq {

// ------------------------------------------------------------------------------------
// complex numbers in the compute precision
// ------------------------------------------------------------------------------------
template <typename R> struct cplx { R re, im; };

template <typename R> LQ_HD cplx<R> cmk(R a, R b) { return {a, b}; }
template <typename R> LQ_HD cplx<R> cadd(cplx<R> a, cplx<R> b) { return {a.re + b.re, a.im + b.im}; }
template <typename R> LQ_HD cplx<R> csub(cplx<R> a, cplx<R> b) { return {a.re - b.re, a.im - b.im}; }
// i*a and -i*a
template <typename R> LQ_HD cplx<R> ctimes_i(cplx<R> a) { return {-a.im, a.re}; }
template <typename R> LQ_HD cplx<R> ctimes_mi(cplx<R> a) { return {a.im, -a.re}; }
template <typename R> LQ_HD cplx<R> cconj(cplx<R> a) { return {a.re, -a.im}; }
template <typename R> LQ_HD cplx<R> cmul(cplx<R> a, cplx<R> b) {
    return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
// c + a*b
template <typename R> LQ_HD cplx<R> cfma(cplx<R> a, cplx<R> b, cplx<R> c) {
    return {fma(a.re, b.re, fma(-a.im, b.im, c.re)), fma(a.re, b.im, fma(a.im, b.re, c.im))};
}
// c + conj(a)*b
template <typename R> LQ_HD cplx<R> cfmac(cplx<R> a, cplx<R> b, cplx<R> c) {
    return {fma(a.re, b.re, fma(a.im, b.im, c.re)), fma(a.re, b.im, fma(-a.im, b.re, c.im))};
}
template <typename R> LQ_HD cplx<R> cscale(R s, cplx<R> a) { return {s * a.re, s * a.im}; }
// c + s*a
template <typename R> LQ_HD cplx<R> caxpy(R s, cplx<R> a, cplx<R> c) {
    return {fma(s, a.re, c.re), fma(s, a.im, c.im)};
}

// A spinor in registers: 12 complex numbers, index spin*3 + colour.
template <typename R> struct Spinor { cplx<R> v[12]; };
// A link in registers: u[row][col].
template <typename R> struct Link { cplx<R> u[3][3]; };

// ------------------------------------------------------------------------------------
// precision traits
// ------------------------------------------------------------------------------------
template <int PREC> struct PrecT;
template <> struct PrecT<LQ_F64> { using Real = double; };
template <> struct PrecT<LQ_F32> { using Real = float; };
template <> struct PrecT<LQ_F16S> { using Real = float; };
template <> struct PrecT<LQ_F64X> { using Real = dd; };
template <> struct PrecT<LQ_I32S> { using Real = float; };

LQ_HD float to_float(float x) { return x; }
LQ_HD float to_float(double x) { return (float)x; }
LQ_HD float to_float(dd x) { return f_add(x.hi, x.lo); }

// ------------------------------------------------------------------------------------
// lattice geometry
// ------------------------------------------------------------------------------------
// Division by a run-time constant d >= 1 for 0 <= n < 2^31 with one multiply-high:
// q = (umulhi(n, mul) + n) >> shift, mul = floor(2^32 (2^shift - d) / d) + 1,
// shift = ceil(log2 d) (the round-up method of Granlund and Montgomery, 1994).
struct FastDiv {
    uint32_t d, mul, shift;
};

inline FastDiv make_fastdiv(uint32_t d) {
    uint32_t l = 0;
    while ((1ull << l) < d) ++l;
    const uint64_t m = ((1ull << 32) * ((1ull << l) - d)) / d + 1;
    return FastDiv{d, (uint32_t)m, l};
}

LQ_HD uint32_t umulhi32(uint32_t a, uint32_t b) {
#ifdef __CUDA_ARCH__
    return __umulhi(a, b);
#else
    return (uint32_t)(((uint64_t)a * b) >> 32);
#endif
}

LQ_HD uint32_t fdiv(uint32_t n, const FastDiv& f) { return (umulhi32(n, f.mul) + n) >> f.shift; }

struct Geom {
    int L[4];       // extents x, y, z, t
    int S[4];       // lexicographic strides 1, Lx, Lx*Ly, Lx*Ly*Lz
    int V, Vh;
    int Lxh;        // Lx / 2
    FastDiv fLx, fLy, fLz, fLxh;
};

inline Geom make_geom(const int32_t d[4]) {
    Geom g;
    for (int i = 0; i < 4; ++i) g.L[i] = d[i];
    g.S[0] = 1;
    g.S[1] = d[0];
    g.S[2] = d[0] * d[1];
    g.S[3] = d[0] * d[1] * d[2];
    g.V = d[0] * d[1] * d[2] * d[3];
    g.Vh = g.V / 2;
    g.Lxh = d[0] / 2;
    g.fLx = make_fastdiv((uint32_t)d[0]);
    g.fLy = make_fastdiv((uint32_t)d[1]);
    g.fLz = make_fastdiv((uint32_t)d[2]);
    g.fLxh = make_fastdiv((uint32_t)(d[0] / 2));
    return g;
}

// A site seen from every layout: lexicographic index, parity and checkerboard index, and
// the right-hand side it is processed for (0 for single-field operations).
struct Site { int lex, p, cb, rhs; };

LQ_HD void coords_from_lex(const Geom& g, int lex, int c[4]) {
    const uint32_t r0 = (uint32_t)lex;
    const uint32_t r1 = fdiv(r0, g.fLx);
    const uint32_t r2 = fdiv(r1, g.fLy);
    const uint32_t r3 = fdiv(r2, g.fLz);
    c[0] = (int)(r0 - r1 * (uint32_t)g.L[0]);
    c[1] = (int)(r1 - r2 * (uint32_t)g.L[1]);
    c[2] = (int)(r2 - r3 * (uint32_t)g.L[2]);
    c[3] = (int)r3;
}

LQ_HD Site site_from_lex(const Geom& g, int lex, int c[4], int rhs = 0) {
    coords_from_lex(g, lex, c);
    return Site{lex, (c[0] + c[1] + c[2] + c[3]) & 1, lex >> 1, rhs};
}

// (p, cb) -> coordinates: cb = x/2 + (Lx/2)*(y + Ly*(z + Lz*t)), x's low bit fixed by p.
LQ_HD Site site_from_eo(const Geom& g, int p, int cb, int c[4], int rhs = 0) {
    const uint32_t r0 = (uint32_t)cb;
    const uint32_t r1 = fdiv(r0, g.fLxh);
    const uint32_t r2 = fdiv(r1, g.fLy);
    const uint32_t r3 = fdiv(r2, g.fLz);
    const int xh = (int)(r0 - r1 * (uint32_t)g.Lxh);
    c[1] = (int)(r1 - r2 * (uint32_t)g.L[1]);
    c[2] = (int)(r2 - r3 * (uint32_t)g.L[2]);
    c[3] = (int)r3;
    c[0] = 2 * xh + ((p + c[1] + c[2] + c[3]) & 1);
    const int lex = 2 * cb + (c[0] & 1);
    return Site{lex, p, cb, rhs};
}

// lexicographic index of n + mu (fwd) and n - mu (bwd), periodic
LQ_HD int lex_fwd(const Geom& g, int lex, const int c[4], int mu) {
    return (c[mu] == g.L[mu] - 1) ? lex - (g.L[mu] - 1) * g.S[mu] : lex + g.S[mu];
}
LQ_HD int lex_bwd(const Geom& g, int lex, const int c[4], int mu) {
    return (c[mu] == 0) ? lex + (g.L[mu] - 1) * g.S[mu] : lex - g.S[mu];
}
LQ_HD Site nb_site(int lexn, int p, int rhs) { return Site{lexn, p ^ 1, lexn >> 1, rhs}; }

// ------------------------------------------------------------------------------------
// load helpers (read-only path for fields that are constant during a kernel)
// ------------------------------------------------------------------------------------
template <bool RO, typename T> LQ_HD T ld(const T* p) {
#ifdef __CUDA_ARCH__
    if constexpr (RO) return __ldg(p);
    else return *p;
#else
    return *p;
#endif
}

// ------------------------------------------------------------------------------------
// Bounds-checked debug build (compiled with LQ_BOUNDS_CHECK): every slot a field accessor
// touches is checked against the slots its buffer holds.  An access out of range is
// skipped (a load yields zero) and counted in a record of its translation unit; the host
// reads the records back through lq_bounds_violations().  Nothing traps or faults.  In the
// normal build the checks compile to nothing.
// ------------------------------------------------------------------------------------
#ifdef LQ_BOUNDS_CHECK
using OobReaderFn = unsigned int (*)(unsigned long long* first);
void register_oob_reader(OobReaderFn r);
namespace {
__device__ unsigned int g_oob_count;
__device__ unsigned long long g_oob_first;
unsigned int read_oob(unsigned long long* first) {
    unsigned int c = 0;
    unsigned long long f = 0;
    const unsigned int zero = 0;
    if (cudaMemcpyFromSymbol(&c, g_oob_count, sizeof(c)) != cudaSuccess) return 0;
    if (c && first && cudaMemcpyFromSymbol(&f, g_oob_first, sizeof(f)) == cudaSuccess && *first == ~0ull) *first = f;
    if (c) cudaMemcpyToSymbol(g_oob_count, &zero, sizeof(zero));
    return c;
}
struct OobRegistrar {
    OobRegistrar() { register_oob_reader(&read_oob); }
} g_oob_registrar;
}  // namespace
LQ_HD bool oob_ok(uint32_t i, uint32_t n) {
    if (i < n) return true;
#ifdef __CUDA_ARCH__
    if (atomicAdd(&g_oob_count, 1u) == 0u) g_oob_first = i;
#endif
    return false;
}
#endif

// The slot bounds of a field accessor (checked only in the debug build).
struct SlotBounds {
#ifdef LQ_BOUNDS_CHECK
    uint32_t nslots = 0xffffffffu, nscales = 0xffffffffu;
    LQ_HD bool slot_ok(uint32_t i) const { return oob_ok(i, nslots); }
    LQ_HD bool scale_ok(uint32_t i) const { return oob_ok(i, nscales); }
#else
    LQ_HD static constexpr bool slot_ok(uint32_t) { return true; }
    LQ_HD static constexpr bool scale_ok(uint32_t) { return true; }
#endif
    // slot b + off of p; the address is formed as (p + b) + off, as the accessors always did,
    // so that the compiler keeps its 64-bit address arithmetic
    template <bool RO, typename T> LQ_HD T at(const T* p, uint32_t b, uint32_t off) const {
        return slot_ok(b + off) ? ld<RO>(p + b + off) : T{};
    }
    template <typename T> LQ_HD void set(T* p, uint32_t b, uint32_t off, const T& v) const {
        if (slot_ok(b + off)) p[b + off] = v;
    }
    template <bool RO> LQ_HD float scale_at(const float* p, uint32_t i) const { return scale_ok(i) ? ld<RO>(p + i) : 0.f; }
    LQ_HD void scale_set(float* p, uint32_t i, float v) const {
        if (scale_ok(i)) p[i] = v;
    }
};

// Brings the cache line holding p into L1 ahead of its load (no register is written, so a
// warp can ask for data it will use later without stalling on it now).
LQ_HD void prefetch_l1(const void* p) {
#ifdef __CUDA_ARCH__
    asm volatile("prefetch.global.L1 [%0];" ::"l"(p));
#else
    (void)p;
#endif
}

// x / y in FP32, correctly rounded
LQ_HD float div_rn(float x, float y) {
#ifdef __CUDA_ARCH__
    return __fdiv_rn(x, y);
#else
    return x / y;
#endif
}

LQ_HD float2 h2f2(uint32_t w) {
    __half2 h = *reinterpret_cast<__half2*>(&w);
    return __half22float2(h);
}
LQ_HD uint32_t f22h2(float a, float b) {
    __half2 h = __halves2half2(__float2half_rn(a), __float2half_rn(b));
    return *reinterpret_cast<uint32_t*>(&h);
}

// ------------------------------------------------------------------------------------
// Spinor field accessors, for nr right-hand sides (nr = 1 for a single field).
//   LEX: nr consecutive fields; chunk k of site n of field r at slot (r*V + n)*K + k.
//   EO : chunk k of (p, cb, r) at slot ((p*K + k)*Vh + cb)*nr + r, i.e. base
//        (p*pstride + cb)*nr + r and stride Vh*nr per chunk (pstride = K*Vh for a full
//        field, 0 for a half field holding one parity); the right-hand sides of a site
//        sit next to each other, so the threads of one site read contiguous memory.
// F16S scales: LEX at r*V + n, EO at (p*sstride + cb)*nr + r (sstride = Vh full, 0 half).
// ------------------------------------------------------------------------------------
template <int PREC, int LAYOUT, bool RO> struct SpinorAcc;

// Slot indices are 32-bit: the ABI caps V at 10^8 sites and V * nrhs at 2^28 site-fields
// per call, so every slot index of every field format (at most 36 V for FP64 18-real LEX
// links, 12 V nrhs for FP64 spinors) stays below 2^32.
struct EoIdx {
    uint32_t Vh, pstride, sstride;
    uint32_t nr;    // right-hand sides interleaved per site (EO) or stacked fields (LEX)
    uint32_t V;     // sites per field (LEX stacking)
};

template <int LAYOUT> LQ_HD uint32_t sp_base(const Site& s, int K, const EoIdx& e) {
    if constexpr (LAYOUT == LQ_LAYOUT_LEX) return ((uint32_t)s.rhs * e.V + (uint32_t)s.lex) * (uint32_t)K;
    else return ((uint32_t)s.p * e.pstride + (uint32_t)s.cb) * e.nr + (uint32_t)s.rhs;
}
template <int LAYOUT> LQ_HD uint32_t sp_kstride(const EoIdx& e) {
    if constexpr (LAYOUT == LQ_LAYOUT_LEX) return 1u;
    else return e.Vh * e.nr;
}
template <int LAYOUT> LQ_HD uint32_t sp_sidx(const Site& s, const EoIdx& e) {
    if constexpr (LAYOUT == LQ_LAYOUT_LEX) return (uint32_t)s.rhs * e.V + (uint32_t)s.lex;
    else return ((uint32_t)s.p * e.sstride + (uint32_t)s.cb) * e.nr + (uint32_t)s.rhs;
}

template <int LAYOUT, bool RO> struct SpinorAcc<LQ_F64, LAYOUT, RO> : SlotBounds {
    using Real = double;
    static constexpr int K = 12;
    static constexpr bool kScaled = false;
    double2* ptr;
    EoIdx e;
    LQ_HD void prefetch(const Site& s) const {
        const uint32_t b = sp_base<LAYOUT>(s, K, e), ks = sp_kstride<LAYOUT>(e);
#pragma unroll
        for (int k = 0; k < K; ++k)
            if (slot_ok(b + k * ks)) prefetch_l1(ptr + b + k * ks);
    }
    template <typename T> LQ_HD void load(const Site& s, Spinor<T>& out) const {
        const uint32_t b = sp_base<LAYOUT>(s, K, e), ks = sp_kstride<LAYOUT>(e);
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            double2 v = at<RO>(ptr, b, k * ks);
            out.v[k] = {from_double<T>(v.x), from_double<T>(v.y)};
        }
    }
    template <typename T> LQ_HD void store(const Site& s, const Spinor<T>& in) const {
        const uint32_t b = sp_base<LAYOUT>(s, K, e), ks = sp_kstride<LAYOUT>(e);
#pragma unroll
        for (int k = 0; k < 12; ++k) set(ptr, b, k * ks, make_double2(to_double(in.v[k].re), to_double(in.v[k].im)));
    }
    LQ_HD void load_raw(const Site& s, Spinor<double>& out, double& sc) const {
        load(s, out);
        sc = 1.0;
    }
};

template <int LAYOUT, bool RO> struct SpinorAcc<LQ_F32, LAYOUT, RO> : SlotBounds {
    using Real = float;
    static constexpr int K = 6;
    static constexpr bool kScaled = false;
    float4* ptr;
    EoIdx e;
    LQ_HD void prefetch(const Site& s) const {
        const uint32_t b = sp_base<LAYOUT>(s, K, e), ks = sp_kstride<LAYOUT>(e);
#pragma unroll
        for (int k = 0; k < K; ++k)
            if (slot_ok(b + k * ks)) prefetch_l1(ptr + b + k * ks);
    }
    template <typename T> LQ_HD void load(const Site& s, Spinor<T>& out) const {
        const uint32_t b = sp_base<LAYOUT>(s, K, e), ks = sp_kstride<LAYOUT>(e);
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            float4 v = at<RO>(ptr, b, k * ks);
            out.v[2 * k] = {(T)v.x, (T)v.y};
            out.v[2 * k + 1] = {(T)v.z, (T)v.w};
        }
    }
    template <typename T> LQ_HD void store(const Site& s, const Spinor<T>& in) const {
        const uint32_t b = sp_base<LAYOUT>(s, K, e), ks = sp_kstride<LAYOUT>(e);
#pragma unroll
        for (int k = 0; k < 6; ++k)
            set(ptr, b, k * ks, make_float4(to_float(in.v[2 * k].re), to_float(in.v[2 * k].im),
                                          to_float(in.v[2 * k + 1].re), to_float(in.v[2 * k + 1].im)));
    }
    LQ_HD void load_raw(const Site& s, Spinor<float>& out, float& sc) const {
        load(s, out);
        sc = 1.0f;
    }
};

// Scaled FP16: value = half * scale, scale = max |fl32(v)| of the site.  Loads compute
// half * scale in T (exact when T = double); stores round to FP32 first, then divide by
// the scale in FP32 (correctly rounded) and round to FP16.
template <int LAYOUT, bool RO> struct SpinorAcc<LQ_F16S, LAYOUT, RO> : SlotBounds {
    using Real = float;
    static constexpr int K = 3;
    static constexpr bool kScaled = true, kHalf2 = true;
    uint4* ptr;
    float* scale;
    EoIdx e;
    LQ_HD void prefetch(const Site& s) const {
        const uint32_t b = sp_base<LAYOUT>(s, K, e), ks = sp_kstride<LAYOUT>(e);
#pragma unroll
        for (int k = 0; k < K; ++k)
            if (slot_ok(b + k * ks)) prefetch_l1(ptr + b + k * ks);
        if (scale_ok(sp_sidx<LAYOUT>(s, e))) prefetch_l1(scale + sp_sidx<LAYOUT>(s, e));
    }
    // the stored halves as floats, without the site's scale (returned separately)
    LQ_HD void load_raw(const Site& s, Spinor<float>& out, float& sc) const {
        const uint32_t b = sp_base<LAYOUT>(s, K, e), ks = sp_kstride<LAYOUT>(e);
        sc = scale_at<RO>(scale, sp_sidx<LAYOUT>(s, e));
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            uint4 w = at<RO>(ptr, b, k * ks);
            const uint32_t ww[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                float2 a = h2f2(ww[j]);
                out.v[4 * k + j] = {a.x, a.y};
            }
        }
    }
    // the stored complex numbers as half2 words (re low, im high), without the scale
    LQ_HD void load_h2(const Site& s, uint32_t out[12], float& sc) const {
        const uint32_t b = sp_base<LAYOUT>(s, K, e), ks = sp_kstride<LAYOUT>(e);
        sc = scale_at<RO>(scale, sp_sidx<LAYOUT>(s, e));
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const uint4 w = at<RO>(ptr, b, k * ks);
            out[4 * k] = w.x;
            out[4 * k + 1] = w.y;
            out[4 * k + 2] = w.z;
            out[4 * k + 3] = w.w;
        }
    }
    template <typename T> LQ_HD void load(const Site& s, Spinor<T>& out) const {
        const uint32_t b = sp_base<LAYOUT>(s, K, e), ks = sp_kstride<LAYOUT>(e);
        const T sc = (T)scale_at<RO>(scale, sp_sidx<LAYOUT>(s, e));
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            uint4 w = at<RO>(ptr, b, k * ks);
            const uint32_t ww[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                float2 a = h2f2(ww[j]);
                out.v[4 * k + j] = {(T)a.x * sc, (T)a.y * sc};
            }
        }
    }
    template <typename T> LQ_HD void store(const Site& s, const Spinor<T>& in) const {
        const uint32_t b = sp_base<LAYOUT>(s, K, e), ks = sp_kstride<LAYOUT>(e);
        float f[24];
#pragma unroll
        for (int k = 0; k < 12; ++k) { f[2 * k] = to_float(in.v[k].re); f[2 * k + 1] = to_float(in.v[k].im); }
        float m = 0.f;
#pragma unroll
        for (int k = 0; k < 24; ++k) m = fmaxf(m, fabsf(f[k]));
        scale_set(scale, sp_sidx<LAYOUT>(s, e), m);
        // one correctly rounded reciprocal per site, then products (kernel outputs; the
        // bit-exact format conversion in convert.cu divides every component)
        const float inv = (m > 0.f) ? div_rn(1.0f, m) : 0.f;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            float q[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) q[j] = f[8 * k + j] * inv;
            set(ptr, b, k * ks, make_uint4(f22h2(q[0], q[1]), f22h2(q[2], q[3]), f22h2(q[4], q[5]), f22h2(q[6], q[7])));
        }
    }
};

// 32-bit fixed point (Q1.30): an integer q stands for q * 2^-30, times the site's FP32
// scale s = max |fl32(v)| for spinors.  Loads convert q to FP32 (rounding to 24 bits) and
// fold s * 2^-30 into the caller's accumulation; stores scale by the correctly rounded
// 2^30 / s and round to the nearest integer (ties to even).
constexpr float kQ30 = 1073741824.0f;           // 2^30
constexpr float kInvQ30 = 9.31322574615478515625e-10f;   // 2^-30

LQ_HD int f2i_rn(float x) {
#ifdef __CUDA_ARCH__
    return __float2int_rn(x);
#else
    return (int)nearbyintf(x);
#endif
}

template <int LAYOUT, bool RO> struct SpinorAcc<LQ_I32S, LAYOUT, RO> : SlotBounds {
    using Real = float;
    static constexpr int K = 6;
    static constexpr bool kScaled = true;
    int4* ptr;
    float* scale;
    EoIdx e;
    LQ_HD void prefetch(const Site& s) const {
        const uint32_t b = sp_base<LAYOUT>(s, K, e), ks = sp_kstride<LAYOUT>(e);
#pragma unroll
        for (int k = 0; k < K; ++k)
            if (slot_ok(b + k * ks)) prefetch_l1(ptr + b + k * ks);
        if (scale_ok(sp_sidx<LAYOUT>(s, e))) prefetch_l1(scale + sp_sidx<LAYOUT>(s, e));
    }
    // the stored integers as floats, and s * 2^-30 separately
    LQ_HD void load_raw(const Site& s, Spinor<float>& out, float& sc) const {
        const uint32_t b = sp_base<LAYOUT>(s, K, e), ks = sp_kstride<LAYOUT>(e);
        sc = scale_at<RO>(scale, sp_sidx<LAYOUT>(s, e)) * kInvQ30;
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            const int4 w = at<RO>(ptr, b, k * ks);
            out.v[2 * k] = {(float)w.x, (float)w.y};
            out.v[2 * k + 1] = {(float)w.z, (float)w.w};
        }
    }
    template <typename T> LQ_HD void load(const Site& s, Spinor<T>& out) const {
        const uint32_t b = sp_base<LAYOUT>(s, K, e), ks = sp_kstride<LAYOUT>(e);
        const T sc = (T)scale_at<RO>(scale, sp_sidx<LAYOUT>(s, e)) * (T)kInvQ30;
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            const int4 w = at<RO>(ptr, b, k * ks);
            out.v[2 * k] = {(T)w.x * sc, (T)w.y * sc};
            out.v[2 * k + 1] = {(T)w.z * sc, (T)w.w * sc};
        }
    }
    template <typename T> LQ_HD void store(const Site& s, const Spinor<T>& in) const {
        const uint32_t b = sp_base<LAYOUT>(s, K, e), ks = sp_kstride<LAYOUT>(e);
        float f[24];
#pragma unroll
        for (int k = 0; k < 12; ++k) { f[2 * k] = to_float(in.v[k].re); f[2 * k + 1] = to_float(in.v[k].im); }
        float m = 0.f;
#pragma unroll
        for (int k = 0; k < 24; ++k) m = fmaxf(m, fabsf(f[k]));
        scale_set(scale, sp_sidx<LAYOUT>(s, e), m);
        const float inv = (m > 0.f) ? div_rn(kQ30, m) : 0.f;
#pragma unroll
        for (int k = 0; k < 6; ++k)
            set(ptr, b, k * ks, make_int4(f2i_rn(f[4 * k] * inv), f2i_rn(f[4 * k + 1] * inv), f2i_rn(f[4 * k + 2] * inv),
                                        f2i_rn(f[4 * k + 3] * inv)));
    }
};

// FP32 pairs: the LQ_F64 layout with every double replaced by (hi, lo); one float4 chunk
// is one complex number (re.hi, re.lo, im.hi, im.lo).
template <int LAYOUT, bool RO> struct SpinorAcc<LQ_F64X, LAYOUT, RO> : SlotBounds {
    using Real = dd;
    static constexpr int K = 12;
    static constexpr bool kScaled = false;
    float4* ptr;
    EoIdx e;
    LQ_HD void prefetch(const Site& s) const {
        const uint32_t b = sp_base<LAYOUT>(s, K, e), ks = sp_kstride<LAYOUT>(e);
#pragma unroll
        for (int k = 0; k < K; ++k)
            if (slot_ok(b + k * ks)) prefetch_l1(ptr + b + k * ks);
    }
    template <typename T> LQ_HD void load(const Site& s, Spinor<T>& out) const {
        const uint32_t b = sp_base<LAYOUT>(s, K, e), ks = sp_kstride<LAYOUT>(e);
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            float4 v = at<RO>(ptr, b, k * ks);
            out.v[k] = {from_pair<T>(v.x, v.y), from_pair<T>(v.z, v.w)};
        }
    }
    template <typename T> LQ_HD void store(const Site& s, const Spinor<T>& in) const {
        const uint32_t b = sp_base<LAYOUT>(s, K, e), ks = sp_kstride<LAYOUT>(e);
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            const dd re = to_pair(in.v[k].re), im = to_pair(in.v[k].im);
            set(ptr, b, k * ks, make_float4(re.hi, re.lo, im.hi, im.lo));
        }
    }
    LQ_HD void load_raw(const Site& s, Spinor<dd>& out, dd& sc) const {
        load(s, out);
        sc = dd(1.0f);
    }
};

// ------------------------------------------------------------------------------------
// Gauge field accessors.
//   LEX: chunk k of link (n, mu) at slot (n*4 + mu)*K + k.
//   EO : chunk k of link (mu, p, cb) at slot ((mu*2 + p)*K + k)*Vh + cb.
// LINK12 rebuilds row 2 = conj(row0 x row1).
// ------------------------------------------------------------------------------------
template <typename R> LQ_HD void reconstruct_row2(Link<R>& U) {
    const cplx<R>* a = U.u[0];
    const cplx<R>* b = U.u[1];
    // (a x b)_0 = a1 b2 - a2 b1 etc.; row 2 is the complex conjugate
    cplx<R> c0 = csub(cmul(a[1], b[2]), cmul(a[2], b[1]));
    cplx<R> c1 = csub(cmul(a[2], b[0]), cmul(a[0], b[2]));
    cplx<R> c2 = csub(cmul(a[0], b[1]), cmul(a[1], b[0]));
    U.u[2][0] = cconj(c0);
    U.u[2][1] = cconj(c1);
    U.u[2][2] = cconj(c2);
}

template <int LAYOUT> LQ_HD uint32_t lk_base(const Site& s, int mu, int K, uint32_t Vh) {
    if constexpr (LAYOUT == LQ_LAYOUT_LEX) return ((uint32_t)s.lex * 4u + (uint32_t)mu) * (uint32_t)K;
    else return ((uint32_t)(mu * 2 + s.p) * (uint32_t)K) * Vh + (uint32_t)s.cb;
}
template <int LAYOUT> LQ_HD uint32_t lk_kstride(uint32_t Vh) {
    if constexpr (LAYOUT == LQ_LAYOUT_LEX) return 1u;
    else return Vh;
}

template <int PREC, int FMT, int LAYOUT> struct GaugeAcc;

// FP64: double2 chunks (one complex), 9 or 6 per link
template <int FMT, int LAYOUT> struct GaugeAcc<LQ_F64, FMT, LAYOUT> : SlotBounds {
    using Real = double;
    static constexpr int K = FMT / 2;
    const double2* ptr;
    uint32_t Vh;
    LQ_HD void load(const Site& s, int mu, Link<double>& U) const {
        const uint32_t b = lk_base<LAYOUT>(s, mu, K, Vh), ks = lk_kstride<LAYOUT>(Vh);
#pragma unroll
        for (int k = 0; k < K; ++k) {
            double2 v = at<true>(ptr, b, k * ks);
            U.u[k / 3][k % 3] = {v.x, v.y};
        }
        if constexpr (FMT == 12) reconstruct_row2(U);
    }
};

// FP32 18: float2 chunks; FP32 12: float4 chunks (two complex)
template <int LAYOUT> struct GaugeAcc<LQ_F32, 18, LAYOUT> : SlotBounds {
    using Real = float;
    static constexpr int K = 9;
    const float2* ptr;
    uint32_t Vh;
    LQ_HD void load(const Site& s, int mu, Link<float>& U) const {
        const uint32_t b = lk_base<LAYOUT>(s, mu, K, Vh), ks = lk_kstride<LAYOUT>(Vh);
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            float2 v = at<true>(ptr, b, k * ks);
            U.u[k / 3][k % 3] = {v.x, v.y};
        }
    }
};
template <int LAYOUT> struct GaugeAcc<LQ_F32, 12, LAYOUT> : SlotBounds {
    using Real = float;
    static constexpr int K = 3;
    const float4* ptr;
    uint32_t Vh;
    LQ_HD void load(const Site& s, int mu, Link<float>& U) const {
        const uint32_t b = lk_base<LAYOUT>(s, mu, K, Vh), ks = lk_kstride<LAYOUT>(Vh);
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            float4 v = at<true>(ptr, b, k * ks);
            const int c0 = 2 * k, c1 = 2 * k + 1;
            U.u[c0 / 3][c0 % 3] = {v.x, v.y};
            U.u[c1 / 3][c1 % 3] = {v.z, v.w};
        }
        reconstruct_row2(U);
    }
};

// FP16 18: one half2 (one complex) per chunk; FP16 12: uint2 = four halves (two complex)
template <int LAYOUT> struct GaugeAcc<LQ_F16S, 18, LAYOUT> : SlotBounds {
    using Real = float;
    static constexpr int K = 9;
    const uint32_t* ptr;
    uint32_t Vh;
    LQ_HD void load(const Site& s, int mu, Link<float>& U) const {
        const uint32_t b = lk_base<LAYOUT>(s, mu, K, Vh), ks = lk_kstride<LAYOUT>(Vh);
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            float2 v = h2f2(at<true>(ptr, b, k * ks));
            U.u[k / 3][k % 3] = {v.x, v.y};
        }
    }
};
template <int LAYOUT> struct GaugeAcc<LQ_F16S, 12, LAYOUT> : SlotBounds {
    using Real = float;
    static constexpr int K = 3;
    static constexpr bool kRowsH2 = true;
    const uint2* ptr;
    uint32_t Vh;
    // the stored rows 0 and 1 as half2 words (w[3 r + c] = U[r][c], re low, im high)
    LQ_HD void load_rows_h2(const Site& s, int mu, uint32_t w[6]) const {
        const uint32_t b = lk_base<LAYOUT>(s, mu, K, Vh), ks = lk_kstride<LAYOUT>(Vh);
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const uint2 v = at<true>(ptr, b, k * ks);
            w[2 * k] = v.x;
            w[2 * k + 1] = v.y;
        }
    }
    LQ_HD void load(const Site& s, int mu, Link<float>& U) const {
        const uint32_t b = lk_base<LAYOUT>(s, mu, K, Vh), ks = lk_kstride<LAYOUT>(Vh);
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            uint2 w = at<true>(ptr, b, k * ks);
            float2 a = h2f2(w.x), c = h2f2(w.y);
            const int c0 = 2 * k, c1 = 2 * k + 1;
            U.u[c0 / 3][c0 % 3] = {a.x, a.y};
            U.u[c1 / 3][c1 % 3] = {c.x, c.y};
        }
        reconstruct_row2(U);
    }
};

// Q1.30 links (no scale; |entries| < 2): int2 chunks (LINK18) or int4 chunks (LINK12)
template <int LAYOUT> struct GaugeAcc<LQ_I32S, 18, LAYOUT> : SlotBounds {
    using Real = float;
    static constexpr int K = 9;
    const int2* ptr;
    uint32_t Vh;
    LQ_HD void load(const Site& s, int mu, Link<float>& U) const {
        const uint32_t b = lk_base<LAYOUT>(s, mu, K, Vh), ks = lk_kstride<LAYOUT>(Vh);
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            const int2 v = at<true>(ptr, b, k * ks);
            U.u[k / 3][k % 3] = {(float)v.x * kInvQ30, (float)v.y * kInvQ30};
        }
    }
};
template <int LAYOUT> struct GaugeAcc<LQ_I32S, 12, LAYOUT> : SlotBounds {
    using Real = float;
    static constexpr int K = 3;
    const int4* ptr;
    uint32_t Vh;
    LQ_HD void load(const Site& s, int mu, Link<float>& U) const {
        const uint32_t b = lk_base<LAYOUT>(s, mu, K, Vh), ks = lk_kstride<LAYOUT>(Vh);
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const int4 w = at<true>(ptr, b, k * ks);
            const int c0 = 2 * k, c1 = 2 * k + 1;
            U.u[c0 / 3][c0 % 3] = {(float)w.x * kInvQ30, (float)w.y * kInvQ30};
            U.u[c1 / 3][c1 % 3] = {(float)w.z * kInvQ30, (float)w.w * kInvQ30};
        }
        reconstruct_row2(U);
    }
};

// ------------------------------------------------------------------------------------
// 10-real links: row 0 and the two entries of row 1 outside column k, one complex number
// per chunk (K = 5 in every precision).  k is the column of row 0 whose larger component
// max(|Re|, |Im|) is the largest (the lowest on ties), found from the stored values in
// their own exact domain, so that every decoder makes the encoder's choice.  Row 1's entry
// k follows from the orthogonality of rows 0 and 1 of a unitary matrix,
//   u1k = -(sum_{j != k} u1j conj(u0j)) / conj(u0k),   |u0k| >= 1/sqrt(6),
// and row 2 = conj(row0 x row1) as for LINK12.
// ------------------------------------------------------------------------------------
template <typename M> LQ_HD int link10_column(M m0, M m1, M m2) {
    int k = 0;
    M mk = m0;
    if (m1 > mk) {
        k = 1;
        mk = m1;
    }
    if (m2 > mk) k = 2;
    return k;
}

// U.u[0] holds row 0; b0, b1 are row 1's stored entries (columns other than k, in order)
template <typename R> LQ_HD void reconstruct10(Link<R>& U, cplx<R> b0, cplx<R> b1, int k) {
    const cplx<R> a0 = U.u[0][0], a1 = U.u[0][1], a2 = U.u[0][2];
    const cplx<R> ak = k == 0 ? a0 : (k == 1 ? a1 : a2);
    const cplx<R> aj1 = k == 0 ? a1 : a0;
    const cplx<R> aj2 = k == 2 ? a1 : a2;
    // x = -(b0 conj(aj1) + b1 conj(aj2)) / conj(ak) = -(...) ak / |ak|^2
    const cplx<R> S = cfma(b1, cconj(aj2), cmul(b0, cconj(aj1)));
    const R inv = R(1) / fma(ak.re, ak.re, ak.im * ak.im);
    const cplx<R> x = cscale(-inv, cmul(S, ak));
    U.u[1][0] = k == 0 ? x : b0;
    U.u[1][1] = k == 0 ? b0 : (k == 1 ? x : b1);
    U.u[1][2] = k == 2 ? x : b1;
    reconstruct_row2(U);
}

template <typename T> LQ_HD T abs_max(T a, T b) {
    const T x = a < T(0) ? -a : a, y = b < T(0) ? -b : b;
    return x > y ? x : y;
}

template <int LAYOUT> struct GaugeAcc<LQ_F64, 10, LAYOUT> : SlotBounds {
    using Real = double;
    static constexpr int K = 5;
    const double2* ptr;
    uint32_t Vh;
    LQ_HD void load(const Site& s, int mu, Link<double>& U) const {
        const uint32_t b = lk_base<LAYOUT>(s, mu, K, Vh), ks = lk_kstride<LAYOUT>(Vh);
        double2 w[5];
#pragma unroll
        for (int k = 0; k < 5; ++k) w[k] = at<true>(ptr, b, k * ks);
        const int c = link10_column(abs_max(w[0].x, w[0].y), abs_max(w[1].x, w[1].y), abs_max(w[2].x, w[2].y));
#pragma unroll
        for (int j = 0; j < 3; ++j) U.u[0][j] = {w[j].x, w[j].y};
        reconstruct10(U, cplx<double>{w[3].x, w[3].y}, cplx<double>{w[4].x, w[4].y}, c);
    }
};

template <int LAYOUT> struct GaugeAcc<LQ_F32, 10, LAYOUT> : SlotBounds {
    using Real = float;
    static constexpr int K = 5;
    const float2* ptr;
    uint32_t Vh;
    LQ_HD void load(const Site& s, int mu, Link<float>& U) const {
        const uint32_t b = lk_base<LAYOUT>(s, mu, K, Vh), ks = lk_kstride<LAYOUT>(Vh);
        float2 w[5];
#pragma unroll
        for (int k = 0; k < 5; ++k) w[k] = at<true>(ptr, b, k * ks);
        const int c = link10_column(abs_max(w[0].x, w[0].y), abs_max(w[1].x, w[1].y), abs_max(w[2].x, w[2].y));
#pragma unroll
        for (int j = 0; j < 3; ++j) U.u[0][j] = {w[j].x, w[j].y};
        reconstruct10(U, cplx<float>{w[3].x, w[3].y}, cplx<float>{w[4].x, w[4].y}, c);
    }
};

// FP16: one half2 word per complex entry; the halves widen to FP32 exactly, so the column
// choice compares the stored values
template <int LAYOUT> struct GaugeAcc<LQ_F16S, 10, LAYOUT> : SlotBounds {
    using Real = float;
    static constexpr int K = 5;
    const uint32_t* ptr;
    uint32_t Vh;
    LQ_HD void load(const Site& s, int mu, Link<float>& U) const {
        const uint32_t b = lk_base<LAYOUT>(s, mu, K, Vh), ks = lk_kstride<LAYOUT>(Vh);
        float2 w[5];
#pragma unroll
        for (int k = 0; k < 5; ++k) w[k] = h2f2(at<true>(ptr, b, k * ks));
        const int c = link10_column(abs_max(w[0].x, w[0].y), abs_max(w[1].x, w[1].y), abs_max(w[2].x, w[2].y));
#pragma unroll
        for (int j = 0; j < 3; ++j) U.u[0][j] = {w[j].x, w[j].y};
        reconstruct10(U, cplx<float>{w[3].x, w[3].y}, cplx<float>{w[4].x, w[4].y}, c);
    }
};

// Q1.30: the column choice compares the stored integers (their FP32 images may round
// together)
template <int LAYOUT> struct GaugeAcc<LQ_I32S, 10, LAYOUT> : SlotBounds {
    using Real = float;
    static constexpr int K = 5;
    const int2* ptr;
    uint32_t Vh;
    LQ_HD void load(const Site& s, int mu, Link<float>& U) const {
        const uint32_t b = lk_base<LAYOUT>(s, mu, K, Vh), ks = lk_kstride<LAYOUT>(Vh);
        int2 w[5];
#pragma unroll
        for (int k = 0; k < 5; ++k) w[k] = at<true>(ptr, b, k * ks);
        const int c = link10_column(abs_max(w[0].x, w[0].y), abs_max(w[1].x, w[1].y), abs_max(w[2].x, w[2].y));
#pragma unroll
        for (int j = 0; j < 3; ++j) U.u[0][j] = {(float)w[j].x * kInvQ30, (float)w[j].y * kInvQ30};
        reconstruct10(U, cplx<float>{(float)w[3].x * kInvQ30, (float)w[3].y * kInvQ30},
                      cplx<float>{(float)w[4].x * kInvQ30, (float)w[4].y * kInvQ30}, c);
    }
};

// FP32 pairs: one float4 chunk = one complex entry; 9 (LINK18) or 6 (LINK12) per link
template <int FMT, int LAYOUT> struct GaugeAcc<LQ_F64X, FMT, LAYOUT> : SlotBounds {
    using Real = dd;
    static constexpr int K = FMT / 2;
    const float4* ptr;
    uint32_t Vh;
    LQ_HD void load(const Site& s, int mu, Link<dd>& U) const {
        const uint32_t b = lk_base<LAYOUT>(s, mu, K, Vh), ks = lk_kstride<LAYOUT>(Vh);
#pragma unroll
        for (int k = 0; k < K; ++k) {
            float4 v = at<true>(ptr, b, k * ks);
            U.u[k / 3][k % 3] = {dd{v.x, v.y}, dd{v.z, v.w}};
        }
        if constexpr (FMT == 12) reconstruct_row2(U);
    }
};

// ------------------------------------------------------------------------------------
// Solver state in device memory (part of the caller's workspace), one slot per
// right-hand side of a batch.  Written only by the last block of a reducing kernel (the
// "finisher"), read by later kernels.
// ------------------------------------------------------------------------------------
constexpr int kMaxRhs = 8;         // right-hand sides per solver batch (a power of two)

// Algorithm 1's outer loop as data: the quantities of the reliable updates per right-hand
// side and the parameters of the next cycle's kernels.  The same functions advance it on the
// host (host-driven solves) or in one-thread kernels inside a solve's CUDA graph.
struct CycleCtl {
    double eta_norm[kMaxRhs];   // ||eta||
    double s[kMaxRhs];          // ||r^high|| of the current iterate (Algorithm 1's s_l)
    double s_prev[kMaxRhs];     // s of the previous cycle
    double rho_k[kMaxRhs];      // the last cycle's final inner ||r||^2 (in that cycle's units)
    double target[kMaxRhs];     // tol * ||eta||
    double best[kMaxRhs];       // smallest s so far (stagnation test)
    double is[kMaxRhs];         // next cycle: 1/s
    double stop_rho[kMaxRhs];   // next cycle: inner stop at rho <= stop_rho
    double b0[kMaxRhs];         // next cycle: beta_0 of a continued direction
    double xs[kMaxRhs];         // this cycle's solution update psi^high += xs psi
    int done[kMaxRhs], first[kMaxRhs], stagnant[kMaxRhs], status[kMaxRhs];
    int total[kMaxRhs], cycles[kMaxRhs];
    int act[kMaxRhs];           // next cycle: takes part
    int cont[kMaxRhs];          // next cycle: continues its direction (act and not first)
    int xact[kMaxRhs];          // this cycle: solution updated and residual to collect
    int nb, l, k_max, any_cont, high_applies, launches;
    int max_cycles, max_iter, per_cycle;
    int want;                   // another cycle is needed (device-driven lattice batches)
    double delta;
};

struct SolverState {
    double rho[kMaxRhs];        // ||r||^2 of the inner iterate, in the cycle's units
    double alpha[kMaxRhs], beta[kMaxRhs];
    double sigma[kMaxRhs];      // <p, D^dag D p> = ||D p||^2 of the last iteration
    double stop_rho[kMaxRhs];   // inner loop stops when rho <= stop_rho
    double red[4][kMaxRhs];     // results of standalone reductions
    int iter[kMaxRhs];          // inner iterations in the current cycle
    int stop[kMaxRhs];          // 0 running; 1 criterion met / cap / idle; 2 breakdown; 3 non-finite
    int p_iter[kMaxRhs];        // iteration whose search-direction update has been written
    int k_max;                  // inner iteration cap for the current cycle
    int nr;                     // right-hand sides in the batch
    int all_stop;               // every right-hand side has stop != 0
    int trips;                  // inner-loop graph trips in the current cycle
    int loop_base, loop_trips, loop_cap, loop_pad;   // lattice-batch loop (first lattice only)
    unsigned int ticket[4];
    CycleCtl ctl;
};

// Tile order of a grid-stride kernel: an epilogue or site operation may walk its tiles from
// the last to the first (reverse_tiles() const, read once per thread after init()).
template <class E, class = void> struct HasTileOrder : std::false_type {};
template <class E>
struct HasTileOrder<E, std::void_t<decltype(std::declval<const E&>().reverse_tiles())>> : std::true_type {};
template <class E> LQ_HD bool reverse_tiles(const E& e) {
    if constexpr (HasTileOrder<E>::value) return e.reverse_tiles();
    else return false;
}

constexpr int kMaxPartials = 4096;     // blocks per reducing kernel
constexpr int kMaxRedValues = 4;       // values reduced per thread
constexpr int kTicketK1 = 0, kTicketK2 = 1, kTicketK3 = 2, kTicketMisc = 3;

// The blocks a kernel body sees as its grid: the hardware grid, or one lattice's share of
// a launch that serves several lattices (bid in [0, nblk)).
struct VGrid {
    int bid, nblk;
};
#ifdef __CUDACC__
__device__ __forceinline__ VGrid hw_grid() { return VGrid{(int)blockIdx.x, (int)gridDim.x}; }
#endif

struct RedCtx {
    SolverState* st;
    double* partials;   // kMaxRedValues * kMaxRhs * kMaxPartials doubles
};

// Sum of v over the block (deterministic tree); result valid in thread 0.
template <int BS> __device__ __forceinline__ double block_sum(double v, double* sh) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) sh[w] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0) {
#pragma unroll
        for (int i = 0; i < BS / 32; ++i) t += sh[i];
    }
    return t;
}

// Grid-wide deterministic reduction of NV values per thread, segmented by right-hand side:
// thread t contributes to segment t mod nr (nr a power of two, nr <= 8).  Every block
// stores its per-segment partial sums; the block that arrives last sums them in block
// order and calls fin(tot) from thread 0 with tot[j * kMaxRhs + r] = the total of value j
// over segment r.  No block waits for another.
template <int BS, int NV, class Fin>
__device__ __forceinline__ void grid_reduce_seg(const RedCtx& rc, int ticket_id, const double (&v)[NV], int nr,
                                                const VGrid& vg, Fin fin) {
    __shared__ double shw[NV][BS / 32][kMaxRhs];
    __shared__ double shb[BS / 32];
    __shared__ double tot[NV * kMaxRhs];
    __shared__ bool last;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int j = 0; j < NV; ++j) {
        double x = v[j];
        for (int o = 16; o >= nr; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
        if (lane < nr) shw[j][w][lane] = x;
    }
    __syncthreads();
    if ((int)threadIdx.x < NV * nr) {
        const int j = threadIdx.x / nr, r = threadIdx.x % nr;
        double t = 0.0;
#pragma unroll
        for (int i = 0; i < BS / 32; ++i) t += shw[j][i][r];
        rc.partials[(size_t)(j * kMaxRhs + r) * vg.nblk + vg.bid] = t;
        __threadfence();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned int t = atomicAdd(&rc.st->ticket[ticket_id], 1u);
        last = (t == (unsigned int)vg.nblk - 1u);
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    for (int q = 0; q < NV * nr; ++q) {
        const int j = q / nr, r = q % nr;
        double x = 0.0;
        for (int i = threadIdx.x; i < vg.nblk; i += BS)
            x += __ldcg(rc.partials + (size_t)(j * kMaxRhs + r) * vg.nblk + i);
        x = block_sum<BS>(x, shb);
        if (threadIdx.x == 0) tot[j * kMaxRhs + r] = x;
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        rc.st->ticket[ticket_id] = 0u;
        fin(tot);
    }
}

// The unsegmented case (one field): tot[j] is the total of value j.
template <int BS, int NV, class Fin>
__device__ __forceinline__ void grid_reduce(const RedCtx& rc, int ticket_id, const double (&v)[NV], const VGrid& vg,
                                            Fin fin) {
    grid_reduce_seg<BS, NV>(rc, ticket_id, v, 1, vg, [&](const double* t) {
        double u[NV];
#pragma unroll
        for (int j = 0; j < NV; ++j) u[j] = t[j * kMaxRhs];
        fin(u);
    });
}

}  // namespace lq
