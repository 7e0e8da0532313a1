// FP32-pair ("double-float") numbers for FP64-class arithmetic on FP32 pipes.
//
// A value is hi + lo with two floats.  Sums use Knuth's TwoSum (the rounding error of a
// float addition is recovered exactly), products Dekker's TwoProduct in its FMA form
// (e = fma(a, b, -fl(a*b)) is the exact error of the product), following Dekker (1971) and
// Knuth (TAOCP vol. 2, 4.2.2).  Sums are left unnormalised (lo may grow to a few ulps of
// hi) and renormalised with FastTwoSum where a result is stored; the relative precision
// is about 2^-47.
//
// All operations use the _rn intrinsics so that the compiler cannot contract a product
// and a sum into one FMA, which would break the error-free transformations.
#pragma once

#include <cuda_runtime.h>

#ifndef LQ_HD
#define LQ_HD __host__ __device__ __forceinline__
#endif

namespace lq {

struct dd {
    float hi, lo;
    dd() = default;
    LQ_HD constexpr dd(float h, float l) : hi(h), lo(l) {}
    LQ_HD constexpr dd(float h) : hi(h), lo(0.f) {}
    LQ_HD constexpr explicit dd(int h) : hi((float)h), lo(0.f) {}
    // a double must be split (dd_from_double / from_double<dd>), never truncated to float
    dd(double) = delete;
};

LQ_HD float f_add(float a, float b) {
#ifdef __CUDA_ARCH__
    return __fadd_rn(a, b);
#else
    volatile float s = a + b;
    return s;
#endif
}
LQ_HD float f_sub(float a, float b) {
#ifdef __CUDA_ARCH__
    return __fsub_rn(a, b);
#else
    volatile float s = a - b;
    return s;
#endif
}
LQ_HD float f_mul(float a, float b) {
#ifdef __CUDA_ARCH__
    return __fmul_rn(a, b);
#else
    volatile float s = a * b;
    return s;
#endif
}
LQ_HD float f_fma(float a, float b, float c) {
#ifdef __CUDA_ARCH__
    return __fmaf_rn(a, b, c);
#else
    return fmaf(a, b, c);
#endif
}

// s + e = a + b exactly (TwoSum, 6 operations, no ordering requirement)
LQ_HD void two_sum(float a, float b, float& s, float& e) {
    s = f_add(a, b);
    const float bb = f_sub(s, a);
    e = f_add(f_sub(a, f_sub(s, bb)), f_sub(b, bb));
}

// renormalise: |lo| <= ulp(hi)/2 afterwards.  TwoSum, not FastTwoSum: after a cancellation
// (a residual eta - A x near convergence) lo can be as large as hi or larger.
LQ_HD dd dd_renorm(dd a) {
    float s, e;
    two_sum(a.hi, a.lo, s, e);
    return dd{s, e};
}

LQ_HD dd operator+(dd a, dd b) {
    float s, e;
    two_sum(a.hi, b.hi, s, e);
    return dd{s, f_add(e, f_add(a.lo, b.lo))};
}
LQ_HD dd operator-(dd a) { return dd{-a.hi, -a.lo}; }
LQ_HD dd operator-(dd a, dd b) { return a + (-b); }

// product: hi*hi exactly as p + e, plus the two cross terms; lo*lo is dropped, which is
// ~2^-48 relative for normalised operands (normalise cancelled values before squaring)
LQ_HD dd operator*(dd a, dd b) {
    const float p = f_mul(a.hi, b.hi);
    float e = f_fma(a.hi, b.hi, -p);
    e = f_fma(a.hi, b.lo, e);
    e = f_fma(a.lo, b.hi, e);
    return dd{p, e};
}

// fused multiply-add for every arithmetic type the kernels use (an overload for dd in this
// namespace would otherwise hide the float and double ones)
LQ_HD float fma(float a, float b, float c) { return fmaf(a, b, c); }
LQ_HD double fma(double a, double b, double c) { return ::fma(a, b, c); }

// a*b + c with one TwoSum
LQ_HD dd fma(dd a, dd b, dd c) {
    const float p = f_mul(a.hi, b.hi);
    float e = f_fma(a.hi, b.hi, -p);
    e = f_fma(a.hi, b.lo, e);
    e = f_fma(a.lo, b.hi, e);
    float s, t;
    two_sum(c.hi, p, s, t);
    return dd{s, f_add(t, f_add(e, c.lo))};
}

// FP64 <-> pair (host or set-up code; uses FP64 arithmetic)
LQ_HD dd dd_from_double(double x) {
    const float h = (float)x;
    return dd{h, (float)(x - (double)h)};
}
LQ_HD double dd_to_double(dd a) { return (double)a.hi + (double)a.lo; }

// Generic conversions used by the type-generic kernels (R = float, double or dd).
LQ_HD double to_double(float x) { return (double)x; }
LQ_HD double to_double(double x) { return x; }
LQ_HD double to_double(dd x) { return dd_to_double(x); }

template <typename R> LQ_HD R from_double(double x) { return (R)x; }
template <> LQ_HD dd from_double<dd>(double x) { return dd_from_double(x); }

// a value stored as a float pair, read in type T (float: rounded sum; dd: as is)
template <typename T> LQ_HD T from_pair(float h, float l);
template <> LQ_HD float from_pair<float>(float h, float l) { return f_add(h, l); }
template <> LQ_HD double from_pair<double>(float h, float l) { return (double)h + (double)l; }
template <> LQ_HD dd from_pair<dd>(float h, float l) { return dd{h, l}; }

// a value of type T written as a normalised float pair
LQ_HD dd to_pair(dd x) { return dd_renorm(x); }
LQ_HD dd to_pair(float x) { return dd{x, 0.f}; }
LQ_HD dd to_pair(double x) { return dd_from_double(x); }

}  // namespace lq
