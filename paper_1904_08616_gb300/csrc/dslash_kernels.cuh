// The Wilson-Dirac stencil of Eq. (1) and the kernel templates built on it.
//
// Per output site n the stencil forms, for each of the 8 hops, the rank-2 spin
// projection of the neighbour spinor (Section 1, stage 2: adds and subtracts of spin
// components), multiplies the resulting two colour vectors by the link or its adjoint
// (stage 3: the SU(3) x vector products, 12-real links rebuilt in registers), and
// expands the two products back into four spin components while accumulating
// (stage 4).  The diagonal (m_q + 4) term and the 1/2 of Eq. (1) are applied by the
// epilogue, which is also where the solver kernels fuse their vector updates and norms.
//
// Chiral basis: gamma_mu = [[0, B_mu], [B_mu^dag, 0]] with B_0 = -i sigma_1,
// B_1 = -i sigma_2, B_2 = -i sigma_3, B_3 = 1.  For P = 1 + S gamma_mu (S = +/-1):
//   upper(P psi) = psi_up + S B psi_dn =: h,   lower(P psi) = S B^dag h,
// so U P psi = [U h ; S B^dag (U h)] and only the two colour vectors of h need the link.
#pragma once

#include <type_traits>

#include "lq_internal.cuh"

namespace lq {

template <int S, typename R> LQ_HD cplx<R> pm(cplx<R> a, cplx<R> b) {
    if constexpr (S > 0) return cadd(a, b);
    else return csub(a, b);
}

// acc + S*sc*x  (SCALED) or acc + S*x
template <int S, bool SCALED, typename R> LQ_HD cplx<R> acc_add(cplx<R> acc, cplx<R> x, R sc) {
    if constexpr (SCALED) {
        const R f = S > 0 ? sc : -sc;
        return {fma(f, x.re, acc.re), fma(f, x.im, acc.im)};
    } else {
        return pm<S>(acc, x);
    }
}

// One hop in three stages: the rank-2 spin projection h = (1 + S gamma_MU) q reduced to its
// upper half (h0, h1 = up + S B_MU dn), the colour mat-vec g = U' h with U' = U (BACK = false)
// or U^dag (BACK = true), and the accumulation acc += sc * (g0, g1, S B_MU^dag (g0, g1)).
template <int MU, int S, typename R>
LQ_HD void hop_project(const Spinor<R>& q, cplx<R> h0[3], cplx<R> h1[3]) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const cplx<R> p0 = q.v[c], p1 = q.v[3 + c], p2 = q.v[6 + c], p3 = q.v[9 + c];
        if constexpr (MU == 0) {          // B psi_dn = (-i p3, -i p2)
            h0[c] = pm<S>(p0, ctimes_mi(p3));
            h1[c] = pm<S>(p1, ctimes_mi(p2));
        } else if constexpr (MU == 1) {   // B psi_dn = (-p3, p2)
            h0[c] = pm<-S>(p0, p3);
            h1[c] = pm<S>(p1, p2);
        } else if constexpr (MU == 2) {   // B psi_dn = (-i p2, i p3)
            h0[c] = pm<S>(p0, ctimes_mi(p2));
            h1[c] = pm<S>(p1, ctimes_i(p3));
        } else {                          // B psi_dn = (p2, p3)
            h0[c] = pm<S>(p0, p2);
            h1[c] = pm<S>(p1, p3);
        }
    }
}

template <bool BACK, typename R>
LQ_HD void hop_matvec(const Link<R>& U, const cplx<R> h0[3], const cplx<R> h1[3], cplx<R> g0[3], cplx<R> g1[3]) {
#pragma unroll
    for (int A = 0; A < 3; ++A) {
        if constexpr (!BACK) {
            g0[A] = cmul(U.u[A][0], h0[0]);
            g1[A] = cmul(U.u[A][0], h1[0]);
#pragma unroll
            for (int B = 1; B < 3; ++B) {
                g0[A] = cfma(U.u[A][B], h0[B], g0[A]);
                g1[A] = cfma(U.u[A][B], h1[B], g1[A]);
            }
        } else {
            g0[A] = cmul(cconj(U.u[0][A]), h0[0]);
            g1[A] = cmul(cconj(U.u[0][A]), h1[0]);
#pragma unroll
            for (int B = 1; B < 3; ++B) {
                g0[A] = cfmac(U.u[B][A], h0[B], g0[A]);
                g1[A] = cfmac(U.u[B][A], h1[B], g1[A]);
            }
        }
    }
}

template <int MU, int S, bool SCALED, typename R>
LQ_HD void hop_accumulate(Spinor<R>& acc, const cplx<R> g0[3], const cplx<R> g1[3], R sc) {
#pragma unroll
    for (int A = 0; A < 3; ++A) {
        acc.v[A] = acc_add<1, SCALED>(acc.v[A], g0[A], sc);
        acc.v[3 + A] = acc_add<1, SCALED>(acc.v[3 + A], g1[A], sc);
        // lower components: S B^dag (g0, g1)
        if constexpr (MU == 0) {          // B^dag g = (i g1, i g0)
            acc.v[6 + A] = acc_add<S, SCALED>(acc.v[6 + A], ctimes_i(g1[A]), sc);
            acc.v[9 + A] = acc_add<S, SCALED>(acc.v[9 + A], ctimes_i(g0[A]), sc);
        } else if constexpr (MU == 1) {   // B^dag g = (g1, -g0)
            acc.v[6 + A] = acc_add<S, SCALED>(acc.v[6 + A], g1[A], sc);
            acc.v[9 + A] = acc_add<-S, SCALED>(acc.v[9 + A], g0[A], sc);
        } else if constexpr (MU == 2) {   // B^dag g = (i g0, -i g1)
            acc.v[6 + A] = acc_add<S, SCALED>(acc.v[6 + A], ctimes_i(g0[A]), sc);
            acc.v[9 + A] = acc_add<S, SCALED>(acc.v[9 + A], ctimes_mi(g1[A]), sc);
        } else {                          // B^dag g = (g0, g1)
            acc.v[6 + A] = acc_add<S, SCALED>(acc.v[6 + A], g0[A], sc);
            acc.v[9 + A] = acc_add<S, SCALED>(acc.v[9 + A], g1[A], sc);
        }
    }
}

// acc += sc * U' (1 + S gamma_MU) q,  U' = U (BACK = false) or U^dag (BACK = true);
// sc is the neighbour's storage scale (1 unless SCALED), folded into the accumulation.
template <int MU, int S, bool BACK, bool SCALED, typename R>
LQ_HD void hop_dir(Spinor<R>& acc, const Spinor<R>& q, const Link<R>& U, R sc) {
    cplx<R> h0[3], h1[3];
    hop_project<MU, S>(q, h0, h1);
    cplx<R> g0[3], g1[3];
    hop_matvec<BACK>(U, h0, h1, g0, g1);
    hop_accumulate<MU, S, SCALED>(acc, g0, g1, sc);
}

// The same hop with the direction MU, the projector sign and the link orientation known
// only at run time.  Used by the rolled stencil below: one copy of the mat-vec serves all
// eight hops, which keeps long FP32-pair kernels inside the instruction cache.
template <typename R> LQ_HD cplx<R> cneg(cplx<R> a) { return {-a.re, -a.im}; }
template <typename R> LQ_HD cplx<R> csel(bool c, cplx<R> a, cplx<R> b) { return c ? a : b; }

template <bool SCALED, typename R>
LQ_HD void hop_dir_rt(Spinor<R>& acc, const Spinor<R>& q, const Link<R>& U, R sc, int mu, bool plus, bool back) {
    cplx<R> h0[3], h1[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const cplx<R> p0 = q.v[c], p1 = q.v[3 + c], p2 = q.v[6 + c], p3 = q.v[9 + c];
        cplx<R> b0, b1;                       // B_mu psi_dn
        switch (mu) {
            case 0: b0 = ctimes_mi(p3); b1 = ctimes_mi(p2); break;
            case 1: b0 = cneg(p3); b1 = p2; break;
            case 2: b0 = ctimes_mi(p2); b1 = ctimes_i(p3); break;
            default: b0 = p2; b1 = p3; break;
        }
        h0[c] = cadd(p0, csel(plus, b0, cneg(b0)));
        h1[c] = cadd(p1, csel(plus, b1, cneg(b1)));
    }
    // W = U or U^dag
    cplx<R> W[3][3];
#pragma unroll
    for (int A = 0; A < 3; ++A)
#pragma unroll
        for (int B = 0; B < 3; ++B) W[A][B] = csel(back, cconj(U.u[B][A]), U.u[A][B]);
    cplx<R> g0[3], g1[3];
#pragma unroll
    for (int A = 0; A < 3; ++A) {
        g0[A] = cmul(W[A][0], h0[0]);
        g1[A] = cmul(W[A][0], h1[0]);
#pragma unroll
        for (int B = 1; B < 3; ++B) {
            g0[A] = cfma(W[A][B], h0[B], g0[A]);
            g1[A] = cfma(W[A][B], h1[B], g1[A]);
        }
    }
    const R sp = sc, sl = plus ? sc : -sc;    // upper and lower accumulation factors
#pragma unroll
    for (int A = 0; A < 3; ++A) {
        cplx<R> l2, l3;                       // B_mu^dag (g0, g1)
        switch (mu) {
            case 0: l2 = ctimes_i(g1[A]); l3 = ctimes_i(g0[A]); break;
            case 1: l2 = g1[A]; l3 = cneg(g0[A]); break;
            case 2: l2 = ctimes_i(g0[A]); l3 = ctimes_mi(g1[A]); break;
            default: l2 = g0[A]; l3 = g1[A]; break;
        }
        if constexpr (SCALED) {
            acc.v[A] = caxpy(sp, g0[A], acc.v[A]);
            acc.v[3 + A] = caxpy(sp, g1[A], acc.v[3 + A]);
            acc.v[6 + A] = caxpy(sl, l2, acc.v[6 + A]);
            acc.v[9 + A] = caxpy(sl, l3, acc.v[9 + A]);
        } else {
            acc.v[A] = cadd(acc.v[A], g0[A]);
            acc.v[3 + A] = cadd(acc.v[3 + A], g1[A]);
            acc.v[6 + A] = cadd(acc.v[6 + A], csel(plus, l2, cneg(l2)));
            acc.v[9 + A] = cadd(acc.v[9 + A], csel(plus, l3, cneg(l3)));
        }
    }
}

// Scaled-FP16 hops: the spin projection runs in half2 arithmetic on the stored words (a
// complex number is one half2 word, re low, im high; each projected component is one add of
// two stored values, rounded once to FP16), so the neighbour spinor is never widened in
// full: only the two projected colour vectors are.  The link mat-vec and the accumulation
// over the eight hops, with the neighbour's scale, are FP32.  The stored values are scaled
// to |v| <= 1 per site, so the projected components stay within |h| <= 2.
namespace h2 {
__device__ __forceinline__ __half2 w2h(uint32_t w) { return *reinterpret_cast<const __half2*>(&w); }
__device__ __forceinline__ uint32_t h2w(__half2 h) { return *reinterpret_cast<const uint32_t*>(&h); }
// i a = (-a.im, a.re),  -i a = (a.im, -a.re)
__device__ __forceinline__ __half2 mul_i(__half2 a) { return w2h(__byte_perm(h2w(a), 0u, 0x1032u) ^ 0x00008000u); }
__device__ __forceinline__ __half2 mul_mi(__half2 a) { return w2h(__byte_perm(h2w(a), 0u, 0x1032u) ^ 0x80000000u); }
template <int S> __device__ __forceinline__ __half2 pm(__half2 a, __half2 b) {
    if constexpr (S > 0) return __hadd2(a, b);
    else return __hsub2(a, b);
}

// the rank-2 projection of hop_project on half2 words
template <int MU, int S>
__device__ __forceinline__ void project(const uint32_t q[12], __half2 h0[3], __half2 h1[3]) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const __half2 p0 = w2h(q[c]), p1 = w2h(q[3 + c]), p2 = w2h(q[6 + c]), p3 = w2h(q[9 + c]);
        if constexpr (MU == 0) {
            h0[c] = pm<S>(p0, mul_mi(p3));
            h1[c] = pm<S>(p1, mul_mi(p2));
        } else if constexpr (MU == 1) {
            h0[c] = pm<-S>(p0, p3);
            h1[c] = pm<S>(p1, p2);
        } else if constexpr (MU == 2) {
            h0[c] = pm<S>(p0, mul_mi(p2));
            h1[c] = pm<S>(p1, mul_i(p3));
        } else {
            h0[c] = pm<S>(p0, p2);
            h1[c] = pm<S>(p1, p3);
        }
    }
}

// acc += sc * U' (1 + S gamma_MU) q for a stored scaled-FP16 neighbour q
template <int MU, int S, bool BACK>
__device__ __forceinline__ void hop(Spinor<float>& acc, const uint32_t q[12], const Link<float>& U, float sc) {
    __half2 h0[3], h1[3];
    project<MU, S>(q, h0, h1);
    cplx<float> f0[3], f1[3], g0[3], g1[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const float2 a = __half22float2(h0[c]), b = __half22float2(h1[c]);
        f0[c] = {a.x, a.y};
        f1[c] = {b.x, b.y};
    }
    hop_matvec<BACK>(U, f0, f1, g0, g1);
    hop_accumulate<MU, S, true>(acc, g0, g1, sc);
}

// The same hop with the stored FP16 rows 0 and 1 of a 12-real link used as they are: each
// product of two FP16 values is exact in FP32, so an FP32 fused multiply-add with FP16
// multiplicands (one rounding, as after exact widening) replaces the widening of the twelve
// link halves.  Row 2 = conj(row 0 x row 1) is rebuilt in FP32 the same way, and only the
// projected components that meet row 2 are widened.
struct hw {
    uint16_t re, im;
};
__device__ __forceinline__ hw split(uint32_t w) {
    hw h;
    asm("mov.b32 {%0, %1}, %2;" : "=h"(h.re), "=h"(h.im) : "r"(w));
    return h;
}
// c + a b  (a, b FP16, c and the result FP32)
__device__ __forceinline__ float fmah(uint16_t a, uint16_t b, float c) {
    float d;
    asm("fma.rn.f32.f16 %0, %1, %2, %3;" : "=f"(d) : "h"(a), "h"(b), "f"(c));
    return d;
}
// -a for an FP16 value (folded into the multiply-add that consumes it)
__device__ __forceinline__ uint16_t hneg(uint16_t a) {
    uint16_t d;
    asm("neg.f16 %0, %1;" : "=h"(d) : "h"(a));
    return d;
}
// c + u h and c + conj(u) h for an FP16 link entry u and an FP16 value h
__device__ __forceinline__ cplx<float> cfmah(hw u, hw h, cplx<float> c) {
    return {fmah(u.re, h.re, fmah(hneg(u.im), h.im, c.re)), fmah(u.re, h.im, fmah(u.im, h.re, c.im))};
}
__device__ __forceinline__ cplx<float> cfmach(hw u, hw h, cplx<float> c) {
    return {fmah(u.re, h.re, fmah(u.im, h.im, c.re)), fmah(u.re, h.im, fmah(hneg(u.im), h.re, c.im))};
}

template <int MU, int S, bool BACK>
__device__ __forceinline__ void hop_rows(Spinor<float>& acc, const uint32_t q[12], const uint32_t lw[6], float sc) {
    __half2 h0[3], h1[3];
    project<MU, S>(q, h0, h1);
    hw u[2][3], a0[3], a1[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        u[0][c] = split(lw[c]);
        u[1][c] = split(lw[3 + c]);
        a0[c] = split(h2w(h0[c]));
        a1[c] = split(h2w(h1[c]));
    }
    // row 2: r[k] = conj(u0[i] u1[j] - u0[j] u1[i]), (i, j, k) cyclic
    cplx<float> r2[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const int i = (k + 1) % 3, j = (k + 2) % 3;
        const hw ai = u[0][i], aj = u[0][j], bi = u[1][i], bj = u[1][j];
        r2[k].re = fmah(ai.re, bj.re, fmah(hneg(ai.im), bj.im, fmah(hneg(aj.re), bi.re, fmah(aj.im, bi.im, 0.f))));
        r2[k].im = fmah(hneg(ai.re), bj.im, fmah(hneg(ai.im), bj.re, fmah(aj.re, bi.im, fmah(aj.im, bi.re, 0.f))));
    }
    const cplx<float> z{0.f, 0.f};
    cplx<float> g0[3], g1[3];
    if constexpr (!BACK) {
        // g[A] = sum_B U[A][B] h[B]; row 2 meets every component, widened
        cplx<float> f0[3], f1[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const float2 a = __half22float2(h0[c]), b = __half22float2(h1[c]);
            f0[c] = {a.x, a.y};
            f1[c] = {b.x, b.y};
        }
#pragma unroll
        for (int A = 0; A < 2; ++A) {
            g0[A] = cfmah(u[A][2], a0[2], cfmah(u[A][1], a0[1], cfmah(u[A][0], a0[0], z)));
            g1[A] = cfmah(u[A][2], a1[2], cfmah(u[A][1], a1[1], cfmah(u[A][0], a1[0], z)));
        }
        g0[2] = cfma(r2[2], f0[2], cfma(r2[1], f0[1], cmul(r2[0], f0[0])));
        g1[2] = cfma(r2[2], f1[2], cfma(r2[1], f1[1], cmul(r2[0], f1[0])));
    } else {
        // g[A] = sum_B conj(U[B][A]) h[B]; row 2 meets h[2] only
        const float2 a = __half22float2(h0[2]), b = __half22float2(h1[2]);
        const cplx<float> f02{a.x, a.y}, f12{b.x, b.y};
#pragma unroll
        for (int A = 0; A < 3; ++A) {
            g0[A] = cfmac(r2[A], f02, cfmach(u[1][A], a0[1], cfmach(u[0][A], a0[0], z)));
            g1[A] = cfmac(r2[A], f12, cfmach(u[1][A], a1[1], cfmach(u[0][A], a1[0], z)));
        }
    }
    hop_accumulate<MU, S, true>(acc, g0, g1, sc);
}
}  // namespace h2

// gauge accessors that expose the stored FP16 rows of 12-real links (load_rows_h2)
template <class A, class = void> struct HasRowsH2 : std::false_type {};
template <class A> struct HasRowsH2<A, std::void_t<decltype(A::kRowsH2)>> : std::bool_constant<A::kRowsH2> {};

// spinor accessors of scaled-FP16 fields expose their stored half2 words (load_h2)
template <class A, class = void> struct HasHalf2 : std::false_type {};
template <class A> struct HasHalf2<A, std::void_t<decltype(A::kHalf2)>> : std::bool_constant<A::kHalf2> {};

// The hopping sum  sum_mu [ U_mu(n) P_f psi(n+mu) + U_mu(n-mu)^dag P_b psi(n-mu) ]
// (without the 1/2), P_f = 1 - gamma (D) or 1 + gamma (D^dag), P_b the other one.
// GA: gauge accessor (full field), SA: spinor accessor of the neighbours.
template <class GA, class SA, bool DAG>
struct Stencil {
    using Real = typename GA::Real;
    // FP32-pair arithmetic is ~10k instructions per site: roll the eight hops so the
    // kernel's code fits the instruction cache; the FP32 / FP16 stencils stay unrolled
    static constexpr bool kRolled = std::is_same<Real, dd>::value;
    Geom g;
    GA ga;
    SA sa;

    static constexpr bool kHalf = HasHalf2<SA>::value;

    template <int MU>
    LQ_HD void dir(const Site& s, const int c[4], Spinor<Real>& acc) const {
        constexpr int SF = DAG ? +1 : -1;
        const Site nf = nb_site(lex_fwd(g, s.lex, c, MU), s.p, s.rhs);
        const Site nb = nb_site(lex_bwd(g, s.lex, c, MU), s.p, s.rhs);
        constexpr bool SC = SA::kScaled;
#ifdef __CUDA_ARCH__
        if constexpr (kHalf && HasRowsH2<GA>::value) {
            uint32_t q[12], lw[6];
            float sc;
            sa.load_h2(nf, q, sc);
            ga.load_rows_h2(s, MU, lw);
            h2::hop_rows<MU, SF, false>(acc, q, lw, sc);
            sa.load_h2(nb, q, sc);
            ga.load_rows_h2(nb, MU, lw);
            h2::hop_rows<MU, -SF, true>(acc, q, lw, sc);
            return;
        } else if constexpr (kHalf) {
            uint32_t q[12];
            float sc;
            Link<float> U;
            sa.load_h2(nf, q, sc);
            ga.load(s, MU, U);
            h2::hop<MU, SF, false>(acc, q, U, sc);
            sa.load_h2(nb, q, sc);
            ga.load(nb, MU, U);
            h2::hop<MU, -SF, true>(acc, q, U, sc);
            return;
        }
#endif
        Spinor<Real> q;
        Link<Real> U;
        Real sc;
        sa.load_raw(nf, q, sc);
        ga.load(s, MU, U);
        hop_dir<MU, SF, false, SC>(acc, q, U, sc);
        sa.load_raw(nb, q, sc);
        ga.load(nb, MU, U);
        hop_dir<MU, -SF, true, SC>(acc, q, U, sc);
    }

    LQ_HD void apply(const Site& s, const int c[4], Spinor<Real>& acc) const {
#pragma unroll
        for (int k = 0; k < 12; ++k) acc.v[k] = {Real(0), Real(0)};
        if constexpr (kRolled) {
            // one hop per trip: forward (h even) and backward (h odd) in each direction
#pragma unroll 1
            for (int h = 0; h < 8; ++h) {
                const int mu = h >> 1;
                const bool back = (h & 1) != 0;
                const int cm = mu == 0 ? c[0] : (mu == 1 ? c[1] : (mu == 2 ? c[2] : c[3]));
                const int L = mu == 0 ? g.L[0] : (mu == 1 ? g.L[1] : (mu == 2 ? g.L[2] : g.L[3]));
                const int St = mu == 0 ? g.S[0] : (mu == 1 ? g.S[1] : (mu == 2 ? g.S[2] : g.S[3]));
                int ln;
                if (!back) ln = (cm == L - 1) ? s.lex - (L - 1) * St : s.lex + St;
                else ln = (cm == 0) ? s.lex + (L - 1) * St : s.lex - St;
                const Site nb = nb_site(ln, s.p, s.rhs);
                Spinor<Real> q;
                Link<Real> U;
                Real sc;
                sa.load_raw(nb, q, sc);
                ga.load(back ? nb : s, mu, U);
                // forward hops use 1 + SF gamma, backward hops 1 - SF gamma (SF = +1 for D^dag)
                const bool plus = back ? !DAG : DAG;
                hop_dir_rt<SA::kScaled>(acc, q, U, sc, mu, plus, back);
            }
        } else {
            dir<0>(s, c, acc);
            dir<1>(s, c, acc);
            dir<2>(s, c, acc);
            dir<3>(s, c, acc);
        }
    }

    // Register blocking over right-hand sides: the hopping sums of RB consecutive right-hand
    // sides s.rhs .. s.rhs + RB - 1 of one site.  Each link is loaded, decoded and rebuilt
    // once per direction and applied to all RB neighbour spinors (unrolled stencils only).
    template <int MU, int RB>
    LQ_HD void dir_rb(const Site& s, const int c[4], Spinor<Real> (&acc)[RB]) const {
        constexpr int SF = DAG ? +1 : -1;
        const Site nf = nb_site(lex_fwd(g, s.lex, c, MU), s.p, s.rhs);
        const Site nb = nb_site(lex_bwd(g, s.lex, c, MU), s.p, s.rhs);
        constexpr bool SC = SA::kScaled;
        Link<Real> U;
        ga.load(s, MU, U);
#pragma unroll
        for (int i = 0; i < RB; ++i) {
            const Site q = Site{nf.lex, nf.p, nf.cb, nf.rhs + i};
#ifdef __CUDA_ARCH__
            if constexpr (kHalf) {
                uint32_t w[12];
                float sc;
                sa.load_h2(q, w, sc);
                h2::hop<MU, SF, false>(acc[i], w, U, sc);
                continue;
            }
#endif
            Spinor<Real> v;
            Real sc;
            sa.load_raw(q, v, sc);
            hop_dir<MU, SF, false, SC>(acc[i], v, U, sc);
        }
        ga.load(nb, MU, U);
#pragma unroll
        for (int i = 0; i < RB; ++i) {
            const Site q = Site{nb.lex, nb.p, nb.cb, nb.rhs + i};
#ifdef __CUDA_ARCH__
            if constexpr (kHalf) {
                uint32_t w[12];
                float sc;
                sa.load_h2(q, w, sc);
                h2::hop<MU, -SF, true>(acc[i], w, U, sc);
                continue;
            }
#endif
            Spinor<Real> v;
            Real sc;
            sa.load_raw(q, v, sc);
            hop_dir<MU, -SF, true, SC>(acc[i], v, U, sc);
        }
    }

    template <int RB>
    LQ_HD void apply_rb(const Site& s, const int c[4], Spinor<Real> (&acc)[RB]) const {
        static_assert(!kRolled, "register blocking is for the unrolled stencils");
#pragma unroll
        for (int i = 0; i < RB; ++i)
#pragma unroll
            for (int k = 0; k < 12; ++k) acc[i].v[k] = {Real(0), Real(0)};
        dir_rb<0, RB>(s, c, acc);
        dir_rb<1, RB>(s, c, acc);
        dir_rb<2, RB>(s, c, acc);
        dir_rb<3, RB>(s, c, acc);
    }
};

// ------------------------------------------------------------------------------------
// Site maps: tile -> sites.  A tile is one block's worth of consecutive sites.
// ------------------------------------------------------------------------------------
// With nr right-hand sides a map covers (site, rhs) pairs, rhs fastest: the nr threads of
// one site are adjacent, so their link loads coincide.  nr is a power of two (lnr = log2)
// dividing BS, so a thread keeps the same rhs = threadIdx.x mod nr in every tile.  With
// register blocking (MapEoFullRB, lrb = log2 RB > 0) a thread takes RB consecutive right-hand
// sides of its site, the first being RB (threadIdx.x mod nr / RB).
template <int BS> struct MapLex {            // all V sites, lexicographic
    Geom g;
    int lnr = 0;
    __host__ __device__ int ntiles() const { return (int)(((int64_t)g.V << lnr) + BS - 1) / BS; }
    __device__ __forceinline__ bool site(int tile, Site& s, int c[4]) const {
        const int f = tile * BS + (int)threadIdx.x;
        if (f >= (g.V << lnr)) return false;
        s = site_from_lex(g, f >> lnr, c, f & ((1 << lnr) - 1));
        return true;
    }
};

template <int BS> struct MapEoFull {         // all V sites; tiles alternate parity over the same cb range
    Geom g;
    int lnr = 0;
    __host__ __device__ int ntiles() const { return 2 * (int)((((int64_t)g.Vh << lnr) + BS - 1) / BS); }
    __device__ __forceinline__ bool site(int tile, Site& s, int c[4]) const {
        const int f = (tile >> 1) * BS + (int)threadIdx.x;
        if (f >= (g.Vh << lnr)) return false;
        s = site_from_eo(g, tile & 1, f >> lnr, c, f & ((1 << lnr) - 1));
        return true;
    }
};

template <int BS> struct MapEoFullRB {       // the same with 2^lrb right-hand sides per thread
    Geom g;
    int lnr = 0;
    int lrb = 0;
    __host__ __device__ int ntiles() const {
        return 2 * (int)((((int64_t)g.Vh << (lnr - lrb)) + BS - 1) / BS);
    }
    __device__ __forceinline__ bool site(int tile, Site& s, int c[4]) const {
        const int f = (tile >> 1) * BS + (int)threadIdx.x, lg = lnr - lrb;
        if (f >= (g.Vh << lg)) return false;
        s = site_from_eo(g, tile & 1, f >> lg, c, (f & ((1 << lg) - 1)) << lrb);
        return true;
    }
};

template <int BS> struct MapEoHalf {         // the Vh sites of one parity
    Geom g;
    int p;
    int lnr = 0;
    __host__ __device__ int ntiles() const { return (int)((((int64_t)g.Vh << lnr) + BS - 1) / BS); }
    __device__ __forceinline__ bool site(int tile, Site& s, int c[4]) const {
        const int f = tile * BS + (int)threadIdx.x;
        if (f >= (g.Vh << lnr)) return false;
        s = site_from_eo(g, p, f >> lnr, c, f & ((1 << lnr) - 1));
        return true;
    }
};

template <typename R> LQ_HD R norm2(const Spinor<R>& a) {
    R s = R(0);
#pragma unroll
    for (int k = 0; k < 12; ++k) s = fma(a.v[k].re, a.v[k].re, fma(a.v[k].im, a.v[k].im, s));
    return s;
}
// FP32 pairs: normalise each component first, so that a value whose lo carries most of it
// (after a cancellation) is squared correctly
LQ_HD dd norm2(const Spinor<dd>& a) {
    dd s = dd(0.f);
#pragma unroll
    for (int k = 0; k < 12; ++k) {
        const dd re = dd_renorm(a.v[k].re), im = dd_renorm(a.v[k].im);
        s = fma(re, re, fma(im, im, s));
    }
    return s;
}

// ------------------------------------------------------------------------------------
// Epilogues.  init() runs once per thread before the site loop and returns false to skip
// the whole kernel (uniformly); active() says whether this thread's right-hand side has
// work (its sites are skipped otherwise, but the thread still joins the reduction);
// apply() consumes the hopping sum of one site; finish() performs the grid reduction.
// ------------------------------------------------------------------------------------

// out = a * y(n) + b * hop(n)        (y = the centre input for the full operator)
// NORM: also reduce ||out||^2 into st->red[slot].
template <class OutA, class YA, bool HASY, bool NORM>
struct EpiAxpby {
    using Real = typename OutA::Real;
    static constexpr int NRED = NORM ? 1 : 0;
    OutA out;
    YA y;
    Real a, b;
    RedCtx rc;
    int slot;
    LQ_HD bool init() { return true; }
    LQ_HD bool active() const { return true; }
    template <typename R>
    LQ_HD void apply(const Site& s, const Spinor<R>& acc, double* red) const {
        Spinor<R> o;
        if constexpr (HASY) {
            Spinor<R> yv;
            y.load(s, yv);
#pragma unroll
            for (int k = 0; k < 12; ++k)
                o.v[k] = {fma((R)b, acc.v[k].re, (R)a * yv.v[k].re), fma((R)b, acc.v[k].im, (R)a * yv.v[k].im)};
        } else {
#pragma unroll
            for (int k = 0; k < 12; ++k) o.v[k] = cscale((R)b, acc.v[k]);
        }
        out.store(s, o);
        if constexpr (NORM) red[0] += to_double(norm2(o));
    }
    template <int BS>
    __device__ __forceinline__ void finish(const double (&red)[NRED > 0 ? NRED : 1], const VGrid& vg) const {
        if constexpr (NORM) {
            const double v[1] = {red[0]};
            SolverState* st = rc.st;
            const int sl = slot;
            grid_reduce<BS, 1>(rc, kTicketMisc, v, vg, [st, sl](const double* t) { st->red[sl][0] = t[0]; });
        }
    }
};

// right-hand sides per thread of an epilogue (1 unless it declares kRB)
template <class E, class = void> struct RhsBlock { static constexpr int value = 1; };
template <class E> struct RhsBlock<E, std::void_t<decltype(E::kRB)>> { static constexpr int value = E::kRB; };

template <class E, class = void> struct HasPrefetch : std::false_type {};
template <class E> struct HasPrefetch<E, std::void_t<decltype(&E::prefetch)>> : std::true_type {};

// Optional minimum resident blocks per SM requested from the compiler (its register
// budget) for the FP32-arithmetic and the FP32-pair stencils; 0 leaves the choice to ptxas.
#ifndef LQ_STENCIL_MINB_F32
#define LQ_STENCIL_MINB_F32 0
#endif
#ifndef LQ_STENCIL_MINB_PAIR
#define LQ_STENCIL_MINB_PAIR 0
#endif
// Optional cap on the resident blocks per SM of the FP32-arithmetic stencils (the grid of the
// grid-stride kernels is sized to it); 0: the occupancy limit.
#ifndef LQ_STENCIL_MAXB_F32
#define LQ_STENCIL_MAXB_F32 0
#endif
template <class Real> struct StencilMaxBlocks { static constexpr int value = 0; };
template <> struct StencilMaxBlocks<float> { static constexpr int value = LQ_STENCIL_MAXB_F32; };
template <class Real> struct StencilMinBlocks { static constexpr int value = 0; };
template <> struct StencilMinBlocks<float> { static constexpr int value = LQ_STENCIL_MINB_F32; };
template <> struct StencilMinBlocks<dd> { static constexpr int value = LQ_STENCIL_MINB_PAIR; };
// Resident blocks per SM asked of ptxas for one stencil kernel (0: ptxas chooses): by default
// by arithmetic type; the solver specialises it for its K1 and K2 beside their epilogues.
template <class Sten, class Epi> struct KernelMinBlocks {
    static constexpr int value = StencilMinBlocks<typename Sten::Real>::value;
};

// Generic stencil kernel: grid-stride over tiles, one thread per site.
template <int BS, class Map, class Sten, class Epi>
__device__ __forceinline__ void stencil_body(const Map& map, const Sten& sten, Epi& epi, const VGrid& vg) {
    if (!epi.init()) return;
    constexpr int NR = Epi::NRED > 0 ? Epi::NRED : 1;
    double red[NR];
#pragma unroll
    for (int j = 0; j < NR; ++j) red[j] = 0.0;
    const int nt = epi.active() ? map.ntiles() : 0;
    const bool rev = reverse_tiles(epi);
    for (int k = vg.bid; k < nt; k += vg.nblk) {
        const int tile = rev ? nt - 1 - k : k;
        Site s;
        int c[4];
        if (!map.site(tile, s, c)) continue;
        // an epilogue may ask for its site-local inputs ahead of the stencil (their loads
        // then hit L1 instead of waiting on DRAM after the eight hops)
        if constexpr (HasPrefetch<Epi>::value) epi.prefetch(s);
        constexpr int RB = RhsBlock<Epi>::value;
        if constexpr (RB > 1) {
            Spinor<typename Sten::Real> acc[RB];
            sten.template apply_rb<RB>(s, c, acc);
            epi.apply_rb(s, acc, red);
        } else {
            Spinor<typename Sten::Real> acc;
            sten.apply(s, c, acc);
            epi.apply(s, acc, red);
        }
    }
    epi.template finish<BS>(red, vg);
}

template <int BS, class Map, class Sten, class Epi>
__global__ void __launch_bounds__(BS) stencil_kernel(Map map, Sten sten, Epi epi) {
    stencil_body<BS>(map, sten, epi, hw_grid());
}

template <int BS, int MINB, class Map, class Sten, class Epi>
__global__ void __launch_bounds__(BS, MINB) stencil_kernel_minb(Map map, Sten sten, Epi epi) {
    stencil_body<BS>(map, sten, epi, hw_grid());
}

// Grid size for a grid-stride kernel: every SM filled to its occupancy, never more
// blocks than tiles, never more than the partial-sum buffer holds.
template <class KernelPtr>
inline int grid_for(KernelPtr k, int bs, int ntiles, int max_per_sm = 0) {
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, bs, 0);
    if (max_per_sm > 0 && per_sm > max_per_sm) per_sm = max_per_sm;
    if (per_sm < 1) per_sm = 1;
    long long g = (long long)sms * per_sm;
    if (g > ntiles) g = ntiles;
    if (g > kMaxPartials) g = kMaxPartials;
    if (g < 1) g = 1;
    return (int)g;
}

template <int BS, class Map, class Sten, class Epi>
inline cudaError_t launch_stencil(const Map& map, const Sten& sten, const Epi& epi, cudaStream_t st) {
    constexpr int MINB = KernelMinBlocks<Sten, Epi>::value;
    auto k = [] {
        if constexpr (MINB > 0) return stencil_kernel_minb<BS, MINB, Map, Sten, Epi>;
        else return stencil_kernel<BS, Map, Sten, Epi>;
    }();
    static thread_local int cached_grid_tiles = -1, cached_grid = 0;
    const int nt = map.ntiles();
    int grid;
    if (cached_grid_tiles == nt) {
        grid = cached_grid;
    } else {
        grid = grid_for(k, BS, nt, StencilMaxBlocks<typename Sten::Real>::value);
        cached_grid_tiles = nt;
        cached_grid = grid;
    }
    k<<<grid, BS, 0, st>>>(map, sten, epi);
    return cudaGetLastError();
}

// EoIdx for a full EO field of K chunks per site, and for a half field of one parity.
inline EoIdx eo_full(const Geom& g, int K, int nr = 1) {
    return EoIdx{(uint32_t)g.Vh, (uint32_t)K * (uint32_t)g.Vh, (uint32_t)g.Vh, (uint32_t)nr, (uint32_t)g.V};
}
inline EoIdx eo_half(const Geom& g, int nr = 1) { return EoIdx{(uint32_t)g.Vh, 0u, 0u, (uint32_t)nr, (uint32_t)g.V}; }
inline EoIdx lex_idx(const Geom& g, int nr = 1) { return EoIdx{0u, 0u, 0u, (uint32_t)nr, (uint32_t)g.V}; }

}  // namespace lq
