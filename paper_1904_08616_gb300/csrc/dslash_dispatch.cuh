// Host-side builders of the public operator kernels: full-lattice D / D^dag in either
// layout, and the parity-to-parity hopping term in the EO layout.  Each precision's
// instances are compiled in their own translation unit (dslash_f64.cu, dslash_f32.cu,
// dslash_f16.cu).
#pragma once

#include "dslash_kernels.cuh"

namespace lq {

constexpr int kApplyBS = 128;

// Spinor accessor over a caller buffer holding nr fields of nsites sites each (V: full
// fields, Vh: half fields), in the layout's multi-field order.
template <int PREC, int LAYOUT, bool RO>
inline SpinorAcc<PREC, LAYOUT, RO> make_spinor(const void* buf, const Geom& g, bool half, int nr = 1) {
    SpinorAcc<PREC, LAYOUT, RO> a;
    const int64_t nsites = (int64_t)(half ? g.Vh : g.V) * nr;
    a.e = (LAYOUT == LQ_LAYOUT_LEX) ? lex_idx(g, nr)
                                    : (half ? eo_half(g, nr) : eo_full(g, SpinorAcc<PREC, LAYOUT, RO>::K, nr));
    if constexpr (PREC == LQ_F64) {
        a.ptr = (double2*)buf;
    } else if constexpr (PREC == LQ_F32 || PREC == LQ_F64X) {
        a.ptr = (float4*)buf;
    } else if constexpr (PREC == LQ_I32S) {
        a.ptr = (int4*)buf;
        a.scale = (float*)((char*)buf + 96 * nsites);
    } else {
        a.ptr = (uint4*)buf;
        a.scale = (float*)((char*)buf + 48 * nsites);
    }
#ifdef LQ_BOUNDS_CHECK
    a.nslots = (uint32_t)(SpinorAcc<PREC, LAYOUT, RO>::K * nsites);
    a.nscales = (uint32_t)nsites;
#endif
    return a;
}

template <int PREC, int FMT, int LAYOUT>
inline GaugeAcc<PREC, FMT, LAYOUT> make_gauge(const void* buf, const Geom& g) {
    GaugeAcc<PREC, FMT, LAYOUT> a;
    a.ptr = (decltype(a.ptr))buf;
    a.Vh = (uint32_t)g.Vh;
#ifdef LQ_BOUNDS_CHECK
    a.nslots = (uint32_t)(4 * GaugeAcc<PREC, FMT, LAYOUT>::K * (int64_t)g.V);
#endif
    return a;
}

// out = D psi (DAG = false) or D^dag psi on the whole lattice, for 2^lnr fields at once
// (LEX: stacked fields; EO: right-hand sides interleaved per site)
template <int PREC, int FMT, int LAYOUT, bool DAG>
cudaError_t run_apply(const Geom& g, double m_q, const void* U, const void* psi, void* out, cudaStream_t st,
                      int lnr = 0) {
    using InA = SpinorAcc<PREC, LAYOUT, true>;
    using OutA = SpinorAcc<PREC, LAYOUT, false>;
    using GA = GaugeAcc<PREC, FMT, LAYOUT>;
    using Real = typename GA::Real;
    const int nr = 1 << lnr;
    Stencil<GA, InA, DAG> sten{g, make_gauge<PREC, FMT, LAYOUT>(U, g), make_spinor<PREC, LAYOUT, true>(psi, g, false, nr)};
    EpiAxpby<OutA, InA, true, false> epi;
    epi.out = make_spinor<PREC, LAYOUT, false>(out, g, false, nr);
    epi.y = sten.sa;
    epi.a = from_double<Real>(m_q + 4.0);
    epi.b = from_double<Real>(0.5);
    epi.rc = RedCtx{nullptr, nullptr};
    epi.slot = 0;
    if constexpr (LAYOUT == LQ_LAYOUT_LEX) return launch_stencil<kApplyBS>(MapLex<kApplyBS>{g, lnr}, sten, epi, st);
    else return launch_stencil<kApplyBS>(MapEoFull<kApplyBS>{g, lnr}, sten, epi, st);
}

// out_p = a y_p + b H_{p,1-p} psi_{1-p}  (EO half fields)
template <int PREC, int FMT, bool DAG, bool HASY>
cudaError_t run_hop(const Geom& g, int p, double a, double b, const void* U, const void* psi_other,
                    const void* y, void* out, cudaStream_t st) {
    constexpr int LAYOUT = LQ_LAYOUT_EO;
    using InA = SpinorAcc<PREC, LAYOUT, true>;
    using OutA = SpinorAcc<PREC, LAYOUT, false>;
    using GA = GaugeAcc<PREC, FMT, LAYOUT>;
    using Real = typename GA::Real;
    Stencil<GA, InA, DAG> sten{g, make_gauge<PREC, FMT, LAYOUT>(U, g), make_spinor<PREC, LAYOUT, true>(psi_other, g, true)};
    EpiAxpby<OutA, InA, HASY, false> epi;
    epi.out = make_spinor<PREC, LAYOUT, false>(out, g, true);
    epi.y = make_spinor<PREC, LAYOUT, true>(HASY ? y : psi_other, g, true);
    epi.a = from_double<Real>(a);
    epi.b = from_double<Real>(0.5 * b);   // the stencil sum excludes the 1/2 of Eq. (1)
    epi.rc = RedCtx{nullptr, nullptr};
    epi.slot = 0;
    return launch_stencil<kApplyBS>(MapEoHalf<kApplyBS>{g, p}, sten, epi, st);
}

// Dispatch entry points, one set per precision (defined in dslash_f64/f32/f16/f64x/i32.cu);
// the applies act on 2^lnr fields.
cudaError_t apply_f64(const Geom& g, double m_q, int fmt, int layout, bool dag, const void* U, const void* psi, void* out, cudaStream_t st, int lnr);
cudaError_t apply_f32(const Geom& g, double m_q, int fmt, int layout, bool dag, const void* U, const void* psi, void* out, cudaStream_t st, int lnr);
cudaError_t apply_f16(const Geom& g, double m_q, int fmt, int layout, bool dag, const void* U, const void* psi, void* out, cudaStream_t st, int lnr);
cudaError_t hop_f64(const Geom& g, int p, bool dag, double a, double b, int fmt, const void* U, const void* psi_other, const void* y, void* out, cudaStream_t st);
cudaError_t hop_f32(const Geom& g, int p, bool dag, double a, double b, int fmt, const void* U, const void* psi_other, const void* y, void* out, cudaStream_t st);
cudaError_t hop_f16(const Geom& g, int p, bool dag, double a, double b, int fmt, const void* U, const void* psi_other, const void* y, void* out, cudaStream_t st);
cudaError_t apply_f64x(const Geom& g, double m_q, int fmt, int layout, bool dag, const void* U, const void* psi, void* out, cudaStream_t st, int lnr);
cudaError_t hop_f64x(const Geom& g, int p, bool dag, double a, double b, int fmt, const void* U, const void* psi_other, const void* y, void* out, cudaStream_t st);
cudaError_t apply_i32(const Geom& g, double m_q, int fmt, int layout, bool dag, const void* U, const void* psi, void* out, cudaStream_t st, int lnr);
cudaError_t hop_i32(const Geom& g, int p, bool dag, double a, double b, int fmt, const void* U, const void* psi_other, const void* y, void* out, cudaStream_t st);

}  // namespace lq

// Defines apply_<name> / hop_<name> for precision PREC.
#define LQ_DEFINE_PREC_DISPATCH(NAME, PREC)                                                            \
    namespace lq {                                                                                   \
    cudaError_t apply_##NAME(const Geom& g, double m_q, int fmt, int layout, bool dag, const void* U, \
                             const void* psi, void* out, cudaStream_t st, int lnr) {                  \
        const bool lex = layout == LQ_LAYOUT_LEX;                                                     \
        if (fmt == 10) {                                                                              \
            if (lex) return dag ? run_apply<PREC, 10, LQ_LAYOUT_LEX, true>(g, m_q, U, psi, out, st, lnr)   \
                                : run_apply<PREC, 10, LQ_LAYOUT_LEX, false>(g, m_q, U, psi, out, st, lnr); \
            return dag ? run_apply<PREC, 10, LQ_LAYOUT_EO, true>(g, m_q, U, psi, out, st, lnr)             \
                       : run_apply<PREC, 10, LQ_LAYOUT_EO, false>(g, m_q, U, psi, out, st, lnr);           \
        }                                                                                             \
        if (fmt == 18) {                                                                              \
            if (lex) return dag ? run_apply<PREC, 18, LQ_LAYOUT_LEX, true>(g, m_q, U, psi, out, st, lnr)   \
                                : run_apply<PREC, 18, LQ_LAYOUT_LEX, false>(g, m_q, U, psi, out, st, lnr); \
            return dag ? run_apply<PREC, 18, LQ_LAYOUT_EO, true>(g, m_q, U, psi, out, st, lnr)             \
                       : run_apply<PREC, 18, LQ_LAYOUT_EO, false>(g, m_q, U, psi, out, st, lnr);           \
        }                                                                                             \
        if (lex) return dag ? run_apply<PREC, 12, LQ_LAYOUT_LEX, true>(g, m_q, U, psi, out, st, lnr)       \
                            : run_apply<PREC, 12, LQ_LAYOUT_LEX, false>(g, m_q, U, psi, out, st, lnr);     \
        return dag ? run_apply<PREC, 12, LQ_LAYOUT_EO, true>(g, m_q, U, psi, out, st, lnr)                 \
                   : run_apply<PREC, 12, LQ_LAYOUT_EO, false>(g, m_q, U, psi, out, st, lnr);               \
    }                                                                                                 \
    cudaError_t hop_##NAME(const Geom& g, int p, bool dag, double a, double b, int fmt, const void* U, \
                           const void* psi_other, const void* y, void* out, cudaStream_t st) {        \
        const bool hy = y != nullptr;                                                                 \
        if (fmt == 10) {                                                                              \
            if (dag) return hy ? run_hop<PREC, 10, true, true>(g, p, a, b, U, psi_other, y, out, st)  \
                               : run_hop<PREC, 10, true, false>(g, p, a, b, U, psi_other, y, out, st); \
            return hy ? run_hop<PREC, 10, false, true>(g, p, a, b, U, psi_other, y, out, st)          \
                      : run_hop<PREC, 10, false, false>(g, p, a, b, U, psi_other, y, out, st);        \
        }                                                                                             \
        if (fmt == 18) {                                                                              \
            if (dag) return hy ? run_hop<PREC, 18, true, true>(g, p, a, b, U, psi_other, y, out, st)  \
                               : run_hop<PREC, 18, true, false>(g, p, a, b, U, psi_other, y, out, st); \
            return hy ? run_hop<PREC, 18, false, true>(g, p, a, b, U, psi_other, y, out, st)          \
                      : run_hop<PREC, 18, false, false>(g, p, a, b, U, psi_other, y, out, st);        \
        }                                                                                             \
        if (dag) return hy ? run_hop<PREC, 12, true, true>(g, p, a, b, U, psi_other, y, out, st)      \
                           : run_hop<PREC, 12, true, false>(g, p, a, b, U, psi_other, y, out, st);    \
        return hy ? run_hop<PREC, 12, false, true>(g, p, a, b, U, psi_other, y, out, st)              \
                  : run_hop<PREC, 12, false, false>(g, p, a, b, U, psi_other, y, out, st);            \
    }                                                                                                 \
    }
