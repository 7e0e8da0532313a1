// Conjugate gradient on A = D^dag D (arXiv 1904.08616, Algorithm 1).
//
// One driver serves all three modes.  The outer loop is Algorithm 1's: FP64 solution
// psi^high (the caller's x), FP64 residual r^high = eta - A psi^high recomputed with the
// FP64 operator (lines 2 and 23), s = ||r^high||, and an inner CG (lines 13-20) on the
// unit-norm residual r_0 = r^high / s in the inner precision.  The inner loop uses
// three fused kernels per iteration:
//   K1  t = D p                       + ||t||^2 = <p, A p>  -> alpha = rho / <p, A p>
//   K2  q = D^dag t (in registers); psi += alpha p; r -= alpha q  + ||r||^2 -> beta, stop
//   K3  p = r + beta p
// Scalars live in a device-side state record written by the last block of each
// reducing kernel; the host only reads that record between chunks of iterations.
//
// Readings of Algorithm 1 (the text has index garbles):
//   * at the start of cycle l, r_0 = r^high_l / s_l;
//   * the first cycle starts from p_0 = r_0, later ones continue the old direction:
//       p_0 = r_0 + beta_0 (p_k - <r_0, p_k> r_0),  beta_0 = s_l / (s_{l-1} rho_k);
//   * rho_0 = ||r_0||^2; psi^high += s_l psi_k;
//   * the inner loop stops when rho_n <= max(delta^2, (tol ||eta|| / s_l)^2) or n = k;
//   * the outer loop stops when s <= tol ||eta|| (relative criterion).
// LQ_CG_F64 runs the same driver with an FP64 inner loop on the caller's links and
// delta = 0, i.e. plain CG followed by an FP64 true-residual check (and, if rounding
// drift left the true residual above tol, another cycle that continues the direction).
//
// The outer (FP64-class) quantities have their own precision HP: native FP64 on the
// caller's LEX fields, or FP32 pairs (LQ_F64X) in EO copies held in the workspace, which
// on GB300 run the residual operator about six times faster than native FP64.
#pragma once

#include <math.h>
#include <string.h>

#include <type_traits>
#include <vector>

#include "lq_abi_internal.h"
#include "dslash_dispatch.cuh"

namespace lq {

namespace solver_detail {

constexpr int kBS = 128;      // stencil kernels
constexpr int kSiteBS = 256;  // site-local kernels

template <typename T> LQ_HD void zero(Spinor<T>& a) {
#pragma unroll
    for (int k = 0; k < 12; ++k) a.v[k] = {T(0), T(0)};
}

// ------------------------------------------------------------------------------------
// site-local kernel: grid-stride over tiles of a map, op.apply per site
// ------------------------------------------------------------------------------------
template <int BS, class Map, class Op>
__global__ void __launch_bounds__(BS) site_kernel(Map map, Op op) {
    if (!op.init()) return;
    constexpr int NR = Op::NRED > 0 ? Op::NRED : 1;
    double red[NR];
#pragma unroll
    for (int j = 0; j < NR; ++j) red[j] = 0.0;
    const int nt = map.ntiles();
    for (int tile = blockIdx.x; tile < nt; tile += gridDim.x) {
        Site s;
        int c[4];
        if (!map.site(tile, s, c)) continue;
        op.apply(s, red);
    }
    op.template finish<BS>(red);
}

template <int BS, class Map, class Op>
cudaError_t launch_site(const Map& map, const Op& op, cudaStream_t st) {
    auto k = site_kernel<BS, Map, Op>;
    static thread_local int cached_tiles = -1, cached_grid = 0;
    const int nt = map.ntiles();
    if (cached_tiles != nt) {
        cached_grid = grid_for(k, BS, nt);
        cached_tiles = nt;
    }
    k<<<cached_grid, BS, 0, st>>>(map, op);
    return cudaGetLastError();
}

// ------------------------------------------------------------------------------------
// inner-loop kernels
// ------------------------------------------------------------------------------------
// K1: t = a p + b hop(p), ||t||^2 -> alpha
template <class TA, class PA>
struct EpiK1 {
    using Real = typename TA::Real;
    static constexpr int NRED = 1;
    TA t;
    PA p;
    Real a, b;
    RedCtx rc;
    LQ_HD bool init() { return rc.st->stop == 0; }
    template <typename R>
    LQ_HD void apply(const Site& s, const Spinor<R>& acc, double* red) const {
        Spinor<R> pv, o;
        p.load(s, pv);
#pragma unroll
        for (int k = 0; k < 12; ++k)
            o.v[k] = {fma((R)b, acc.v[k].re, (R)a * pv.v[k].re), fma((R)b, acc.v[k].im, (R)a * pv.v[k].im)};
        t.store(s, o);
        red[0] += to_double(norm2(o));
    }
    template <int BS> __device__ __forceinline__ void finish(const double (&red)[1]) const {
        SolverState* st = rc.st;
        grid_reduce<BS, 1>(rc, kTicketK1, red, [st](const double* tot) {
            const double sg = tot[0];
            st->sigma = sg;
            if (!isfinite(sg)) {
                st->stop = 3;
                st->alpha = 0.0;
            } else if (!(sg > 0.0)) {
                st->stop = 2;
                st->alpha = 0.0;
            } else {
                st->alpha = st->rho / sg;
            }
        });
    }
};

// K2: q = a t + b hop^dag(t); psi += alpha p; r -= alpha q; ||r||^2 -> beta, stop test
template <class TA, class PA, class XA, class RA>
struct EpiK2 {
    using Real = typename RA::Real;
    static constexpr int NRED = 1;
    TA t;
    PA p;
    XA x;
    RA r;
    Real a, b;
    RedCtx rc;
    Real alpha;
    LQ_HD bool init() {
        if (rc.st->stop) return false;
        alpha = from_double<Real>(rc.st->alpha);
        return true;
    }
    template <typename R>
    LQ_HD void apply(const Site& s, const Spinor<R>& acc, double* red) const {
        Spinor<R> tv, pv, xv, rv;
        t.load(s, tv);
        p.load(s, pv);
        x.load(s, xv);
        r.load(s, rv);
        const R al = (R)alpha;
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            const R qre = fma((R)b, acc.v[k].re, (R)a * tv.v[k].re);
            const R qim = fma((R)b, acc.v[k].im, (R)a * tv.v[k].im);
            xv.v[k] = {fma(al, pv.v[k].re, xv.v[k].re), fma(al, pv.v[k].im, xv.v[k].im)};
            rv.v[k] = {fma(-al, qre, rv.v[k].re), fma(-al, qim, rv.v[k].im)};
        }
        x.store(s, xv);
        r.store(s, rv);
        red[0] += to_double(norm2(rv));
    }
    template <int BS> __device__ __forceinline__ void finish(const double (&red)[1]) const {
        SolverState* st = rc.st;
        grid_reduce<BS, 1>(rc, kTicketK2, red, [st](const double* tot) {
            const double rn = tot[0];
            st->iter += 1;
            if (!isfinite(rn)) {
                st->stop = 3;
                return;
            }
            st->beta = rn / st->rho;
            st->rho = rn;
            if (rn <= st->stop_rho || st->iter >= st->k_max) st->stop = 1;
        });
    }
};

// K3: p = r + beta p, once per completed iteration
template <class PA, class RA>
struct OpK3 {
    using Real = typename PA::Real;
    static constexpr int NRED = 1;
    PA p;
    RA r;
    RedCtx rc;
    Real beta;
    LQ_HD bool init() {
        if (rc.st->p_iter == rc.st->iter) return false;
        beta = from_double<Real>(rc.st->beta);
        return true;
    }
    LQ_HD void apply(const Site& s, double*) const {
        Spinor<Real> pv, rv;
        p.load(s, pv);
        r.load(s, rv);
#pragma unroll
        for (int k = 0; k < 12; ++k) pv.v[k] = {fma(beta, pv.v[k].re, rv.v[k].re), fma(beta, pv.v[k].im, rv.v[k].im)};
        p.store(s, pv);
    }
    template <int BS> __device__ __forceinline__ void finish(const double (&red)[1]) const {
        SolverState* st = rc.st;
        grid_reduce<BS, 1>(rc, kTicketK3, red, [st](const double*) { st->p_iter = st->iter; });
    }
};

// ------------------------------------------------------------------------------------
// cycle start (Algorithm 1 lines 8-12)
// ------------------------------------------------------------------------------------
// r = fl_low(r^high / s); FIRST: p = r; psi = 0.  Otherwise reduce <r, p> and ||r||^2.
template <class RHA, class RA, class PA, class XA, bool FIRST>
struct OpRestart {
    using Real = typename RA::Real;
    static constexpr int NRED = FIRST ? 1 : 3;
    RHA rh;
    RA r;
    PA p;
    XA x;
    double stop_rho;
    int k_max;
    RedCtx rc;
    LQ_HD bool init() { return true; }
    Real is;   // 1/s in the inner arithmetic
    LQ_HD void apply(const Site& s, double* red) const {
        Spinor<Real> w;
        rh.load(s, w);
#pragma unroll
        for (int k = 0; k < 12; ++k) w.v[k] = {is * w.v[k].re, is * w.v[k].im};
        r.store(s, w);
        if constexpr (FIRST) {
            p.store(s, w);
            Spinor<Real> z;
            zero(z);
            x.store(s, z);
            red[0] += to_double(norm2(w));
        } else {
            Spinor<Real> pv;
            p.load(s, pv);
            Real re = Real(0), im = Real(0);
#pragma unroll
            for (int k = 0; k < 12; ++k) {
                re = fma(w.v[k].re, pv.v[k].re, fma(w.v[k].im, pv.v[k].im, re));
                im = fma(w.v[k].re, pv.v[k].im, fma(-w.v[k].im, pv.v[k].re, im));
            }
            red[0] += to_double(re);
            red[1] += to_double(im);
            red[2] += to_double(norm2(w));
        }
    }
    template <int BS> __device__ __forceinline__ void finish(const double (&red)[NRED]) const {
        SolverState* st = rc.st;
        const double sr = stop_rho;
        const int km = k_max;
        grid_reduce<BS, NRED>(rc, kTicketMisc, red, [st, sr, km](const double* tot) {
            if constexpr (FIRST) {
                st->rho = tot[0];
            } else {
                st->red[0] = tot[0];
                st->red[1] = tot[1];
                st->rho = tot[2];
            }
            st->iter = 0;
            st->p_iter = 0;
            st->stop = 0;
            st->stop_rho = sr;
            st->k_max = km;
        });
    }
};

// p = r + beta0 (p - c r), c = <r, p> from the previous kernel; psi = 0
template <class RA, class PA, class XA>
struct OpRestartP {
    using Real = typename RA::Real;
    static constexpr int NRED = 0;
    RA r;
    PA p;
    XA x;
    Real b0;
    RedCtx rc;
    Real cre, cim;
    LQ_HD bool init() {
        cre = from_double<Real>(rc.st->red[0]);
        cim = from_double<Real>(rc.st->red[1]);
        return true;
    }
    LQ_HD void apply(const Site& s, double*) const {
        Spinor<Real> rv, pv;
        r.load(s, rv);
        p.load(s, pv);
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            const cplx<Real> cr = cmul(cplx<Real>{cre, cim}, rv.v[k]);
            pv.v[k] = {fma(b0, pv.v[k].re - cr.re, rv.v[k].re), fma(b0, pv.v[k].im - cr.im, rv.v[k].im)};
        }
        p.store(s, pv);
        Spinor<Real> z;
        zero(z);
        x.store(s, z);
    }
    template <int BS> __device__ __forceinline__ void finish(const double (&)[1]) const {}
};

// psi^high += s psi  (Algorithm 1 line 22 as read above), in the outer arithmetic
template <class XA, class PsiA>
struct OpXUpdate {
    using Real = typename XA::Real;
    static constexpr int NRED = 0;
    XA x;
    PsiA psi;
    Real s;
    LQ_HD bool init() { return true; }
    LQ_HD void apply(const Site& st, double*) const {
        Spinor<Real> xv, pv;
        x.load(st, xv);
        psi.load(st, pv);
#pragma unroll
        for (int k = 0; k < 12; ++k) xv.v[k] = {fma(s, pv.v[k].re, xv.v[k].re), fma(s, pv.v[k].im, xv.v[k].im)};
        x.store(st, xv);
    }
    template <int BS> __device__ __forceinline__ void finish(const double (&)[1]) const {}
};

// ||a||^2 -> st->red[slot] (FP64)
template <class A>
struct OpNorm {
    static constexpr int NRED = 1;
    A a;
    RedCtx rc;
    int slot;
    LQ_HD bool init() { return true; }
    LQ_HD void apply(const Site& s, double* red) const {
        Spinor<double> v;
        a.load(s, v);
        red[0] += norm2(v);
    }
    template <int BS> __device__ __forceinline__ void finish(const double (&red)[1]) const {
        SolverState* st = rc.st;
        const int sl = slot;
        grid_reduce<BS, 1>(rc, kTicketMisc, red, [st, sl](const double* t) { st->red[sl] = t[0]; });
    }
};

// x = 0
template <class XA>
struct OpZero {
    static constexpr int NRED = 0;
    XA x;
    LQ_HD bool init() { return true; }
    LQ_HD void apply(const Site& s, double*) const {
        Spinor<double> z;
        zero(z);
        x.store(s, z);
    }
    template <int BS> __device__ __forceinline__ void finish(const double (&)[1]) const {}
};

// r^high = eta - (a t + b hop^dag(t)), ||r^high||^2 -> st->red[slot]  (outer arithmetic)
template <class EtaA, class TA, class RA>
struct EpiResid {
    using Real = typename RA::Real;
    static constexpr int NRED = 1;
    EtaA eta;
    TA t;
    RA r;
    Real a, b;
    RedCtx rc;
    int slot;
    LQ_HD bool init() { return true; }
    LQ_HD void apply(const Site& s, const Spinor<Real>& acc, double* red) const {
        Spinor<Real> tv, ev, o;
        t.load(s, tv);
        eta.load(s, ev);
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            o.v[k].re = ev.v[k].re - fma(b, acc.v[k].re, a * tv.v[k].re);
            o.v[k].im = ev.v[k].im - fma(b, acc.v[k].im, a * tv.v[k].im);
        }
        r.store(s, o);
        red[0] += to_double(norm2(o));
    }
    template <int BS> __device__ __forceinline__ void finish(const double (&red)[1]) const {
        SolverState* st = rc.st;
        const int sl = slot;
        grid_reduce<BS, 1>(rc, kTicketMisc, red, [st, sl](const double* tt) { st->red[sl] = tt[0]; });
    }
};

// ------------------------------------------------------------------------------------
// workspace layout
// ------------------------------------------------------------------------------------
inline size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

// Workspace: state record, partial sums, then the outer fields, then the inner fields.
// With FP32-pair outer arithmetic (HP = LQ_F64X) the outer fields are EO copies of U, eta
// and x plus r^high and t^high, all as pairs; with native FP64 only r^high and t^high are
// needed (U, eta, x are the caller's).  The query returns the larger of the two.
struct WsLayout {
    size_t state, partials, r_high, t_high, u_x, eta_x, x_x, u_low, psi, r, p, t, total;
};

inline int inner_prec(int mode) {
    switch (mode) {
        case LQ_CG_MIXED_F32: return LQ_F32;
        case LQ_CG_MIXED_F16: return LQ_F16S;
        case LQ_CG_F64X: return LQ_F64X;
        default: return LQ_F64;
    }
}

inline WsLayout ws_layout(const Geom& g, int mode, bool pair_outer, int inner_fmt) {
    WsLayout w{};
    size_t o = 0;
    auto take = [&](size_t bytes) {
        const size_t at = o;
        o += align256(bytes);
        return at;
    };
    w.state = take(sizeof(SolverState));
    w.partials = take(sizeof(double) * 3 * kMaxPartials);
    w.r_high = take(spinor_bytes(g.V, LQ_F64));
    w.t_high = take(spinor_bytes(g.V, LQ_F64));
    if (pair_outer) {
        w.u_x = take(gauge_bytes(g.V, LQ_F64X, 18));
        w.eta_x = take(spinor_bytes(g.V, LQ_F64X));
        w.x_x = take(spinor_bytes(g.V, LQ_F64X));
    }
    const int ip = inner_prec(mode);
    if (mode == LQ_CG_MIXED_F32 || mode == LQ_CG_MIXED_F16) w.u_low = take(gauge_bytes(g.V, ip, inner_fmt));
    const size_t lo = spinor_bytes(g.V, ip);
    w.psi = take(lo);
    w.r = take(lo);
    w.p = take(lo);
    w.t = take(lo);
    w.total = o;
    return w;
}

inline size_t ws_bytes_for_mode(const Geom& g, int mode) {
    size_t m = 0;
    // native FP64 CG never uses pair copies; the FP32-pair CG always does; the mixed modes
    // may use either (LQ_CG_NATIVE_F64)
    const int pair_lo = (mode == LQ_CG_F64X) ? 1 : 0, pair_hi = (mode == LQ_CG_F64) ? 0 : 1;
    for (int pair = pair_lo; pair <= pair_hi; ++pair)
        for (int fmt : {12, 18}) {
            const size_t t = ws_layout(g, mode, pair != 0, fmt).total;
            if (t > m) m = t;
        }
    return m;
}

// ------------------------------------------------------------------------------------
// the driver: inner precision IP / link format IF / layout IL, outer precision HP
// ------------------------------------------------------------------------------------
template <int HP> struct Outer;
template <> struct Outer<LQ_F64> {      // the caller's FP64 LEX fields
    static constexpr int L = LQ_LAYOUT_LEX;
};
template <> struct Outer<LQ_F64X> {     // FP32-pair EO copies in the workspace
    static constexpr int L = LQ_LAYOUT_EO;
};

template <int IP, int IF, int IL, int HP>
int run_solver(const Geom& g, double m_q, const void* U, const void* eta, void* x, const lq_cg_params& prm,
               double delta, const WsLayout& w, char* ws, lq_cg_info* info, cudaStream_t st) {
    using Real = typename PrecT<IP>::Real;
    using HReal = typename PrecT<HP>::Real;
    constexpr int HL = Outer<HP>::L;
    using SpRO = SpinorAcc<IP, IL, true>;
    using SpRW = SpinorAcc<IP, IL, false>;
    using GA = GaugeAcc<IP, IF, IL>;
    using HiRO = SpinorAcc<HP, HL, true>;
    using HiRW = SpinorAcc<HP, HL, false>;
    using HiGA = GaugeAcc<HP, 18, HL>;
    using CallerRO = SpinorAcc<LQ_F64, LQ_LAYOUT_LEX, true>;
    using IMap = typename std::conditional<IL == LQ_LAYOUT_LEX, MapLex<kBS>, MapEoFull<kBS>>::type;
    using ISiteMap = typename std::conditional<IL == LQ_LAYOUT_LEX, MapLex<kSiteBS>, MapEoFull<kSiteBS>>::type;
    using HMap = typename std::conditional<HL == LQ_LAYOUT_LEX, MapLex<kBS>, MapEoFull<kBS>>::type;
    using HSiteMap = typename std::conditional<HL == LQ_LAYOUT_LEX, MapLex<kSiteBS>, MapEoFull<kSiteBS>>::type;
    constexpr bool kPairs = (HP == LQ_F64X);

    SolverState* dstate = (SolverState*)(ws + w.state);
    const RedCtx rc{dstate, (double*)(ws + w.partials)};
    const double a = m_q + 4.0, b = 0.5;

    // outer fields: the caller's arrays (native FP64) or pair copies in the workspace
    const void* Uo = kPairs ? (const void*)(ws + w.u_x) : U;
    const void* etao = kPairs ? (const void*)(ws + w.eta_x) : eta;
    void* xo = kPairs ? (void*)(ws + w.x_x) : x;
    const HiGA Uh = make_gauge<HP, 18, HL>(Uo, g);
    const HiRO eta_ro = make_spinor<HP, HL, true>(etao, g, false);
    const HiRO x_ro = make_spinor<HP, HL, true>(xo, g, false);
    const HiRW x_rw = make_spinor<HP, HL, false>(xo, g, false);
    const HiRO rh_ro = make_spinor<HP, HL, true>(ws + w.r_high, g, false);
    const HiRW rh_rw = make_spinor<HP, HL, false>(ws + w.r_high, g, false);
    const HiRO th_ro = make_spinor<HP, HL, true>(ws + w.t_high, g, false);
    const HiRW th_rw = make_spinor<HP, HL, false>(ws + w.t_high, g, false);
    const CallerRO eta_caller = make_spinor<LQ_F64, LQ_LAYOUT_LEX, true>(eta, g, false);
    const SpinorAcc<LQ_F64, LQ_LAYOUT_LEX, false> x_caller = make_spinor<LQ_F64, LQ_LAYOUT_LEX, false>(x, g, false);

    // inner fields; an FP64-class inner loop shares the outer links
    const void* Ulow = (IP == LQ_F64) ? U : (IP == LQ_F64X ? Uo : (const void*)(ws + w.u_low));
    const GA Ui = make_gauge<IP, IF, IL>(Ulow, g);
    const SpRO psi_ro = make_spinor<IP, IL, true>(ws + w.psi, g, false);
    const SpRW psi_rw = make_spinor<IP, IL, false>(ws + w.psi, g, false);
    const SpRO r_ro = make_spinor<IP, IL, true>(ws + w.r, g, false);
    const SpRW r_rw = make_spinor<IP, IL, false>(ws + w.r, g, false);
    const SpRO p_ro = make_spinor<IP, IL, true>(ws + w.p, g, false);
    const SpRW p_rw = make_spinor<IP, IL, false>(ws + w.p, g, false);
    const SpRO t_ro = make_spinor<IP, IL, true>(ws + w.t, g, false);
    const SpRW t_rw = make_spinor<IP, IL, false>(ws + w.t, g, false);

    const MapLex<kSiteBS> lexsite{g};
    const HMap hmap{g};
    const HSiteMap hsite{g};
    const IMap imap{g};
    const ISiteMap isite{g};

    cudaError_t e;
    SolverState hs;
    lq_cg_info out{};
    const bool prof = (prm.flags & LQ_CG_PROFILE) != 0;
    const int chunk = prm.chunk > 0 ? prm.chunk : (g.V >= (1 << 18) ? 8 : 32);
    // CUDA events around the inner kernels (3 roles x chunk) and the outer residual
    struct Events {
        std::vector<cudaEvent_t> ev;
        ~Events() {
            for (cudaEvent_t x : ev) cudaEventDestroy(x);
        }
    } evs;
    if (prof) {
        evs.ev.resize(6 * chunk + 2);
        for (auto& ev : evs.ev)
            if ((e = cudaEventCreate(&ev)) != cudaSuccess) return cuda_fail(e, "event create");
    }
    auto ev_at = [&](int role, int j, int end) { return evs.ev[(role * chunk + j) * 2 + end]; };
    auto elapsed = [&](cudaEvent_t a0, cudaEvent_t a1) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, a0, a1);
        return (double)ms;
    };
    auto read_state = [&]() -> cudaError_t {
        cudaError_t er = cudaMemcpyAsync(&hs, dstate, sizeof(hs), cudaMemcpyDeviceToHost, st);
        if (er != cudaSuccess) return er;
        return cudaStreamSynchronize(st);
    };

    // r^high = eta - A x, s^2 -> red[2]   (Algorithm 1 lines 2 and 23)
    auto high_residual = [&]() -> cudaError_t {
        Stencil<HiGA, HiRO, false> s1{g, Uh, x_ro};
        EpiAxpby<HiRW, HiRO, true, false> e1;
        e1.out = th_rw;
        e1.y = x_ro;
        e1.a = from_double<HReal>(a);
        e1.b = from_double<HReal>(b);
        e1.rc = rc;
        e1.slot = 0;
        if (prof) cudaEventRecord(evs.ev[6 * chunk], st);
        cudaError_t er = launch_stencil<kBS>(hmap, s1, e1, st);
        if (er != cudaSuccess) return er;
        Stencil<HiGA, HiRO, true> s2{g, Uh, th_ro};
        EpiResid<HiRO, HiRO, HiRW> e2{eta_ro, th_ro, rh_rw, from_double<HReal>(a), from_double<HReal>(b), rc, 2};
        er = launch_stencil<kBS>(hmap, s2, e2, st);
        out.launches += 2;
        if (prof) cudaEventRecord(evs.ev[6 * chunk + 1], st);
        return er;
    };
    // after the stream has been synchronised: add the residual's event time
    auto account_high = [&]() {
        if (!prof) return;
        out.kernel_ms[LQ_K_HIGH] += elapsed(evs.ev[6 * chunk], evs.ev[6 * chunk + 1]);
        out.kernel_calls[LQ_K_HIGH] += 2;
    };
    // the pair copy of x back into the caller's FP64 x
    auto write_back_x = [&]() -> cudaError_t {
        if constexpr (kPairs) {
            out.launches += 1;
            return convert_spinor(g, LQ_F64X, LQ_LAYOUT_EO, xo, LQ_F64, LQ_LAYOUT_LEX, x, st);
        }
        return cudaSuccess;
    };

    if ((e = cudaMemsetAsync(dstate, 0, sizeof(SolverState), st)) != cudaSuccess) return cuda_fail(e, "state init");
    if constexpr (kPairs) {
        if ((e = convert_gauge(g, LQ_F64, LQ_LAYOUT_LEX, U, LQ_F64X, 18, LQ_LAYOUT_EO, ws + w.u_x, st)) != cudaSuccess ||
            (e = convert_spinor(g, LQ_F64, LQ_LAYOUT_LEX, eta, LQ_F64X, LQ_LAYOUT_EO, ws + w.eta_x, st)) != cudaSuccess ||
            (e = convert_spinor(g, LQ_F64, LQ_LAYOUT_LEX, x, LQ_F64X, LQ_LAYOUT_EO, ws + w.x_x, st)) != cudaSuccess)
            return cuda_fail(e, "FP32-pair copies");
        out.launches += 3;
    }
    if constexpr (IP == LQ_F32 || IP == LQ_F16S) {
        if ((e = convert_gauge(g, LQ_F64, LQ_LAYOUT_LEX, U, IP, IF, IL, ws + w.u_low, st)) != cudaSuccess)
            return cuda_fail(e, "link pack");
        out.launches += 1;
    }
    // ||eta||^2 -> red[3], from the caller's FP64 eta
    if ((e = launch_site<kSiteBS>(lexsite, OpNorm<CallerRO>{eta_caller, rc, 3}, st)) != cudaSuccess)
        return cuda_fail(e, "norm");
    out.launches += 1;
    if ((e = read_state()) != cudaSuccess) return cuda_fail(e, "norm");
    const double eta_norm = sqrt(hs.red[3]);
    out.eta_norm = eta_norm;
    if (!isfinite(eta_norm)) return fail(LQ_ERR_NONFINITE, "eta has non-finite entries");
    if (eta_norm == 0.0) {
        if ((e = launch_site<kSiteBS>(lexsite, OpZero<SpinorAcc<LQ_F64, LQ_LAYOUT_LEX, false>>{x_caller}, st)) != cudaSuccess)
            return cuda_fail(e, "zero");
        out.launches += 1;
        if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return cuda_fail(e, "zero");
        out.status = LQ_OK;
        if (info) *info = out;
        return LQ_OK;
    }

    if ((e = high_residual()) != cudaSuccess) return cuda_fail(e, "residual");
    if ((e = read_state()) != cudaSuccess) return cuda_fail(e, "residual");
    account_high();
    double s = sqrt(hs.red[2]);
    out.high_applies = 1;
    const double target = prm.tol * eta_norm;
    double s_prev = 0.0, rho_k = 0.0;
    int l = 0, total = 0, stagnant = 0, status = LQ_OK;
    const int max_cycles = prm.max_cycles > 0 ? prm.max_cycles : 1000;

    while (true) {
        if (!isfinite(s)) {
            status = fail(LQ_ERR_NONFINITE, "FP64 residual became non-finite");
            break;
        }
        if (s <= target) break;
        if (l >= max_cycles || total >= prm.max_iter || stagnant >= 5) {
            status = LQ_NOT_CONVERGED;
            break;
        }
        const double rel_target = target / s;
        const double stop_rho = fmax(delta * delta, rel_target * rel_target);
        const int k_max = prm.max_iter - total;
        // cycle start: both fields of the restart live on the outer map's sites
        if (l == 0) {
            OpRestart<HiRO, SpRW, SpRW, SpRW, true> op{rh_ro, r_rw, p_rw, psi_rw, stop_rho, k_max, rc,
                                                       from_double<Real>(1.0 / s)};
            e = launch_site<kSiteBS>(hsite, op, st);
            out.launches += 1;
        } else {
            OpRestart<HiRO, SpRW, SpRO, SpRW, false> op{rh_ro, r_rw, p_ro, psi_rw, stop_rho, k_max, rc,
                                                        from_double<Real>(1.0 / s)};
            e = launch_site<kSiteBS>(hsite, op, st);
            if (e == cudaSuccess) {
                OpRestartP<SpRO, SpRW, SpRW> op2;
                op2.r = r_ro;
                op2.p = p_rw;
                op2.x = psi_rw;
                op2.b0 = from_double<Real>(s / (s_prev * rho_k));
                op2.rc = rc;
                e = launch_site<kSiteBS>(isite, op2, st);
            }
            out.launches += 2;
        }
        if (e != cudaSuccess) return cuda_fail(e, "cycle start");

        // inner CG: chunks of K1, K2, K3 until the device-side stop flag is set
        Stencil<GA, SpRO, false> sK1{g, Ui, p_ro};
        EpiK1<SpRW, SpRO> eK1{t_rw, p_ro, from_double<Real>(a), from_double<Real>(b), rc};
        Stencil<GA, SpRO, true> sK2{g, Ui, t_ro};
        EpiK2<SpRO, SpRO, SpRW, SpRW> eK2{t_ro, p_ro, psi_rw, r_rw, from_double<Real>(a), from_double<Real>(b), rc,
                                          Real(0)};
        OpK3<SpRW, SpRO> oK3{p_rw, r_ro, rc, Real(0)};
        int guard = 0, iter_before = 0;
        while (true) {
            for (int j = 0; j < chunk; ++j) {
                if (prof) cudaEventRecord(ev_at(0, j, 0), st);
                if ((e = launch_stencil<kBS>(imap, sK1, eK1, st)) != cudaSuccess) return cuda_fail(e, "K1");
                if (prof) cudaEventRecord(ev_at(0, j, 1), st);
                if ((e = launch_stencil<kBS>(imap, sK2, eK2, st)) != cudaSuccess) return cuda_fail(e, "K2");
                if (prof) cudaEventRecord(ev_at(1, j, 1), st);
                if ((e = launch_site<kSiteBS>(isite, oK3, st)) != cudaSuccess) return cuda_fail(e, "K3");
                if (prof) cudaEventRecord(ev_at(2, j, 1), st);
            }
            out.launches += 3 * chunk;
            if ((e = read_state()) != cudaSuccess) return cuda_fail(e, "inner loop");
            if (prof) {
                // only the iterations that ran in this chunk; later launches found the stop flag
                const int ran = hs.iter - iter_before;
                for (int j = 0; j < ran && j < chunk; ++j) {
                    out.kernel_ms[LQ_K_APPLY_D] += elapsed(ev_at(0, j, 0), ev_at(0, j, 1));
                    out.kernel_ms[LQ_K_APPLY_DDAG] += elapsed(ev_at(0, j, 1), ev_at(1, j, 1));
                    out.kernel_ms[LQ_K_UPDATE_P] += elapsed(ev_at(1, j, 1), ev_at(2, j, 1));
                    out.kernel_calls[LQ_K_APPLY_D] += 1;
                    out.kernel_calls[LQ_K_APPLY_DDAG] += 1;
                    out.kernel_calls[LQ_K_UPDATE_P] += 1;
                }
            }
            iter_before = hs.iter;
            if (hs.stop) break;
            if (++guard > (k_max / chunk) + 2) break;   // cannot happen: K2 stops at k_max
        }
        if (hs.stop >= 2) {
            // breakdown or non-finite: keep x as it is (the last reliable iterate)
            status = fail(hs.stop == 2 ? LQ_ERR_BREAKDOWN : LQ_ERR_NONFINITE,
                          hs.stop == 2 ? "CG breakdown: <p, D^dag D p> <= 0" : "inner CG produced non-finite values");
            total += hs.iter;
            break;
        }
        total += hs.iter;
        rho_k = hs.rho;
        // psi^high += s psi_k; then the outer residual
        OpXUpdate<HiRW, SpinorAcc<IP, IL, true>> xu{x_rw, psi_ro, from_double<HReal>(s)};
        if constexpr (HL == IL) e = launch_site<kSiteBS>(hsite, xu, st);
        else e = launch_site<kSiteBS>(lexsite, xu, st);
        if (e != cudaSuccess) return cuda_fail(e, "x update");
        out.launches += 1;
        if ((e = high_residual()) != cudaSuccess) return cuda_fail(e, "residual");
        if ((e = read_state()) != cudaSuccess) return cuda_fail(e, "residual");
        account_high();
        out.high_applies += 1;
        const double s_new = sqrt(hs.red[2]);
        stagnant = (s_new > 0.999 * s) ? stagnant + 1 : 0;
        s_prev = s;
        s = s_new;
        ++l;
    }
    if ((e = write_back_x()) != cudaSuccess) return cuda_fail(e, "x write-back");
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return cuda_fail(e, "x write-back");
    out.iters = total;
    out.cycles = l;
    out.true_rel_resid = s / eta_norm;
    out.status = status;
    if (info) *info = out;
    return status;
}

// Instantiations live in solver_f64.cu (FP64 and FP32-pair inner loops), solver_f32.cu
// and solver_f16.cu (mixed inner loops with either outer arithmetic and link format).
int solve_f64(const Geom& g, double m_q, const void* U, const void* eta, void* x, const lq_cg_params& prm,
              double delta, const WsLayout& w, char* ws, lq_cg_info* info, cudaStream_t st);
int solve_f64x(const Geom& g, double m_q, const void* U, const void* eta, void* x, const lq_cg_params& prm,
               double delta, const WsLayout& w, char* ws, lq_cg_info* info, cudaStream_t st);
int solve_mixed_f32(const Geom& g, double m_q, const void* U, const void* eta, void* x, const lq_cg_params& prm,
                    double delta, const WsLayout& w, char* ws, lq_cg_info* info, cudaStream_t st, bool pairs,
                    int fmt);
int solve_mixed_f16(const Geom& g, double m_q, const void* U, const void* eta, void* x, const lq_cg_params& prm,
                    double delta, const WsLayout& w, char* ws, lq_cg_info* info, cudaStream_t st, bool pairs,
                    int fmt);

}  // namespace solver_detail

}  // namespace lq
