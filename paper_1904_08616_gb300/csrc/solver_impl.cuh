// Conjugate gradient on A = D^dag D (arXiv 1904.08616, Algorithm 1), for a batch of up to
// kMaxRhs right-hand sides solved as independent CGs that share every link load.
//
// One driver serves all modes.  The outer loop is Algorithm 1's: FP64-class solution
// psi^high, FP64-class residual r^high = eta - A psi^high recomputed with the FP64-class
// operator at the start and after every cycle, s = ||r^high||, and an inner CG on the
// unit-norm residual r_0 = r^high / s in the inner precision.  The inner loop uses
// three fused kernels per iteration:
//   K1  t = D p                       + ||t||^2 = <p, A p>  -> alpha = rho / <p, A p>
//   K2  q = D^dag t (in registers); psi += alpha p; r -= alpha q  + ||r||^2 -> beta, stop
//   K3  p = r + beta p
// Scalars live in a device-side state record (one slot per right-hand side) written by
// the last block of each reducing kernel; the host reads that record once per cycle (or
// between chunks of iterations when it drives the inner loop itself).  A right-hand side whose inner loop has stopped is skipped by
// the kernels while the others go on; the cycles (reliable updates) are taken together.
//
// Readings of Algorithm 1 (the text has index garbles):
//   * at the start of cycle l, r_0 = r^high_l / s_l;
//   * the first cycle starts from p_0 = r_0, later ones continue the old direction:
//       p_0 = r_0 + beta_0 (p_k - <r_0, p_k> r_0),  beta_0 = s_l / (s_{l-1} rho_k),
//     unless the new true residual exceeds twice the inner recurrence's prediction
//     (s_l > 2 s_{l-1} sqrt(rho_k), as below the resolution of the outer arithmetic), when
//     the cycle starts afresh from p_0 = r_0;
//   * the inner loop takes at most k iterations per cycle (lq_cg_params.max_inner, 1000);
//   * rho_0 = ||r_0||^2; psi^high += s_l psi_k;
//   * the inner loop stops when rho_n <= max(delta^2, (tol ||eta|| / s_l)^2) or n = k;
//   * the outer loop stops when s <= tol ||eta|| (relative criterion).
// LQ_CG_F64 runs the same driver with an FP64 inner loop on the caller's links and
// delta = 0, i.e. plain CG followed by an FP64 true-residual check (and, if rounding
// drift left the true residual above tol, another cycle that continues the direction).
//
// The outer (FP64-class) quantities have their own precision HP: native FP64 on the
// caller's LEX fields, or FP32 pairs (LQ_F64X) in EO copies held in the workspace, which
// on GB300 run the residual operator about four times faster than native FP64.
#pragma once

#include <math.h>
#include <string.h>

#include <string>
#include <type_traits>
#include <vector>

#include "lq_abi_internal.h"
#include "dslash_dispatch.cuh"

namespace lq {

namespace solver_detail {

// Precision of the inner solution psi (the sum of the cycle's alpha p updates): FP32 when
// the inner vectors are scaled FP16.  psi is read and written once per iteration (by K2), and
// its FP16 quantisation, repeated every iteration, had capped the residual reduction one
// cycle could reach (delta 0.1 instead of 0.01, twice the cycles).
constexpr int psi_prec(int ip) { return ip == LQ_F16S ? LQ_F32 : ip; }


constexpr int kBS = 128;      // stencil kernels
constexpr int kSiteBS = 256;  // site-local kernels

template <typename T> LQ_HD void zero(Spinor<T>& a) {
#pragma unroll
    for (int k = 0; k < 12; ++k) a.v[k] = {T(0), T(0)};
}

// this thread's right-hand side (the maps give every thread a fixed one)
LQ_HD int thread_rhs(int nr) {
#ifdef __CUDA_ARCH__
    return (int)threadIdx.x & (nr - 1);
#else
    (void)nr;
    return 0;
#endif
}

// ------------------------------------------------------------------------------------
// site-local kernel: grid-stride over tiles of a map, op.apply per site
// ------------------------------------------------------------------------------------
template <int BS, class Map, class Op>
__device__ __forceinline__ void site_body(const Map& map, Op& op, const VGrid& vg) {
    if (!op.init()) return;
    constexpr int NR = Op::NRED > 0 ? Op::NRED : 1;
    double red[NR];
#pragma unroll
    for (int j = 0; j < NR; ++j) red[j] = 0.0;
    const int nt = op.active() ? map.ntiles() : 0;
    for (int tile = vg.bid; tile < nt; tile += vg.nblk) {
        Site s;
        int c[4];
        if (!map.site(tile, s, c)) continue;
        op.apply(s, red);
    }
    op.template finish<BS>(red, vg);
}

template <int BS, class Map, class Op>
__global__ void __launch_bounds__(BS) site_kernel(Map map, Op op) {
    site_body<BS>(map, op, hw_grid());
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

// Per-right-hand-side scalars handed to a kernel as a parameter.
template <typename T> struct PerRhs { T v[kMaxRhs]; };

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
    int nr;
    bool on;
    LQ_HD bool init() {
        if (rc.st->all_stop) return false;
        on = rc.st->stop[thread_rhs(nr)] == 0;
        return true;
    }
    LQ_HD bool active() const { return on; }
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
    template <int BS> __device__ __forceinline__ void finish(const double (&red)[1], const VGrid& vg) const {
        SolverState* st = rc.st;
        const int n = nr;
        grid_reduce_seg<BS, 1>(rc, kTicketK1, red, n, vg, [st, n](const double* tot) {
            for (int j = 0; j < n; ++j) {
                if (st->stop[j]) continue;
                const double sg = tot[j];
                st->sigma[j] = sg;
                if (!isfinite(sg)) {
                    st->stop[j] = 3;
                    st->alpha[j] = 0.0;
                } else if (!(sg > 0.0)) {
                    st->stop[j] = 2;
                    st->alpha[j] = 0.0;
                } else {
                    st->alpha[j] = st->rho[j] / sg;
                }
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
    int nr;
    Real alpha;
    bool on;
    LQ_HD bool init() {
        if (rc.st->all_stop) return false;
        const int j = thread_rhs(nr);
        on = rc.st->stop[j] == 0;
        alpha = from_double<Real>(rc.st->alpha[j]);
        return true;
    }
    LQ_HD bool active() const { return on; }
    // K2 walks its tiles from the last to the first: it starts on the sites K1 wrote last,
    // whose t, links and p are still in L2, and ends on the ones K3 reads first, leaving
    // their r and p in L2 (32^4 scaled FP16: K2 96.5 -> 94.6 us, K3 32.9 -> 30.8 us).
    // Alternating all three kernels' order every iteration, so that K1 would start on
    // K3's last sites as well, made K1 slower on its backward sweeps and is not used.
    LQ_HD bool reverse_tiles() const { return true; }
    // psi is read once per site and never by a neighbour: asked for before the stencil, its
    // load after the eight hops hits L1 (K2 6% faster on the 32^4 workload; prefetching the
    // other fields as well gained nothing more)
    LQ_HD void prefetch(const Site& s) const { x.prefetch(s); }
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
    template <int BS> __device__ __forceinline__ void finish(const double (&red)[1], const VGrid& vg) const {
        SolverState* st = rc.st;
        const int n = nr;
        grid_reduce_seg<BS, 1>(rc, kTicketK2, red, n, vg, [st, n](const double* tot) {
            int all = 1;
            for (int j = 0; j < n; ++j) {
                if (!st->stop[j]) {
                    const double rn = tot[j];
                    st->iter[j] += 1;
                    if (!isfinite(rn)) {
                        st->stop[j] = 3;
                    } else {
                        st->beta[j] = rn / st->rho[j];
                        st->rho[j] = rn;
                        if (rn <= st->stop_rho[j] || st->iter[j] >= st->k_max) st->stop[j] = 1;
                    }
                }
                all &= (st->stop[j] != 0);
            }
            st->all_stop = all;
        });
    }
};

}  // namespace solver_detail

// stored precision of a spinor accessor and link format of a gauge accessor
template <class A> struct SpinorPrec { static constexpr int value = -1; };
template <int P, int L, bool RO> struct SpinorPrec<SpinorAcc<P, L, RO>> { static constexpr int value = P; };
template <class A> struct GaugeFmt { static constexpr int value = -1; };
template <int P, int F, int L> struct GaugeFmt<GaugeAcc<P, F, L>> { static constexpr int value = F; };

// The inner K1 and K2 with 12-real links ask for at least 5 resident blocks of 128 threads (at
// most 102 registers).  On the 32^4 solves: FP32 fields K1 96.5 / K2 141.5 us against 102.0 /
// 153.8 with ptxas's own choice (104 registers, 4 blocks); scaled FP16 K1 75.1 against 78.7
// (ptxas's 80 registers, 6 blocks), while its K2 is faster as ptxas leaves it (96.2 against
// 100.7 us at 5 blocks).
template <class GA, class SA, bool DAG, class TA, class PA>
struct KernelMinBlocks<Stencil<GA, SA, DAG>, solver_detail::EpiK1<TA, PA>> {
    static constexpr bool kSet = GaugeFmt<GA>::value == 12 &&
                                 (SpinorPrec<SA>::value == LQ_F32 || SpinorPrec<SA>::value == LQ_F16S);
    static constexpr int value = kSet ? 5 : StencilMinBlocks<typename GA::Real>::value;
};
template <class GA, class SA, bool DAG, class TA, class PA, class XA, class RA>
struct KernelMinBlocks<Stencil<GA, SA, DAG>, solver_detail::EpiK2<TA, PA, XA, RA>> {
    static constexpr bool kSet = GaugeFmt<GA>::value == 12 && SpinorPrec<SA>::value == LQ_F32;
    static constexpr int value = kSet ? 5 : StencilMinBlocks<typename GA::Real>::value;
};

namespace solver_detail {

// The right-hand sides a thread serves: RB consecutive ones starting at this value (the
// maps give every thread a fixed group).
LQ_HD int thread_rhs0(int nr, int rb) {
#ifdef __CUDA_ARCH__
    return ((int)threadIdx.x & (nr / rb - 1)) * rb;
#else
    (void)nr;
    (void)rb;
    return 0;
#endif
}

// K1 with RB > 1 right-hand sides per thread (register blocking: the stencil has applied
// each link to all of them); the single-right-hand-side form EpiK1 is above.
template <class TA, class PA, int RB>
struct EpiK1Blk {
    using Real = typename TA::Real;
    static constexpr int kRB = RB;
    static constexpr int NRED = RB;
    TA t;
    PA p;
    Real a, b;
    RedCtx rc;
    int nr;
    bool on[RB];
    LQ_HD bool init() {
        if (rc.st->all_stop) return false;
        const int j0 = thread_rhs0(nr, RB);
#pragma unroll
        for (int i = 0; i < RB; ++i) on[i] = rc.st->stop[j0 + i] == 0;
        return true;
    }
    LQ_HD bool active() const {
        bool any = false;
#pragma unroll
        for (int i = 0; i < RB; ++i) any |= on[i];
        return any;
    }
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
    template <typename R>
    LQ_HD void apply_rb(const Site& s, const Spinor<R> (&acc)[RB], double* red) const {
#pragma unroll
        for (int i = 0; i < RB; ++i) {
            if (!on[i]) continue;
            const Site si{s.lex, s.p, s.cb, s.rhs + i};
            Spinor<R> pv, o;
            p.load(si, pv);
#pragma unroll
            for (int k = 0; k < 12; ++k)
                o.v[k] = {fma((R)b, acc[i].v[k].re, (R)a * pv.v[k].re), fma((R)b, acc[i].v[k].im, (R)a * pv.v[k].im)};
            t.store(si, o);
            red[i] += to_double(norm2(o));
        }
    }
    template <int BS> __device__ __forceinline__ void finish(const double (&red)[RB], const VGrid& vg) const {
        SolverState* st = rc.st;
        const int n = nr;
        grid_reduce_seg<BS, RB>(rc, kTicketK1, red, n / RB, vg, [st, n](const double* tot) {
            for (int j = 0; j < n; ++j) {
                if (st->stop[j]) continue;
                const double sg = tot[(j % RB) * kMaxRhs + j / RB];
                st->sigma[j] = sg;
                if (!isfinite(sg)) {
                    st->stop[j] = 3;
                    st->alpha[j] = 0.0;
                } else if (!(sg > 0.0)) {
                    st->stop[j] = 2;
                    st->alpha[j] = 0.0;
                } else {
                    st->alpha[j] = st->rho[j] / sg;
                }
            }
        });
    }
};

// K2 with RB > 1 right-hand sides per thread; the single-right-hand-side form EpiK2 is above.
template <class TA, class PA, class XA, class RA, int RB>
struct EpiK2Blk {
    using Real = typename RA::Real;
    static constexpr int kRB = RB;
    static constexpr int NRED = RB;
    TA t;
    PA p;
    XA x;
    RA r;
    Real a, b;
    RedCtx rc;
    int nr;
    Real alpha[RB];
    bool on[RB];
    LQ_HD bool init() {
        if (rc.st->all_stop) return false;
        const int j0 = thread_rhs0(nr, RB);
#pragma unroll
        for (int i = 0; i < RB; ++i) {
            on[i] = rc.st->stop[j0 + i] == 0;
            alpha[i] = from_double<Real>(rc.st->alpha[j0 + i]);
        }
        return true;
    }
    LQ_HD bool active() const {
        bool any = false;
#pragma unroll
        for (int i = 0; i < RB; ++i) any |= on[i];
        return any;
    }
    // psi is read once per site and never by a neighbour: asked for before the stencil, its
    // load after the eight hops hits L1 (K2 6% faster on the 32^4 workload; prefetching the
    // other fields as well gained nothing more)
    LQ_HD void prefetch(const Site& s) const {
#pragma unroll
        for (int i = 0; i < RB; ++i) x.prefetch(Site{s.lex, s.p, s.cb, s.rhs + i});
    }
    template <typename R>
    LQ_HD void update(const Site& s, const Spinor<R>& acc, R al, double& red) const {
        Spinor<R> tv, pv, xv, rv;
        t.load(s, tv);
        p.load(s, pv);
        x.load(s, xv);
        r.load(s, rv);
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            const R qre = fma((R)b, acc.v[k].re, (R)a * tv.v[k].re);
            const R qim = fma((R)b, acc.v[k].im, (R)a * tv.v[k].im);
            xv.v[k] = {fma(al, pv.v[k].re, xv.v[k].re), fma(al, pv.v[k].im, xv.v[k].im)};
            rv.v[k] = {fma(-al, qre, rv.v[k].re), fma(-al, qim, rv.v[k].im)};
        }
        x.store(s, xv);
        r.store(s, rv);
        red += to_double(norm2(rv));
    }
    template <typename R>
    LQ_HD void apply(const Site& s, const Spinor<R>& acc, double* red) const {
        update(s, acc, (R)alpha[0], red[0]);
    }
    template <typename R>
    LQ_HD void apply_rb(const Site& s, const Spinor<R> (&acc)[RB], double* red) const {
#pragma unroll
        for (int i = 0; i < RB; ++i)
            if (on[i]) update(Site{s.lex, s.p, s.cb, s.rhs + i}, acc[i], (R)alpha[i], red[i]);
    }
    template <int BS> __device__ __forceinline__ void finish(const double (&red)[RB], const VGrid& vg) const {
        SolverState* st = rc.st;
        const int n = nr;
        grid_reduce_seg<BS, RB>(rc, kTicketK2, red, n / RB, vg, [st, n](const double* tot) {
            int all = 1;
            for (int j = 0; j < n; ++j) {
                if (!st->stop[j]) {
                    const double rn = tot[(j % RB) * kMaxRhs + j / RB];
                    st->iter[j] += 1;
                    if (!isfinite(rn)) {
                        st->stop[j] = 3;
                    } else {
                        st->beta[j] = rn / st->rho[j];
                        st->rho[j] = rn;
                        if (rn <= st->stop_rho[j] || st->iter[j] >= st->k_max) st->stop[j] = 1;
                    }
                }
                all &= (st->stop[j] != 0);
            }
            st->all_stop = all;
        });
    }
};

// K3: p = r + beta p, once per completed iteration of each right-hand side
template <class PA, class RA>
struct OpK3 {
    using Real = typename PA::Real;
    static constexpr int NRED = 1;
    PA p;
    RA r;
    RedCtx rc;
    int nr;
    Real beta;
    bool on;
    LQ_HD bool init() {
        bool any = false;
        for (int j = 0; j < nr; ++j) any |= (rc.st->p_iter[j] != rc.st->iter[j]);
        if (!any) return false;
        const int j = thread_rhs(nr);
        on = rc.st->p_iter[j] != rc.st->iter[j];
        beta = from_double<Real>(rc.st->beta[j]);
        return true;
    }
    LQ_HD bool active() const { return on; }
    LQ_HD void apply(const Site& s, double*) const {
        Spinor<Real> pv, rv;
        p.load(s, pv);
        r.load(s, rv);
#pragma unroll
        for (int k = 0; k < 12; ++k) pv.v[k] = {fma(beta, pv.v[k].re, rv.v[k].re), fma(beta, pv.v[k].im, rv.v[k].im)};
        p.store(s, pv);
    }
    template <int BS> __device__ __forceinline__ void finish(const double (&red)[1], const VGrid& vg) const {
        SolverState* st = rc.st;
        const int n = nr;
        grid_reduce_seg<BS, 1>(rc, kTicketK3, red, n, vg, [st, n](const double*) {
            for (int j = 0; j < n; ++j) st->p_iter[j] = st->iter[j];
        });
    }
};

// ------------------------------------------------------------------------------------
// cycle start (Algorithm 1), per right-hand side that takes part (act)
// ------------------------------------------------------------------------------------
// r = fl_low(r^high / s); first cycle: p = r; psi = 0.  Reduces <r, p> and ||r||^2.
template <class RHA, class RA, class PA, class XA>
struct OpRestart {
    using Real = typename RA::Real;
    static constexpr int NRED = 3;
    RHA rh;
    RA r;
    PA p;
    XA x;
    RedCtx rc;
    int nr;
    Real my_is;
    bool on, my_first;
    // the cycle's parameters (act, first, 1/s, stop_rho, k_max) come from rc.st->ctl
    LQ_HD bool init() {
        const int j = thread_rhs(nr);
        const CycleCtl& c = rc.st->ctl;
        on = c.act[j] != 0;
        my_first = c.first[j] != 0;
        my_is = from_double<Real>(c.is[j]);
        return true;
    }
    LQ_HD bool active() const { return on; }
    LQ_HD void apply(const Site& s, double* red) const {
        Spinor<Real> w;
        rh.load(s, w);
#pragma unroll
        for (int k = 0; k < 12; ++k) w.v[k] = {my_is * w.v[k].re, my_is * w.v[k].im};
        r.store(s, w);
        Spinor<Real> pv;
        if (my_first) {
            p.store(s, w);
            Spinor<Real> z;
            zero(z);
            x.store(s, z);
        } else {
            p.load(s, pv);
            Real re = Real(0), im = Real(0);
#pragma unroll
            for (int k = 0; k < 12; ++k) {
                re = fma(w.v[k].re, pv.v[k].re, fma(w.v[k].im, pv.v[k].im, re));
                im = fma(w.v[k].re, pv.v[k].im, fma(-w.v[k].im, pv.v[k].re, im));
            }
            red[0] += to_double(re);
            red[1] += to_double(im);
        }
        red[2] += to_double(norm2(w));
    }
    template <int BS> __device__ __forceinline__ void finish(const double (&red)[3], const VGrid& vg) const {
        SolverState* st = rc.st;
        const int n = nr;
        grid_reduce_seg<BS, 3>(rc, kTicketMisc, red, n, vg, [st, n](const double* tot) {
            int all = 1;
            for (int j = 0; j < n; ++j) {
                if (st->ctl.act[j]) {
                    st->red[0][j] = tot[0 * kMaxRhs + j];
                    st->red[1][j] = tot[1 * kMaxRhs + j];
                    st->rho[j] = tot[2 * kMaxRhs + j];
                    st->stop[j] = 0;
                    all = 0;
                } else {
                    st->stop[j] = 1;    // idle this cycle
                }
                st->iter[j] = 0;
                st->p_iter[j] = 0;
                st->stop_rho[j] = st->ctl.stop_rho[j];
            }
            st->k_max = st->ctl.k_max;
            st->trips = 0;
            st->all_stop = all;
        });
    }
};

// later cycles: p = r + beta0 (p - c r), c = <r, p> from the previous kernel; psi = 0
template <class RA, class PA, class XA>
struct OpRestartP {
    using Real = typename RA::Real;
    static constexpr int NRED = 0;
    RA r;
    PA p;
    XA x;
    RedCtx rc;
    int nr;
    Real cre, cim, my_b0;
    bool on;
    // beta_0 and whether the right-hand side continues its direction come from rc.st->ctl
    LQ_HD bool init() {
        const int j = thread_rhs(nr);
        const CycleCtl& c = rc.st->ctl;
        on = c.cont[j] != 0;
        cre = from_double<Real>(rc.st->red[0][j]);
        cim = from_double<Real>(rc.st->red[1][j]);
        my_b0 = from_double<Real>(c.b0[j]);
        return true;
    }
    LQ_HD bool active() const { return on; }
    LQ_HD void apply(const Site& s, double*) const {
        Spinor<Real> rv, pv;
        r.load(s, rv);
        p.load(s, pv);
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            const cplx<Real> cr = cmul(cplx<Real>{cre, cim}, rv.v[k]);
            pv.v[k] = {fma(my_b0, pv.v[k].re - cr.re, rv.v[k].re), fma(my_b0, pv.v[k].im - cr.im, rv.v[k].im)};
        }
        p.store(s, pv);
        Spinor<Real> z;
        zero(z);
        x.store(s, z);
    }
    template <int BS> __device__ __forceinline__ void finish(const double (&)[1], const VGrid& vg) const {}
};

// psi^high += s psi  (the cycle's update of Algorithm 1 as read above), in the outer
// arithmetic, for the right-hand sides that ctl marks (xact, with s in xs)
template <class XA, class PsiA>
struct OpXUpdate {
    using Real = typename XA::Real;
    static constexpr int NRED = 0;
    XA x;
    PsiA psi;
    int nr;
    const CycleCtl* ctl;
    Real my_s;
    bool on;
    LQ_HD bool init() {
        const int j = thread_rhs(nr);
        on = ctl->xact[j] != 0;
        my_s = from_double<Real>(ctl->xs[j]);
        return true;
    }
    LQ_HD bool active() const { return on; }
    LQ_HD void apply(const Site& st, double*) const {
        Spinor<Real> xv, pv;
        x.load(st, xv);
        psi.load(st, pv);
#pragma unroll
        for (int k = 0; k < 12; ++k)
            xv.v[k] = {fma(my_s, pv.v[k].re, xv.v[k].re), fma(my_s, pv.v[k].im, xv.v[k].im)};
        x.store(st, xv);
    }
    template <int BS> __device__ __forceinline__ void finish(const double (&)[1], const VGrid& vg) const {}
};

// ||a||^2 -> st->red[slot][rhs] (FP64)
template <class A>
struct OpNorm {
    static constexpr int NRED = 1;
    A a;
    RedCtx rc;
    int nr, slot;
    LQ_HD bool init() { return true; }
    LQ_HD bool active() const { return true; }
    LQ_HD void apply(const Site& s, double* red) const {
        Spinor<double> v;
        a.load(s, v);
        red[0] += norm2(v);
    }
    template <int BS> __device__ __forceinline__ void finish(const double (&red)[1], const VGrid& vg) const {
        SolverState* st = rc.st;
        const int n = nr, sl = slot;
        grid_reduce_seg<BS, 1>(rc, kTicketMisc, red, n, vg, [st, n, sl](const double* t) {
            for (int j = 0; j < n; ++j) st->red[sl][j] = t[j];
        });
    }
};

// ||eta||^2 -> st->red[3][rhs] and the number of nonzero components of x -> st->red[1][rhs]:
// for a zero starting guess the first outer residual is eta itself
template <class A>
struct OpNormEtaX {
    static constexpr int NRED = 2;
    A eta, x;
    RedCtx rc;
    int nr;
    LQ_HD bool init() { return true; }
    LQ_HD bool active() const { return true; }
    LQ_HD void apply(const Site& s, double* red) const {
        Spinor<double> v;
        eta.load(s, v);
        red[0] += norm2(v);
        x.load(s, v);
        double nz = 0.0;
#pragma unroll
        for (int k = 0; k < 12; ++k) nz += (v.v[k].re != 0.0 ? 1.0 : 0.0) + (v.v[k].im != 0.0 ? 1.0 : 0.0);
        red[1] += nz;
    }
    template <int BS> __device__ __forceinline__ void finish(const double (&red)[2], const VGrid& vg) const {
        SolverState* st = rc.st;
        const int n = nr;
        grid_reduce_seg<BS, 2>(rc, kTicketMisc, red, n, vg, [st, n](const double* t) {
            for (int j = 0; j < n; ++j) {
                st->red[3][j] = t[j];
                st->red[1][j] = t[kMaxRhs + j];
            }
        });
    }
};

// x = 0 for the right-hand sides marked in act
template <class XA>
struct OpZero {
    static constexpr int NRED = 0;
    XA x;
    int nr;
    PerRhs<int> act;
    bool on;
    LQ_HD bool init() {
        on = act.v[thread_rhs(nr)] != 0;
        return true;
    }
    LQ_HD bool active() const { return on; }
    LQ_HD void apply(const Site& s, double*) const {
        Spinor<double> z;
        zero(z);
        x.store(s, z);
    }
    template <int BS> __device__ __forceinline__ void finish(const double (&)[1], const VGrid& vg) const {}
};

// r^high = eta - (a t + b hop^dag(t)), ||r^high||^2 -> st->red[slot][rhs]  (outer arithmetic)
template <class EtaA, class TA, class RA>
struct EpiResid {
    using Real = typename RA::Real;
    static constexpr int NRED = 1;
    EtaA eta;
    TA t;
    RA r;
    Real a, b;
    RedCtx rc;
    int nr, slot;
    LQ_HD bool init() { return true; }
    LQ_HD bool active() const { return true; }
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
    template <int BS> __device__ __forceinline__ void finish(const double (&red)[1], const VGrid& vg) const {
        SolverState* st = rc.st;
        const int n = nr, sl = slot;
        grid_reduce_seg<BS, 1>(rc, kTicketMisc, red, n, vg, [st, n, sl](const double* tt) {
            for (int j = 0; j < n; ++j) st->red[sl][j] = tt[j];
        });
    }
};

// out = b hop(in) on the other parity: the first half of the Schur operator inside the
// inner loop, skipped like K1/K2 for right-hand sides (and whole launches) that have stopped
template <class OutA>
struct EpiPreHop {
    using Real = typename OutA::Real;
    static constexpr int NRED = 0;
    OutA out;
    Real b;
    RedCtx rc;
    int nr;
    bool on;
    LQ_HD bool init() {
        if (rc.st->all_stop) return false;
        on = rc.st->stop[thread_rhs(nr)] == 0;
        return true;
    }
    LQ_HD bool active() const { return on; }
    template <typename R>
    LQ_HD void apply(const Site& s, const Spinor<R>& acc, double*) const {
        Spinor<R> o;
#pragma unroll
        for (int k = 0; k < 12; ++k) o.v[k] = cscale((R)b, acc.v[k]);
        out.store(s, o);
    }
    template <int BS> __device__ __forceinline__ void finish(const double (&)[1], const VGrid&) const {}
};

// ------------------------------------------------------------------------------------
// workspace layout
// ------------------------------------------------------------------------------------
inline size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

// Workspace for a batch of nb right-hand sides: state record, partial sums, then the
// outer fields, then the inner fields.  With FP32-pair outer arithmetic (HP = LQ_F64X) the
// outer fields are EO copies of U, eta and x plus r^high and t^high, all as pairs; with
// native FP64 only r^high and t^high are needed (U, eta, x are the caller's).  The query
// returns the largest layout a mode can use.
struct WsLayout {
    size_t state, partials, r_high, t_high, u_x, eta_x, x_x, u_low, psi, r, p, t, total;
    size_t tmp_high, b_x, tmp;   // even-odd Schur solve only
};

inline int inner_prec(int mode) {
    switch (mode) {
        case LQ_CG_MIXED_F32: return LQ_F32;
        case LQ_CG_MIXED_F16: return LQ_F16S;
        case LQ_CG_MIXED_I32: return LQ_I32S;
        case LQ_CG_F64X: return LQ_F64X;
        default: return LQ_F64;
    }
}

// default inner reduction delta of Algorithm 1 per mode (the paper gives none): FP32-class
// inner arithmetic and storage 1e-4, scaled-FP16 storage 0.1, FP64-class inner 0 (run to
// the target)
inline double default_delta(int mode) {
    switch (mode) {
        case LQ_CG_MIXED_F32:
        case LQ_CG_MIXED_I32: return 1e-4;
        case LQ_CG_MIXED_F16: return 0.01;
        default: return 0.0;
    }
}

inline WsLayout ws_layout(const Geom& g, int mode, bool pair_outer, int inner_fmt, int nb) {
    WsLayout w{};
    size_t o = 0;
    auto take = [&](size_t bytes) {
        const size_t at = o;
        o += align256(bytes);
        return at;
    };
    const int64_t Vn = (int64_t)g.V * nb;
    w.state = take(sizeof(SolverState));
    w.partials = take(sizeof(double) * kMaxRedValues * kMaxRhs * kMaxPartials);
    w.r_high = take(spinor_bytes(Vn, LQ_F64));
    w.t_high = take(spinor_bytes(Vn, LQ_F64));
    if (pair_outer) {
        w.u_x = take(gauge_bytes(g.V, LQ_F64X, 18));
        w.eta_x = take(spinor_bytes(Vn, LQ_F64X));
        w.x_x = take(spinor_bytes(Vn, LQ_F64X));
    }
    const int ip = inner_prec(mode);
    if (mode == LQ_CG_MIXED_F32 || mode == LQ_CG_MIXED_F16 || mode == LQ_CG_MIXED_I32)
        w.u_low = take(gauge_bytes(g.V, ip, inner_fmt));
    const size_t lo = spinor_bytes(Vn, ip);
    w.psi = take(spinor_bytes(Vn, psi_prec(ip)));
    w.r = take(lo);
    w.p = take(lo);
    w.t = take(lo);
    w.total = o;
    return w;
}

// Even-odd Schur solve (D x = b through CG on Mhat^dag Mhat over the even sites): FP32-pair
// outer fields (full U, b and x; half r^high, t^high, eta-hat and an odd scratch), then the
// inner links and half inner fields with an odd scratch.
inline WsLayout ws_layout_schur(const Geom& g, int mode, int inner_fmt, int nb) {
    WsLayout w{};
    size_t o = 0;
    auto take = [&](size_t bytes) {
        const size_t at = o;
        o += align256(bytes);
        return at;
    };
    const int64_t Vn = (int64_t)g.V * nb, Hn = (int64_t)g.Vh * nb;
    w.state = take(sizeof(SolverState));
    w.partials = take(sizeof(double) * kMaxRedValues * kMaxRhs * kMaxPartials);
    w.r_high = take(spinor_bytes(Hn, LQ_F64X));
    w.t_high = take(spinor_bytes(Hn, LQ_F64X));
    w.tmp_high = take(spinor_bytes(Hn, LQ_F64X));
    w.u_x = take(gauge_bytes(g.V, LQ_F64X, 18));
    w.eta_x = take(spinor_bytes(Hn, LQ_F64X));
    w.x_x = take(spinor_bytes(Vn, LQ_F64X));
    w.b_x = take(spinor_bytes(Vn, LQ_F64X));
    const int ip = inner_prec(mode);
    if (ip != LQ_F64X) w.u_low = take(gauge_bytes(g.V, ip, inner_fmt));
    const size_t lo = spinor_bytes(Hn, ip);
    w.psi = take(spinor_bytes(Hn, psi_prec(ip)));
    w.r = take(lo);
    w.p = take(lo);
    w.t = take(lo);
    w.tmp = take(lo);
    w.total = o;
    return w;
}

// right-hand sides in the first batch of a multi-field solve (a power of two <= kMaxRhs)
inline int batch_size(int nrhs) {
    int b = 1;
    while (b * 2 <= nrhs && b * 2 <= kMaxRhs) b *= 2;
    return b;
}

inline size_t ws_bytes_for_mode(const Geom& g, int mode, int nrhs) {
    size_t m = 0;
    const int nb = batch_size(nrhs);
    // native FP64 CG never uses pair copies; the FP32-pair CG always does; the mixed modes
    // may use either (LQ_CG_NATIVE_F64)
    const int pair_lo = (mode == LQ_CG_F64X) ? 1 : 0, pair_hi = (mode == LQ_CG_F64) ? 0 : 1;
    for (int pair = pair_lo; pair <= pair_hi; ++pair)
        for (int fmt : {12, 18}) {
            const size_t t = ws_layout(g, mode, pair != 0, fmt, nb).total;
            if (t > m) m = t;
        }
    return m;
}

inline int log2i(int n) {
    int l = 0;
    while ((1 << l) < n) ++l;
    return l;
}
// ------------------------------------------------------------------------------------
// One solve: inner precision IP / link format IF / layout IL, outer precision HP, inner
// stencil block size IBS, for a batch of nb right-hand sides (a power of two <= kMaxRhs)
// given as nb consecutive FP64 LEX fields eta[.], x[.].  The steps of Algorithm 1 are
// methods so that one driver runs a single lattice and another runs several lattices whose
// inner kernels share launches.
// ------------------------------------------------------------------------------------
template <int HP> struct Outer;
template <> struct Outer<LQ_F64> {      // the caller's FP64 LEX fields
    static constexpr int L = LQ_LAYOUT_LEX;
};
template <> struct Outer<LQ_F64X> {     // FP32-pair EO copies in the workspace
    static constexpr int L = LQ_LAYOUT_EO;
};

// The last node of the inner-loop graph: another trip while some right-hand side is running
// and the cycle has not used k_max + 2 trips (K2 stops every right-hand side at k_max, so the
// trip bound only matters if that ever failed; it keeps the loop finite).
static __global__ void inner_loop_cond(cudaGraphConditionalHandle h, SolverState* st) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        const int t = ++st->trips;
        cudaGraphSetConditional(h, (st->all_stop == 0 && t < st->k_max + 2) ? 1u : 0u);
    }
}

// One cycle's inner CG as a CUDA graph: a conditional WHILE node whose body is K1, K2, K3 and
// inner_loop_cond, captured once per solve and launched once per cycle.  Used by host-driven
// cycles when the whole-solve graph (SolveGraph, below) cannot be built.
struct InnerGraph {
    cudaStream_t cs = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    InnerGraph() = default;
    InnerGraph(const InnerGraph&) = delete;
    InnerGraph& operator=(const InnerGraph&) = delete;
    ~InnerGraph() { reset(); }
    void reset() {
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        if (cs) cudaStreamDestroy(cs);
        exec = nullptr;
        graph = nullptr;
        cs = nullptr;
    }
    // body(stream) enqueues one iteration's kernels
    template <class Body>
    cudaError_t build(SolverState* st, Body body) {
        cudaError_t e;
        if ((e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking)) != cudaSuccess) return e;
        if ((e = cudaGraphCreate(&graph, 0)) != cudaSuccess) return e;
        cudaGraphConditionalHandle h;
        if ((e = cudaGraphConditionalHandleCreate(&h, graph, 1, cudaGraphCondAssignDefault)) != cudaSuccess) return e;
        cudaGraphNodeParams p = {};
        p.type = cudaGraphNodeTypeConditional;
        p.conditional.handle = h;
        p.conditional.type = cudaGraphCondTypeWhile;
        p.conditional.size = 1;
        cudaGraphNode_t node;
        if ((e = cudaGraphAddNode(&node, graph, nullptr, nullptr, 0, &p)) != cudaSuccess) return e;
        cudaGraph_t bodyg = p.conditional.phGraph_out[0];
        if ((e = cudaStreamBeginCaptureToGraph(cs, bodyg, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal)) !=
            cudaSuccess)
            return e;
        cudaError_t le = body(cs);
        if (le == cudaSuccess) {
            inner_loop_cond<<<1, 32, 0, cs>>>(h, st);
            le = cudaGetLastError();
        }
        e = cudaStreamEndCapture(cs, &bodyg);
        if (le != cudaSuccess) return le;
        if (e != cudaSuccess) return e;
        return cudaGraphInstantiate(&exec, graph, 0);
    }
};

// ------------------------------------------------------------------------------------
// Algorithm 1's outer loop on a CycleCtl.  Host-driven solves call these on a host copy and
// upload it before the kernels that read it; device-driven solves run them in one-thread
// kernels of the solve's graph, so both follow the same decisions.
// ------------------------------------------------------------------------------------
// convergence and limits per right-hand side, and the next cycle's inner iteration cap;
// true if some right-hand side needs another cycle
LQ_HD bool ctl_plan(CycleCtl& c) {
    int total_max = 0;
    bool any = false;
    for (int j = 0; j < c.nb; ++j) {
        if (c.done[j]) continue;
        if (!isfinite(c.s[j])) {
            c.status[j] = LQ_ERR_NONFINITE;
            c.done[j] = 1;
        } else if (c.s[j] <= c.target[j]) {
            c.done[j] = 1;
        } else if (c.l >= c.max_cycles || c.total[j] >= c.max_iter || c.stagnant[j] >= 5) {
            c.status[j] = LQ_NOT_CONVERGED;
            c.done[j] = 1;
        }
        if (!c.done[j]) {
            any = true;
            if (c.total[j] > total_max) total_max = c.total[j];
        }
    }
    c.k_max = c.max_iter - total_max;
    if (c.k_max > c.per_cycle) c.k_max = c.per_cycle;
    return any;
}

// the next cycle's restart (Algorithm 1): r_0 = r^high / s, the inner stopping point
// rho <= max(delta^2, (tol ||eta|| / s)^2), and beta_0 = s_l / (s_{l-1} rho_k) for a
// right-hand side that continues its direction; right-hand sides that are done take no part
LQ_HD void ctl_params(CycleCtl& c) {
    c.any_cont = 0;
    for (int j = 0; j < kMaxRhs; ++j) {
        const bool in = j < c.nb;
        const int act = in && !c.done[j];
        const double rel = in ? c.target[j] / (c.s[j] > 0 ? c.s[j] : 1.0) : 0.0;
        c.act[j] = act;
        c.is[j] = act ? 1.0 / c.s[j] : 0.0;
        c.stop_rho[j] = fmax(c.delta * c.delta, rel * rel);
        c.cont[j] = act && !c.first[j];
        c.b0[j] = c.cont[j] ? c.s[j] / (c.s_prev[j] * c.rho_k[j]) : 0.0;
        c.any_cont |= c.cont[j];
    }
}

// the end of a cycle's inner loop: its iterations and stop code per right-hand side, and
// the solution update psi^high += s psi to apply
LQ_HD void ctl_mid(CycleCtl& c, const SolverState& st) {
    for (int j = 0; j < kMaxRhs; ++j) {
        c.xact[j] = 0;
        if (j >= c.nb || c.done[j]) continue;
        c.total[j] += st.iter[j];
        if (st.stop[j] >= 2) {
            // breakdown or non-finite: x stays the last reliable iterate
            c.status[j] = st.stop[j] == 2 ? LQ_ERR_BREAKDOWN : LQ_ERR_NONFINITE;
            c.done[j] = 1;
            continue;
        }
        c.rho_k[j] = st.rho[j];
        c.xact[j] = 1;
        c.xs[j] = c.s[j];
    }
}

// the new outer residual s = ||r^high|| (st.red[2]): stagnation (cycles since s last
// improved on its best by 0.1%) and whether the next cycle continues the direction (only
// while the inner recurrence predicted the true residual)
LQ_HD void ctl_collect(CycleCtl& c, const SolverState& st) {
    c.high_applies += 1;
    for (int j = 0; j < c.nb; ++j) {
        if (!c.xact[j]) continue;
        const double s_new = sqrt(st.red[2][j]);
        if (s_new < 0.999 * c.best[j]) {
            c.best[j] = s_new;
            c.stagnant[j] = 0;
        } else {
            c.stagnant[j] += 1;
        }
        c.first[j] = !(s_new <= 2.0 * c.s[j] * sqrt(c.rho_k[j]));
        c.s_prev[j] = c.s[j];
        c.s[j] = s_new;
        c.cycles[j] += 1;
    }
    ++c.l;
}

// The one-thread kernels of a device-driven solve.  ctl_first and ctl_end decide whether
// another cycle runs (the outer WHILE node's condition); ctl_arm opens the cycle's inner
// loop; ctl_end also counts the cycle's launches (fixed ones plus per_trip per inner trip).
static __global__ void ctl_first_kernel(SolverState* st, cudaGraphConditionalHandle outer) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        CycleCtl& c = st->ctl;
        const bool any = ctl_plan(c);
        ctl_params(c);
        c.launches += 1;
        cudaGraphSetConditional(outer, any ? 1u : 0u);
    }
}
static __global__ void ctl_arm_kernel(cudaGraphConditionalHandle inner) {
    if (threadIdx.x == 0 && blockIdx.x == 0) cudaGraphSetConditional(inner, 1u);
}
static __global__ void ctl_mid_kernel(SolverState* st) {
    if (threadIdx.x == 0 && blockIdx.x == 0) ctl_mid(st->ctl, *st);
}
static __global__ void ctl_end_kernel(SolverState* st, cudaGraphConditionalHandle outer, int per_trip, int fixed) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        CycleCtl& c = st->ctl;
        ctl_collect(c, *st);
        c.launches += fixed + per_trip * st->trips;
        const bool any = ctl_plan(c);
        ctl_params(c);
        cudaGraphSetConditional(outer, any ? 1u : 0u);
    }
}

// Adds a conditional node with handle h after the work captured so far on cs (which is
// capturing) and makes later captured work depend on it; *body receives its body graph.
inline cudaError_t capture_conditional(cudaStream_t cs, cudaGraphConditionalHandle h, cudaGraphConditionalNodeType type,
                                       cudaGraph_t* body) {
    cudaStreamCaptureStatus status;
    cudaGraph_t g = nullptr;
    const cudaGraphNode_t* deps = nullptr;
    size_t nd = 0;
    cudaError_t e = cudaStreamGetCaptureInfo(cs, &status, nullptr, &g, &deps, nullptr, &nd);
    if (e != cudaSuccess) return e;
    if (status != cudaStreamCaptureStatusActive) return cudaErrorStreamCaptureInvalidated;
    cudaGraphNodeParams p = {};
    p.type = cudaGraphNodeTypeConditional;
    p.conditional.handle = h;
    p.conditional.type = type;
    p.conditional.size = 1;
    cudaGraphNode_t node;
    if ((e = cudaGraphAddNode(&node, g, deps, nullptr, nd, &p)) != cudaSuccess) return e;
    *body = p.conditional.phGraph_out[0];
    return cudaStreamUpdateCaptureDependencies(cs, &node, nullptr, 1, cudaStreamSetCaptureDependencies);
}

// A whole solve's cycles as one CUDA graph (Algorithm 1 with every decision on the device):
//   ctl_first; WHILE (another cycle) { ctl_arm; restart(); WHILE (inner loop runs)
//   { iteration(); inner_loop_cond }; ctl_mid; tail(); ctl_end }
// restart() enqueues the cycle start, iteration() one inner CG iteration and tail() the
// solution update and the outer residual.  Built once per solve, launched once.
struct SolveGraph {
    cudaStream_t cs = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    SolveGraph() = default;
    SolveGraph(const SolveGraph&) = delete;
    SolveGraph& operator=(const SolveGraph&) = delete;
    ~SolveGraph() { reset(); }
    void reset() {
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        if (cs) cudaStreamDestroy(cs);
        exec = nullptr;
        graph = nullptr;
        cs = nullptr;
    }
    template <class Restart, class Iteration, class Tail>
    cudaError_t build(SolverState* st, int per_trip, int fixed, Restart restart, Iteration iteration, Tail tail) {
        constexpr cudaStreamCaptureMode mode = cudaStreamCaptureModeThreadLocal;
        cudaError_t e, le;
        if ((e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking)) != cudaSuccess) return e;
        if ((e = cudaGraphCreate(&graph, 0)) != cudaSuccess) return e;
        cudaGraphConditionalHandle outer, inner;
        if ((e = cudaGraphConditionalHandleCreate(&outer, graph, 0, cudaGraphCondAssignDefault)) != cudaSuccess)
            return e;
        // top level: the first decision, then the cycle loop
        if ((e = cudaStreamBeginCaptureToGraph(cs, graph, nullptr, nullptr, 0, mode)) != cudaSuccess) return e;
        ctl_first_kernel<<<1, 32, 0, cs>>>(st, outer);
        le = cudaGetLastError();
        cudaGraph_t cycle = nullptr, body = nullptr;
        if (le == cudaSuccess) le = capture_conditional(cs, outer, cudaGraphCondTypeWhile, &cycle);
        e = cudaStreamEndCapture(cs, &graph);
        if (le != cudaSuccess) return le;
        if (e != cudaSuccess) return e;
        // one cycle
        if ((e = cudaGraphConditionalHandleCreate(&inner, cycle, 1, cudaGraphCondAssignDefault)) != cudaSuccess)
            return e;
        if ((e = cudaStreamBeginCaptureToGraph(cs, cycle, nullptr, nullptr, 0, mode)) != cudaSuccess) return e;
        ctl_arm_kernel<<<1, 32, 0, cs>>>(inner);
        le = cudaGetLastError();
        if (le == cudaSuccess) le = restart(cs);
        if (le == cudaSuccess) le = capture_conditional(cs, inner, cudaGraphCondTypeWhile, &body);
        if (le == cudaSuccess) {
            ctl_mid_kernel<<<1, 32, 0, cs>>>(st);
            le = cudaGetLastError();
        }
        if (le == cudaSuccess) le = tail(cs);
        if (le == cudaSuccess) {
            ctl_end_kernel<<<1, 32, 0, cs>>>(st, outer, per_trip, fixed);
            le = cudaGetLastError();
        }
        e = cudaStreamEndCapture(cs, &cycle);
        if (le != cudaSuccess) return le;
        if (e != cudaSuccess) return e;
        // one inner iteration and the loop test
        if ((e = cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, mode)) != cudaSuccess) return e;
        le = iteration(cs);
        if (le == cudaSuccess) {
            inner_loop_cond<<<1, 32, 0, cs>>>(inner, st);
            le = cudaGetLastError();
        }
        e = cudaStreamEndCapture(cs, &body);
        if (le != cudaSuccess) return le;
        if (e != cudaSuccess) return e;
        return cudaGraphInstantiate(&exec, graph, 0);
    }
};

struct EventSet {
    std::vector<cudaEvent_t> ev;
    EventSet() = default;
    EventSet(const EventSet&) = delete;
    EventSet& operator=(const EventSet&) = delete;
    ~EventSet() {
        for (cudaEvent_t x : ev) cudaEventDestroy(x);
    }
};

// SCHUR: the even-odd Schur solve of D x = b (FP32-pair outer arithmetic, EO layout):
// CG on Mhat^dag Mhat over the even sites, Mhat = A - H_eo H_oe / A with A = m_q + 4 and
// H the hopping term of Eq. (1); each operator is a hop to the odd sites and a hop back.
// RB: right-hand sides per thread in the inner stencil kernels K1 and K2 (register blocking;
// EO layout, unrolled stencils, not the Schur solve).
template <int IP, int IF, int IL, int HP, int IBS = kBS, bool SCHUR = false, int RB = 1>
struct Solve {
    static_assert(!SCHUR || (HP == LQ_F64X && IL == LQ_LAYOUT_EO), "the Schur solve runs on FP32-pair EO fields");
    static_assert(RB == 1 || (!SCHUR && IL == LQ_LAYOUT_EO && !std::is_same<typename PrecT<IP>::Real, dd>::value),
                  "register blocking over right-hand sides needs the unrolled EO stencils");
    using Real = typename PrecT<IP>::Real;
    using HReal = typename PrecT<HP>::Real;
    static constexpr int HL = Outer<HP>::L;
    using SpRO = SpinorAcc<IP, IL, true>;
    using SpRW = SpinorAcc<IP, IL, false>;
    using GA = GaugeAcc<IP, IF, IL>;
    using HiRO = SpinorAcc<HP, HL, true>;
    using HiRW = SpinorAcc<HP, HL, false>;
    using HiGA = GaugeAcc<HP, 18, HL>;
    using CallerRO = SpinorAcc<LQ_F64, LQ_LAYOUT_LEX, true>;
    using CallerRW = SpinorAcc<LQ_F64, LQ_LAYOUT_LEX, false>;
    template <int B>
    using FullMap = typename std::conditional<IL == LQ_LAYOUT_LEX, MapLex<B>, MapEoFull<B>>::type;
    template <int B>
    using FullHMap = typename std::conditional<HL == LQ_LAYOUT_LEX, MapLex<B>, MapEoFull<B>>::type;
    using IMap = typename std::conditional<SCHUR, MapEoHalf<IBS>,
                                           typename std::conditional<RB == 1, FullMap<IBS>, MapEoFullRB<IBS>>::type>::type;
    using ISiteMap = typename std::conditional<SCHUR, MapEoHalf<kSiteBS>, FullMap<kSiteBS>>::type;
    using HMap = typename std::conditional<SCHUR, MapEoHalf<kBS>, FullHMap<kBS>>::type;
    using HSiteMap = typename std::conditional<SCHUR, MapEoHalf<kSiteBS>, FullHMap<kSiteBS>>::type;
    using K1Sten = Stencil<GA, SpRO, false>;
    using K1Epi = typename std::conditional<RB == 1, EpiK1<SpRW, SpRO>, EpiK1Blk<SpRW, SpRO, RB>>::type;
    using K2Sten = Stencil<GA, SpRO, true>;
    static constexpr int PSIP = psi_prec(IP);
    using PsiRO = SpinorAcc<PSIP, IL, true>;
    using PsiRW = SpinorAcc<PSIP, IL, false>;
    using K2Epi = typename std::conditional<RB == 1, EpiK2<SpRO, SpRO, PsiRW, SpRW>,
                                            EpiK2Blk<SpRO, SpRO, PsiRW, SpRW, RB>>::type;
    using K3Op = OpK3<SpRW, SpRO>;
    using PreEpi = EpiPreHop<SpRW>;
    static constexpr bool kPairs = (HP == LQ_F64X);
    static constexpr int kBlock = IBS;

    // the problem
    Geom g;
    double m_q = 0.0, delta = 0.0, a = 4.0, b = 0.5;
    int nb = 1;
    const void* U = nullptr;
    const void* eta = nullptr;
    void* x = nullptr;
    lq_cg_params prm{};
    WsLayout w{};
    char* ws = nullptr;
    cudaStream_t st = nullptr;

    // device-side objects
    SolverState* dstate = nullptr;
    RedCtx rc{};
    const void* Uo = nullptr;
    const void* etao = nullptr;
    void* xo = nullptr;
    HiGA Uh;
    HiRO eta_ro, x_ro, rh_ro, th_ro;
    HiRW x_rw, rh_rw, th_rw;
    CallerRO eta_caller;
    CallerRW x_caller;
    GA Ui;
    SpRO r_ro, p_ro, t_ro;
    SpRW r_rw, p_rw, t_rw;
    PsiRO psi_ro;
    PsiRW psi_rw;
    MapLex<kSiteBS> lexsite;
    HMap hmap;
    HSiteMap hsite;
    IMap imap;
    ISiteMap isite;
    K1Sten sK1;
    K1Epi eK1;
    K2Sten sK2;
    K2Epi eK2;
    K3Op oK3;
    // Schur solve: odd-site maps, odd scratch fields, the pre-hops and the FP32-pair b
    IMap omap;
    HMap hmap_odd;
    SpRO tmp_ro;
    SpRW tmp_rw;
    HiRO tmh_ro, b_ro;
    HiRW tmh_rw;
    K1Sten sPre1;
    K2Sten sPre2;
    PreEpi ePre;

    // host-side state; hc is Algorithm 1's outer loop (the device copy, dstate->ctl, is what
    // the cycle kernels read: uploaded by host-driven solves, advanced in place by the graph)
    SolverState hs{};
    CycleCtl hc{};
    lq_cg_info out[kMaxRhs];
    bool prof = false;
    int chunk = 8, launches = 0, k_max = 0, guard = 0;
    double kms[4] = {0, 0, 0, 0};
    int kcalls[4] = {0, 0, 0, 0};
    EventSet evs;
    InnerGraph igraph;
    bool graph_off = false;   // the inner-loop graph could not be built

    Solve() = default;
    Solve(const Solve&) = delete;
    Solve& operator=(const Solve&) = delete;

    void init(const Geom& g_, double m_q_, int nb_, const void* U_, const void* eta_, void* x_,
              const lq_cg_params& prm_, double delta_, const WsLayout& w_, char* ws_, cudaStream_t st_) {
        g = g_;
        m_q = m_q_;
        nb = nb_;
        U = U_;
        eta = eta_;
        x = x_;
        prm = prm_;
        delta = delta_;
        w = w_;
        ws = ws_;
        st = st_;
        a = m_q + 4.0;
        b = 0.5;
        const int lnr = log2i(nb);
        dstate = (SolverState*)(ws + w.state);
        rc = RedCtx{dstate, (double*)(ws + w.partials)};
        // outer fields: the caller's arrays (native FP64) or pair copies in the workspace
        Uo = kPairs ? (const void*)(ws + w.u_x) : U;
        etao = kPairs ? (const void*)(ws + w.eta_x) : eta;
        xo = kPairs ? (void*)(ws + w.x_x) : x;
        // Schur: eta-hat, r^high, t^high and the inner fields are even half fields; x stays full
        constexpr bool H = SCHUR;
        Uh = make_gauge<HP, 18, HL>(Uo, g);
        eta_ro = make_spinor<HP, HL, true>(etao, g, H, nb);
        x_ro = make_spinor<HP, HL, true>(xo, g, false, nb);
        x_rw = make_spinor<HP, HL, false>(xo, g, false, nb);
        rh_ro = make_spinor<HP, HL, true>(ws + w.r_high, g, H, nb);
        rh_rw = make_spinor<HP, HL, false>(ws + w.r_high, g, H, nb);
        th_ro = make_spinor<HP, HL, true>(ws + w.t_high, g, H, nb);
        th_rw = make_spinor<HP, HL, false>(ws + w.t_high, g, H, nb);
        eta_caller = make_spinor<LQ_F64, LQ_LAYOUT_LEX, true>(eta, g, false, nb);
        x_caller = make_spinor<LQ_F64, LQ_LAYOUT_LEX, false>(x, g, false, nb);
        // inner fields; an FP64-class inner loop shares the outer links
        const void* Ulow = (IP == LQ_F64) ? U : (IP == LQ_F64X ? Uo : (const void*)(ws + w.u_low));
        Ui = make_gauge<IP, IF, IL>(Ulow, g);
        psi_ro = make_spinor<PSIP, IL, true>(ws + w.psi, g, H, nb);
        psi_rw = make_spinor<PSIP, IL, false>(ws + w.psi, g, H, nb);
        r_ro = make_spinor<IP, IL, true>(ws + w.r, g, H, nb);
        r_rw = make_spinor<IP, IL, false>(ws + w.r, g, H, nb);
        p_ro = make_spinor<IP, IL, true>(ws + w.p, g, H, nb);
        p_rw = make_spinor<IP, IL, false>(ws + w.p, g, H, nb);
        t_ro = make_spinor<IP, IL, true>(ws + w.t, g, H, nb);
        t_rw = make_spinor<IP, IL, false>(ws + w.t, g, H, nb);
        lexsite = MapLex<kSiteBS>{g, lnr};
        // the inner and outer operators: a t + b hop(t) with (a, b) = (m_q + 4, 1/2) for
        // D^dag D, (A, -1/(2A)) for the second hop of the Schur operator
        const double ka = a, kb = SCHUR ? -0.5 / a : b;
        if constexpr (SCHUR) {
            hmap = HMap{g, 0, lnr};
            hmap_odd = HMap{g, 1, lnr};
            hsite = HSiteMap{g, 0, lnr};
            imap = IMap{g, 0, lnr};
            omap = IMap{g, 1, lnr};
            isite = ISiteMap{g, 0, lnr};
            tmp_ro = make_spinor<IP, IL, true>(ws + w.tmp, g, true, nb);
            tmp_rw = make_spinor<IP, IL, false>(ws + w.tmp, g, true, nb);
            tmh_ro = make_spinor<HP, HL, true>(ws + w.tmp_high, g, true, nb);
            tmh_rw = make_spinor<HP, HL, false>(ws + w.tmp_high, g, true, nb);
            b_ro = make_spinor<HP, HL, true>(ws + w.b_x, g, false, nb);
            sPre1 = K1Sten{g, Ui, p_ro};
            sPre2 = K2Sten{g, Ui, t_ro};
            ePre = PreEpi{tmp_rw, from_double<Real>(0.5), rc, nb, false};
            sK1 = K1Sten{g, Ui, tmp_ro};
            sK2 = K2Sten{g, Ui, tmp_ro};
        } else {
            hmap = HMap{g, lnr};
            hsite = HSiteMap{g, lnr};
            imap = IMap{g, lnr};
            if constexpr (RB > 1) imap.lrb = log2i(RB);
            isite = ISiteMap{g, lnr};
            sK1 = K1Sten{g, Ui, p_ro};
            sK2 = K2Sten{g, Ui, t_ro};
        }
        eK1 = K1Epi{t_rw, p_ro, from_double<Real>(ka), from_double<Real>(kb), rc, nb, false};
        eK2 = K2Epi{t_ro, p_ro, psi_rw, r_rw, from_double<Real>(ka), from_double<Real>(kb), rc, nb, Real(0), false};
        oK3 = K3Op{p_rw, r_ro, rc, nb, Real(0), false};
        memset(out, 0, sizeof(out));
        prof = (prm.flags & LQ_CG_PROFILE) != 0;
        const int64_t Vn = (int64_t)g.V * nb;
        chunk = prm.chunk > 0 ? prm.chunk : (Vn >= (1 << 18) ? 8 : 32);
    }

    cudaEvent_t ev_at(int role, int j, int end) const { return evs.ev[(role * chunk + j) * 2 + end]; }
    static double elapsed(cudaEvent_t a0, cudaEvent_t a1) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, a0, a1);
        return (double)ms;
    }
    cudaError_t read_state_async() { return cudaMemcpyAsync(&hs, dstate, sizeof(hs), cudaMemcpyDeviceToHost, st); }
    cudaError_t read_state() {
        const cudaError_t er = read_state_async();
        if (er != cudaSuccess) return er;
        return cudaStreamSynchronize(st);
    }

    // out = ya y + hb hop(in) over the sites of map, in the outer arithmetic (Schur set-up,
    // residual and reconstruction steps)
    template <class Map, class OutA, class InA, class YA, bool DAG, bool HASY>
    cudaError_t outer_hop(const Map& map, const OutA& out, const InA& in, const YA& y, double ya, double hb,
                          cudaStream_t s) {
        Stencil<HiGA, InA, DAG> sten{g, Uh, in};
        EpiAxpby<OutA, YA, HASY, false> e;
        e.out = out;
        e.y = y;
        e.a = from_double<HReal>(ya);
        e.b = from_double<HReal>(hb);
        e.rc = rc;
        e.slot = 0;
        launches += 1;
        return launch_stencil<kBS>(map, sten, e, s);
    }

    // r^high = eta - A x, s^2 -> red[2][.]   (Algorithm 1: the high-precision residual)
    cudaError_t high_residual(cudaStream_t s) {
        if constexpr (SCHUR) {
            // tmp_o = H_oe x_e;  t_e = A x_e - H_eo tmp_o / A;  tmp_o = H^dag_oe t_e;
            // r_e = eta-hat - (A t_e - H^dag_eo tmp_o / A)
            if (prof) cudaEventRecord(evs.ev[6 * chunk], s);
            cudaError_t er;
            if ((er = outer_hop<HMap, HiRW, HiRO, HiRO, false, false>(hmap_odd, tmh_rw, x_ro, x_ro, 0.0, 0.5, s)) !=
                    cudaSuccess ||
                (er = outer_hop<HMap, HiRW, HiRO, HiRO, false, true>(hmap, th_rw, tmh_ro, x_ro, a, -0.5 / a, s)) !=
                    cudaSuccess ||
                (er = outer_hop<HMap, HiRW, HiRO, HiRO, true, false>(hmap_odd, tmh_rw, th_ro, th_ro, 0.0, 0.5, s)) !=
                    cudaSuccess)
                return er;
            Stencil<HiGA, HiRO, true> s4{g, Uh, tmh_ro};
            EpiResid<HiRO, HiRO, HiRW> e4{eta_ro, th_ro, rh_rw, from_double<HReal>(a), from_double<HReal>(-0.5 / a), rc, nb, 2};
            er = launch_stencil<kBS>(hmap, s4, e4, s);
            launches += 1;
            if (prof) cudaEventRecord(evs.ev[6 * chunk + 1], s);
            return er;
        }
        Stencil<HiGA, HiRO, false> s1{g, Uh, x_ro};
        EpiAxpby<HiRW, HiRO, true, false> e1;
        e1.out = th_rw;
        e1.y = x_ro;
        e1.a = from_double<HReal>(a);
        e1.b = from_double<HReal>(b);
        e1.rc = rc;
        e1.slot = 0;
        if (prof) cudaEventRecord(evs.ev[6 * chunk], s);
        cudaError_t er = launch_stencil<kBS>(hmap, s1, e1, s);
        if (er != cudaSuccess) return er;
        Stencil<HiGA, HiRO, true> s2{g, Uh, th_ro};
        EpiResid<HiRO, HiRO, HiRW> e2{eta_ro, th_ro, rh_rw, from_double<HReal>(a), from_double<HReal>(b), rc, nb, 2};
        er = launch_stencil<kBS>(hmap, s2, e2, s);
        launches += 2;
        if (prof) cudaEventRecord(evs.ev[6 * chunk + 1], s);
        return er;
    }
    // after the stream has been synchronised: add the residual's event time
    void account_high() {
        if (!prof) return;
        kms[LQ_K_HIGH] += elapsed(evs.ev[6 * chunk], evs.ev[6 * chunk + 1]);
        kcalls[LQ_K_HIGH] += SCHUR ? 4 : 2;
    }

    // state record, field conversions, ||eta||, x = 0 for zero right-hand sides, and the
    // first outer residual
    int begin() {
        NvtxRange nvtx("lq solve: set-up (conversions, norms, first residual)");
        cudaError_t e;
        if (prof) {
            evs.ev.resize(6 * chunk + 2);
            for (auto& ev : evs.ev)
                if ((e = cudaEventCreate(&ev)) != cudaSuccess) return cuda_fail(e, "event create");
        }
        // state zeroed, with the inner loop marked stopped until a cycle starts (inner
        // launches shared with other lattices then skip this one)
        if ((e = cudaMemsetAsync(dstate, 0, sizeof(SolverState), st)) != cudaSuccess ||
            (e = cudaMemsetAsync(&dstate->all_stop, 1, sizeof(dstate->all_stop), st)) != cudaSuccess)
            return cuda_fail(e, "state init");
        constexpr bool kLowLinks = IP != LQ_F64 && IP != LQ_F64X;   // reduced-precision inner links
        if constexpr (kPairs) {
            // pair links and the inner links from one pass over U.  Schur: the caller's
            // right-hand side is b (full, kept as pairs in b_x); eta-hat is built from it below
            if ((e = convert_gauge(g, LQ_F64, LQ_LAYOUT_LEX, U, LQ_F64X, 18, LQ_LAYOUT_EO, ws + w.u_x, st, IP, IF, IL,
                                   kLowLinks ? (void*)(ws + w.u_low) : nullptr)) != cudaSuccess ||
                (e = convert_spinor(g, LQ_F64, LQ_LAYOUT_LEX, eta, LQ_F64X, LQ_LAYOUT_EO,
                                    ws + (SCHUR ? w.b_x : w.eta_x), st, nb)) != cudaSuccess ||
                (e = convert_spinor(g, LQ_F64, LQ_LAYOUT_LEX, x, LQ_F64X, LQ_LAYOUT_EO, ws + w.x_x, st, nb)) !=
                    cudaSuccess)
                return cuda_fail(e, "FP32-pair copies");
            launches += 3;
        } else if constexpr (kLowLinks) {
            if ((e = convert_gauge(g, LQ_F64, LQ_LAYOUT_LEX, U, IP, IF, IL, ws + w.u_low, st)) != cudaSuccess)
                return cuda_fail(e, "link pack");
            launches += 1;
        }
        if constexpr (SCHUR) {
            // bhat_e = b_e - H_eo b_o / A (in t^high);  tmp_o = H^dag_oe bhat_e;
            // eta-hat = Mhat^dag bhat_e = A bhat_e - H^dag_eo tmp_o / A;  ||eta-hat||^2 -> red[3]
            if ((e = outer_hop<HMap, HiRW, HiRO, HiRO, false, true>(hmap, th_rw, b_ro, b_ro, 1.0, -0.5 / a, st)) !=
                    cudaSuccess ||
                (e = outer_hop<HMap, HiRW, HiRO, HiRO, true, false>(hmap_odd, tmh_rw, th_ro, th_ro, 0.0, 0.5, st)) !=
                    cudaSuccess ||
                (e = outer_hop<HMap, HiRW, HiRO, HiRO, true, true>(hmap, make_spinor<HP, HL, false>(etao, g, true, nb),
                                                                   tmh_ro, th_ro, a, -0.5 / a, st)) != cudaSuccess ||
                (e = launch_site<kSiteBS>(hsite, OpNorm<HiRO>{eta_ro, rc, nb, 3}, st)) != cudaSuccess)
                return cuda_fail(e, "Schur right-hand side");
            launches += 1;
        } else {
            // ||eta||^2 -> red[3][.] from the caller's FP64 eta; nonzero count of x -> red[1][.]
            const CallerRO x_caller_ro = make_spinor<LQ_F64, LQ_LAYOUT_LEX, true>(x, g, false, nb);
            if ((e = launch_site<kSiteBS>(lexsite, OpNormEtaX<CallerRO>{eta_caller, x_caller_ro, rc, nb}, st)) !=
                cudaSuccess)
                return cuda_fail(e, "norm");
            launches += 1;
        }
        if ((e = read_state()) != cudaSuccess) return cuda_fail(e, "norm");

        PerRhs<int> zero_rhs{};
        bool any_zero = false;
        memset(&hc, 0, sizeof(hc));
        hc.nb = nb;
        hc.delta = delta;
        hc.max_cycles = prm.max_cycles > 0 ? prm.max_cycles : 1000;
        hc.max_iter = prm.max_iter;
        hc.per_cycle = prm.max_inner > 0 ? prm.max_inner : 1000;
        for (int j = 0; j < nb; ++j) {
            // first[j]: the next cycle starts from p_0 = r_0 (the first cycle, or after the
            // true residual left the inner recurrence's prediction)
            hc.eta_norm[j] = sqrt(hs.red[3][j]);
            out[j].eta_norm = hc.eta_norm[j];
            hc.first[j] = 1;
            hc.status[j] = LQ_OK;
            hc.target[j] = prm.tol * hc.eta_norm[j];
            if (!isfinite(hc.eta_norm[j])) {
                hc.status[j] = LQ_ERR_NONFINITE;
                hc.done[j] = 1;
            } else if (hc.eta_norm[j] == 0.0) {
                zero_rhs.v[j] = 1;
                any_zero = true;
                hc.done[j] = 1;
            }
        }
        if (any_zero) {
            if ((e = launch_site<kSiteBS>(lexsite, OpZero<CallerRW>{x_caller, nb, zero_rhs, false}, st)) !=
                cudaSuccess)
                return cuda_fail(e, "zero");
            launches += 1;
            if constexpr (kPairs) {
                if ((e = convert_spinor(g, LQ_F64, LQ_LAYOUT_LEX, x, LQ_F64X, LQ_LAYOUT_EO, ws + w.x_x, st, nb)) !=
                    cudaSuccess)
                    return cuda_fail(e, "zero");
                launches += 1;
            }
        }
        // Algorithm 1 starts from r = eta - D^dag D x0; a zero x0 (every right-hand side still
        // to solve) makes that eta itself, so the outer operator is not applied
        bool x0_zero = !SCHUR;
        if constexpr (!SCHUR)
            for (int j = 0; j < nb; ++j) x0_zero = x0_zero && (hc.done[j] || hs.red[1][j] == 0.0);
        if (x0_zero) {
            if ((e = cudaMemcpyAsync(ws + w.r_high, etao, spinor_bytes((int64_t)g.V * nb, HP),
                                     cudaMemcpyDeviceToDevice, st)) != cudaSuccess)
                return cuda_fail(e, "residual");
            for (int j = 0; j < nb; ++j) hc.s[j] = hc.eta_norm[j];
            hc.high_applies = 0;
        } else {
            if ((e = high_residual(st)) != cudaSuccess) return cuda_fail(e, "residual");
            if ((e = read_state()) != cudaSuccess) return cuda_fail(e, "residual");
            account_high();
            for (int j = 0; j < nb; ++j) hc.s[j] = sqrt(hs.red[2][j]);
            hc.high_applies = 1;
        }
        for (int j = 0; j < nb; ++j) hc.best[j] = hc.s[j];
        return LQ_OK;
    }

    // the host copy of the outer loop's state to the device (the cycle kernels read it there)
    cudaError_t upload_ctl() { return cudaMemcpyAsync(&dstate->ctl, &hc, sizeof(hc), cudaMemcpyHostToDevice, st); }

    // convergence and limits, per right-hand side; true if some right-hand side needs a cycle
    bool plan() {
        const bool any = ctl_plan(hc);
        k_max = hc.k_max;
        return any;
    }

    // the cycle-start kernels (Algorithm 1's restart), reading their parameters from
    // dstate->ctl; any_cont: some right-hand side continues its direction
    cudaError_t launch_restart(cudaStream_t s, bool any_cont) {
        OpRestart<HiRO, SpRW, SpRW, PsiRW> op{rh_ro, r_rw, p_rw, psi_rw, rc, nb, Real(0), false, false};
        cudaError_t e = launch_site<kSiteBS>(hsite, op, s);
        if (e != cudaSuccess || !any_cont) return e;
        OpRestartP<SpRO, SpRW, PsiRW> op2{r_ro, p_rw, psi_rw, rc, nb, Real(0), Real(0), Real(0), false};
        return launch_site<kSiteBS>(isite, op2, s);
    }

    // cycle start (Algorithm 1)
    int start_cycle() {
        NvtxRange nvtx("lq solve: cycle start (Algorithm 1 restart)");
        ctl_params(hc);
        cudaError_t e = upload_ctl();
        if (e == cudaSuccess) e = launch_restart(st, hc.any_cont != 0);
        if (e != cudaSuccess) return cuda_fail(e, "cycle start");
        launches += hc.any_cont ? 2 : 1;
        guard = 0;
        return LQ_OK;
    }

    // K1 alone (the block-size tuner times it)
    cudaError_t launch_k1(cudaStream_t s) const { return launch_stencil<IBS>(imap, sK1, eK1, s); }
    cudaError_t launch_k2(cudaStream_t s) const { return launch_stencil<IBS>(imap, sK2, eK2, s); }
    // one inner CG iteration (K1, K2, K3; Schur: with the two hops to the odd sites)
    cudaError_t launch_iteration(cudaStream_t s) const {
        cudaError_t r;
        if constexpr (SCHUR)
            if ((r = launch_stencil<IBS>(omap, sPre1, ePre, s)) != cudaSuccess) return r;
        if ((r = launch_stencil<IBS>(imap, sK1, eK1, s)) != cudaSuccess) return r;
        if constexpr (SCHUR)
            if ((r = launch_stencil<IBS>(omap, sPre2, ePre, s)) != cudaSuccess) return r;
        if ((r = launch_stencil<IBS>(imap, sK2, eK2, s)) != cudaSuccess) return r;
        return launch_site<kSiteBS>(isite, oK3, s);
    }

    // the inner CG of one lattice: chunks of K1, K2, K3 until every right-hand side has
    // stopped; leaves the final state record in hs
    int inner_single() {
        NvtxRange nvtx("lq solve: inner CG");
        cudaError_t e;
        if (!prof && !graph_off && (prm.flags & LQ_CG_NO_GRAPH) == 0) {
            // the whole inner loop on the device: one graph launch, one read-back
            if (!igraph.exec) {
                e = igraph.build(dstate, [&](cudaStream_t s) { return launch_iteration(s); });
                if (e != cudaSuccess) {
                    // no conditional graph here (driver or capture refused it): the host
                    // drives the same kernels below for the rest of the solve
                    (void)cudaGetLastError();
                    igraph.reset();
                    graph_off = true;
                }
            }
            if (!graph_off) {
                if ((e = cudaGraphLaunch(igraph.exec, st)) != cudaSuccess) return cuda_fail(e, "inner-loop graph");
                if ((e = read_state()) != cudaSuccess) return cuda_fail(e, "inner loop");
                launches += ((SCHUR ? 5 : 3) + 1) * hs.trips;
                return LQ_OK;
            }
        }
        int iter_before = 0;
        while (true) {
            for (int j = 0; j < chunk; ++j) {
                if (prof) cudaEventRecord(ev_at(0, j, 0), st);
                if constexpr (SCHUR)
                    if ((e = launch_stencil<IBS>(omap, sPre1, ePre, st)) != cudaSuccess) return cuda_fail(e, "K1 hop");
                if ((e = launch_stencil<IBS>(imap, sK1, eK1, st)) != cudaSuccess) return cuda_fail(e, "K1");
                if (prof) cudaEventRecord(ev_at(0, j, 1), st);
                if constexpr (SCHUR)
                    if ((e = launch_stencil<IBS>(omap, sPre2, ePre, st)) != cudaSuccess) return cuda_fail(e, "K2 hop");
                if ((e = launch_stencil<IBS>(imap, sK2, eK2, st)) != cudaSuccess) return cuda_fail(e, "K2");
                if (prof) cudaEventRecord(ev_at(1, j, 1), st);
                if ((e = launch_site<kSiteBS>(isite, oK3, st)) != cudaSuccess) return cuda_fail(e, "K3");
                if (prof) cudaEventRecord(ev_at(2, j, 1), st);
            }
            launches += (SCHUR ? 5 : 3) * chunk;
            if ((e = read_state()) != cudaSuccess) return cuda_fail(e, "inner loop");
            int iter_max = 0;
            for (int j = 0; j < nb; ++j)
                if (hs.iter[j] > iter_max) iter_max = hs.iter[j];
            if (prof) {
                // only the iterations that ran in this chunk; later launches found the stop flags
                const int ran = iter_max - iter_before;
                for (int j = 0; j < ran && j < chunk; ++j) {
                    kms[LQ_K_APPLY_D] += elapsed(ev_at(0, j, 0), ev_at(0, j, 1));
                    kms[LQ_K_APPLY_DDAG] += elapsed(ev_at(0, j, 1), ev_at(1, j, 1));
                    kms[LQ_K_UPDATE_P] += elapsed(ev_at(1, j, 1), ev_at(2, j, 1));
                    kcalls[LQ_K_APPLY_D] += 1;
                    kcalls[LQ_K_APPLY_DDAG] += 1;
                    kcalls[LQ_K_UPDATE_P] += 1;
                }
            }
            iter_before = iter_max;
            if (hs.all_stop) break;
            if (++guard > (k_max / chunk) + 2) break;   // cannot happen: K2 stops at k_max
        }
        return LQ_OK;
    }

    // outcome of the cycle (hs holds the final inner state), psi^high += s psi_k, and the
    // outer residual
    // The outcome of the cycle (hs holds the final inner state): psi^high += s psi_k and the
    // outer residual are enqueued here; end_cycle_collect() takes the residual once the state
    // record has been read back (several lattices share that one read); end_cycle() does both.
    // x^high += s psi for the right-hand sides dstate->ctl marks, then the outer residual
    cudaError_t launch_tail(cudaStream_t s) {
        OpXUpdate<HiRW, PsiRO> xu{x_rw, psi_ro, nb, &dstate->ctl, HReal(0), false};
        cudaError_t e = launch_site<kSiteBS>(hsite, xu, s);
        if (e != cudaSuccess) return e;
        return high_residual(s);
    }
    int end_cycle_launch() {
        NvtxRange nvtx("lq solve: reliable update (solution, FP64-class residual)");
        ctl_mid(hc, hs);
        cudaError_t e = upload_ctl();
        if (e == cudaSuccess) e = launch_tail(st);
        if (e != cudaSuccess) return cuda_fail(e, "reliable update");
        launches += 1;
        return LQ_OK;
    }
    void end_cycle_collect() {
        account_high();
        ctl_collect(hc, hs);
    }
    int end_cycle() {
        int r;
        if ((r = end_cycle_launch()) != LQ_OK) return r;
        cudaError_t e;
        if ((e = read_state()) != cudaSuccess) return cuda_fail(e, "residual");
        end_cycle_collect();
        return LQ_OK;
    }

    // Every cycle on the device: one graph (SolveGraph) holds Algorithm 1's loop with its
    // decisions, launched once; the host reads the state back at the end.  Returns false
    // (nothing launched) if the graph cannot be built here; the host then drives the cycles.
    bool device_cycles(int* r) {
        if (prof || graph_off || (prm.flags & LQ_CG_NO_GRAPH) != 0) return false;
        NvtxRange nvtx("lq solve: cycles (one graph)");
        SolveGraph sg;
        const int counted = launches;   // the builders count their launches while captured
        const int per_trip = (SCHUR ? 5 : 3) + 1, fixed = 2 + 1 + 1 + 1 + (SCHUR ? 4 : 2) + 1;
        cudaError_t e = sg.build(
            dstate, per_trip, fixed, [&](cudaStream_t s) { return launch_restart(s, true); },
            [&](cudaStream_t s) { return launch_iteration(s); }, [&](cudaStream_t s) { return launch_tail(s); });
        launches = counted;
        if (e != cudaSuccess) {
            (void)cudaGetLastError();
            return false;
        }
        *r = LQ_OK;
        if ((e = upload_ctl()) != cudaSuccess || (e = cudaGraphLaunch(sg.exec, st)) != cudaSuccess ||
            (e = read_state()) != cudaSuccess) {
            *r = cuda_fail(e, "solve graph");
            return true;
        }
        hc = hs.ctl;
        launches += hc.launches;
        k_max = hc.k_max;
        return true;
    }

    // write-back, per-right-hand-side records; returns the worst status
    int finish(lq_cg_info* info) {
        NvtxRange nvtx("lq solve: write-back");
        cudaError_t e;
        if constexpr (SCHUR) {
            // x_o = (b_o - H_oe x_e) / A
            if ((e = outer_hop<HMap, HiRW, HiRO, HiRO, false, true>(hmap_odd, x_rw, x_ro, b_ro, 1.0 / a, -0.5 / a, st)) !=
                cudaSuccess)
                return cuda_fail(e, "odd-site solution");
        }
        if constexpr (kPairs) {
            if ((e = convert_spinor(g, LQ_F64X, LQ_LAYOUT_EO, xo, LQ_F64, LQ_LAYOUT_LEX, x, st, nb)) != cudaSuccess)
                return cuda_fail(e, "x write-back");
            launches += 1;
        }
        if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return cuda_fail(e, "x write-back");
        int worst = LQ_OK;
        for (int j = 0; j < nb; ++j) {
            const int sj = hc.status[j];
            if (sj == LQ_ERR_BREAKDOWN) fail(sj, "CG breakdown: <p, D^dag D p> <= 0");
            if (sj == LQ_ERR_NONFINITE) fail(sj, "non-finite values (in eta, or produced by the solve)");
            out[j].iters = hc.total[j];
            out[j].cycles = hc.cycles[j];
            out[j].high_applies = hc.high_applies;
            out[j].true_rel_resid = hc.eta_norm[j] > 0 ? hc.s[j] / hc.eta_norm[j] : 0.0;
            out[j].status = sj;
            out[j].launches = launches;
            out[j].block = IBS;
            out[j].rhs_block = RB;
            for (int q = 0; q < 4; ++q) {
                out[j].kernel_ms[q] = kms[q];
                out[j].kernel_calls[q] = kcalls[q];
            }
            if (info) info[j] = out[j];
            if (sj < 0 && (worst >= 0 || sj < worst)) worst = sj;
            if (sj == LQ_NOT_CONVERGED && worst == LQ_OK) worst = LQ_NOT_CONVERGED;
        }
        return worst;
    }
};

// The single-lattice driver: one batch of nb right-hand sides (SCHUR: eta is b of D x = b),
// with RB right-hand sides per thread in the inner stencil kernels.
template <int IP, int IF, int IL, int HP, bool SCHUR = false, int RB = 1>
int run_solver_rb(const Geom& g, double m_q, int nb, const void* U, const void* eta, void* x, const lq_cg_params& prm,
                  double delta, const WsLayout& w, char* ws, lq_cg_info* info, cudaStream_t st) {
    Solve<IP, IF, IL, HP, kBS, SCHUR, RB> sv;
    sv.init(g, m_q, nb, U, eta, x, prm, delta, w, ws, st);
    int r;
    if ((r = sv.begin()) != LQ_OK) return r;
    if (sv.device_cycles(&r)) {
        if (r != LQ_OK) return r;
    } else {
        while (sv.plan()) {
            if ((r = sv.start_cycle()) != LQ_OK) return r;
            if ((r = sv.inner_single()) != LQ_OK) return r;
            if ((r = sv.end_cycle()) != LQ_OK) return r;
        }
    }
    return sv.finish(info);
}

// Right-hand sides per thread for a batch of nb: the LQ_CG_RHS_BLOCK_* flag if one is set
// (capped at nb), else 1.  Measured on the 24^3 x 48 workload with 12 right-hand sides (one
// GB300): scaled FP16 114.1 / 119.0 / 140.2 ms and FP32 127.4 / 130.7 / 174.8 ms for 1 / 2 /
// 4 right-hand sides per thread.  The link is decoded once per direction for all of them,
// but their accumulators raise the kernels' registers (scaled FP16 K1 96 -> 168 -> 251, K2
// 128 -> 168 -> 249), which costs resident warps; since the scaled-FP16 hop multiplies with
// the stored FP16 link rows directly, its link decode is too small a part of a hop for
// blocking to pay.
inline int rhs_block(const lq_cg_params& prm, int nb) {
    int rb = (prm.flags & LQ_CG_RHS_BLOCK_4) ? 4 : (prm.flags & LQ_CG_RHS_BLOCK_2) ? 2 : 1;
    while (rb > nb) rb >>= 1;
    return rb;
}

// The tuning cache (lattices.cu): tuned values by key, kept for the life of the process and
// appended to the file named by LQ_TUNE_CACHE.
bool tune_lookup(const std::string& key, int* value);
void tune_store(const std::string& key, int value);
std::string tune_key_rhs_block(int ip, int fmt, int hp, const Geom& g, int nb);

// Mean device time of K1 + K2 (the two stencil kernels; K3 does not depend on the blocking)
// with RB right-hand sides per thread on this batch: the inner links converted from U, p, r and
// psi filled with a small constant, and the state record zeroed before each pair, so that K1
// finds alpha = 0, K2 leaves psi and r as they are and every repetition does the same work on
// the same finite values; ms, or < 0 on error.  The solve that follows re-initialises
// everything the probe writes.
template <int IP, int IF, int IL, int HP, int RB>
double time_k12_rb(const Geom& g, double m_q, int nb, const void* U, const void* eta, void* x, const lq_cg_params& prm,
                   const WsLayout& w, char* ws, cudaStream_t st) {
    Solve<IP, IF, IL, HP, kBS, false, RB> sv;
    sv.init(g, m_q, nb, U, eta, x, prm, 0.0, w, ws, st);
    const int64_t vn = (int64_t)g.V * nb;
    if (cudaMemsetAsync(ws + w.p, 0x3c, spinor_bytes(vn, IP), st) != cudaSuccess ||
        cudaMemsetAsync(ws + w.r, 0x3c, spinor_bytes(vn, IP), st) != cudaSuccess ||
        cudaMemsetAsync(ws + w.psi, 0x3c, spinor_bytes(vn, psi_prec(IP)), st) != cudaSuccess ||
        convert_gauge(g, LQ_F64, LQ_LAYOUT_LEX, U, IP, IF, IL, ws + w.u_low, st) != cudaSuccess)
        return -1.0;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess) return -1.0;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return -1.0;
    }
    auto pair = [&] {
        return cudaMemsetAsync(sv.dstate, 0, sizeof(SolverState), st) == cudaSuccess &&
               sv.launch_k1(st) == cudaSuccess && sv.launch_k2(st) == cudaSuccess;
    };
    constexpr int kWarm = 2, kReps = 6;
    bool ok = true;
    for (int i = 0; i < kWarm; ++i) ok &= pair();
    ok &= cudaEventRecord(e0, st) == cudaSuccess;
    for (int i = 0; i < kReps; ++i) ok &= pair();
    ok &= cudaEventRecord(e1, st) == cudaSuccess;
    ok &= cudaEventSynchronize(e1) == cudaSuccess;
    float ms = 0.f;
    ok &= cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return ok ? ms / kReps : -1.0;
}

// Right-hand sides per thread chosen by timing (LQ_CG_AUTOTUNE without an LQ_CG_RHS_BLOCK_*
// flag): K1 + K2 with 1, 2 and 4 (at most nb), the fastest kept in the tuning cache per GPU,
// link format, precisions, lattice and batch size; 0 if a probe failed.
template <int IP, int IF, int IL, int HP>
int tuned_rhs_block(const Geom& g, double m_q, int nb, const void* U, const void* eta, void* x,
                    const lq_cg_params& prm, const WsLayout& w, char* ws, cudaStream_t st) {
    const std::string key = tune_key_rhs_block(IP, IF, HP, g, nb);
    int rb = 1;
    if (tune_lookup(key, &rb) && rb >= 1 && rb <= nb) return rb;
    const double t[3] = {time_k12_rb<IP, IF, IL, HP, 1>(g, m_q, nb, U, eta, x, prm, w, ws, st),
                         nb >= 2 ? time_k12_rb<IP, IF, IL, HP, 2>(g, m_q, nb, U, eta, x, prm, w, ws, st) : -1.0,
                         nb >= 4 ? time_k12_rb<IP, IF, IL, HP, 4>(g, m_q, nb, U, eta, x, prm, w, ws, st) : -1.0};
    if (t[0] < 0.0 || (nb >= 2 && t[1] < 0.0) || (nb >= 4 && t[2] < 0.0)) return 0;
    int best = 0;
    for (int i = 1; i < 3; ++i)
        if (t[i] >= 0.0 && t[i] < t[best]) best = i;
    rb = 1 << best;
    tune_store(key, rb);
    return rb;
}

template <int IP, int IF, int IL, int HP, bool SCHUR = false>
int run_solver(const Geom& g, double m_q, int nb, const void* U, const void* eta, void* x, const lq_cg_params& prm,
               double delta, const WsLayout& w, char* ws, lq_cg_info* info, cudaStream_t st) {
    if constexpr (!SCHUR && IL == LQ_LAYOUT_EO && IF == 12 && !std::is_same<typename PrecT<IP>::Real, dd>::value) {
        int rb = rhs_block(prm, nb);
        const int rsel = prm.flags & (LQ_CG_RHS_BLOCK_1 | LQ_CG_RHS_BLOCK_2 | LQ_CG_RHS_BLOCK_4);
        if ((prm.flags & LQ_CG_AUTOTUNE) && rsel == 0 && nb > 1) {
            rb = tuned_rhs_block<IP, IF, IL, HP>(g, m_q, nb, U, eta, x, prm, w, ws, st);
            if (rb == 0) return fail(LQ_ERR_CUDA, "right-hand-side block tuning failed: %s",
                                     cudaGetErrorString(cudaGetLastError()));
        }
        if (rb == 4) return run_solver_rb<IP, IF, IL, HP, SCHUR, 4>(g, m_q, nb, U, eta, x, prm, delta, w, ws, info, st);
        if (rb == 2) return run_solver_rb<IP, IF, IL, HP, SCHUR, 2>(g, m_q, nb, U, eta, x, prm, delta, w, ws, info, st);
    }
    return run_solver_rb<IP, IF, IL, HP, SCHUR, 1>(g, m_q, nb, U, eta, x, prm, delta, w, ws, info, st);
}

// Instantiations live in solver_f64.cu (FP64 and FP32-pair inner loops), solver_f32.cu,
// solver_f16.cu and solver_i32.cu (mixed inner loops with either outer arithmetic and link
// format).
int solve_f64(const Geom& g, double m_q, int nb, const void* U, const void* eta, void* x, const lq_cg_params& prm,
              double delta, const WsLayout& w, char* ws, lq_cg_info* info, cudaStream_t st);
int solve_f64x(const Geom& g, double m_q, int nb, const void* U, const void* eta, void* x, const lq_cg_params& prm,
               double delta, const WsLayout& w, char* ws, lq_cg_info* info, cudaStream_t st);
int solve_mixed_f32(const Geom& g, double m_q, int nb, const void* U, const void* eta, void* x,
                    const lq_cg_params& prm, double delta, const WsLayout& w, char* ws, lq_cg_info* info,
                    cudaStream_t st, bool pairs, int fmt);
int solve_mixed_f16(const Geom& g, double m_q, int nb, const void* U, const void* eta, void* x,
                    const lq_cg_params& prm, double delta, const WsLayout& w, char* ws, lq_cg_info* info,
                    cudaStream_t st, bool pairs, int fmt);
int solve_mixed_i32(const Geom& g, double m_q, int nb, const void* U, const void* eta, void* x,
                    const lq_cg_params& prm, double delta, const WsLayout& w, char* ws, lq_cg_info* info,
                    cudaStream_t st, bool pairs, int fmt);
// even-odd Schur solves of D x = b (solver_schur_a.cu, solver_schur_b.cu)
int schur_f64x(const Geom& g, double m_q, int nb, const void* U, const void* b, void* x, const lq_cg_params& prm,
               double delta, const WsLayout& w, char* ws, lq_cg_info* info, cudaStream_t st, int fmt);
int schur_f32(const Geom& g, double m_q, int nb, const void* U, const void* b, void* x, const lq_cg_params& prm,
              double delta, const WsLayout& w, char* ws, lq_cg_info* info, cudaStream_t st, int fmt);
int schur_f16(const Geom& g, double m_q, int nb, const void* U, const void* b, void* x, const lq_cg_params& prm,
              double delta, const WsLayout& w, char* ws, lq_cg_info* info, cudaStream_t st, int fmt);
int schur_i32(const Geom& g, double m_q, int nb, const void* U, const void* b, void* x, const lq_cg_params& prm,
              double delta, const WsLayout& w, char* ws, lq_cg_info* info, cudaStream_t st, int fmt);

}  // namespace solver_detail

}  // namespace lq
