// Gradient of Re <g, D psi> with respect to the links (Eq. 1 differentiated; the paper
// does not differentiate the operator, this is the library's adjoint support):
//   G_mu(n) = 1/2 sum_spin [ g(n) (P^{-mu} psi(n+mu))^H + (P^{+mu} psi(n)) g(n+mu)^H ],
// one 3x3 complex matrix per link, in the convention grad = dL/dRe + i dL/dIm.
// out = scale * G (+ out when accumulating).  FP64, LEX layout, one thread per site.
#include "lq_abi_internal.h"
#include "dslash_dispatch.cuh"

namespace lq {

namespace {

constexpr int kGradBS = 128;

// (1 + S gamma_MU) q as a full four-spin spinor: upper h = up + S B dn, lower S B^dag h
template <int MU, int S>
__device__ __forceinline__ void project_full(const Spinor<double>& q, Spinor<double>& o) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const cplx<double> p0 = q.v[c], p1 = q.v[3 + c], p2 = q.v[6 + c], p3 = q.v[9 + c];
        cplx<double> h0, h1, l2, l3;
        if constexpr (MU == 0) {
            h0 = pm<S>(p0, ctimes_mi(p3));
            h1 = pm<S>(p1, ctimes_mi(p2));
            l2 = ctimes_i(h1);
            l3 = ctimes_i(h0);
        } else if constexpr (MU == 1) {
            h0 = pm<-S>(p0, p3);
            h1 = pm<S>(p1, p2);
            l2 = h1;
            l3 = cneg(h0);
        } else if constexpr (MU == 2) {
            h0 = pm<S>(p0, ctimes_mi(p2));
            h1 = pm<S>(p1, ctimes_i(p3));
            l2 = ctimes_i(h0);
            l3 = ctimes_mi(h1);
        } else {
            h0 = pm<S>(p0, p2);
            h1 = pm<S>(p1, p3);
            l2 = h0;
            l3 = h1;
        }
        o.v[c] = h0;
        o.v[3 + c] = h1;
        o.v[6 + c] = (S > 0) ? l2 : cneg(l2);
        o.v[9 + c] = (S > 0) ? l3 : cneg(l3);
    }
}

// M[A][B] += sum_spin a_A conj(b_B)
__device__ __forceinline__ void outer_acc(const Spinor<double>& a, const Spinor<double>& b, cplx<double> M[3][3]) {
#pragma unroll
    for (int s = 0; s < 4; ++s)
#pragma unroll
        for (int A = 0; A < 3; ++A)
#pragma unroll
            for (int B = 0; B < 3; ++B) M[A][B] = cfmac(b.v[3 * s + B], a.v[3 * s + A], M[A][B]);
}

template <int MU>
__device__ __forceinline__ void grad_dir(const Geom& g, const SpinorAcc<LQ_F64, LQ_LAYOUT_LEX, true>& G,
                                         const SpinorAcc<LQ_F64, LQ_LAYOUT_LEX, true>& P, const Site& s,
                                         const int c[4], const Spinor<double>& gn, const Spinor<double>& pn,
                                         double scale, bool accumulate, double2* out) {
    const Site nf = nb_site(lex_fwd(g, s.lex, c, MU), s.p, 0);
    Spinor<double> gf, pf, w, v;
    G.load(nf, gf);
    P.load(nf, pf);
    project_full<MU, -1>(pf, w);   // P^{-mu} psi(n + mu)
    project_full<MU, +1>(pn, v);   // P^{+mu} psi(n)
    cplx<double> M[3][3];
#pragma unroll
    for (int A = 0; A < 3; ++A)
#pragma unroll
        for (int B = 0; B < 3; ++B) M[A][B] = {0.0, 0.0};
    outer_acc(gn, w, M);
    outer_acc(v, gf, M);
    double2* o = out + ((size_t)s.lex * 4 + MU) * 9;
    const double f = 0.5 * scale;
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        double2 r = make_double2(f * M[k / 3][k % 3].re, f * M[k / 3][k % 3].im);
        if (accumulate) {
            const double2 old = o[k];
            r.x += old.x;
            r.y += old.y;
        }
        o[k] = r;
    }
}

__global__ void __launch_bounds__(kGradBS) link_grad_kernel(Geom g, SpinorAcc<LQ_F64, LQ_LAYOUT_LEX, true> G,
                                                            SpinorAcc<LQ_F64, LQ_LAYOUT_LEX, true> P, double scale,
                                                            int accumulate, double2* out) {
    for (int lex = blockIdx.x * kGradBS + threadIdx.x; lex < g.V; lex += gridDim.x * kGradBS) {
        int c[4];
        const Site s = site_from_lex(g, lex, c);
        Spinor<double> gn, pn;
        G.load(s, gn);
        P.load(s, pn);
        grad_dir<0>(g, G, P, s, c, gn, pn, scale, accumulate != 0, out);
        grad_dir<1>(g, G, P, s, c, gn, pn, scale, accumulate != 0, out);
        grad_dir<2>(g, G, P, s, c, gn, pn, scale, accumulate != 0, out);
        grad_dir<3>(g, G, P, s, c, gn, pn, scale, accumulate != 0, out);
    }
}

}  // namespace

cudaError_t link_grad(const Geom& g, const void* gf, const void* psi, double scale, bool accumulate, void* out,
                      cudaStream_t st) {
    auto k = link_grad_kernel;
    const int nt = (g.V + kGradBS - 1) / kGradBS;
    const int grid = grid_for(k, kGradBS, nt);
    k<<<grid, kGradBS, 0, st>>>(g, make_spinor<LQ_F64, LQ_LAYOUT_LEX, true>(gf, g, false),
                                make_spinor<LQ_F64, LQ_LAYOUT_LEX, true>(psi, g, false), scale, accumulate ? 1 : 0,
                                (double2*)out);
    return cudaGetLastError();
}

}  // namespace lq
