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

// The spin sums collapse onto the rank-2 projections: for P = 1 + S gamma_mu, whose lower
// spin half is S B^dag times its upper half h (chiral basis), sum_s a_s conj((P b)_s) equals
// sum_{k=0,1} (P a)_k conj((P b)_k) with (P a)_k the upper half of P a.  So
//   G_mu(n) = 1/2 sum_{k=0,1} [ (P^- g(n))_k (P^- psi(n+mu))_k^H + (P^+ psi(n))_k (P^+ g(n+mu))_k^H ],
// two 3x3 outer products of colour vectors per term instead of four.

// M[A][B] += a0_A conj(b0_B) + a1_A conj(b1_B)
__device__ __forceinline__ void outer_acc2(const cplx<double> a0[3], const cplx<double> a1[3],
                                           const cplx<double> b0[3], const cplx<double> b1[3],
                                           cplx<double> M[3][3]) {
#pragma unroll
    for (int A = 0; A < 3; ++A)
#pragma unroll
        for (int B = 0; B < 3; ++B) M[A][B] = cfmac(b1[B], a1[A], cfmac(b0[B], a0[A], M[A][B]));
}

template <int MU>
__device__ __forceinline__ void grad_dir(const Geom& g, const SpinorAcc<LQ_F64, LQ_LAYOUT_LEX, true>& G,
                                         const SpinorAcc<LQ_F64, LQ_LAYOUT_LEX, true>& P, const Site& s,
                                         const int c[4], const Spinor<double>& gn, const Spinor<double>& pn,
                                         double scale, bool accumulate, double2* out) {
    const Site nf = nb_site(lex_fwd(g, s.lex, c, MU), s.p, 0);
    Spinor<double> gf, pf;
    G.load(nf, gf);
    P.load(nf, pf);
    cplx<double> a0[3], a1[3], b0[3], b1[3];
    cplx<double> M[3][3];
#pragma unroll
    for (int A = 0; A < 3; ++A)
#pragma unroll
        for (int B = 0; B < 3; ++B) M[A][B] = {0.0, 0.0};
    hop_project<MU, -1>(gn, a0, a1);   // P^{-mu} g(n)
    hop_project<MU, -1>(pf, b0, b1);   // P^{-mu} psi(n + mu)
    outer_acc2(a0, a1, b0, b1, M);
    hop_project<MU, +1>(pn, a0, a1);   // P^{+mu} psi(n)
    hop_project<MU, +1>(gf, b0, b1);   // P^{+mu} g(n + mu)
    outer_acc2(a0, a1, b0, b1, M);
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
