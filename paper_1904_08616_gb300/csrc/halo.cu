// The Wilson-Dirac operator of Eq. (1) on one t-slab of a lattice split across domains
// (ranks), with the hops that cross the slab's two t-faces fed by face buffers from the
// neighbouring domains.  The paper exchanges boundary data between FPGAs over their
// transceivers; here a domain packs, for each face, what the neighbour's hop needs, the
// caller moves the buffers (a device copy between virtual ranks on one GPU, or a
// point-to-point transfer between processes), and the domain kernel consumes them.
//
//   to_prev[s] = (1 + S_f gamma_t) psi at t = 0, reduced to its upper spin half (h0, h1):
//                the forward t-hop of the previous domain's top slice projects with
//                S_f = -1 (D) or +1 (D^dag) and applies its own link U_t.
//   to_next[s] = U_t(n)^dag (1 - S_f gamma_t) psi(n) at t = Lt - 1, upper half (g0, g1):
//                the backward t-hop of the next domain's bottom slice, whose link U_t(n - t)
//                lives here.
// Face site s = x + Lx (y + Ly z); each face is Lx Ly Lz half spinors of 6 complex FP64
// numbers (96 bytes).  The stage arithmetic is the one of the full-lattice kernel, so a
// decomposed apply equals the single-domain one bit for bit.
#include "lq_abi_internal.h"
#include "dslash_dispatch.cuh"

namespace lq {

namespace {

constexpr int kHaloBS = 128;

using HSpin = SpinorAcc<LQ_F64, LQ_LAYOUT_LEX, true>;
using HGauge = GaugeAcc<LQ_F64, 18, LQ_LAYOUT_LEX>;

struct HalfSpinor {
    cplx<double> a[3], b[3];
};

__device__ __forceinline__ void face_store(double2* f, int s, const cplx<double> a[3], const cplx<double> b[3]) {
    double2* o = f + (size_t)s * 6;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        o[c] = make_double2(a[c].re, a[c].im);
        o[3 + c] = make_double2(b[c].re, b[c].im);
    }
}
__device__ __forceinline__ void face_load(const double2* f, int s, cplx<double> a[3], cplx<double> b[3]) {
    const double2* o = f + (size_t)s * 6;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const double2 u = __ldg(o + c), v = __ldg(o + 3 + c);
        a[c] = {u.x, u.y};
        b[c] = {v.x, v.y};
    }
}

template <bool DAG>
__global__ void __launch_bounds__(kHaloBS) halo_pack_kernel(Geom g, HGauge U, HSpin psi, double2* to_prev,
                                                            double2* to_next) {
    constexpr int SF = DAG ? +1 : -1;
    const int vs = g.S[3];   // sites per t-slice
    for (int i = blockIdx.x * kHaloBS + threadIdx.x; i < 2 * vs; i += gridDim.x * kHaloBS) {
        const bool top = i >= vs;
        const int s = top ? i - vs : i;
        const int lex = top ? s + (g.L[3] - 1) * vs : s;
        int c[4];
        const Site site = site_from_lex(g, lex, c);
        Spinor<double> q;
        psi.load(site, q);
        cplx<double> h0[3], h1[3];
        if (!top) {
            hop_project<3, SF>(q, h0, h1);
            face_store(to_prev, s, h0, h1);
        } else {
            hop_project<3, -SF>(q, h0, h1);
            Link<double> L;
            U.load(site, 3, L);
            cplx<double> g0[3], g1[3];
            hop_matvec<true>(L, h0, h1, g0, g1);
            face_store(to_next, s, g0, g1);
        }
    }
}

template <bool DAG>
__global__ void __launch_bounds__(kHaloBS) halo_dslash_kernel(Geom g, HGauge U, HSpin psi, const double2* from_next,
                                                              const double2* from_prev, double a, double b,
                                                              double2* out) {
    constexpr int SF = DAG ? +1 : -1;
    const int vs = g.S[3];
    for (int lex = blockIdx.x * kHaloBS + threadIdx.x; lex < g.V; lex += gridDim.x * kHaloBS) {
        int c[4];
        const Site s = site_from_lex(g, lex, c);
        Spinor<double> acc;
#pragma unroll
        for (int k = 0; k < 12; ++k) acc.v[k] = {0.0, 0.0};
        // x, y, z: the full-lattice stencil's hops
        Stencil<HGauge, HSpin, DAG> st{g, U, psi};
        st.template dir<0>(s, c, acc);
        st.template dir<1>(s, c, acc);
        st.template dir<2>(s, c, acc);
        // t: inside the slab as usual, across a face from the neighbour's buffer
        const int fs = lex - c[3] * vs;
        cplx<double> h0[3], h1[3], g0[3], g1[3];
        if (c[3] < g.L[3] - 1) {
            Spinor<double> q;
            psi.load(nb_site(lex + vs, s.p, 0), q);
            hop_project<3, SF>(q, h0, h1);
        } else {
            face_load(from_next, fs, h0, h1);
        }
        {
            Link<double> L;
            U.load(s, 3, L);
            hop_matvec<false>(L, h0, h1, g0, g1);
            hop_accumulate<3, SF, false>(acc, g0, g1, 1.0);
        }
        if (c[3] > 0) {
            const Site nb = nb_site(lex - vs, s.p, 0);
            Spinor<double> q;
            psi.load(nb, q);
            hop_project<3, -SF>(q, h0, h1);
            Link<double> L;
            U.load(nb, 3, L);
            hop_matvec<true>(L, h0, h1, g0, g1);
        } else {
            face_load(from_prev, fs, g0, g1);
        }
        hop_accumulate<3, -SF, false>(acc, g0, g1, 1.0);
        // out = a psi + b hop
        Spinor<double> y;
        psi.load(s, y);
        double2* o = out + (size_t)lex * 12;
#pragma unroll
        for (int k = 0; k < 12; ++k)
            o[k] = make_double2(fma(b, acc.v[k].re, a * y.v[k].re), fma(b, acc.v[k].im, a * y.v[k].im));
    }
}

int halo_grid(int n) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    long long want = ((long long)n + kHaloBS - 1) / kHaloBS, cap = (long long)sms * 8;
    return (int)(want < cap ? (want > 0 ? want : 1) : cap);
}

}  // namespace

cudaError_t halo_pack(const Geom& g, bool dag, const void* U, const void* psi, void* to_prev, void* to_next,
                      cudaStream_t st) {
    const HGauge ga = make_gauge<LQ_F64, 18, LQ_LAYOUT_LEX>(U, g);
    const HSpin sa = make_spinor<LQ_F64, LQ_LAYOUT_LEX, true>(psi, g, false);
    const int grid = halo_grid(2 * g.S[3]);
    if (dag) halo_pack_kernel<true><<<grid, kHaloBS, 0, st>>>(g, ga, sa, (double2*)to_prev, (double2*)to_next);
    else halo_pack_kernel<false><<<grid, kHaloBS, 0, st>>>(g, ga, sa, (double2*)to_prev, (double2*)to_next);
    return cudaGetLastError();
}

cudaError_t halo_dslash(const Geom& g, double m_q, bool dag, const void* U, const void* psi, const void* from_next,
                        const void* from_prev, void* out, cudaStream_t st) {
    const HGauge ga = make_gauge<LQ_F64, 18, LQ_LAYOUT_LEX>(U, g);
    const HSpin sa = make_spinor<LQ_F64, LQ_LAYOUT_LEX, true>(psi, g, false);
    const int grid = halo_grid(g.V);
    const double a = m_q + 4.0, b = 0.5;
    if (dag)
        halo_dslash_kernel<true><<<grid, kHaloBS, 0, st>>>(g, ga, sa, (const double2*)from_next,
                                                           (const double2*)from_prev, a, b, (double2*)out);
    else
        halo_dslash_kernel<false><<<grid, kHaloBS, 0, st>>>(g, ga, sa, (const double2*)from_next,
                                                            (const double2*)from_prev, a, b, (double2*)out);
    return cudaGetLastError();
}

}  // namespace lq
