// Operator kernels for FP32-pair (LQ_F64X) fields, 18-real links only: full-lattice D,
// D^dag and the EO hopping term.
#include "dslash_dispatch.cuh"

namespace lq {

cudaError_t apply_f64x(const Geom& g, double m_q, int fmt, int layout, bool dag, const void* U, const void* psi,
                       void* out, cudaStream_t st, int lnr) {
    if (fmt != 18) return cudaErrorInvalidValue;
    if (layout == LQ_LAYOUT_LEX)
        return dag ? run_apply<LQ_F64X, 18, LQ_LAYOUT_LEX, true>(g, m_q, U, psi, out, st, lnr)
                   : run_apply<LQ_F64X, 18, LQ_LAYOUT_LEX, false>(g, m_q, U, psi, out, st, lnr);
    return dag ? run_apply<LQ_F64X, 18, LQ_LAYOUT_EO, true>(g, m_q, U, psi, out, st, lnr)
               : run_apply<LQ_F64X, 18, LQ_LAYOUT_EO, false>(g, m_q, U, psi, out, st, lnr);
}

cudaError_t hop_f64x(const Geom& g, int p, bool dag, double a, double b, int fmt, const void* U,
                     const void* psi_other, const void* y, void* out, cudaStream_t st) {
    if (fmt != 18) return cudaErrorInvalidValue;
    const bool hy = y != nullptr;
    if (dag) return hy ? run_hop<LQ_F64X, 18, true, true>(g, p, a, b, U, psi_other, y, out, st)
                       : run_hop<LQ_F64X, 18, true, false>(g, p, a, b, U, psi_other, y, out, st);
    return hy ? run_hop<LQ_F64X, 18, false, true>(g, p, a, b, U, psi_other, y, out, st)
              : run_hop<LQ_F64X, 18, false, false>(g, p, a, b, U, psi_other, y, out, st);
}

}  // namespace lq
