// Even-odd Schur solve of D x = b with scaled-FP16 and 32-bit fixed-point inner storage
// (FP32 arithmetic, FP32-pair outer loop); see solver_schur_a.cu.
#include "solver_impl.cuh"

namespace lq {

namespace solver_detail {

int schur_f16(const Geom& g, double m_q, int nb, const void* U, const void* b, void* x, const lq_cg_params& prm,
              double delta, const WsLayout& w, char* ws, lq_cg_info* info, cudaStream_t st, int fmt) {
    return fmt == 18 ? run_solver<LQ_F16S, 18, LQ_LAYOUT_EO, LQ_F64X, true>(g, m_q, nb, U, b, x, prm, delta, w, ws, info, st)
                     : run_solver<LQ_F16S, 12, LQ_LAYOUT_EO, LQ_F64X, true>(g, m_q, nb, U, b, x, prm, delta, w, ws, info, st);
}

int schur_i32(const Geom& g, double m_q, int nb, const void* U, const void* b, void* x, const lq_cg_params& prm,
              double delta, const WsLayout& w, char* ws, lq_cg_info* info, cudaStream_t st, int fmt) {
    return fmt == 18 ? run_solver<LQ_I32S, 18, LQ_LAYOUT_EO, LQ_F64X, true>(g, m_q, nb, U, b, x, prm, delta, w, ws, info, st)
                     : run_solver<LQ_I32S, 12, LQ_LAYOUT_EO, LQ_F64X, true>(g, m_q, nb, U, b, x, prm, delta, w, ws, info, st);
}

}  // namespace solver_detail

}  // namespace lq
