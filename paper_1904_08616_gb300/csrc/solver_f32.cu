// Mixed-precision CG drivers (Algorithm 1) with a LQ_F32 inner loop: FP32-pair or native
// FP64 outer arithmetic, 12-, 18- or (with FP32-pair outer arithmetic) 10-real inner links.
#include "solver_impl.cuh"

namespace lq {

namespace solver_detail {

int solve_mixed_f32(const Geom& g, double m_q, int nb, const void* U, const void* eta, void* x,
                    const lq_cg_params& prm, double delta, const WsLayout& w, char* ws, lq_cg_info* info,
                    cudaStream_t st, bool pairs, int fmt) {
    if (pairs && fmt == 10)
        return run_solver<LQ_F32, 10, LQ_LAYOUT_EO, LQ_F64X>(g, m_q, nb, U, eta, x, prm, delta, w, ws, info, st);
    if (pairs)
        return fmt == 18 ? run_solver<LQ_F32, 18, LQ_LAYOUT_EO, LQ_F64X>(g, m_q, nb, U, eta, x, prm, delta, w, ws, info, st)
                         : run_solver<LQ_F32, 12, LQ_LAYOUT_EO, LQ_F64X>(g, m_q, nb, U, eta, x, prm, delta, w, ws, info, st);
    return fmt == 18 ? run_solver<LQ_F32, 18, LQ_LAYOUT_EO, LQ_F64>(g, m_q, nb, U, eta, x, prm, delta, w, ws, info, st)
                     : run_solver<LQ_F32, 12, LQ_LAYOUT_EO, LQ_F64>(g, m_q, nb, U, eta, x, prm, delta, w, ws, info, st);
}

}  // namespace solver_detail

}  // namespace lq
