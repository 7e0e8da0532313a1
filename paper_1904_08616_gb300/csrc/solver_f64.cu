// CG drivers with an FP64-class inner loop (native FP64, or FP32 pairs) and the mode
// dispatch of lq_cg_solve.
#include "solver_impl.cuh"

namespace lq {

namespace solver_detail {

int solve_f64(const Geom& g, double m_q, const void* U, const void* eta, void* x, const lq_cg_params& prm,
              double delta, const WsLayout& w, char* ws, lq_cg_info* info, cudaStream_t st) {
    return run_solver<LQ_F64, 18, LQ_LAYOUT_LEX, LQ_F64>(g, m_q, U, eta, x, prm, delta, w, ws, info, st);
}

int solve_f64x(const Geom& g, double m_q, const void* U, const void* eta, void* x, const lq_cg_params& prm,
               double delta, const WsLayout& w, char* ws, lq_cg_info* info, cudaStream_t st) {
    return run_solver<LQ_F64X, 18, LQ_LAYOUT_EO, LQ_F64X>(g, m_q, U, eta, x, prm, delta, w, ws, info, st);
}

}  // namespace solver_detail

size_t cg_workspace_bytes(const Geom& g, int mode) { return solver_detail::ws_bytes_for_mode(g, mode); }

int cg_solve(const Geom& g, double m_q, int mode, const void* U, const void* eta, void* x, const lq_cg_params& prm,
             void* ws, size_t ws_bytes, lq_cg_info* info, cudaStream_t st) {
    using namespace solver_detail;
    const bool native = (prm.flags & LQ_CG_NATIVE_F64) != 0;
    if (mode == LQ_CG_F64X && native) return fail(LQ_ERR_ARG, "LQ_CG_NATIVE_F64 does not apply to LQ_CG_F64X");
    const bool pairs = (mode == LQ_CG_F64X) || ((mode == LQ_CG_MIXED_F32 || mode == LQ_CG_MIXED_F16) && !native);
    const int fmt = (prm.flags & LQ_CG_LINK18) ? 18 : 12;
    const WsLayout w = ws_layout(g, mode, pairs, fmt);
    if (ws == nullptr || ws_bytes < w.total)
        return fail(LQ_ERR_WORKSPACE, "workspace of %zu bytes needed, %zu given", w.total, ws_bytes);
    char* base = (char*)ws;
    double delta = prm.delta;
    switch (mode) {
        case LQ_CG_F64:
            if (!(delta > 0.0)) delta = 0.0;
            return solve_f64(g, m_q, U, eta, x, prm, delta, w, base, info, st);
        case LQ_CG_F64X:
            if (!(delta > 0.0)) delta = 0.0;
            return solve_f64x(g, m_q, U, eta, x, prm, delta, w, base, info, st);
        case LQ_CG_MIXED_F32:
            if (!(delta > 0.0)) delta = 1e-4;
            return solve_mixed_f32(g, m_q, U, eta, x, prm, delta, w, base, info, st, pairs, fmt);
        case LQ_CG_MIXED_F16:
            if (!(delta > 0.0)) delta = 0.1;
            return solve_mixed_f16(g, m_q, U, eta, x, prm, delta, w, base, info, st, pairs, fmt);
        default:
            return fail(LQ_ERR_ARG, "unknown CG mode %d", mode);
    }
}

}  // namespace lq
