// CG drivers with an FP64-class inner loop (native FP64, or FP32 pairs) and the mode
// dispatch of lq_cg_solve.
#include "solver_impl.cuh"

namespace lq {

namespace solver_detail {

int solve_f64(const Geom& g, double m_q, int nb, const void* U, const void* eta, void* x, const lq_cg_params& prm,
              double delta, const WsLayout& w, char* ws, lq_cg_info* info, cudaStream_t st) {
    return run_solver<LQ_F64, 18, LQ_LAYOUT_LEX, LQ_F64>(g, m_q, nb, U, eta, x, prm, delta, w, ws, info, st);
}

int solve_f64x(const Geom& g, double m_q, int nb, const void* U, const void* eta, void* x, const lq_cg_params& prm,
               double delta, const WsLayout& w, char* ws, lq_cg_info* info, cudaStream_t st) {
    return run_solver<LQ_F64X, 18, LQ_LAYOUT_EO, LQ_F64X>(g, m_q, nb, U, eta, x, prm, delta, w, ws, info, st);
}

}  // namespace solver_detail

size_t cg_workspace_bytes(const Geom& g, int mode, int nrhs) { return solver_detail::ws_bytes_for_mode(g, mode, nrhs); }

int cg_solve(const Geom& g, double m_q, int mode, int nrhs, const void* U, const void* eta, void* x,
             const lq_cg_params& prm, void* ws, size_t ws_bytes, lq_cg_info* info, cudaStream_t st) {
    using namespace solver_detail;
    const bool native = (prm.flags & LQ_CG_NATIVE_F64) != 0;
    if (mode == LQ_CG_F64X && native) return fail(LQ_ERR_ARG, "LQ_CG_NATIVE_F64 does not apply to LQ_CG_F64X");
    const bool mixed = mode == LQ_CG_MIXED_F32 || mode == LQ_CG_MIXED_F16 || mode == LQ_CG_MIXED_I32;
    const bool pairs = (mode == LQ_CG_F64X) || (mixed && !native);
    if ((prm.flags & LQ_CG_LINK10) && (prm.flags & LQ_CG_LINK18))
        return fail(LQ_ERR_ARG, "LQ_CG_LINK10 and LQ_CG_LINK18 exclude each other");
    if ((prm.flags & LQ_CG_LINK10) && mixed && !pairs)
        return fail(LQ_ERR_ARG, "LQ_CG_LINK10 runs with the FP32-pair outer loop (not with LQ_CG_NATIVE_F64)");
    const int fmt = (prm.flags & LQ_CG_LINK18) ? 18 : ((prm.flags & LQ_CG_LINK10) ? 10 : 12);
    {
        const WsLayout w = ws_layout(g, mode, pairs, fmt, batch_size(nrhs));
        if (ws == nullptr || ws_bytes < w.total)
            return fail(LQ_ERR_WORKSPACE, "workspace of %zu bytes needed, %zu given", w.total, ws_bytes);
    }
    double delta = prm.delta;
    if (!(delta > 0.0)) delta = default_delta(mode);
    // batches of a power of two <= kMaxRhs right-hand sides, each sharing the link loads
    const size_t field = spinor_bytes(g.V, LQ_F64);
    int worst = LQ_OK;
    for (int first = 0; first < nrhs;) {
        const int nb = batch_size(nrhs - first);
        const WsLayout w = ws_layout(g, mode, pairs, fmt, nb);
        const void* eb = (const char*)eta + field * first;
        void* xb = (char*)x + field * first;
        lq_cg_info* ib = info ? info + first : nullptr;
        int r;
        switch (mode) {
            case LQ_CG_F64: r = solve_f64(g, m_q, nb, U, eb, xb, prm, delta, w, (char*)ws, ib, st); break;
            case LQ_CG_F64X: r = solve_f64x(g, m_q, nb, U, eb, xb, prm, delta, w, (char*)ws, ib, st); break;
            case LQ_CG_MIXED_F32:
                r = solve_mixed_f32(g, m_q, nb, U, eb, xb, prm, delta, w, (char*)ws, ib, st, pairs, fmt);
                break;
            case LQ_CG_MIXED_F16:
                r = solve_mixed_f16(g, m_q, nb, U, eb, xb, prm, delta, w, (char*)ws, ib, st, pairs, fmt);
                break;
            case LQ_CG_MIXED_I32:
                r = solve_mixed_i32(g, m_q, nb, U, eb, xb, prm, delta, w, (char*)ws, ib, st, pairs, fmt);
                break;
            default: return fail(LQ_ERR_ARG, "unknown CG mode %d", mode);
        }
        if (r == LQ_ERR_CUDA || r == LQ_ERR_WORKSPACE || r == LQ_ERR_ARG) return r;
        if (r < 0 && (worst >= 0 || r < worst)) worst = r;
        if (r == LQ_NOT_CONVERGED && worst == LQ_OK) worst = LQ_NOT_CONVERGED;
        first += nb;
    }
    return worst;
}

}  // namespace lq
