// Even-odd Schur solve of D x = b (not in the paper, which inverts D^dag D): CG, or
// Algorithm 1, on Mhat^dag Mhat x_e = Mhat^dag bhat_e over the even sites with
// Mhat = A - H_eo H_oe / A, bhat_e = b_e - H_eo b_o / A (A = m_q + 4, H the hopping term of
// Eq. 1), then x_o = (b_o - H_oe x_e) / A.  FP32-pair and FP32 inner loops, and the mode
// dispatch; solver_schur_b.cu holds the scaled-FP16 and fixed-point inner loops.
#include "solver_impl.cuh"

namespace lq {

namespace solver_detail {

int schur_f64x(const Geom& g, double m_q, int nb, const void* U, const void* b, void* x, const lq_cg_params& prm,
               double delta, const WsLayout& w, char* ws, lq_cg_info* info, cudaStream_t st, int) {
    return run_solver<LQ_F64X, 18, LQ_LAYOUT_EO, LQ_F64X, true>(g, m_q, nb, U, b, x, prm, delta, w, ws, info, st);
}

int schur_f32(const Geom& g, double m_q, int nb, const void* U, const void* b, void* x, const lq_cg_params& prm,
              double delta, const WsLayout& w, char* ws, lq_cg_info* info, cudaStream_t st, int fmt) {
    return fmt == 18 ? run_solver<LQ_F32, 18, LQ_LAYOUT_EO, LQ_F64X, true>(g, m_q, nb, U, b, x, prm, delta, w, ws, info, st)
                     : run_solver<LQ_F32, 12, LQ_LAYOUT_EO, LQ_F64X, true>(g, m_q, nb, U, b, x, prm, delta, w, ws, info, st);
}

size_t schur_ws_bytes(const Geom& g, int mode, int nrhs) {
    size_t m = 0;
    for (int fmt : {12, 18}) {
        const size_t t = ws_layout_schur(g, mode, fmt, batch_size(nrhs)).total;
        if (t > m) m = t;
    }
    return m;
}

}  // namespace solver_detail

size_t cg_workspace_bytes_schur(const Geom& g, int mode, int nrhs) {
    return solver_detail::schur_ws_bytes(g, mode, nrhs);
}

int cg_solve_schur(const Geom& g, double m_q, int mode, int nrhs, const void* U, const void* b, void* x,
                   const lq_cg_params& prm, void* ws, size_t ws_bytes, lq_cg_info* info, cudaStream_t st) {
    using namespace solver_detail;
    if (mode == LQ_CG_F64) return fail(LQ_ERR_ARG, "the Schur solve runs its outer loop in FP32 pairs: use LQ_CG_F64X");
    if (prm.flags & LQ_CG_NATIVE_F64) return fail(LQ_ERR_ARG, "LQ_CG_NATIVE_F64 does not apply to the Schur solve");
    if (prm.flags & LQ_CG_LINK10) return fail(LQ_ERR_ARG, "LQ_CG_LINK10 does not apply to the Schur solve");
    const int fmt = (mode == LQ_CG_F64X || (prm.flags & LQ_CG_LINK18)) ? 18 : 12;
    {
        const WsLayout w = ws_layout_schur(g, mode, fmt, batch_size(nrhs));
        if (ws == nullptr || ws_bytes < w.total)
            return fail(LQ_ERR_WORKSPACE, "workspace of %zu bytes needed, %zu given", w.total, ws_bytes);
    }
    double delta = prm.delta;
    if (!(delta > 0.0)) delta = default_delta(mode);
    const size_t field = spinor_bytes(g.V, LQ_F64);
    int worst = LQ_OK;
    for (int first = 0; first < nrhs;) {
        const int nb = batch_size(nrhs - first);
        const WsLayout w = ws_layout_schur(g, mode, fmt, nb);
        const void* bb = (const char*)b + field * first;
        void* xb = (char*)x + field * first;
        lq_cg_info* ib = info ? info + first : nullptr;
        int r;
        switch (mode) {
            case LQ_CG_F64X: r = schur_f64x(g, m_q, nb, U, bb, xb, prm, delta, w, (char*)ws, ib, st, fmt); break;
            case LQ_CG_MIXED_F32: r = schur_f32(g, m_q, nb, U, bb, xb, prm, delta, w, (char*)ws, ib, st, fmt); break;
            case LQ_CG_MIXED_F16: r = schur_f16(g, m_q, nb, U, bb, xb, prm, delta, w, (char*)ws, ib, st, fmt); break;
            case LQ_CG_MIXED_I32: r = schur_i32(g, m_q, nb, U, bb, xb, prm, delta, w, (char*)ws, ib, st, fmt); break;
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
