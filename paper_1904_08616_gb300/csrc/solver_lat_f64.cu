// Multi-lattice CG with an FP64-class inner loop: native FP64, or FP32 pairs.
#include "solver_lattices.cuh"

namespace lq {

namespace solver_detail {

int lattices_f64(int n, const LatticeJob* jobs, const lq_cg_params& prm, double delta, char* ws, lq_cg_info* info,
                 cudaStream_t st) {
    return run_lattices<LQ_F64, 18, LQ_LAYOUT_LEX, LQ_F64>(LQ_CG_F64, n, jobs, prm, delta, ws, info, st);
}

int lattices_f64x(int n, const LatticeJob* jobs, const lq_cg_params& prm, double delta, char* ws, lq_cg_info* info,
                  cudaStream_t st) {
    return run_lattices<LQ_F64X, 18, LQ_LAYOUT_EO, LQ_F64X>(LQ_CG_F64X, n, jobs, prm, delta, ws, info, st);
}

}  // namespace solver_detail

}  // namespace lq
