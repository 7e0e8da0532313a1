// Multi-lattice mixed-precision CG (Algorithm 1): FP32 inner loop on 12-real links,
// FP32-pair outer arithmetic.
#include "solver_lattices.cuh"

namespace lq {

namespace solver_detail {

int lattices_mixed_f32(int n, const LatticeJob* jobs, const lq_cg_params& prm, double delta, char* ws,
                       lq_cg_info* info, cudaStream_t st) {
    return run_lattices<LQ_F32, 12, LQ_LAYOUT_EO, LQ_F64X>(LQ_CG_MIXED_F32, n, jobs, prm, delta, ws, info, st);
}

}  // namespace solver_detail

}  // namespace lq
