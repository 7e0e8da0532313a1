// Operator kernels (full-lattice D, D^dag, EO hopping term) for precision LQ_F32.
#include "dslash_dispatch.cuh"

LQ_DEFINE_PREC_DISPATCH(f32, LQ_F32)
