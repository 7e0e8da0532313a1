// Operator kernels (full-lattice D, D^dag, EO hopping term) for precision LQ_F64.
#include "dslash_dispatch.cuh"

LQ_DEFINE_PREC_DISPATCH(f64, LQ_F64)
