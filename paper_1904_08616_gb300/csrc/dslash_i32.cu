// Operator kernels (full-lattice D, D^dag, EO hopping term) for precision LQ_I32S.
#include "dslash_dispatch.cuh"

LQ_DEFINE_PREC_DISPATCH(i32, LQ_I32S)
