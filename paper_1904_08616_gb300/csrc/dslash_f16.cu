// Operator kernels (full-lattice D, D^dag, EO hopping term) for precision LQ_F16S.
#include "dslash_dispatch.cuh"

LQ_DEFINE_PREC_DISPATCH(f16, LQ_F16S)
