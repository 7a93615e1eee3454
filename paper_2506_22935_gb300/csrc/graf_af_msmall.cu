// Instantiates the row kernels for M = 8, 16, 32, 64.
#include "graf_af_impl.cuh"

GRAF_INSTANTIATE_M(8)
GRAF_INSTANTIATE_M(16)
GRAF_INSTANTIATE_M(32)
GRAF_INSTANTIATE_M(64)
