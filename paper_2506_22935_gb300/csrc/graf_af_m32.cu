// Instantiates the row kernels for M = 32.
#include "graf_af_impl.cuh"

GRAF_INSTANTIATE_M(32)
