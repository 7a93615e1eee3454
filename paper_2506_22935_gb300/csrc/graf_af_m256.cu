// Instantiates the row kernels for M = 256.
#include "graf_af_impl.cuh"

GRAF_INSTANTIATE_M(256)
