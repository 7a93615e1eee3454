// Instantiates the row kernels for M = 128.
#include "graf_af_impl.cuh"

GRAF_INSTANTIATE_M(128)
