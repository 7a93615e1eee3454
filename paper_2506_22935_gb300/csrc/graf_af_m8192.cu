// Instantiates the row kernels for M = 8192.
#include "graf_af_impl.cuh"

GRAF_INSTANTIATE_M(8192)
