// Instantiates the row kernels for M = 512.
#include "graf_af_impl.cuh"

GRAF_INSTANTIATE_M(512)
