// Instantiates the row kernels for M = 2048.
#include "graf_af_impl.cuh"

GRAF_INSTANTIATE_M(2048)
