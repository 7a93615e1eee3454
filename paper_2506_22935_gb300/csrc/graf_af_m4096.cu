// Instantiates the row kernels for M = 4096.
#include "graf_af_impl.cuh"

GRAF_INSTANTIATE_M(4096)
