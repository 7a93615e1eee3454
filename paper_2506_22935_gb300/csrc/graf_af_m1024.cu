// Instantiates the row kernels for M = 1024.
#include "graf_af_impl.cuh"

GRAF_INSTANTIATE_M(1024)
