// Instantiates the row kernels for M = 128, 256, 512.
#include "graf_af_impl.cuh"

GRAF_INSTANTIATE_M(128)
GRAF_INSTANTIATE_M(256)
GRAF_INSTANTIATE_M(512)
