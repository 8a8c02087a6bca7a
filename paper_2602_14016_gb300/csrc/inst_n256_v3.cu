// Kernels and launchers for n = 256, plan variant 3.
#include "ops_impl.cuh"
DA_INSTANTIATE(256, 3)
