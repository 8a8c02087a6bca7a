// Kernels and launchers for n = 256, plan variant 2.
#include "ops_impl.cuh"
DA_INSTANTIATE(256, 2)
