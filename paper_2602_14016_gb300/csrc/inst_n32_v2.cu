// Kernels and launchers for n = 32, plan variant 2.
#include "ops_impl.cuh"
DA_INSTANTIATE(32, 2)
