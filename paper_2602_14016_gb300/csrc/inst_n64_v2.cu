// Kernels and launchers for n = 64, plan variant 2.
#include "ops_impl.cuh"
DA_INSTANTIATE(64, 2)
