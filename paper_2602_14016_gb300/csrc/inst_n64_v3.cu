// Kernels and launchers for n = 64, plan variant 3.
#include "ops_impl.cuh"
DA_INSTANTIATE(64, 3)
