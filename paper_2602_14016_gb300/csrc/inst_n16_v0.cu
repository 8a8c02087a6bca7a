// Kernels and launchers for n = 16, plan variant 0.
#include "ops_impl.cuh"
DA_INSTANTIATE(16, 0)
