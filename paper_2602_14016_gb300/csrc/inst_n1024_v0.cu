// Kernels and launchers for n = 1024, plan variant 0.
#include "ops_impl.cuh"
DA_INSTANTIATE(1024, 0)
