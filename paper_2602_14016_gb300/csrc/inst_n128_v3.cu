// Kernels and launchers for n = 128, plan variant 3.
#include "ops_impl.cuh"
DA_INSTANTIATE(128, 3)
