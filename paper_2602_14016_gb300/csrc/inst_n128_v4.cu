// Kernels and launchers for n = 128, plan variant 4.
#include "ops_impl.cuh"
DA_INSTANTIATE(128, 4)
