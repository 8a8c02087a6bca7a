// Kernels and launchers for n = 512, plan variant 2.
#include "ops_impl.cuh"
DA_INSTANTIATE(512, 2)
