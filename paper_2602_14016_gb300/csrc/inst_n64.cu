// Kernels and launchers for n = 64.
#include "ops_impl.cuh"
DA_INSTANTIATE(64)
