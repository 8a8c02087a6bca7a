// Kernels and launchers for n = 32.
#include "ops_impl.cuh"
DA_INSTANTIATE(32)
