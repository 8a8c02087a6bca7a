// Kernels and launchers for n = 16.
#include "ops_impl.cuh"
DA_INSTANTIATE(16)
