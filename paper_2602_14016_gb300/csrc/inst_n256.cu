// Kernels and launchers for n = 256.
#include "ops_impl.cuh"
DA_INSTANTIATE(256)
