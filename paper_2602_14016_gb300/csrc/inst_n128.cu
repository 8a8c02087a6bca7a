// Kernels and launchers for n = 128.
#include "ops_impl.cuh"
DA_INSTANTIATE(128)
