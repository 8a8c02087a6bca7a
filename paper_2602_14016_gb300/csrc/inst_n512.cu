// Kernels and launchers for n = 512.
#include "ops_impl.cuh"
DA_INSTANTIATE(512)
