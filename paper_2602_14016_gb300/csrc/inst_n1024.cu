// Kernels and launchers for n = 1024.
#include "ops_impl.cuh"
DA_INSTANTIATE(1024)
