// blas.cuh -- per-member vector kernels of the optimiser.  Every member of a
// batch has its own vectors, addressed through device arrays of B pointers
// (a NULL pointer skips that member).  Reductions run in a fixed order, so
// dot products are bitwise reproducible.
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>

namespace da {

constexpr int kDotChunk = 8192;
inline int dot_chunks(size_t len) { return (int)((len + kDotChunk - 1) / kDotChunk); }

// part[b][chunk] = sum over the chunk of a_b[i] * c_b[i].  grid (chunks, B), block 256.
__global__ void k_dot_partial(const double* const* __restrict__ A, const double* const* __restrict__ C,
                              double* __restrict__ part, size_t len);
// out[b] = sum over chunks of part[b][chunk], in chunk order.  grid B, block 256.
__global__ void k_dot_final(const double* __restrict__ part, double* __restrict__ out, int chunks);
// y_b = alpha_b x_b + beta_b y_b.  grid (ceil(len/1024), B), block 256.
__global__ void k_axpby(const double* const* __restrict__ X, double* const* __restrict__ Y,
                        const double* __restrict__ alpha, const double* __restrict__ beta, size_t len);

}  // namespace da
