// blas.cu -- per-member vector kernels of the optimiser (see blas.cuh).
#include "blas.cuh"

namespace da {

__global__ void k_dot_partial(const double* const* __restrict__ A, const double* const* __restrict__ C,
                              double* __restrict__ part, size_t len) {
  const int b = blockIdx.y, chunk = blockIdx.x;
  const double* a = A[b];
  const double* c = C[b];
  __shared__ double red[256];
  double acc = 0.0;
  if (a && c) {
    const size_t lo = (size_t)chunk * kDotChunk;
    const size_t hi = lo + kDotChunk < len ? lo + kDotChunk : len;
    for (size_t i = lo + threadIdx.x; i < hi; i += blockDim.x) acc = fma(a[i], c[i], acc);
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[(size_t)b * gridDim.x + chunk] = red[0];
}

__global__ void k_dot_final(const double* __restrict__ part, double* __restrict__ out, int chunks) {
  const int b = blockIdx.x;
  __shared__ double red[256];
  double acc = 0.0;
  for (int i = threadIdx.x; i < chunks; i += blockDim.x) acc += part[(size_t)b * chunks + i];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[b] = red[0];
}

__global__ void k_axpby(const double* const* __restrict__ X, double* const* __restrict__ Y,
                        const double* __restrict__ alpha, const double* __restrict__ beta, size_t len) {
  const int b = blockIdx.y;
  const double* x = X[b];
  double* y = Y[b];
  if (!x || !y) return;
  const double al = alpha[b], be = beta[b];
  const size_t lo = (size_t)blockIdx.x * 1024;
  for (size_t i = lo + threadIdx.x; i < lo + 1024 && i < len; i += blockDim.x) y[i] = fma(al, x[i], be * y[i]);
}

}  // namespace da
