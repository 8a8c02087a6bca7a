// residual.cu -- observation residual and cost of each member.
#include "kernels.cuh"

namespace da {

// r = model observations - data and J = 1/2 sum r^2 per member, in a fixed
// order (deterministic).  grid B, block 256.
__global__ void k_residual(Dev d) {
  const int bm = blockIdx.x;
  const int cnt = d.nt * d.px * d.px * 2;
  const double* o = d.obs + (size_t)bm * cnt;
  const double* m = d.mobs + (size_t)bm * cnt;
  double* r = d.res + (size_t)bm * cnt;
  double acc = 0.0;
  for (int i = threadIdx.x; i < cnt; i += blockDim.x) {
    const double v = o[i] - m[i];
    r[i] = v;
    acc = fma(v, v, acc);
  }
  __shared__ double red[256];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) d.J[bm] = 0.5 * red[0];
}

}  // namespace da
