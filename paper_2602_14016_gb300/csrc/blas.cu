// blas.cu -- per-member vector kernels of the optimiser (see blas.cuh).
#include "blas.cuh"

namespace da {

namespace {

__device__ __forceinline__ double* bank(const LbfgsArgs& a, int k, int b) {
  return a.V + ((size_t)k * a.B + b) * a.len;
}

// Sum of v over the CTA in a fixed tree order; every thread gets the result.
__device__ double block_sum(double v, double* red) {
  red[threadIdx.x] = v;
  __syncthreads();
#pragma unroll 1
  for (int s = kBlasThreads / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  const double r = red[0];
  __syncthreads();  // red is reused by the next reduction
  return r;
}

__device__ double block_dot(const double* __restrict__ x, const double* __restrict__ y, size_t len, double* red) {
  double acc = 0.0;
  for (size_t i = threadIdx.x; i < len; i += kBlasThreads) acc = fma(x[i], y[i], acc);
  return block_sum(acc, red);
}

constexpr int kChunk = 4096;  // elements per CTA of the element-wise kernels

}  // namespace

__global__ void __launch_bounds__(kBlasThreads) k_two_loop(LbfgsArgs a) {
  const int b = blockIdx.x;
  if (!a.mask[b]) return;
  __shared__ double red[kBlasThreads];
  __shared__ double alpha[64];
  const size_t len = a.len;
  const double* g = bank(a, BANK_G, b);
  double* d = bank(a, BANK_D, b);
  const int h = a.cnt[b];
  const int* ps = a.pslot + (size_t)b * a.mem;
  const double* rho = a.prho + (size_t)b * a.mem;
  // d carries -q: q = g, then q -= alpha_j y_j from the newest pair back
  for (size_t i = threadIdx.x; i < len; i += kBlasThreads) d[i] = -g[i];
  for (int j = h - 1; j >= 0; --j) {
    const double* s = bank(a, BANK_S0 + ps[j], b);
    const double* y = bank(a, BANK_S0 + a.slots + ps[j], b);
    const double al = -rho[j] * block_dot(s, d, len, red);  // rho s.q
    if (threadIdx.x == 0) alpha[j] = al;
    for (size_t i = threadIdx.x; i < len; i += kBlasThreads) d[i] = fma(al, y[i], d[i]);
  }
  if (h > 0) {  // H0 = (s.y / y.y) I from the newest pair
    const double* y = bank(a, BANK_S0 + a.slots + ps[h - 1], b);
    const double gam = 1.0 / (rho[h - 1] * block_dot(y, y, len, red));
    for (size_t i = threadIdx.x; i < len; i += kBlasThreads) d[i] *= gam;
  }
  __syncthreads();  // alpha[] written by thread 0
  for (int j = 0; j < h; ++j) {  // r += (alpha_j - beta_j) s_j, oldest first
    const double* s = bank(a, BANK_S0 + ps[j], b);
    const double* y = bank(a, BANK_S0 + a.slots + ps[j], b);
    const double coef = -(alpha[j] + rho[j] * block_dot(y, d, len, red));
    for (size_t i = threadIdx.x; i < len; i += kBlasThreads) d[i] = fma(coef, s[i], d[i]);
  }
  const double gd = block_dot(g, d, len, red);
  if (threadIdx.x == 0) a.scal[(size_t)b * SC_COUNT + SC_GD] = gd;
}

__global__ void k_neg_grad(LbfgsArgs a) {
  const int b = blockIdx.y;
  if (!a.mask[b]) return;
  const double* g = bank(a, BANK_G, b);
  double* d = bank(a, BANK_D, b);
  const size_t lo = (size_t)blockIdx.x * kChunk;
  for (size_t i = lo + threadIdx.x; i < lo + kChunk && i < a.len; i += blockDim.x) d[i] = -g[i];
}

__global__ void k_trial(LbfgsArgs a) {
  const int b = blockIdx.y;
  const double* x = bank(a, BANK_X, b);
  const double* d = bank(a, BANK_D, b);
  double* xt = bank(a, BANK_XT, b);
  const bool on = a.mask[b] != 0;
  const double st = on ? a.stp[b] : 0.0;
  const size_t lo = (size_t)blockIdx.x * kChunk;
  for (size_t i = lo + threadIdx.x; i < lo + kChunk && i < a.len; i += blockDim.x)
    xt[i] = on ? fma(st, d[i], x[i]) : x[i];
}

__global__ void __launch_bounds__(kBlasThreads) k_dot_gt_d(LbfgsArgs a) {
  const int b = blockIdx.x;
  if (!a.mask[b]) return;
  __shared__ double red[kBlasThreads];
  const double r = block_dot(bank(a, BANK_GT, b), bank(a, BANK_D, b), a.len, red);
  if (threadIdx.x == 0) a.scal[(size_t)b * SC_COUNT + SC_DG] = r;
}

__global__ void __launch_bounds__(kBlasThreads) k_accept(LbfgsArgs a) {
  const int b = blockIdx.x;
  if (!a.mask[b]) return;
  __shared__ double red[kBlasThreads];
  double* x = bank(a, BANK_X, b);
  double* g = bank(a, BANK_G, b);
  const double* xt = bank(a, BANK_XT, b);
  const double* gt = bank(a, BANK_GT, b);
  double* s = bank(a, BANK_S0 + a.aslot[b], b);
  double* y = bank(a, BANK_S0 + a.slots + a.aslot[b], b);
  double sy = 0.0, yy = 0.0;
  for (size_t i = threadIdx.x; i < a.len; i += kBlasThreads) {
    const double si = xt[i] - x[i], yi = gt[i] - g[i];
    s[i] = si;
    y[i] = yi;
    sy = fma(si, yi, sy);
    yy = fma(yi, yi, yy);
    x[i] = xt[i];
    g[i] = gt[i];
  }
  sy = block_sum(sy, red);
  yy = block_sum(yy, red);
  if (threadIdx.x == 0) {
    a.scal[(size_t)b * SC_COUNT + SC_SY] = sy;
    a.scal[(size_t)b * SC_COUNT + SC_YY] = yy;
  }
}

__global__ void __launch_bounds__(kBlasThreads) k_gnorm2(LbfgsArgs a) {
  const int b = blockIdx.x;
  __shared__ double red[kBlasThreads];
  const double* g = bank(a, BANK_G, b);
  const double r = block_dot(g, g, a.len, red);
  if (threadIdx.x == 0) a.scal[(size_t)b * SC_COUNT + SC_GG] = r;
}

__global__ void k_take_gradient(LbfgsArgs a) {
  const int b = blockIdx.y;
  if (!a.mask[b]) return;
  const double* gt = bank(a, BANK_GT, b);
  double* g = bank(a, BANK_G, b);
  const size_t lo = (size_t)blockIdx.x * kChunk;
  for (size_t i = lo + threadIdx.x; i < lo + kChunk && i < a.len; i += blockDim.x) g[i] = gt[i];
}

}  // namespace da
