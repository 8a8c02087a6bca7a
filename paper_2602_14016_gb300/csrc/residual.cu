// residual.cu -- observation residual and cost of each member.
#include "kernels.cuh"

namespace da {

// r = model observations - data and J = 1/2 sum r^2 per member, in a fixed
// order (deterministic).  grid B, block 256.
__global__ void k_residual(Dev d) {
  const int bm = blockIdx.x;
  const int cnt = d.ragged ? d.mnt[bm] * d.mpx[bm] * d.mpx[bm] * 2 : d.nt * d.px * d.px * 2;
  const double* o = d.obs + bm * d.obs_stride;
  const double* m = d.mobs + bm * d.obs_stride;
  double* r = d.res + bm * d.obs_stride;
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

__global__ void k_sobolev_cost(double* J, const double2* w0, double lambda, int N, int Kr, int Kc) {
  const int bm = blockIdx.x;
  const double2* w = w0 + (size_t)bm * Kr * Kc;
  double acc = 0.0;
  for (int i = threadIdx.x; i < Kr * Kc; i += blockDim.x) {
    const double wt = i < Kr ? 1.0 : 2.0;  // column-major: i < Kr is kx = 0; kx > 0 stands for +-kx
    acc = fma(wt, w[i].x * w[i].x + w[i].y * w[i].y, acc);
  }
  __shared__ double red[256];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) J[bm] += 0.5 * lambda * red[0] / ((double)N * N);
}

__global__ void k_sobolev_grad(double2* lam, const double2* w0, double lambda, int count) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x)
    lam[i] = make_double2(fma(lambda, w0[i].x, lam[i].x), fma(lambda, w0[i].y, lam[i].y));
}

// Shell energies of the adjoint velocity u_dagger = (d lambda/dy, -d lambda/dx)
// from the compact DFT of lambda: for shell k (k <= |k| < k+1),
// E(k) = 1/2 sum_{modes} |u_dagger_hat|^2 with normalised coefficients, i.e.
// sum of wgt[m] |lambda_hat(m)|^2, wgt = (1 or 2) k^2 / (2 N^4) precomputed.
// Modes of shell s are mode[off[s]..off[s+1]).  grid (nshell, B), block 128.
__global__ void k_shell_member(const double2* lam, const int* off, const int* mode, const double* wgt, int nmodes,
                               double* out, int nshell) {
  const int sh = blockIdx.x, bm = blockIdx.y;
  const double2* l = lam + (size_t)bm * nmodes;
  double acc = 0.0;
  for (int i = off[sh] + threadIdx.x; i < off[sh + 1]; i += blockDim.x) {
    const double2 v = l[mode[i]];
    acc = fma(wgt[i], v.x * v.x + v.y * v.y, acc);
  }
  __shared__ double red[128];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[(size_t)bm * nshell + sh] = red[0];
}

// Shell energy of the ensemble-mean adjoint (members averaged in index
// order).  grid nshell, block 128.
__global__ void k_shell_mean(const double2* lam, int B, const int* off, const int* mode, const double* wgt, int nmodes,
                             double* out) {
  const int sh = blockIdx.x;
  double acc = 0.0;
  for (int i = off[sh] + threadIdx.x; i < off[sh + 1]; i += blockDim.x) {
    double mx = 0.0, my = 0.0;
    for (int b = 0; b < B; ++b) {
      const double2 v = lam[(size_t)b * nmodes + mode[i]];
      mx += v.x;
      my += v.y;
    }
    mx /= B;
    my /= B;
    acc = fma(wgt[i], mx * mx + my * my, acc);
  }
  __shared__ double red[128];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[sh] = red[0];
}

}  // namespace da
