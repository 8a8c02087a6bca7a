// static_ctrl.cu -- control map s -> w0_hat for callers that cannot allocate
// device memory.
//
// It computes what da_omega_from_control computes for one member, without a
// context: the intermediate rows (the transform along x of s) live in a
// file-scope static device array instead of a context buffer, the FFT
// twiddles in a second one, and the multiplier |k| W(k)^{1/2} is evaluated
// in the kernel.  Every GPU that loads the library holds both arrays
// (about 356 KB) until the process exits.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>

#include "../../include/da.h"
#include "kernels.cuh"

namespace da {
namespace st {

constexpr int kMaxN = 256;
constexpr int kMaxKc = (kMaxN - 1) / 3 + 1;

// Scratch shared by every call: mixed rows [y][kx], y < n, kx <= (n-1)/3.
static __device__ __align__(256) double2 g_rows[kMaxN * kMaxKc];
// exp(-2 pi i t / 256), t < 256; length n uses every (256/n)-th entry.
static __device__ __align__(256) double2 g_tw[kMaxN];

template <int N>
__device__ __forceinline__ void load_tw(double2* tw, const double2* __restrict__ g) {
  for (int i = threadIdx.x; i < N; i += blockDim.x) tw[i] = g[i * (kMaxN / N)];
}

// Real rows of s -> rows[y][kx], kx <= K, two rows per complex transform.
template <int N>
__global__ void __launch_bounds__(Geo<N>::THREADS) k_rows(const double* __restrict__ s, double2* __restrict__ rows,
                                                          const double2* __restrict__ tw256) {
  using G = Geo<N>;
  extern __shared__ double2 sm[];
  double2 *tw = sm, *a = tw + N;
  const int y0 = 2 * blockIdx.x;
  load_tw<N>(tw, tw256);
  const double* r0 = s + (size_t)y0 * N;
  for (int x = threadIdx.x; x < N; x += blockDim.x) a[x] = make_double2(r0[x], r0[N + x]);
  __syncthreads();
  fft_batch<N, -1, 1>(a, tw);
  double2* M = rows + (size_t)y0 * G::Kc;
  for (int kx = threadIdx.x; kx < G::Kc; kx += blockDim.x) {
    double2 A, Bv;
    unpack_pair<N>(a, kx, A, Bv);
    M[kx] = A;
    M[G::Kc + kx] = Bv;
  }
}

// Column kx of the half spectrum: transform of rows[.][kx] along y times
// |k| W^{1/2} on the retained set, zero elsewhere.  grid N/2+1 columns.
template <int N>
__global__ void __launch_bounds__(Geo<N>::THREADS) k_cols(const double2* __restrict__ rows,
                                                          const double2* __restrict__ tw256, int kind, double param,
                                                          double nu, double2* __restrict__ out) {
  using G = Geo<N>;
  extern __shared__ double2 sm[];
  double2 *tw = sm, *a = tw + N;
  const int kx = blockIdx.x;
  if (kx > G::K) {  // outside the retained set: zero column
    for (int q = threadIdx.x; q < N; q += blockDim.x) out[(size_t)q * G::NH + kx] = make_double2(0.0, 0.0);
    return;
  }
  load_tw<N>(tw, tw256);
  for (int y = threadIdx.x; y < N; y += blockDim.x) a[y] = rows[(size_t)y * G::Kc + kx];
  __syncthreads();
  fft_batch<N, -1, 1>(a, tw);
  const double2* r = a;
  for (int q = threadIdx.x; q < N; q += blockDim.x) {
    const int ky = q < N / 2 ? q : q - N;
    double2 v = make_double2(0.0, 0.0);
    if (ky >= -G::K && ky <= G::K && !(kx == 0 && ky == 0)) {
      const double k2 = (double)(kx * kx + ky * ky);
      const double k = sqrt(k2);
      double W;
      if (kind == 0) W = 1.0;
      else if (kind == 1) W = exp(-param * k);
      else if (kind == 2) W = pow(k, -2.0 * param);
      else W = exp(-nu * param * k2);
      v = cscale(r[q], k * sqrt(W));
    }
    out[(size_t)q * G::NH + kx] = v;
  }
}

template <int N>
cudaError_t launch(const double* s, double* omega0, double2* rows, const double2* tw, int kind, double param,
                   double nu, cudaStream_t stream) {
  using G = Geo<N>;
  cudaError_t e = cudaFuncSetAttribute((const void*)k_rows<N>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)G::SMEM);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute((const void*)k_cols<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)G::SMEM);
  if (e != cudaSuccess) return e;
  k_rows<N><<<N / 2, G::THREADS, G::SMEM, stream>>>(s, rows, tw);
  k_cols<N><<<G::NH, G::THREADS, G::SMEM, stream>>>(rows, tw, kind, param, nu, (double2*)omega0);
  return cudaGetLastError();
}

// Per-device set-up: device addresses of the two arrays and the twiddles.
// The states live in a fixed array that never moves, and a caller gets a
// copy taken under the lock, so concurrent first calls on different devices
// cannot invalidate each other's view.
constexpr int kMaxDevices = 64;
struct DeviceState {
  bool ready = false;
  double2* rows = nullptr;
  double2* tw = nullptr;
};
static std::mutex g_mu;
static DeviceState g_dev[kMaxDevices];

static cudaError_t setup_current_device(DeviceState* out, const char** msg) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) {
    *msg = "device ordinal beyond the 64 devices the static control map keeps state for";
    return cudaErrorInvalidDevice;
  }
  std::lock_guard<std::mutex> lock(g_mu);
  DeviceState& d = g_dev[dev];
  if (!d.ready) {
    DeviceState t;
    e = cudaGetSymbolAddress((void**)&t.rows, g_rows);
    if (e != cudaSuccess) return e;
    e = cudaGetSymbolAddress((void**)&t.tw, g_tw);
    if (e != cudaSuccess) return e;
    double2 host[kMaxN];
    const long double pi = 3.141592653589793238462643383279502884L;
    for (int i = 0; i < kMaxN; ++i) {
      const long double a = -2.0L * pi * (long double)i / (long double)kMaxN;
      host[i] = make_double2((double)cosl(a), (double)sinl(a));
    }
    e = cudaMemcpyToSymbol(g_tw, host, sizeof(host));
    if (e != cudaSuccess) return e;
    t.ready = true;
    d = t;
  }
  *out = d;
  return cudaSuccess;
}

// W(k) of kinds 1..3 is monotone in |k|, so it is finite and non-negative on
// the retained set (1 <= |k| <= sqrt(2) K) iff it is at both ends.
static bool kernel_finite_on_retained_set(int kind, double param, double nu, int n) {
  const double K = (double)((n - 1) / 3);
  const double ks[2] = {1.0, std::sqrt(2.0) * K};
  for (double k : ks) {
    double W = 1.0;
    if (kind == 1) W = std::exp(-param * k);
    else if (kind == 2) W = std::pow(k, -2.0 * param);
    else if (kind == 3) W = std::exp(-nu * param * k * k);
    const double m = k * std::sqrt(W);
    if (!std::isfinite(W) || !(W >= 0.0) || !std::isfinite(m)) return false;
  }
  return true;
}

}  // namespace st
}  // namespace da

extern "C" da_status da_omega_from_control_static(int n, double nu, const da_kernel* kernel, const double* s,
                                                  double* omega0, void* stream, const char** message) {
  const char* dummy;
  const char** msg = message ? message : &dummy;
  *msg = "";
  if (!kernel || !s || !omega0) {
    *msg = "kernel, s and omega0 must not be NULL";
    return DA_EINVAL;
  }
  if (n != 16 && n != 32 && n != 64 && n != 128 && n != 256) {
    *msg = "n must be a power of two in [16, 256]: the static scratch holds at most a 256 x 86 mixed field";
    return DA_EINVAL;
  }
  if (kernel->kind < DA_KERNEL_IDENTITY || kernel->kind > DA_KERNEL_EXP_SQ) {
    *msg = "kernel kind must be identity, exp_abs, frac or exp_sq (tables need device memory)";
    return DA_EINVAL;
  }
  if (!std::isfinite(kernel->param) || !(nu >= 0.0) || !std::isfinite(nu)) {
    *msg = "kernel parameter must be finite and nu >= 0";
    return DA_EINVAL;
  }
  if (!da::st::kernel_finite_on_retained_set(kernel->kind, kernel->param, nu, n)) {
    *msg = "kernel W is not finite and non-negative on the retained set";
    return DA_EINVAL;
  }
  da::st::DeviceState dst;
  const char* setup_msg = nullptr;
  cudaError_t e = da::st::setup_current_device(&dst, &setup_msg);
  if (e != cudaSuccess) {
    *msg = setup_msg ? setup_msg : cudaGetErrorString(e);
    return DA_ECUDA;
  }
  const da::st::DeviceState* d = &dst;
  cudaStream_t st = (cudaStream_t)stream;
  const int kind = kernel->kind;
  const double a = kernel->param;
  switch (n) {
    case 16: e = da::st::launch<16>(s, omega0, d->rows, d->tw, kind, a, nu, st); break;
    case 32: e = da::st::launch<32>(s, omega0, d->rows, d->tw, kind, a, nu, st); break;
    case 64: e = da::st::launch<64>(s, omega0, d->rows, d->tw, kind, a, nu, st); break;
    case 128: e = da::st::launch<128>(s, omega0, d->rows, d->tw, kind, a, nu, st); break;
    default: e = da::st::launch<256>(s, omega0, d->rows, d->tw, kind, a, nu, st); break;
  }
  if (e != cudaSuccess) {
    *msg = cudaGetErrorString(e);
    return DA_ECUDA;
  }
  return DA_OK;
}
