// fp64_probe.cu -- FP64 pipe throughput probe (da_fp64_probe of
// include/da.h): the measurement behind the roofline denominator of the pass
// kernels, which are bound by FP64 arithmetic rather than by HBM.
//
// Every thread runs 8 independent dependency chains of one FP64 operation
// for `iters` x 4 rounds; 4 CTAs of 256 threads per SM keep 32 warps per SM
// in flight, so the chains' latency is hidden and the pipe's issue rate
// shows.  Kinds: 0 DFMA with a register multiplicand and a constant addend,
// 1 DFMA with three register operands, 2 DADD, 3 DMUL.  Thread 0 of CTA 0
// reads clock64 and %globaltimer around its loop, which gives the SM clock
// the probe ran at.
#include <cuda_runtime.h>

#include <string>

#include "../../include/da.h"

namespace da {
namespace probe {

constexpr int kThreads = 256, kCtasPerSm = 4, kChains = 8, kUnroll = 4;

__device__ __forceinline__ unsigned long long globaltimer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

template <int KIND>
__global__ void __launch_bounds__(kThreads) k_probe(double* out, int iters, double x0, double y0,
                                                    unsigned long long* clk) {
  double a[kChains];
  const double x = x0 + 1e-12 * threadIdx.x, y = y0 - 1e-12 * blockIdx.x;
#pragma unroll
  for (int i = 0; i < kChains; ++i) a[i] = 1.0 + 1e-3 * i + 1e-9 * threadIdx.x;
  const long long c0 = clock64();
  const unsigned long long g0 = globaltimer_ns();
#pragma unroll 1
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
#pragma unroll
      for (int i = 0; i < kChains; ++i) {
        if constexpr (KIND == 0) a[i] = fma(a[i], x, 0.5);
        if constexpr (KIND == 1) a[i] = fma(a[i], x, y);
        if constexpr (KIND == 2) a[i] = a[i] + x;
        if constexpr (KIND == 3) a[i] = a[i] * x;
      }
    }
  }
  const long long c1 = clock64();
  const unsigned long long g1 = globaltimer_ns();
  double s = 0.0;
#pragma unroll
  for (int i = 0; i < kChains; ++i) s += a[i];
  out[(size_t)blockIdx.x * kThreads + threadIdx.x] = s;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    clk[0] = (unsigned long long)(c1 - c0);
    clk[1] = g1 - g0;
  }
}

}  // namespace probe
}  // namespace da

extern "C" da_status da_fp64_probe(int kind, int iters, double* gflops, double* ops_per_clk_per_sm, double* sm_mhz,
                                   void* stream) {
  using namespace da::probe;
  if (kind < 0 || kind > 3 || iters < 1 || !gflops) return DA_EINVAL;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return DA_ECUDA;
  const int ctas = sms * kCtasPerSm;
  cudaStream_t st = (cudaStream_t)stream;
  double* out = nullptr;
  unsigned long long* clk = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  da_status r = DA_OK;
  if (cudaMalloc(&out, (size_t)ctas * kThreads * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&clk, 2 * sizeof(unsigned long long)) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
      cudaEventCreate(&e1) != cudaSuccess) {
    r = DA_ENOMEM;
  } else {
    auto launch = [&](int n_it) {
      switch (kind) {
        case 0: k_probe<0><<<ctas, kThreads, 0, st>>>(out, n_it, 0.999999999, 0.25, clk); break;
        case 1: k_probe<1><<<ctas, kThreads, 0, st>>>(out, n_it, 0.999999999, 0.25, clk); break;
        case 2: k_probe<2><<<ctas, kThreads, 0, st>>>(out, n_it, 1e-9, 0.25, clk); break;
        default: k_probe<3><<<ctas, kThreads, 0, st>>>(out, n_it, 0.999999999, 0.25, clk); break;
      }
    };
    launch(iters / 10 + 1);  // warm-up: clocks up, module loaded
    cudaEventRecord(e0, st);
    launch(iters);
    cudaEventRecord(e1, st);
    unsigned long long hclk[2] = {0, 0};
    float ms = 0.f;
    if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess ||
        cudaMemcpy(hclk, clk, sizeof(hclk), cudaMemcpyDeviceToHost) != cudaSuccess) {
      r = DA_ECUDA;
    } else {
      const double ops = (double)ctas * kThreads * iters * kUnroll * kChains;
      const double flop_per_op = kind <= 1 ? 2.0 : 1.0;
      *gflops = ops * flop_per_op / (ms * 1e-3) / 1e9;
      const double mhz = hclk[1] ? (double)hclk[0] / (double)hclk[1] * 1e3 : 0.0;
      if (sm_mhz) *sm_mhz = mhz;
      if (ops_per_clk_per_sm) *ops_per_clk_per_sm = mhz > 0 ? ops / (ms * 1e-3) / (mhz * 1e6) / sms : 0.0;
    }
  }
  if (out) cudaFree(out);
  if (clk) cudaFree(clk);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (r != DA_OK) cudaGetLastError();
  return r;
}
