// fft.cuh -- FP64 shared-memory FFT engine for the pass kernels.
//
// A CTA transforms a batch of F complex sequences of length N held in shared
// memory, with a mixed-radix Stockham auto-sort algorithm: stage s with
// radix R and current sub-length L loads the R points x[i + m N/R] of
// butterfly i, twiddles them by W_{LR}^{m (i mod L)}, applies an R-point DFT
// in registers and stores them to y[(i - i mod L) R + i mod L + m L].  After
// the last stage (L = N) the output is in natural order.  Stages ping-pong
// between two buffers.  Twiddles come from a per-N table of
// W_N^t = exp(-2 pi i t / N) in shared memory; the inverse sign uses the
// conjugate.  The R-point DFTs (R = 4, 8, 16) are written out by even/odd
// splitting so that multiplications by +-i and +-1 cost nothing.
//
// GB300's FP64 pipe is the bottleneck of every kernel here (about 2 DFMA per
// clock per SM), so the engine counts FP64 instructions: complex products
// use two FMAs and two multiplies, twiddles are loaded rather than computed.
#pragma once
#include <cuda_runtime.h>

namespace da {

__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ double2 conjd(double2 a) { return make_double2(a.x, -a.y); }
__device__ __forceinline__ double2 cscale(double2 a, double s) { return make_double2(a.x * s, a.y * s); }

// (S i) * a, S = +-1
template <int S>
__device__ __forceinline__ double2 mul_si(double2 a) {
  return S > 0 ? make_double2(-a.y, a.x) : make_double2(a.y, -a.x);
}

// X_k = sum_m a_m exp(S 2 pi i m k / R), in place, natural order.
template <int S>
__device__ __forceinline__ void dft4(double2* a) {
  const double2 t0 = cadd(a[0], a[2]), t1 = csub(a[0], a[2]);
  const double2 t2 = cadd(a[1], a[3]), t3 = mul_si<S>(csub(a[1], a[3]));
  a[0] = cadd(t0, t2);
  a[2] = csub(t0, t2);
  a[1] = cadd(t1, t3);
  a[3] = csub(t1, t3);
}

template <int S>
__device__ __forceinline__ void dft2(double2* a) {
  const double2 t = a[0];
  a[0] = cadd(t, a[1]);
  a[1] = csub(t, a[1]);
}

// cos(pi/4), cos(pi/8), sin(pi/8)
constexpr double kR2 = 0.70710678118654752440;
constexpr double kC8 = 0.92387953251128675613;
constexpr double kS8 = 0.38268343236508977173;

template <int S>
__device__ __forceinline__ void dft8(double2* a) {
  double2 e[4] = {a[0], a[2], a[4], a[6]};
  double2 o[4] = {a[1], a[3], a[5], a[7]};
  dft4<S>(e);
  dft4<S>(o);
  // o_k *= exp(S i pi k / 4)
  o[1] = make_double2((o[1].x - S * o[1].y) * kR2, (o[1].y + S * o[1].x) * kR2);
  o[2] = mul_si<S>(o[2]);
  o[3] = make_double2((-o[3].x - S * o[3].y) * kR2, (-o[3].y + S * o[3].x) * kR2);
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    a[k] = cadd(e[k], o[k]);
    a[k + 4] = csub(e[k], o[k]);
  }
}

template <int S>
__device__ __forceinline__ void dft16(double2* a) {
  double2 e[8], o[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    e[k] = a[2 * k];
    o[k] = a[2 * k + 1];
  }
  dft8<S>(e);
  dft8<S>(o);
  // o_k *= exp(S i pi k / 8)
  o[1] = cmul(o[1], make_double2(kC8, S * kS8));
  o[2] = make_double2((o[2].x - S * o[2].y) * kR2, (o[2].y + S * o[2].x) * kR2);
  o[3] = cmul(o[3], make_double2(kS8, S * kC8));
  o[4] = mul_si<S>(o[4]);
  o[5] = cmul(o[5], make_double2(-kS8, S * kC8));
  o[6] = make_double2((-o[6].x - S * o[6].y) * kR2, (-o[6].y + S * o[6].x) * kR2);
  o[7] = cmul(o[7], make_double2(-kC8, S * kS8));
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    a[k] = cadd(e[k], o[k]);
    a[k + 8] = csub(e[k], o[k]);
  }
}

template <int R, int S>
__device__ __forceinline__ void dftR(double2* a) {
  if constexpr (R == 2) dft2<S>(a);
  if constexpr (R == 4) dft4<S>(a);
  if constexpr (R == 8) dft8<S>(a);
  if constexpr (R == 16) dft16<S>(a);
}

// Radix plan per length: R1 x R2 (x R3).
template <int N> struct Plan;
template <> struct Plan<16> { static constexpr int R1 = 4, R2 = 4, R3 = 1; };
template <> struct Plan<32> { static constexpr int R1 = 4, R2 = 8, R3 = 1; };
template <> struct Plan<64> { static constexpr int R1 = 8, R2 = 8, R3 = 1; };
template <> struct Plan<128> { static constexpr int R1 = 8, R2 = 16, R3 = 1; };
template <> struct Plan<256> { static constexpr int R1 = 16, R2 = 16, R3 = 1; };
template <> struct Plan<512> { static constexpr int R1 = 8, R2 = 8, R3 = 8; };
template <> struct Plan<1024> { static constexpr int R1 = 16, R2 = 8, R3 = 8; };

// One Stockham stage on F sequences (leading dimension ld) by all CTA threads.
template <int N, int R, int S>
__device__ __forceinline__ void stockham_stage(const double2* __restrict__ src, double2* __restrict__ dst, int F,
                                               int ld, int L, const double2* __restrict__ tw) {
  constexpr int NB = N / R;
  const int step = N / (L * R);
  for (int u = threadIdx.x; u < F * NB; u += blockDim.x) {
    const int f = u / NB;
    const int i = u - f * NB;
    const int k = i & (L - 1);
    const double2* s = src + f * ld;
    double2* d = dst + f * ld;
    double2 a[R];
#pragma unroll
    for (int m = 0; m < R; ++m) a[m] = s[i + m * NB];
    if (L > 1) {
#pragma unroll
      for (int m = 1; m < R; ++m) {
        double2 w = tw[m * k * step];
        if (S > 0) w.y = -w.y;
        a[m] = cmul(a[m], w);
      }
    }
    dftR<R, S>(a);
    const int j = (i - k) * R + k;
#pragma unroll
    for (int m = 0; m < R; ++m) d[j + m * L] = a[m];
  }
}

// Transform F sequences in `a` (each N points, leading dimension ld); `b` is
// scratch of the same shape.  Returns the buffer that holds the result.
// Must be called by every thread of the CTA with `a` already synchronised;
// returns after a final __syncthreads().
template <int N, int S>
__device__ __forceinline__ double2* fft_batch(double2* a, double2* b, int F, int ld, const double2* tw) {
  using P = Plan<N>;
  stockham_stage<N, P::R1, S>(a, b, F, ld, 1, tw);
  __syncthreads();
  stockham_stage<N, P::R2, S>(b, a, F, ld, P::R1, tw);
  __syncthreads();
  if constexpr (P::R3 > 1) {
    stockham_stage<N, P::R3, S>(a, b, F, ld, P::R1 * P::R2, tw);
    __syncthreads();
    return b;
  } else {
    return a;
  }
}

}  // namespace da
