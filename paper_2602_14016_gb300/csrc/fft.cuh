// fft.cuh -- FP64 shared-memory FFT engine for the pass kernels.
//
// A CTA transforms a batch of F complex sequences of length N held in shared
// memory, with a mixed-radix Stockham auto-sort algorithm: stage s with
// radix R and current sub-length L loads the R points x[i + m N/R] of
// butterfly i, twiddles them by W_{LR}^{m (i mod L)}, applies an R-point DFT
// in registers and stores them to y[(i - i mod L) R + i mod L + m L].  After
// the last stage (L = N) the output is in natural order.  Stages work in
// place: every thread holds its butterfly in registers across a barrier, so
// one buffer of F sequences suffices.  Twiddles come from a per-N table of
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

// cos(pi/4), cos(pi/8), tan(pi/8)
constexpr double kR2 = 0.70710678118654752440;
constexpr double kC8 = 0.92387953251128675613;
constexpr double kT8 = 0.41421356237309504880;

// Output pair of a radix-2 combination with a scaled twiddle:
// e +- c z, as two FMAs per component.
__device__ __forceinline__ void bfly_scaled(const double2 e, const double2 z, double c, double2& plus, double2& minus) {
  plus = make_double2(fma(c, z.x, e.x), fma(c, z.y, e.y));
  minus = make_double2(fma(-c, z.x, e.x), fma(-c, z.y, e.y));
}

// Every twiddle w = exp(S i theta) of the internal combinations is written as
// c (1 + i t) (or c (t + i)) with a constant tangent t, so that w o = c z
// with z two FMAs (or two adds when t = 1), and e +- w o = e +- c z costs
// four FMAs: six FP64 instructions instead of eight.
template <int S>
__device__ __forceinline__ void dft8(double2* a) {
  double2 e[4] = {a[0], a[2], a[4], a[6]};
  double2 o[4] = {a[1], a[3], a[5], a[7]};
  dft4<S>(e);
  dft4<S>(o);
  // k = 0
  a[0] = cadd(e[0], o[0]);
  a[4] = csub(e[0], o[0]);
  // k = 2: w = S i
  const double2 o2 = mul_si<S>(o[2]);
  a[2] = cadd(e[2], o2);
  a[6] = csub(e[2], o2);
  // k = 1: w = (1 + S i)/sqrt2
  const double2 z1 = make_double2(o[1].x - S * o[1].y, o[1].y + S * o[1].x);
  bfly_scaled(e[1], z1, kR2, a[1], a[5]);
  // k = 3: w = (-1 + S i)/sqrt2 = -(1 - S i)/sqrt2
  const double2 z3 = make_double2(o[3].x + S * o[3].y, o[3].y - S * o[3].x);
  bfly_scaled(e[3], z3, -kR2, a[3], a[7]);
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
  // k = 0 and k = 4 (w = S i)
  a[0] = cadd(e[0], o[0]);
  a[8] = csub(e[0], o[0]);
  const double2 o4 = mul_si<S>(o[4]);
  a[4] = cadd(e[4], o4);
  a[12] = csub(e[4], o4);
  // k = 2, 6: w = (+-1 + S i)/sqrt2
  const double2 z2 = make_double2(o[2].x - S * o[2].y, o[2].y + S * o[2].x);
  bfly_scaled(e[2], z2, kR2, a[2], a[10]);
  const double2 z6 = make_double2(o[6].x + S * o[6].y, o[6].y - S * o[6].x);
  bfly_scaled(e[6], z6, -kR2, a[6], a[14]);
  // k = 1, 3, 5, 7: w = cos(k pi/8) + S i sin(k pi/8) = c z with c = cos(pi/8)
  // and z formed with t = tan(pi/8)
  const double2 z1 = make_double2(fma(-S * kT8, o[1].y, o[1].x), fma(S * kT8, o[1].x, o[1].y));
  bfly_scaled(e[1], z1, kC8, a[1], a[9]);
  const double2 z3 = make_double2(fma(kT8, o[3].x, -S * o[3].y), fma(kT8, o[3].y, S * o[3].x));
  bfly_scaled(e[3], z3, kC8, a[3], a[11]);
  const double2 z5 = make_double2(fma(-kT8, o[5].x, -S * o[5].y), fma(-kT8, o[5].y, S * o[5].x));
  bfly_scaled(e[5], z5, kC8, a[5], a[13]);
  const double2 z7 = make_double2(fma(-S * kT8, o[7].y, -o[7].x), fma(S * kT8, o[7].x, -o[7].y));
  bfly_scaled(e[7], z7, kC8, a[7], a[15]);
}

template <int R, int S>
__device__ __forceinline__ void dftR(double2* a) {
  if constexpr (R == 2) dft2<S>(a);
  if constexpr (R == 4) dft4<S>(a);
  if constexpr (R == 8) dft8<S>(a);
  if constexpr (R == 16) dft16<S>(a);
}

// Radix plans: a list of stage radices whose product is N.
template <int... Rs>
struct Radices {};

// Plan for two concurrent transforms (the pass kernels) and for a single
// transform (control and gradient maps), with the CTA width they run on.
// Wide radices keep the FP64 instruction count low; the width is chosen so
// that the stages of the two-transform plan fill whole warps (a stage with
// more butterflies than threads gives each thread several).
template <int N> struct Plan;
template <> struct Plan<16> { using two = Radices<4, 4>; using one = Radices<4, 4>; static constexpr int threads = 32; };
template <> struct Plan<32> { using two = Radices<4, 8>; using one = Radices<4, 8>; static constexpr int threads = 32; };
template <> struct Plan<64> { using two = Radices<4, 4, 4>; using one = Radices<4, 4, 4>; static constexpr int threads = 32; };
template <> struct Plan<128> { using two = Radices<4, 4, 8>; using one = Radices<4, 4, 8>; static constexpr int threads = 64; };
template <> struct Plan<256> { using two = Radices<8, 8, 4>; using one = Radices<8, 8, 4>; static constexpr int threads = 64; };
template <> struct Plan<512> { using two = Radices<8, 8, 8>; using one = Radices<8, 8, 8>; static constexpr int threads = 128; };
template <> struct Plan<1024> { using two = Radices<16, 8, 8>; using one = Radices<16, 8, 8>; static constexpr int threads = 256; };

template <int N>
struct PlanInfo {
  static constexpr int THREADS = Plan<N>::threads;
};

// One in-place Stockham stage on F sequences of N points stored back to back
// in `buf`: every thread loads the R points of each of its butterflies,
// twiddles and transforms them in registers, waits for all loads, then
// stores.
template <int N, int R, int S, int F>
__device__ __forceinline__ void stockham_stage(double2* buf, int L, const double2* __restrict__ tw) {
  constexpr int NB = N / R, T = PlanInfo<N>::THREADS, TOT = F * NB, J = (TOT + T - 1) / T;
  double2 a[J][R];
  int base[J], dst[J];
#pragma unroll
  for (int jb = 0; jb < J; ++jb) {
    const int u = threadIdx.x + jb * T;
    base[jb] = 0;
    dst[jb] = 0;
    if (TOT % T == 0 || u < TOT) {
      const int f = u / NB;
      const int i = u - f * NB;
      const int k = i & (L - 1);
      base[jb] = f * N;
#pragma unroll
      for (int m = 0; m < R; ++m) a[jb][m] = buf[base[jb] + i + m * NB];
      if (L > 1) {
        const int step = N / (L * R);
#pragma unroll
        for (int m = 1; m < R; ++m) {
          double2 w = tw[m * k * step];
          if (S > 0) w.y = -w.y;
          a[jb][m] = cmul(a[jb][m], w);
        }
      }
      dftR<R, S>(a[jb]);
      dst[jb] = (i - k) * R + k;
    }
  }
  __syncthreads();
#pragma unroll
  for (int jb = 0; jb < J; ++jb) {
    const int u = threadIdx.x + jb * T;
    if (TOT % T == 0 || u < TOT) {
#pragma unroll
      for (int m = 0; m < R; ++m) buf[base[jb] + dst[jb] + m * L] = a[jb][m];
    }
  }
  __syncthreads();
}

template <int N, int S, int F, int L>
__device__ __forceinline__ void run_stages(double2*, const double2*, Radices<>) {}

template <int N, int S, int F, int L, int R, int... Rs>
__device__ __forceinline__ void run_stages(double2* buf, const double2* tw, Radices<R, Rs...>) {
  stockham_stage<N, R, S, F>(buf, L, tw);
  run_stages<N, S, F, L * R>(buf, tw, Radices<Rs...>{});
}

// Transform, in place, F (1 or 2) sequences of N points stored back to back
// in buf.  Called by every thread of a CTA of PlanInfo<N>::THREADS threads,
// with buf already synchronised; returns after a final __syncthreads().
template <int N, int S, int F>
__device__ __forceinline__ void fft_batch(double2* buf, const double2* tw) {
  static_assert(F == 1 || F == 2, "batches of one or two transforms");
  if constexpr (F == 1)
    run_stages<N, S, F, 1>(buf, tw, typename Plan<N>::one{});
  else
    run_stages<N, S, F, 1>(buf, tw, typename Plan<N>::two{});
}

}  // namespace da
