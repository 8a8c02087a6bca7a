// fft.cuh -- FP64 shared-memory FFT engine for the pass kernels.
//
// A CTA transforms a batch of F complex sequences of length N held in shared
// memory, with a mixed-radix Stockham auto-sort algorithm: stage s with
// radix R and current sub-length L loads the R points x[i + m N/R] of
// butterfly i, twiddles them by W_{LR}^{m (i mod L)}, applies an R-point DFT
// in registers and stores them to y[(i - i mod L) R + i mod L + m L].  After
// the last stage (L = N) the output is in natural order.  Stages work in
// place: every thread holds its butterfly in registers across a barrier, so
// one buffer of F sequences suffices.  The R-point DFTs (R = 4, 8, 16) are
// written out by even/odd splitting so that multiplications by +-i and +-1
// cost nothing.
//
// GB300's FP64 pipe is the bottleneck of every kernel here (about 1.6 FP64
// instructions per clock per SM for this mix), so the engine counts FP64
// instructions.  The pass kernels use fft_folded: the twiddles' cosines are
// folded into the butterflies' FMAs (see "Folded twiddles" below), from a
// per-N table in shared memory.  fft_batch, with a plain table of
// W_N^t = exp(-2 pi i t / N) (conjugated for the inverse sign), serves the
// allocation-free control map, whose scratch is static.
#pragma once
#include <cuda_runtime.h>

#include <cmath>

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

// x + y and x - y where ZX, ZY mark an operand known to be zero: a first-stage
// input in the gap of a band-limited sequence, whose load was skipped (its
// register holds nothing).  A known zero costs no FP64 instruction.
template <bool ZX, bool ZY>
__device__ __forceinline__ double2 add_z(double2 x, double2 y) {
  if constexpr (ZX && ZY) return make_double2(0.0, 0.0);
  else if constexpr (ZY) return x;
  else if constexpr (ZX) return y;
  else return cadd(x, y);
}
template <bool ZX, bool ZY>
__device__ __forceinline__ double2 sub_z(double2 x, double2 y) {
  if constexpr (ZX && ZY) return make_double2(0.0, 0.0);
  else if constexpr (ZY) return x;
  else if constexpr (ZX) return make_double2(-y.x, -y.y);
  else return csub(x, y);
}

// Bits 0, 2, 4, ... (even) or 1, 3, 5, ... (odd) of a zero mask of r inputs,
// packed: the masks of the two half-length DFTs of an even/odd split.
__host__ __device__ constexpr int even_bits(int z, int r) {
  int o = 0;
  for (int j = 0; j < r / 2; ++j) o |= ((z >> (2 * j)) & 1) << j;
  return o;
}
__host__ __device__ constexpr int odd_bits(int z, int r) { return even_bits(z >> 1, r); }

// X_k = sum_m a_m exp(S 2 pi i m k / R), in place, natural order.  Bit m of
// Z marks input m as zero (not loaded); Z = 0 is the plain DFT.
template <int S, int Z = 0>
__device__ __forceinline__ void dft4(double2* a) {
  constexpr bool z0 = Z & 1, z1 = (Z >> 1) & 1, z2 = (Z >> 2) & 1, z3 = (Z >> 3) & 1;
  constexpr bool ze = z0 && z2, zo = z1 && z3;
  const double2 t0 = add_z<z0, z2>(a[0], a[2]), t1 = sub_z<z0, z2>(a[0], a[2]);
  const double2 t2 = add_z<z1, z3>(a[1], a[3]), t3 = mul_si<S>(sub_z<z1, z3>(a[1], a[3]));
  a[0] = add_z<ze, zo>(t0, t2);
  a[2] = sub_z<ze, zo>(t0, t2);
  a[1] = add_z<ze, zo>(t1, t3);
  a[3] = sub_z<ze, zo>(t1, t3);
}

template <int S, int Z = 0>
__device__ __forceinline__ void dft2(double2* a) {
  constexpr bool z0 = Z & 1, z1 = (Z >> 1) & 1;
  const double2 t = a[0];
  a[0] = add_z<z0, z1>(t, a[1]);
  a[1] = sub_z<z0, z1>(t, a[1]);
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
template <int S, int Z = 0>
__device__ __forceinline__ void dft8(double2* a) {
  double2 e[4] = {a[0], a[2], a[4], a[6]};
  double2 o[4] = {a[1], a[3], a[5], a[7]};
  dft4<S, even_bits(Z, 8)>(e);
  dft4<S, odd_bits(Z, 8)>(o);
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

template <int S, int Z = 0>
__device__ __forceinline__ void dft16(double2* a) {
  double2 e[8], o[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    e[k] = a[2 * k];
    o[k] = a[2 * k + 1];
  }
  dft8<S, even_bits(Z, 16)>(e);
  dft8<S, odd_bits(Z, 16)>(o);
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

template <int R, int S, int Z = 0>
__device__ __forceinline__ void dftR(double2* a) {
  if constexpr (R == 2) dft2<S, Z>(a);
  if constexpr (R == 4) dft4<S, Z>(a);
  if constexpr (R == 8) dft8<S, Z>(a);
  if constexpr (R == 16) dft16<S, Z>(a);
}

// Radix plans: a list of stage radices whose product is N.
template <int... Rs>
struct Radices {};

// Plans: for each size N, a few variants V of the radix list used for two
// concurrent transforms (the pass kernels; `two`) and for a single transform
// (`one`), with the CTA width they run on.  Wide radices keep the FP64
// instruction count low; narrow ones and wider CTAs keep more warps in
// flight.  A stage with more butterflies than threads gives each thread
// several.  Variant 0 is the default; the autotuner (da_autotune) times the
// variants of a grid on the context's own batch and keeps the fastest.  The
// allocation-free control map uses variant 0.
template <int N, int V = 0> struct Plan;
template <> struct Plan<16, 0> { using two = Radices<4, 4>; using one = Radices<4, 4>; static constexpr int threads = 32; };
template <> struct Plan<32, 0> { using two = Radices<4, 8>; using one = Radices<4, 8>; static constexpr int threads = 32; };
template <> struct Plan<64, 0> { using two = Radices<4, 4, 4>; using one = Radices<4, 4, 4>; static constexpr int threads = 32; };
template <> struct Plan<64, 1> { using two = Radices<8, 8>; using one = Radices<8, 8>; static constexpr int threads = 32; };
// Radix-2 plans: 1.2x the FP64 instructions of the radix-4 ones, but each
// thread's chain is about half as long (34 instead of 60 instructions per
// 64-point transform).  On GB300 a lone warp issues one FP64 instruction per
// ~67 SM clocks whatever its active lanes, so the small grids at small
// batches, whose pass kernels are bound by that chain, run faster on them.
template <> struct Plan<32, 1> { using two = Radices<2, 2, 2, 2, 2>; using one = Radices<2, 2, 2, 2, 2>; static constexpr int threads = 32; };
template <> struct Plan<64, 2> { using two = Radices<2, 2, 2, 2, 2, 2>; using one = Radices<2, 2, 2, 2, 2, 2>; static constexpr int threads = 64; };
template <> struct Plan<128, 0> { using two = Radices<4, 4, 8>; using one = Radices<4, 4, 8>; static constexpr int threads = 64; };
template <> struct Plan<128, 1> { using two = Radices<8, 4, 4>; using one = Radices<8, 4, 4>; static constexpr int threads = 64; };
template <> struct Plan<128, 2> { using two = Radices<4, 4, 8>; using one = Radices<4, 4, 8>; static constexpr int threads = 32; };
template <> struct Plan<128, 3> { using two = Radices<2, 2, 2, 2, 2, 2, 2>; using one = Radices<2, 2, 2, 2, 2, 2, 2>; static constexpr int threads = 128; };
template <> struct Plan<256, 0> { using two = Radices<4, 4, 4, 4>; using one = Radices<4, 4, 4, 4>; static constexpr int threads = 128; };
template <> struct Plan<256, 1> { using two = Radices<8, 8, 4>; using one = Radices<8, 8, 4>; static constexpr int threads = 64; };
template <> struct Plan<256, 2> { using two = Radices<4, 4, 4, 4>; using one = Radices<4, 4, 4, 4>; static constexpr int threads = 64; };
template <> struct Plan<512, 0> { using two = Radices<8, 8, 8>; using one = Radices<8, 8, 8>; static constexpr int threads = 128; };
template <> struct Plan<512, 1> { using two = Radices<8, 4, 4, 4>; using one = Radices<8, 4, 4, 4>; static constexpr int threads = 256; };
template <> struct Plan<512, 2> { using two = Radices<8, 8, 8>; using one = Radices<8, 8, 8>; static constexpr int threads = 64; };
template <> struct Plan<1024, 0> { using two = Radices<16, 8, 8>; using one = Radices<16, 8, 8>; static constexpr int threads = 256; };
template <> struct Plan<1024, 1> { using two = Radices<16, 4, 4, 4>; using one = Radices<16, 4, 4, 4>; static constexpr int threads = 256; };
template <> struct Plan<1024, 2> { using two = Radices<8, 8, 4, 4>; using one = Radices<8, 8, 4, 4>; static constexpr int threads = 256; };

// Number of plan variants of each size (the instantiations in inst_n*.cu).
constexpr int plan_count(int n) {
  return n == 32 ? 2 : n == 64 ? 3 : n == 128 ? 4 : (n == 256 || n == 512 || n == 1024) ? 3 : 1;
}

template <int N, int V = 0>
struct PlanInfo {
  static constexpr int THREADS = Plan<N, V>::threads;
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

// ---------------------------------------------------------------------------
// Folded twiddles
// ---------------------------------------------------------------------------
//
// A twiddle w = exp(S i theta) written as c (1 + i t), c = cos theta,
// t = S tan theta, turns w a into c z with z = (a.x - t a.y, a.y + t a.x):
// two FMAs.  The factor c then rides on the FMAs of the butterfly that
// follows: in a radix-4 butterfly, a0 +- c2 z2 and, with r31 = c3/c1,
// c1 (z1 +- r31 z3); in a radix-8 butterfly the even half is a folded
// radix-4 on (a0, a2, a4, a6) and every output of the odd half carries the
// common factor c1, which joins the last combination (for k = 1, 3 as
// kR2 c1).  A twiddled radix-4 butterfly costs 22 FP64 instructions instead
// of 28 and a twiddled radix-8 one 66 instead of 80.  c is never exactly
// zero (the angles are below pi/2 for c1, and elsewhere cos of a rounded
// angle), and c t, c r reconstitute sin theta and the other cosines to a
// rounding, so every output keeps an error of a few ulps of the inputs.
//
// Per stage with L > 1 the table holds, slot-major (slot j of butterfly
// class k at j * L + k):
//   R = 2: t1, c1;
//   R = 4: t1 t2 t3 (for S = -1), c1, c2, r31;
//   R = 8: t1..t7, c1, c2, c4, r62 = c6/c2, r51 = c5/c1, r73 = c7/c3,
//          r31 = c3/c1, q = cos(pi/4) c1.

template <int R> struct FoldSlots { static constexpr int value = 0; };  // untwiddled first stages only
template <> struct FoldSlots<2> { static constexpr int value = 2; };
template <> struct FoldSlots<4> { static constexpr int value = 6; };
template <> struct FoldSlots<8> { static constexpr int value = 15; };

// Doubles of the folded table of a plan, stages after the first.
template <int L, typename P> struct FoldSize;
template <int L> struct FoldSize<L, Radices<>> { static constexpr int value = 0; };
template <int L, int R, int... Rs> struct FoldSize<L, Radices<R, Rs...>> {
  static constexpr int value = (L > 1 ? FoldSlots<R>::value * L : 0) + FoldSize<L * R, Radices<Rs...>>::value;
};

template <int N, int V = 0>
struct FoldInfo {
  static constexpr int DOUBLES = FoldSize<1, typename Plan<N, V>::two>::value;
  // padded to whole double2 so that the sequences after it stay aligned
  static constexpr int PADDED = (DOUBLES + 1) / 2 * 2;
};

// z = (a.x - t a.y, a.y + t a.x)
__device__ __forceinline__ double2 tan_rot(double2 a, double t) {
  return make_double2(fma(-t, a.y, a.x), fma(t, a.x, a.y));
}

// e +- c z  (plus, minus)
__device__ __forceinline__ void fma_pair(double2 e, double2 z, double c, double2& plus, double2& minus) {
  plus = make_double2(fma(c, z.x, e.x), fma(c, z.y, e.y));
  minus = make_double2(fma(-c, z.x, e.x), fma(-c, z.y, e.y));
}

// e + c z into plus unless output p is masked, e - c z into minus unless
// output q is: the last stage of a forward transform leaves the outputs that
// fall in the gap unformed (the compiler drops what only they would use).
template <int O, int p, int q>
__device__ __forceinline__ void fma_pair_o(double2 e, double2 z, double c, double2& plus, double2& minus) {
  if constexpr (!((O >> p) & 1)) plus = make_double2(fma(c, z.x, e.x), fma(c, z.y, e.y));
  if constexpr (!((O >> q) & 1)) minus = make_double2(fma(-c, z.x, e.x), fma(-c, z.y, e.y));
}

// Twiddled radix-2 butterfly with a folded twiddle: a0 +- c1 z1, six FP64
// instructions.  Bit m of O: output m is not needed (left unformed).
template <int S, int O = 0>
__device__ __forceinline__ void dft2_folded(double2* a, const double* T, int k, int L) {
  const double sg = S < 0 ? 1.0 : -1.0;
  const double2 z1 = tan_rot(a[1], sg * T[k]);
  fma_pair_o<O, 0, 1>(a[0], z1, T[L + k], a[0], a[1]);
}

// Twiddled radix-4 butterfly with folded twiddles (table T, class k, L).
template <int S, int O = 0>
__device__ __forceinline__ void dft4_folded(double2* a, const double* T, int k, int L) {
  const double sg = S < 0 ? 1.0 : -1.0;
  const double t1 = sg * T[k], t2 = sg * T[L + k], t3 = sg * T[2 * L + k];
  const double c1 = T[3 * L + k], c2 = T[4 * L + k], r31 = T[5 * L + k];
  const double2 z1 = tan_rot(a[1], t1), z2 = tan_rot(a[2], t2), z3 = tan_rot(a[3], t3);
  double2 t0, tt1, u, v;
  fma_pair(a[0], z2, c2, t0, tt1);
  fma_pair(z1, z3, r31, u, v);
  fma_pair_o<O, 0, 2>(t0, u, c1, a[0], a[2]);
  fma_pair_o<O, 1, 3>(tt1, mul_si<S>(v), c1, a[1], a[3]);
}

// Twiddled radix-8 butterfly with folded twiddles.
template <int S, int O = 0>
__device__ __forceinline__ void dft8_folded(double2* a, const double* T, int k, int L) {
  const double sg = S < 0 ? 1.0 : -1.0;
  double2 z[8];
#pragma unroll
  for (int m = 1; m < 8; ++m) z[m] = tan_rot(a[m], sg * T[(m - 1) * L + k]);
  const double c1 = T[7 * L + k], c2 = T[8 * L + k], c4 = T[9 * L + k];
  const double r62 = T[10 * L + k], r51 = T[11 * L + k], r73 = T[12 * L + k], r31 = T[13 * L + k];
  const double q = T[14 * L + k];
  // even half: radix 4 on (a0, a2', a4', a6')
  double2 et0, et1, eu, ev, e0, e1, e2, e3;
  fma_pair(a[0], z[4], c4, et0, et1);
  fma_pair(z[2], z[6], r62, eu, ev);
  fma_pair(et0, eu, c2, e0, e2);
  fma_pair(et1, mul_si<S>(ev), c2, e1, e3);
  // odd half on (a1', a3', a5', a7'), outputs c1 p_k
  double2 ou0, ov0, ou1, ov1, p0, p1, p2, p3;
  fma_pair(z[1], z[5], r51, ou0, ov0);
  fma_pair(z[3], z[7], r73, ou1, ov1);
  fma_pair(ou0, ou1, r31, p0, p2);
  fma_pair(ov0, mul_si<S>(ov1), r31, p1, p3);
  // a_k = e_k + W8^k c1 p_k
  fma_pair_o<O, 0, 4>(e0, p0, c1, a[0], a[4]);
  fma_pair_o<O, 2, 6>(e2, mul_si<S>(p2), c1, a[2], a[6]);
  const double2 w1 = make_double2(p1.x - S * p1.y, p1.y + S * p1.x);
  fma_pair_o<O, 1, 5>(e1, w1, q, a[1], a[5]);
  const double2 w3 = make_double2(p3.x + S * p3.y, p3.y - S * p3.x);
  fma_pair_o<O, 3, 7>(e3, w3, -q, a[3], a[7]);
}

// ---------------------------------------------------------------------------
// Band-limited sequences
// ---------------------------------------------------------------------------
//
// The inverse transforms of the pass kernels read sequences that are zero in
// the gap K < q < N - K (the 2/3 rule, K = (N-1)/3), and their forward
// transforms are read back only on the band q <= K, q >= N - K.  Input m of
// butterfly i of the first stage is x[i + m N/R]; output m of butterfly k of
// the last stage is y[k + m N/R].  Where that position lies in the gap for
// all 32 lanes of a warp, the warp skips the load and the additions the zero
// would enter (first stage), or neither forms nor stores the output (last
// stage; the buffer keeps whatever it held there).  The tests are per warp
// because GB300's FP64 pipe spends the same time on a warp instruction
// whatever its active lanes: only whole warp instructions saved count.  A
// warp covers 32 consecutive butterflies of one sequence when N/R is a
// multiple of 32; otherwise only the positions in the gap for every
// butterfly are skipped.

// positions lo..hi all in the gap of band kb (kb < 0: no band)
__host__ __device__ constexpr bool in_gap(int n, int kb, int lo, int hi) {
  return kb >= 0 && lo >= kb + 1 && hi <= n - kb - 1;
}
// m whose position is in the gap for every butterfly of a stage of radix r
__host__ __device__ constexpr int gap_common(int n, int r, int kb) {
  int c = 0;
  for (int m = 0; m < r; ++m)
    if (in_gap(n, kb, m * (n / r), m * (n / r) + n / r - 1)) c |= 1 << m;
  return c;
}
// m in the gap for all lanes of some warps only
__host__ __device__ constexpr int gap_per_warp(int n, int r, int kb) {
  const int nb = n / r;
  int c = 0;
  if (nb % 32) return 0;
  for (int m = 0; m < r; ++m)
    for (int i0 = 0; i0 < nb; i0 += 32)
      if (!((gap_common(n, r, kb) >> m) & 1) && in_gap(n, kb, i0 + m * nb, i0 + 31 + m * nb)) c |= 1 << m;
  return c;
}
__host__ __device__ constexpr int bit_index(int b) {
  int m = 0;
  while (b > 1) {
    b >>= 1;
    ++m;
  }
  return m;
}
__host__ __device__ constexpr int popcount_c(int b) {
  int c = 0;
  for (; b; b &= b - 1) ++c;
  return c;
}

template <int N, int R, int KB>
struct GapMask {
  static constexpr int NB = N / R;
  static constexpr int C = gap_common(N, R, KB), X = gap_per_warp(N, R, KB);
  static constexpr int A = X & -X, B = X & ~A;  // the per-warp bits
  static_assert((B & (B - 1)) == 0, "at most two per-warp gap positions per butterfly");
  // mask of the warp that holds butterfly i
  __host__ __device__ static int warp(int i) {
    int w = C;
    if constexpr (A != 0) {
      const int i0 = i & ~31;
      constexpr int ma = bit_index(A);
      if (in_gap(N, KB, i0 + ma * NB, i0 + 31 + ma * NB)) w |= A;
      if constexpr (B != 0) {
        constexpr int mb = bit_index(B);
        if (in_gap(N, KB, i0 + mb * NB, i0 + 31 + mb * NB)) w |= B;
      }
    }
    return w;
  }
};

// The butterfly of one stage: untwiddled with zero inputs Z (first stage),
// or twiddled with unneeded outputs O.
template <int R, int S, int L, int Z, int O>
__device__ __forceinline__ void stage_butterfly(double2* a, const double* T, int k) {
  if constexpr (L == 1) {
    static_assert(O == 0, "a first stage that is also the last");
    dftR<R, S, Z>(a);
  } else {
    static_assert(Z == 0, "zero inputs in the first stage only");
    static_assert(R == 2 || R == 4 || R == 8, "folded twiddles for radix 2, 4 and 8");
    if constexpr (R == 2) dft2_folded<S, O>(a, T, k, L);
    if constexpr (R == 4) dft4_folded<S, O>(a, T, k, L);
    if constexpr (R == 8) dft8_folded<S, O>(a, T, k, L);
  }
}

// Runs the butterfly for the warp's mask w, one of C, C|A, C|B, C|A|B of
// GapMask G (w is warp-uniform, so the branches do not diverge); IN: w
// masks inputs (Z), else outputs (O).
template <int R, int S, int L, bool IN, typename G>
__device__ __forceinline__ void masked_butterfly(double2* a, const double* T, int k, int w) {
  constexpr int C = G::C, A = G::A, B = G::B;
  if constexpr (A == 0) {
    stage_butterfly<R, S, L, IN ? C : 0, IN ? 0 : C>(a, T, k);
  } else if constexpr (B == 0) {
    if (w & A) stage_butterfly<R, S, L, IN ? C | A : 0, IN ? 0 : C | A>(a, T, k);
    else stage_butterfly<R, S, L, IN ? C : 0, IN ? 0 : C>(a, T, k);
  } else {
    if ((w & (A | B)) == (A | B)) stage_butterfly<R, S, L, IN ? C | A | B : 0, IN ? 0 : C | A | B>(a, T, k);
    else if (w & A) stage_butterfly<R, S, L, IN ? C | A : 0, IN ? 0 : C | A>(a, T, k);
    else if (w & B) stage_butterfly<R, S, L, IN ? C | B : 0, IN ? 0 : C | B>(a, T, k);
    else stage_butterfly<R, S, L, IN ? C : 0, IN ? 0 : C>(a, T, k);
  }
}

// No output pair of a folded butterfly (its two fma_pair_o halves) may be
// masked whole: the flop count of band_transform_flops assumes that every
// masked output saves its own two FMAs and nothing else.
// (pairs: radix 2 (0, 1); radix 4 (0, 2), (1, 3); radix 8 (m, m + 4)).
__host__ __device__ constexpr bool no_whole_pair(int r, int o) {
  if (r == 2) return (o & 3) != 3;
  if (r == 4) return (o & 5) != 5 && (o & 10) != 10;
  if (r == 8) return (o & 0x11) != 0x11 && (o & 0x44) != 0x44 && (o & 0x22) != 0x22 && (o & 0x88) != 0x88;
  return o == 0;
}

// One in-place Stockham stage with folded twiddles (T: this stage's table).
// KIN >= 0: the input is band-limited to KIN (first stage skips the gap);
// KOUT >= 0: only the band KOUT of the output is needed (last stage).
template <int N, int V, int R, int S, int F, int L, int KIN, int KOUT>
__device__ __forceinline__ void stockham_stage_folded(double2* buf, const double* __restrict__ T) {
  constexpr int NB = N / R, Th = PlanInfo<N, V>::THREADS, TOT = F * NB, J = (TOT + Th - 1) / Th;
  constexpr bool FIRST = L == 1, LAST = L * R == N;
  using GI = GapMask<N, R, FIRST ? KIN : -1>;
  using GO = GapMask<N, R, LAST ? KOUT : -1>;
  static_assert(no_whole_pair(R, GO::C | GO::A | GO::B), "a whole output pair in the gap");
  double2 a[J][R];
  int base[J], dst[J], om[J];
#pragma unroll
  for (int jb = 0; jb < J; ++jb) {
    const int u = threadIdx.x + jb * Th;
    base[jb] = 0;
    dst[jb] = 0;
    om[jb] = 0;
    if (TOT % Th == 0 || u < TOT) {
      const int f = u / NB;
      const int i = u - f * NB;
      const int k = i & (L - 1);
      base[jb] = f * N;
      const int zm = GI::warp(i);
#pragma unroll
      for (int m = 0; m < R; ++m)
        if (!((zm >> m) & 1)) a[jb][m] = buf[base[jb] + i + m * NB];
      if constexpr (FIRST) {
        masked_butterfly<R, S, L, true, GI>(a[jb], T, k, zm);
      } else {
        om[jb] = GO::warp(i);
        masked_butterfly<R, S, L, false, GO>(a[jb], T, k, om[jb]);
      }
      dst[jb] = (i - k) * R + k;
    }
  }
  __syncthreads();
#pragma unroll
  for (int jb = 0; jb < J; ++jb) {
    const int u = threadIdx.x + jb * Th;
    if (TOT % Th == 0 || u < TOT) {
#pragma unroll
      for (int m = 0; m < R; ++m)
        if (!((om[jb] >> m) & 1)) buf[base[jb] + dst[jb] + m * L] = a[jb][m];
    }
  }
  __syncthreads();
}

template <int N, int V, int S, int F, int L, int KIN, int KOUT>
__device__ __forceinline__ void run_stages_folded(double2*, const double*, Radices<>) {}

template <int N, int V, int S, int F, int L, int KIN, int KOUT, int R, int... Rs>
__device__ __forceinline__ void run_stages_folded(double2* buf, const double* T, Radices<R, Rs...>) {
  stockham_stage_folded<N, V, R, S, F, L, KIN, KOUT>(buf, T);
  run_stages_folded<N, V, S, F, L * R, KIN, KOUT>(buf, T + (L > 1 ? FoldSlots<R>::value * L : 0), Radices<Rs...>{});
}

// First and last radix of a plan, the plan without its last stage, and
// without its first.
template <typename P> struct FirstRadix;
template <int R, int... Rs> struct FirstRadix<Radices<R, Rs...>> { static constexpr int value = R; };
template <typename P> struct LastRadix;
template <int R> struct LastRadix<Radices<R>> { static constexpr int value = R; };
template <int R, int R2, int... Rs> struct LastRadix<Radices<R, R2, Rs...>> {
  static constexpr int value = LastRadix<Radices<R2, Rs...>>::value;
};
template <int R, typename P> struct Prepend;
template <int R, int... Rs> struct Prepend<R, Radices<Rs...>> { using type = Radices<R, Rs...>; };
template <typename P> struct InitRadices;
template <int R> struct InitRadices<Radices<R>> { using type = Radices<>; };
template <int R, int R2, int... Rs> struct InitRadices<Radices<R, R2, Rs...>> {
  using type = typename Prepend<R, typename InitRadices<Radices<R2, Rs...>>::type>::type;
};
template <typename P> struct TailRadices;
template <int R, int... Rs> struct TailRadices<Radices<R, Rs...>> { using type = Radices<Rs...>; };

// Transform, in place, F (1 or 2) sequences of N points stored back to back
// in buf, with the folded table of Plan<N, V>::two (both lists of a plan
// are the same radices) in shared memory.  Same contract as fft_batch, on a
// CTA of PlanInfo<N, V>::THREADS threads.  KIN >= 0: every sequence is zero
// in the gap KIN < q < N - KIN (the gap must hold zeros: warps that straddle
// it still read it).  KOUT >= 0: the caller reads the result only at
// q <= KOUT and q >= N - KOUT; the gap positions are left undefined.
template <int N, int V, int S, int F, int KIN = -1, int KOUT = -1>
__device__ __forceinline__ void fft_folded(double2* buf, const double* T) {
  static_assert(F == 1 || F == 2, "batches of one or two transforms");
  run_stages_folded<N, V, S, F, 1, KIN, KOUT>(buf, T, typename Plan<N, V>::two{});
}

// Whether an inverse transform, a pointwise map and a forward transform of the
// same sequences can hand the data over in registers: when the plan's first
// and last radix agree, the thread that forms outputs k + m N/R of the last
// inverse stage is the thread that needs inputs i + m N/R (i = k) of the
// first forward stage.
template <int N, int V>
struct Fusable {
  using P = typename Plan<N, V>::two;
  static constexpr bool value = FirstRadix<P>::value == LastRadix<P>::value;
};

// Inverse transform (S = +1, input band-limited to KIN), then op applied to
// every output point, then forward transform (S = -1, output needed on the
// band KOUT) of F sequences in buf: the last inverse stage, op and the first
// forward stage run on registers, between one pair of barriers.  op(f, x, z)
// gets sequence f, position x and the inverse transform's value there, and
// returns the forward transform's input there.  Same contract as two
// fft_folded calls with op applied in between; requires Fusable<N, V>.
template <int N, int V, int F, int KIN, int KOUT, typename Op>
__device__ __forceinline__ void fft_folded_turn(double2* buf, const double* T, Op op) {
  using P = typename Plan<N, V>::two;
  static_assert(Fusable<N, V>::value, "first and last radix must agree");
  constexpr int R = LastRadix<P>::value, NB = N / R, L = N / R;
  constexpr int Th = PlanInfo<N, V>::THREADS, TOT = F * NB, J = (TOT + Th - 1) / Th;
  // inverse stages but the last
  run_stages_folded<N, V, +1, F, 1, KIN, -1>(buf, T, typename InitRadices<P>::type{});
  const double* Tl = T + FoldSize<1, typename InitRadices<P>::type>::value;
  double2 a[J][R];
  int base[J], ii[J];
#pragma unroll
  for (int jb = 0; jb < J; ++jb) {
    const int u = threadIdx.x + jb * Th;
    base[jb] = 0;
    ii[jb] = 0;
    if (TOT % Th == 0 || u < TOT) {
      const int f = u / NB;
      const int i = u - f * NB;
      base[jb] = f * N;
      ii[jb] = i;
#pragma unroll
      for (int m = 0; m < R; ++m) a[jb][m] = buf[base[jb] + i + m * NB];
      stage_butterfly<R, +1, L, 0, 0>(a[jb], Tl, i);  // last inverse stage: class k = i
    }
  }
  __syncthreads();  // every thread has read buf
#pragma unroll
  for (int jb = 0; jb < J; ++jb) {
    const int u = threadIdx.x + jb * Th;
    if (TOT % Th == 0 || u < TOT) {
      const int f = u / NB;
#pragma unroll
      for (int m = 0; m < R; ++m) a[jb][m] = op(f, ii[jb] + m * L, a[jb][m]);
      dftR<R, -1, 0>(a[jb]);  // first forward stage
#pragma unroll
      for (int m = 0; m < R; ++m) buf[base[jb] + ii[jb] * R + m] = a[jb][m];
    }
  }
  __syncthreads();
  // forward stages after the first (its table slots start at 0: the first
  // stage has none)
  run_stages_folded<N, V, -1, F, R, -1, KOUT>(buf, T, typename TailRadices<P>::type{});
}

// Host side: flops of one band-limited transform of N points under Plan<N,
// V> as the pass kernels run it: the nominal 5 N log2 N less the operations
// the gap tests skip (a real addition or multiplication counts one, an FMA
// two).  Inverse: the zero inputs of the first stage; forward: the unformed
// outputs of the last (two FMAs each).

// flops a zero mask z saves in the untwiddled r-point DFT (dft2/4/8/16):
// every add_z / sub_z with a known-zero operand saves one complex addition
constexpr int zero_savings(int r, int z) {
  if (r == 2) return (z & 3) ? 4 : 0;
  if (r == 4) {
    const bool z0 = z & 1, z1 = (z >> 1) & 1, z2 = (z >> 2) & 1, z3 = (z >> 3) & 1;
    return ((z0 || z2) ? 4 : 0) + ((z1 || z3) ? 4 : 0) + (((z0 && z2) || (z1 && z3)) ? 8 : 0);
  }
  return zero_savings(r / 2, even_bits(z, r)) + zero_savings(r / 2, odd_bits(z, r));
}

template <int N, int V, int KB>
inline double band_transform_flops(bool inverse) {
  using P = typename Plan<N, V>::two;
  double saved = 0.0;
  if (inverse) {
    constexpr int R = FirstRadix<P>::value;
    for (int i = 0; i < N / R; ++i) saved += zero_savings(R, GapMask<N, R, KB>::warp(i));
  } else {
    constexpr int R = LastRadix<P>::value;
    for (int i = 0; i < N / R; ++i) saved += 4 * popcount_c(GapMask<N, R, KB>::warp(i));
  }
  return 5.0 * N * std::log2((double)N) - saved;
}

// Host side: fill the folded table of Plan<N, V>::two (FoldInfo<N, V>::DOUBLES
// entries) for S = -1.
template <int L>
inline void fold_fill(double*, int, Radices<>) {}

template <int L, int R, int... Rs>
inline void fold_fill(double* out, int n, Radices<R, Rs...>) {
  if (L > 1) {
    const double pi = 3.14159265358979323846;
    for (int k = 0; k < L; ++k) {
      double c[8], t[8];
      for (int m = 1; m < R; ++m) {
        const double th = -2.0 * pi * (double)(m * k) / (double)(L * R);  // W_{LR}^{mk}, S = -1
        c[m] = std::cos(th);
        t[m] = std::tan(th);
      }
      if (R == 2) {
        out[k] = t[1];
        out[L + k] = c[1];
      } else if (R == 4) {
        const double v[6] = {t[1], t[2], t[3], c[1], c[2], c[3] / c[1]};
        for (int j = 0; j < 6; ++j) out[j * L + k] = v[j];
      } else {
        const double v[15] = {t[1], t[2], t[3], t[4], t[5], t[6], t[7], c[1], c[2], c[4],
                              c[6] / c[2], c[5] / c[1], c[7] / c[3], c[3] / c[1], 0.70710678118654752440 * c[1]};
        for (int j = 0; j < 15; ++j) out[j * L + k] = v[j];
      }
    }
    out += FoldSlots<R>::value * L;
  }
  fold_fill<L * R>(out, n, Radices<Rs...>{});
}

template <int N, int V>
inline void fold_table(double* out) {
  fold_fill<1>(out, N, typename Plan<N, V>::two{});
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
