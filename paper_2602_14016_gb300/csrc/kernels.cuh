// kernels.cuh -- pass kernels of the cost-and-gradient evaluation.
//
// Layout (per member b of a batch):
//   compact spectra  [Kc][Kr] complex, column-major (cidx): the retained
//                    set of the 2/3 rule, kx = 0..K (columns), compact row
//                    r -> ky = r (r <= K) or r - Kr; K = floor((N-1)/3),
//                    Kc = K+1, Kr = 2K+1.  A column pass reads and writes one
//                    contiguous column.
//   mixed fields     physical y, spectral kx (kx = 0..K), two fields: the
//                    column-pass output Mx row-major [2][N][Kc] (a row
//                    pass reads whole rows), the row-pass output Mn
//                    column-major [Kc][2][N] (a column pass reads its
//                    column of both fields as one contiguous block).
//   stage fields     [nsteps][4 stages][2 fields][N][N] double: u, v of
//                    every RK stage state, written by the forward row pass
//                    and read back by the adjoint row pass.
//
// The advection term is evaluated in the divergence form of Basdevant
// (1983): for a divergence-free band-limited velocity,
//   u . grad w = (d_xx - d_yy)(u v) + d_xy (v^2 - u^2),
// and with the 2/3 rule both sides are the same retained coefficients (the
// products of retained fields alias nothing onto the retained set), so the
// discrete right-hand side is the one of the advective form, u w_x + v w_y,
// evaluated with four real transforms instead of five and two stored stage
// fields instead of four.
//
// A forward RK stage is two kernels: a ROW pass (inverse transforms along x
// of the packed mixed rows -> u, v; stage-field store; probe gather; the
// products u v and v^2 - u^2; their forward transforms along x, handed over
// in registers where the plan allows: fft_folded_turn) and a COLUMN
// pass (forward transforms along y of the two products, the advection term,
// RK epilogue with viscosity, forcing and the stage update, then the
// inverse column transforms of the next stage's u and v).  The adjoint
// mirrors this with the transposed operators.  Every transform is an FP64
// shared-memory FFT from fft.cuh; the 1/N^2 of the inverse 2D transform is
// applied once, to the spectral coefficients before the column transform.
// Every inverse transform here reads a sequence that is zero in the gap
// K < q < N - K, and every forward transform is read back only on the band
// q <= K, q >= N - K: the transforms are called band-limited (fft_folded
// with KIN / KOUT = K) and skip that work where whole warps allow.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "fft.cuh"

namespace da {

enum : int {
  F_STORE = 1,     // forward row pass: write stage fields
  F_OBS = 2,       // forward row pass: gather probes into the observation slot
  F_OBS_ONLY = 4,  // forward row pass: only gather probes (final state)
  F_NO_NEXT = 8,   // column pass: skip the inverse transforms of the next stage
  F_SRC = 16       // adjoint column pass: add the observation source at this step
};

// Start of the adjoint sweep (k_adj_init): add the observation source of
// the last step, and/or start from the terminal field already in LamBar; or
// resume from the adjoint stage value in KB after a checkpoint recompute.
enum : int { INIT_SRC = 1, INIT_LAMBAR = 2, INIT_RESUME = 4 };

// Multipliers of the generic spectral-to-mixed column pass.
enum : int { M_ONE = 0, M_CTRL = 1, M_FILTERED = 2, M_INV_CTRL = 3 };

// Per-mode constants of the column passes, column-major [Kc][Kr] (entry
// kx * Kr + r), computed once on the host so that no column pass divides or
// converts integers in FP64:
//   fwd: su = ky/k^2/N^2, sv = kx/k^2/N^2 (u, v columns of a state value),
//        cp = (ky^2 - kx^2)/2, cq = -kx ky/2 (advection symbols; the 1/2 is
//        the one the row pass leaves out when it unpacks two real rows);
//   adj: a1 = ky/k^2/2, c1 = kx/k^2/2 (transposed velocity symbols, same
//        1/2), ca = -2 kx ky/N^2, cb = (ky^2 - kx^2)/N^2 (adjoint-field
//        columns; ca carries the 2 of rho_u, rho_v);
//   k2 = k^2 (the column passes multiply it by the member's viscosity).
struct __align__(32) Sym4 {
  double a, b, c, d;
};

// Everything a kernel needs, passed by value.
struct Dev {
  int B, nsteps, every, include_t0, px, nt;  // nsteps: the evaluation's window (global steps)
  double dt, nu;
  int force;
  double amp;
  int nf;
  // Ragged batches: member b runs its own window, end-aligned in the
  // evaluation's -- live from global step mstart[b] to nsteps, its local step
  // n - mstart[b] -- with its own probe lattice, viscosity and forcing switch;
  // a member with mstart[b] > nsteps is idle.  With ragged == 0 every member
  // runs the context's window and the tables are not read.
  int ragged;
  const int* mstart;                         // [B]
  const int* mnt;                            // [B] observation times of member b
  const int* mpx;                            // [B] probes per side of member b
  const double* mnu;                         // [B]
  const int* mforce;                         // [B] Kolmogorov forcing on (1) or off (0)
  size_t obs_stride;                         // doubles from one member's obs, mobs, res to the next
  double2 *W, *Acc, *Y, *KB, *LamBar, *Sum;  // compact [B][Kc][Kr] (cidx)
  double2* Mx;                               // mixed [B][2][N][Kc]: column-pass output
  double2* Mn;                               // mixed [B][Kc][2][N]: row-pass output
  double* traj;                              // [B][traj_steps][4][2][N][N]
  int traj_steps;                            // steps the stage-field store holds
  int seg0;                                  // step stored in slot 0 of the store
  double* obs;                               // model observations [B][nt][P2][2]
  const double* mobs;                        // data [B][nt][P2][2]
  double* res;                               // residuals [B][nt][P2][2]
  double* J;                                 // [B]
  const double* mult;                        // control multiplier |k| W^1/2, compact [B][Kc][Kr]
  const double* fold;                        // folded twiddles of Plan<N> (fft.cuh)
  const double2* twP;                        // W_64^t, t < 64 (W_P^t = W_64^{t 64/P})
  const Sym4* symF;                          // [Kc][Kr] su, sv, cp, cq
  const Sym4* symA;                          // [Kc][Kr] a1, c1, ca, cb
  const double* k2;                          // [Kc][Kr] k^2 (times nu of the member)
  double dt2, dt3, dt6;                      // dt/2, dt/3, dt/6
};

template <int N, int V = 0>
struct Geo {
  static constexpr int K = (N - 1) / 3;
  static constexpr int Kc = K + 1;
  static constexpr int Kr = 2 * K + 1;
  static constexpr int NH = N / 2 + 1;
  // threads: two transforms at a time (fft.cuh)
  static constexpr int THREADS = PlanInfo<N, V>::THREADS;
  // shared memory: folded twiddle table + one buffer of two sequences +
  // probe sums
  static constexpr int PMAX = 64;
  static constexpr size_t SMEM = sizeof(double) * FoldInfo<N, V>::PADDED + sizeof(double2) * (2 * N + 2 * PMAX);
  // column passes load their epilogue inputs before the transforms (about
  // 60 more registers a thread) where a CTA is at most 128 threads
  static constexpr bool PREFETCH = THREADS <= 128;
};

__device__ __forceinline__ int ky_of_row(int r, int K) { return r <= K ? r : r - (2 * K + 1); }

// Index of mode (row r, column kx) of member bm in a compact array.
template <int N>
__host__ __device__ __forceinline__ size_t cidx(int bm, int r, int kx) {
  return ((size_t)bm * Geo<N>::Kc + kx) * Geo<N>::Kr + r;
}

template <int N, int V = 0>
__device__ __forceinline__ void load_fold(double* T, const double* __restrict__ g) {
  for (int i = threadIdx.x; i < FoldInfo<N, V>::DOUBLES; i += blockDim.x) T[i] = g[i];
}

// The window of member bm in this evaluation (see Dev).
struct MemberWindow {
  int start, P;
  double nu;
  bool forced;
};

__device__ __forceinline__ MemberWindow member_window(const Dev& d, int bm) {
  if (!d.ragged) return {0, d.px, d.nu, d.force != 0};
  return {d.mstart[bm], d.mpx[bm], d.mnu[bm], d.force != 0 && d.mforce[bm] != 0};
}

// Observation slot of local step k, or -1.
__device__ __forceinline__ int obs_slot(const Dev& d, int k) {
  if (k == 0) return d.include_t0 ? 0 : -1;
  if (k % d.every) return -1;
  return k / d.every - 1 + (d.include_t0 ? 1 : 0);
}

// Full-length sequence whose inverse transform is a + i b, for two real rows
// a, b given by their mixed half spectra A, B (kx = 0..K): Z(kx) = A + iB,
// Z(-kx) = conj(A) + i conj(B); the DC bin keeps real parts only.  Every
// coefficient is loaded once and written to kx and -kx; the gap
// K < kx < N-K is zeroed.  Coefficient kx of A and Bv is at [kx * STRIDE].
// Loops run over compile-time trip counts so that a thread's loads are
// issued together.
template <int N, int T, int STRIDE = 1>
__device__ __forceinline__ void pack_rows(double2* seq, const double2* __restrict__ A, const double2* __restrict__ Bv) {
  constexpr int K = Geo<N>::K, GAP = N - 2 * K - 1;
#pragma unroll
  for (int t = 0; t < (GAP + T - 1) / T; ++t) {
    const int u = threadIdx.x + t * T;
    if (u < GAP) seq[K + 1 + u] = make_double2(0.0, 0.0);
  }
#pragma unroll
  for (int t = 0; t < (K + 1 + T - 1) / T; ++t) {
    const int kx = threadIdx.x + t * T;
    if (kx <= K) {
      const double2 p = A[(size_t)kx * STRIDE], q = Bv[(size_t)kx * STRIDE];
      if (kx == 0) {
        seq[0] = make_double2(p.x, q.x);
      } else {
        seq[kx] = make_double2(p.x - q.y, p.y + q.x);
        seq[N - kx] = make_double2(p.x + q.y, q.x - p.y);
      }
    }
  }
}

// The two half spectra packed in a forward transform Z of a + i b:
// A(k) = (Z(k) + conj Z(-k))/2, B(k) = -i (Z(k) - conj Z(-k))/2.
template <int N, int V = 0>
__device__ __forceinline__ void unpack_pair(const double2* Z, int kx, double2& A, double2& Bv) {
  const double2 zk = Z[kx], zm = Z[(N - kx) & (N - 1)];
  const double sx = zk.x + zm.x, sy = zk.y - zm.y;
  const double tx = zk.x - zm.x, ty = zk.y + zm.y;
  A = make_double2(0.5 * sx, 0.5 * sy);
  Bv = make_double2(0.5 * ty, -0.5 * tx);
}

// Twice the two half spectra (no 1/2): the pass kernels fold the 1/2 into
// the per-mode symbols of the column pass that consumes them.
template <int N, int V = 0>
__device__ __forceinline__ void unpack_pair2(const double2* Z, int kx, double2& A, double2& Bv) {
  const double2 zk = Z[kx], zm = Z[(N - kx) & (N - 1)];
  A = make_double2(zk.x + zm.x, zk.y - zm.y);
  Bv = make_double2(zk.y + zm.y, zm.x - zk.x);
}

// ---------------------------------------------------------------------------
// Generic row transforms (control map, gradient map)
// ---------------------------------------------------------------------------

// Real rows in[b][y][x] -> mixed half rows Mn[b][y][kx], kx <= K (forward,
// unnormalised), two rows per complex transform.  grid (N/2, B).
template <int N, int V = 0>
__global__ void __launch_bounds__(Geo<N, V>::THREADS) k_r2c_rows(Dev d, const double* __restrict__ in) {
  using G = Geo<N, V>;
  extern __shared__ double2 sm[];
  double* T = reinterpret_cast<double*>(sm);
  double2* a = sm + FoldInfo<N, V>::PADDED / 2;
  const int bm = blockIdx.y, y0 = 2 * blockIdx.x;
  load_fold<N, V>(T, d.fold);
  const double* r0 = in + ((size_t)bm * N + y0) * N;
  #pragma unroll
  for (int x = threadIdx.x; x < N; x += G::THREADS) a[x] = make_double2(r0[x], r0[N + x]);
  __syncthreads();
  fft_folded<N, V, -1, 1, -1, G::K>(a, T);
  double2* M = d.Mn + (size_t)bm * G::Kc * 2 * N + y0;  // field 0, rows y0 and y0 + 1
  #pragma unroll
  for (int kx = threadIdx.x; kx < G::Kc; kx += G::THREADS) {
    double2 A, Bv;
    unpack_pair<N>(a, kx, A, Bv);
    M[(size_t)kx * 2 * N] = A;
    M[(size_t)kx * 2 * N + 1] = Bv;
  }
}

// Mixed half rows Mn[b][y][kx] -> real rows out[b][y][x] (the inverse along
// x; the 1/N^2 is already in Mn), two rows per complex transform.
template <int N, int V = 0>
__global__ void __launch_bounds__(Geo<N, V>::THREADS) k_c2r_rows(Dev d, double* __restrict__ out) {
  using G = Geo<N, V>;
  extern __shared__ double2 sm[];
  double* T = reinterpret_cast<double*>(sm);
  double2* a = sm + FoldInfo<N, V>::PADDED / 2;
  const int bm = blockIdx.y, y0 = 2 * blockIdx.x;
  load_fold<N, V>(T, d.fold);
  const double2* M = d.Mn + (size_t)bm * G::Kc * 2 * N + y0;  // field 0, rows y0 and y0 + 1
  pack_rows<N, G::THREADS, 2 * N>(a, M, M + 1);
  __syncthreads();
  fft_folded<N, V, +1, 1, G::K>(a, T);
  double* r0 = out + ((size_t)bm * N + y0) * N;
  #pragma unroll
  for (int x = threadIdx.x; x < N; x += G::THREADS) {
    r0[x] = a[x].x;
    r0[N + x] = a[x].y;
  }
}

// Compact spectrum src[b] times a multiplier (and 1/N^2), transformed along
// y -> mixed Mn[b] (first field).  grid (Kc, B).
template <int N, int V = 0>
__global__ void __launch_bounds__(Geo<N, V>::THREADS) k_spec_to_mixed(Dev d, const double2* __restrict__ src, int mode) {
  using G = Geo<N, V>;
  extern __shared__ double2 sm[];
  double* T = reinterpret_cast<double*>(sm);
  double2* a = sm + FoldInfo<N, V>::PADDED / 2;
  const int kx = blockIdx.x, bm = blockIdx.y;
  load_fold<N, V>(T, d.fold);
  const double s = 1.0 / ((double)N * N);
  #pragma unroll
  for (int q = threadIdx.x; q < N; q += G::THREADS) {
    const int ky = q < N / 2 ? q : q - N;
    double2 v = make_double2(0.0, 0.0);
    if (ky >= -G::K && ky <= G::K) {
      const int r = ky >= 0 ? ky : ky + G::Kr;
      const size_t idx = cidx<N>(bm, r, kx);
      const double m = d.mult[idx];
      double f;
      if (mode == M_ONE) f = 1.0;
      else if (mode == M_CTRL) f = m;
      else if (mode == M_FILTERED) f = (kx == 0 && ky == 0) ? 0.0 : m * m / sqrt((double)(kx * kx + ky * ky));
      else f = m != 0.0 ? 1.0 / m : 0.0;
      v = cscale(src[idx], f * s);
    }
    a[q] = v;
  }
  __syncthreads();
  fft_folded<N, V, +1, 1, G::K>(a, T);
  double2* M = d.Mn + ((size_t)bm * G::Kc + kx) * 2 * N;  // field 0 of column kx
  #pragma unroll
  for (int y = threadIdx.x; y < N; y += G::THREADS) M[y] = a[y];
}

// Compact <-> half-spectrum copies.  grid (ceil(N*NH/256), B), block 256.
template <int N, int V = 0>
__global__ void k_compact_to_half(const double2* __restrict__ src, double2* __restrict__ out) {
  using G = Geo<N, V>;
  const int bm = blockIdx.y;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N * G::NH; i += gridDim.x * blockDim.x) {
    const int q = i / G::NH, p = i - q * G::NH;
    const int ky = q < N / 2 ? q : q - N;
    double2 v = make_double2(0.0, 0.0);
    if (p <= G::K && ky >= -G::K && ky <= G::K) {
      const int r = ky >= 0 ? ky : ky + G::Kr;
      v = src[cidx<N>(bm, r, p)];
    }
    out[(size_t)bm * N * G::NH + i] = v;
  }
}

template <int N, int V = 0>
__global__ void k_half_to_compact(const double2* __restrict__ in, double2* __restrict__ dst) {
  using G = Geo<N, V>;
  const int bm = blockIdx.y;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < G::Kr * G::Kc; i += gridDim.x * blockDim.x) {
    const int kx = i / G::Kr, r = i - kx * G::Kr;
    const int ky = ky_of_row(r, G::K);
    dst[(size_t)bm * G::Kr * G::Kc + i] = in[((size_t)bm * N + (ky & (N - 1))) * G::NH + kx];
  }
}

// ---------------------------------------------------------------------------
// Control map and the inverse column transforms of a stage state
// ---------------------------------------------------------------------------

// Writes the two column values u = i ky/k^2 Yv, v = -i kx/k^2 Yv (scaled by
// 1/N^2; f = symF entry of the mode) into position q of seq[0..1][N].
template <int N, int V = 0>
__device__ __forceinline__ void put_stage_columns(double2* seq, int q, const Sym4& f, double2 Yv) {
  seq[q] = make_double2(-f.a * Yv.y, f.a * Yv.x);      // u:  i ky / k^2
  seq[N + q] = make_double2(f.b * Yv.y, -f.b * Yv.x);  // v: -i kx / k^2
}

// Writes the two column values of the adjoint fields of an adjoint stage
// value kb: 2a = 2 d_xy kb = -2 kx ky kb and b = (d_xx - d_yy) kb =
// (ky^2 - kx^2) kb, scaled by 1/N^2 (g = symA entry of the mode), at q.
template <int N, int V = 0>
__device__ __forceinline__ void put_adjoint_columns(double2* seq, int q, const Sym4& g, double2 kb) {
  seq[q] = cscale(kb, g.c);
  seq[N + q] = cscale(kb, g.d);
}

// Zeroes the positions outside the retained set in `nseq` sequences.
template <int N, int V = 0>
__device__ __forceinline__ void zero_outside(double2* seq, int nseq) {
  constexpr int K = Geo<N, V>::K, GAP = N - 2 * K - 1;
  for (int u = threadIdx.x; u < nseq * GAP; u += blockDim.x) {
    const int f = u / GAP, q = K + 1 + (u - f * GAP);
    seq[f * N + q] = make_double2(0.0, 0.0);
  }
}

// The two transformed columns of seq -> column kx of both fields of Mx[bm].
template <int N, int V = 0>
__device__ __forceinline__ void store_mixed2(const Dev& d, const double2* z, int bm, int kx) {
  using G = Geo<N, V>;
  double2* M = d.Mx + (size_t)bm * 2 * N * G::Kc + kx;
#pragma unroll
  for (int t = 0; t < (2 * N + G::THREADS - 1) / G::THREADS; ++t) {
    const int u = threadIdx.x + t * G::THREADS;
    if (u < 2 * N) M[(size_t)u * G::Kc] = z[u];
  }
}

// Column kx of the first F fields of the column-major Mn (M points at the
// column: F * N contiguous entries, field-major) into seq[f*N + y], with a
// compile-time trip count.
template <int N, int T, int F>
__device__ __forceinline__ void load_column(double2* seq, const double2* __restrict__ M) {
#pragma unroll
  for (int t = 0; t < (F * N + T - 1) / T; ++t) {
    const int u = threadIdx.x + t * T;
    if (u < F * N) seq[u] = M[u];
  }
}

// Both rows y0, y0+1 of the two fields of a mixed buffer, packed for the
// inverse transform along x: sequence rr holds row y0+rr of (field 0,
// field 1) as field0 + i field1.
template <int N, int V = 0>
__device__ __forceinline__ void pack_field_pairs(double2* a, const double2* __restrict__ M, int y0) {
  constexpr int Kc = Geo<N, V>::Kc;
#pragma unroll
  for (int rr = 0; rr < 2; ++rr)
    pack_rows<N, Geo<N, V>::THREADS>(a + rr * N, M + (size_t)(y0 + rr) * Kc, M + ((size_t)N + y0 + rr) * Kc);
}

// Forward transforms along x of rows y0, y0+1, sequence rr packed as
// (field 0 of row y0+rr) + i (field 1 of row y0+rr) -> twice the two fields
// of both rows in the column-major mixed buffer O = Mn of the member
// (kx <= K): entry (kx, f, y) at (kx * 2 + f) * N + y.
template <int N, int V = 0>
__device__ __forceinline__ void unpack_row_pairs(const double2* a, double2* __restrict__ O, int y0) {
  using G = Geo<N, V>;
#pragma unroll
  for (int t = 0; t < (2 * G::Kc + G::THREADS - 1) / G::THREADS; ++t) {
    const int u = threadIdx.x + t * G::THREADS;
    if (u < 2 * G::Kc) {
      const int rr = u / G::Kc, kx = u - rr * G::Kc;
      double2 A, Bv;
      unpack_pair2<N>(a + rr * N, kx, A, Bv);
      double2* o = O + (size_t)kx * 2 * N + y0 + rr;
      o[0] = A;
      o[N] = Bv;
    }
  }
}

// s_hat = forward transform along y of the mixed rows in Mn; w0 = mult s_hat
// into W (and Y); then, unless F_NO_NEXT, the inverse column transforms of
// u and v of stage 1.  grid (Kc, B).
template <int N, int V = 0>
__global__ void __launch_bounds__(Geo<N, V>::THREADS) k_ctrl_cols(Dev d, int flags) {
  using G = Geo<N, V>;
  extern __shared__ double2 sm[];
  double* T = reinterpret_cast<double*>(sm);
  double2* a = sm + FoldInfo<N, V>::PADDED / 2;
  const int kx = blockIdx.x, bm = blockIdx.y;
  load_fold<N, V>(T, d.fold);
  load_column<N, G::THREADS, 1>(a, d.Mn + ((size_t)bm * G::Kc + kx) * 2 * N);
  __syncthreads();
  fft_folded<N, V, -1, 1, -1, G::K>(a, T);
  // each retained position is read and rewritten by one thread only
  #pragma unroll
  for (int rr = threadIdx.x; rr < G::Kr; rr += G::THREADS) {
    const int ky = ky_of_row(rr, G::K);
    const size_t idx = cidx<N>(bm, rr, kx);
    const double2 w0 = cscale(a[ky & (N - 1)], d.mult[idx]);
    d.W[idx] = w0;
    d.Y[idx] = w0;
    put_stage_columns<N>(a, ky & (N - 1), d.symF[kx * G::Kr + rr], w0);
  }
  if (flags & F_NO_NEXT) return;
  zero_outside<N>(a, 2);
  __syncthreads();
  fft_folded<N, V, +1, 2, G::K>(a, T);
  store_mixed2<N, V>(d, a, bm, kx);
}

// Restart from the compact state in W (a checkpoint): Y = W and the inverse
// column transforms of u and v of stage 1.  grid (Kc, B).
template <int N, int V = 0>
__global__ void __launch_bounds__(Geo<N, V>::THREADS) k_state_cols(Dev d) {
  using G = Geo<N, V>;
  extern __shared__ double2 sm[];
  double* T = reinterpret_cast<double*>(sm);
  double2* a = sm + FoldInfo<N, V>::PADDED / 2;
  const int kx = blockIdx.x, bm = blockIdx.y;
  load_fold<N, V>(T, d.fold);
  zero_outside<N>(a, 2);
  #pragma unroll
  for (int rr = threadIdx.x; rr < G::Kr; rr += G::THREADS) {
    const int ky = ky_of_row(rr, G::K);
    const size_t idx = cidx<N>(bm, rr, kx);
    const double2 w = d.W[idx];
    d.Y[idx] = w;
    put_stage_columns<N>(a, ky & (N - 1), d.symF[kx * G::Kr + rr], w);
  }
  __syncthreads();
  fft_folded<N, V, +1, 2, G::K>(a, T);
  store_mixed2<N, V>(d, a, bm, kx);
}

// ---------------------------------------------------------------------------
// Forward RK stage
// ---------------------------------------------------------------------------

// Row pass of stage `stage` (1..4) of step n: u, v of rows y0, y0+1; the
// stage-field store and probe gather; the products u v and v^2 - u^2 of
// each row (packed as P + i Q) and their forward transforms along x into
// Mn.  grid (N/2, B).
template <int N, int V = 0>
__global__ void __launch_bounds__(Geo<N, V>::THREADS) k_fwd_rows(Dev d, int n, int stage, int flags) {
  using G = Geo<N, V>;
  extern __shared__ double2 sm[];
  double* T = reinterpret_cast<double*>(sm);
  double2* a = sm + FoldInfo<N, V>::PADDED / 2;
  const int bm = blockIdx.y, y0 = 2 * blockIdx.x;
  const MemberWindow mw = member_window(d, bm);
  if (n < mw.start) return;  // the member's window has not begun
  load_fold<N, V>(T, d.fold);
  pack_field_pairs<N, V>(a, d.Mx + (size_t)bm * 2 * N * G::Kc, y0);
  __syncthreads();
  const int P = mw.P, st = N / P;
  const int slot = (flags & (F_OBS | F_OBS_ONLY)) ? obs_slot(d, n - mw.start) : -1;
  double* trj = (flags & F_STORE)
                    ? d.traj + (((size_t)bm * d.traj_steps + (n - d.seg0)) * 4 + (stage - 1)) * 2 * (size_t)N * N
                    : nullptr;
  // (u, v) at column x of row y0 + rr: stage-field store, probe gather, and
  // the products P = u v, Q = v^2 - u^2 as P + i Q
  auto products = [&](int rr, int x, double2 uv) {
    const int y = y0 + rr;
    if (trj) {
      const size_t o = (size_t)y * N + x;
      trj[o] = uv.x;
      trj[(size_t)N * N + o] = uv.y;
    }
    if (slot >= 0 && (y % st) == 0 && (x % st) == 0) {
      const int p = (y / st) * P + x / st;
      double* o = d.obs + bm * d.obs_stride + ((size_t)slot * P * P + p) * 2;
      o[0] = uv.x;
      o[1] = uv.y;
    }
    return make_double2(uv.x * uv.y, fma(uv.y, uv.y, -uv.x * uv.x));
  };
  if (flags & F_OBS_ONLY) {  // the final state: stage fields and probes only
    fft_folded<N, V, +1, 2, G::K>(a, T);
    for (int u = threadIdx.x; u < 2 * N; u += G::THREADS) products(u / N, u % N, a[u]);
    return;
  }
  if constexpr (Fusable<N, V>::value) {
    fft_folded_turn<N, V, 2, G::K, G::K>(a, T, products);
  } else {
    fft_folded<N, V, +1, 2, G::K>(a, T);
    // each position is read and rewritten by one thread only
#pragma unroll
    for (int t = 0; t < (2 * N + G::THREADS - 1) / G::THREADS; ++t) {
      const int u = threadIdx.x + t * G::THREADS;
      if (u < 2 * N) a[u] = products(u / N, u % N, a[u]);
    }
    __syncthreads();
    fft_folded<N, V, -1, 2, -1, G::K>(a, T);
  }
  unpack_row_pairs<N, V>(a, d.Mn + (size_t)bm * G::Kc * 2 * N, y0);
}

// Column pass of stage `stage`: the advection term
//   n_hat = (ky^2 - kx^2) DFT(u v) - kx ky DFT(v^2 - u^2),
// k_j = -n_hat - nu k^2 y_j + f_hat, the RK4 update, and the inverse column
// transforms of u and v of the next stage state.  Acc holds k1 + 2 k2 +
// 2 k3 (+ k4).  grid (Kc, B).
template <int N, int V = 0>
__global__ void __launch_bounds__(Geo<N, V>::THREADS) k_fwd_cols(Dev d, int n, int stage, int flags) {
  using G = Geo<N, V>;
  extern __shared__ double2 sm[];
  double* T = reinterpret_cast<double*>(sm);
  double2* a = sm + FoldInfo<N, V>::PADDED / 2;
  const int kx = blockIdx.x, bm = blockIdx.y;
  const MemberWindow mw = member_window(d, bm);
  if (n < mw.start) return;
  load_fold<N, V>(T, d.fold);
  load_column<N, G::THREADS, 2>(a, d.Mn + ((size_t)bm * G::Kc + kx) * 2 * N);
  // the epilogue's inputs for this thread's modes; where registers allow
  // (G::PREFETCH), loaded now so that their latency hides behind the
  // column transforms
  constexpr int MT = (G::Kr + G::THREADS - 1) / G::THREADS;
  double2 yv[MT], wv[MT], accv[MT];
  Sym4 f[MT];
  double nk2[MT];
  auto load_inputs = [&](int t) {
    const int rr = threadIdx.x + t * G::THREADS;
    if (rr < G::Kr) {
      const size_t idx = cidx<N>(bm, rr, kx);
      yv[t] = d.Y[idx];
      wv[t] = d.W[idx];
      accv[t] = stage > 1 ? d.Acc[idx] : make_double2(0.0, 0.0);
      f[t] = d.symF[kx * G::Kr + rr];
      nk2[t] = mw.nu * d.k2[kx * G::Kr + rr];
    }
  };
  if constexpr (G::PREFETCH) {
#pragma unroll
    for (int t = 0; t < MT; ++t) load_inputs(t);
  }
  __syncthreads();
  fft_folded<N, V, -1, 2, -1, G::K>(a, T);
  const double dt = d.dt;
  const double fval = -d.amp * d.nf * (double)N * N / 2.0;
  // each retained position is read and rewritten (both sequences) by one
  // thread only
#pragma unroll
  for (int t = 0; t < MT; ++t) {
    const int rr = threadIdx.x + t * G::THREADS;
    if (rr >= G::Kr) break;
    if constexpr (!G::PREFETCH) load_inputs(t);
    const int ky = ky_of_row(rr, G::K);
    const int qi = ky & (N - 1);
    const size_t idx = cidx<N>(bm, rr, kx);
    const double2 ph = a[qi], qh = a[N + qi];
    // F = -(cp P + cq Q) - nu k^2 y
    double2 F = make_double2(-fma(f[t].c, ph.x, fma(f[t].d, qh.x, nk2[t] * yv[t].x)),
                             -fma(f[t].c, ph.y, fma(f[t].d, qh.y, nk2[t] * yv[t].y)));
    if (mw.forced && kx == 0 && (ky == d.nf || ky == -d.nf)) F.x += fval;
    const double2 w = wv[t], acc = accv[t];
    double2 ynext;
    if (stage == 1) {
      d.Acc[idx] = F;
      ynext = make_double2(fma(d.dt2, F.x, w.x), fma(d.dt2, F.y, w.y));
    } else if (stage == 2) {
      d.Acc[idx] = make_double2(fma(2.0, F.x, acc.x), fma(2.0, F.y, acc.y));
      ynext = make_double2(fma(d.dt2, F.x, w.x), fma(d.dt2, F.y, w.y));
    } else if (stage == 3) {
      d.Acc[idx] = make_double2(fma(2.0, F.x, acc.x), fma(2.0, F.y, acc.y));
      ynext = make_double2(fma(dt, F.x, w.x), fma(dt, F.y, w.y));
    } else {
      ynext = make_double2(fma(d.dt6, acc.x + F.x, w.x), fma(d.dt6, acc.y + F.y, w.y));
      d.W[idx] = ynext;
    }
    d.Y[idx] = ynext;
    put_stage_columns<N>(a, qi, f[t], ynext);
  }
  if (flags & F_NO_NEXT) return;
  zero_outside<N>(a, 2);
  __syncthreads();
  fft_folded<N, V, +1, 2, G::K>(a, T);
  store_mixed2<N, V>(d, a, bm, kx);
}

// r = model observations - data and J = 1/2 sum r^2 per member, in a fixed
// order (deterministic).  grid B, block 256.  Defined in residual.cu.
__global__ void k_residual(Dev d);

// Regularisation of Eq. (4): J[b] += lambda/2 sum_grid w0^2, from the compact
// initial spectrum w0 (sum_grid w^2 = 1/N^2 sum over the full spectrum).
// grid B, block 256.  Defined in residual.cu.
__global__ void k_sobolev_cost(double* J, const double2* w0, double lambda, int N, int Kr, int Kc);

// Shell energies of the adjoint velocity, per member and of the ensemble
// mean.  Defined in residual.cu.
__global__ void k_shell_member(const double2* lam, const int* off, const int* mode, const double* wgt, int nmodes,
                               double* out, int nshell);
__global__ void k_shell_mean(const double2* lam, int B, const int* off, const int* mode, const double* wgt, int nmodes,
                             double* out);

// LamBar[b] += lambda w0[b] on the compact set.  Defined in residual.cu.
__global__ void k_sobolev_grad(double2* lam, const double2* w0, double lambda, int count);

// ---------------------------------------------------------------------------
// Adjoint
// ---------------------------------------------------------------------------
//
// The tangent of the advection term at (u, v) is
//   dn = (d_xx - d_yy)(u dv + v du) + d_xy (2 v dv - 2 u du),
// so its transpose applied to kbar is, with a = IDFT(d_xy kbar) and
// b = IDFT((d_xx - d_yy) kbar) on the grid,
//   rho_u = v b - 2 u a,   rho_v = u b + 2 v a,
//   J^T kbar = -P[(-i ky/k^2) DFT(rho_u) + (i kx/k^2) DFT(rho_v)] - nu k^2 kbar,
// the transposes of du = IDFT(i ky/k^2 dw), dv = IDFT(-i kx/k^2 dw).

// Separable DFT of the residual at observation slot `slot` on the probe
// lattice: for each lattice row, T(kx) = sum_q r[row][q] W_P^{kx q}; the
// column pass then sums over rows with W_P^{ky row}.  Fills Tu, Tv [P].
__device__ __forceinline__ void probe_row_sums(const Dev& d, int bm, int P, int slot, int kx, double2* Tu,
                                               double2* Tv) {
  const double* r = d.res + bm * d.obs_stride + (size_t)slot * P * P * 2;
  const int tws = 64 / P;
  for (int row = threadIdx.x; row < P; row += blockDim.x) {
    double2 su = make_double2(0.0, 0.0), sv = make_double2(0.0, 0.0);
    for (int qq = 0; qq < P; ++qq) {
      const double2 w = d.twP[((kx * qq) % P) * tws];
      const double ru = r[(row * P + qq) * 2], rv = r[(row * P + qq) * 2 + 1];
      su = make_double2(fma(ru, w.x, su.x), fma(ru, w.y, su.y));
      sv = make_double2(fma(rv, w.x, sv.x), fma(rv, w.y, sv.y));
    }
    Tu[row] = su;
    Tv[row] = sv;
  }
}

// H^T r at (kx, ky): (-i ky/k^2) R_u + (i kx/k^2) R_v with R the DFT of the
// probe residual scattered onto the grid.
__device__ __forceinline__ double2 probe_source(const Dev& d, int P, int kx, int ky, const double2* Tu,
                                                const double2* Tv) {
  double2 Ru = make_double2(0.0, 0.0), Rv = make_double2(0.0, 0.0);
  const int kyp = ((ky % P) + P) % P;
  const int tws = 64 / P;
  for (int row = 0; row < P; ++row) {
    const double2 w = d.twP[((kyp * row) % P) * tws];
    Ru = cadd(Ru, cmul(Tu[row], w));
    Rv = cadd(Rv, cmul(Tv[row], w));
  }
  const double k2 = (double)(kx * kx + ky * ky);
  const double ik2 = k2 > 0.0 ? 1.0 / k2 : 0.0;
  const double a = ky * ik2, c = kx * ik2;
  // (-i a) Ru + (i c) Rv
  return make_double2(a * Ru.y - c * Rv.y, -a * Ru.x + c * Rv.x);
}

// Start of the adjoint sweep: LamBar = (terminal field in LamBar, with
// INIT_LAMBAR) + (H^T r at the last step, with INIT_SRC), KB = dt/6 LamBar;
// with INIT_RESUME, KB as it stands (after a checkpoint recompute).  Then
// the inverse column transforms of the adjoint fields a, b of KB into Mx.
// grid (Kc, B).
template <int N, int V = 0>
__global__ void __launch_bounds__(Geo<N, V>::THREADS) k_adj_init(Dev d, int mode) {
  using G = Geo<N, V>;
  extern __shared__ double2 sm[];
  double* T = reinterpret_cast<double*>(sm);
  double2 *a = sm + FoldInfo<N, V>::PADDED / 2, *Tu = a + 2 * N, *Tv = Tu + G::PMAX;
  const int kx = blockIdx.x, bm = blockIdx.y;
  load_fold<N, V>(T, d.fold);
  const MemberWindow mw = member_window(d, bm);
  // an idle member starts (and stays) at lambda = 0
  if (mw.start > d.nsteps) mode = 0;
  const bool resume = (mode & INIT_RESUME) != 0;
  const int slot = (!resume && (mode & INIT_SRC)) ? obs_slot(d, d.nsteps - mw.start) : -1;
  if (slot >= 0) probe_row_sums(d, bm, mw.P, slot, kx, Tu, Tv);
  zero_outside<N>(a, 2);
  __syncthreads();
  #pragma unroll
  for (int rr = threadIdx.x; rr < G::Kr; rr += G::THREADS) {
    const int ky = ky_of_row(rr, G::K);
    const size_t idx = cidx<N>(bm, rr, kx);
    double2 kb;
    if (resume) {
      kb = d.KB[idx];
    } else {
      double2 lam = (mode & INIT_LAMBAR) ? d.LamBar[idx] : make_double2(0.0, 0.0);
      if (slot >= 0) lam = cadd(lam, probe_source(d, mw.P, kx, ky, Tu, Tv));
      d.LamBar[idx] = lam;
      kb = cscale(lam, d.dt6);
      d.KB[idx] = kb;
    }
    put_adjoint_columns<N>(a, ky & (N - 1), d.symA[kx * G::Kr + rr], kb);
  }
  __syncthreads();
  fft_folded<N, V, +1, 2, G::K>(a, T);
  store_mixed2<N, V>(d, a, bm, kx);
}

// Adjoint row pass of stage `stage` of step n: 2a, b of rows y0, y0+1
// (inverse transforms along x), rho_u and rho_v with the stored u, v (each
// row packed as rho_u + i rho_v), and their forward transforms along x into
// Mn (twice, as in the forward row pass).  grid (N/2, B).
template <int N, int V = 0>
__global__ void __launch_bounds__(Geo<N, V>::THREADS) k_adj_rows(Dev d, int n, int stage) {
  using G = Geo<N, V>;
  extern __shared__ double2 sm[];
  double* T = reinterpret_cast<double*>(sm);
  double2* a = sm + FoldInfo<N, V>::PADDED / 2;
  const int bm = blockIdx.y, y0 = 2 * blockIdx.x;
  if (d.ragged && n < d.mstart[bm]) return;
  load_fold<N, V>(T, d.fold);
  pack_field_pairs<N, V>(a, d.Mx + (size_t)bm * 2 * N * G::Kc, y0);
  __syncthreads();
  const double* trj = d.traj + (((size_t)bm * d.traj_steps + (n - d.seg0)) * 4 + (stage - 1)) * 2 * (size_t)N * N;
  // (2a, b) at column x of row y0 + rr -> rho_u + i rho_v with the stored u, v
  auto rho = [&](int rr, int x, double2 ab) {
    const size_t o = (size_t)(y0 + rr) * N + x;
    const double fu = trj[o], fv = trj[(size_t)N * N + o];
    return make_double2(fma(fv, ab.y, -fu * ab.x), fma(fu, ab.y, fv * ab.x));
  };
  if constexpr (Fusable<N, V>::value) {
    fft_folded_turn<N, V, 2, G::K, G::K>(a, T, rho);
  } else {
    fft_folded<N, V, +1, 2, G::K>(a, T);
    // each position is read and rewritten by one thread only
#pragma unroll
    for (int t = 0; t < (2 * N + G::THREADS - 1) / G::THREADS; ++t) {
      const int u = threadIdx.x + t * G::THREADS;
      if (u < 2 * N) a[u] = rho(u / N, u % N, a[u]);
    }
    __syncthreads();
    fft_folded<N, V, -1, 2, -1, G::K>(a, T);
  }
  unpack_row_pairs<N, V>(a, d.Mn + (size_t)bm * G::Kc * 2 * N, y0);
}

// Adjoint column pass of stage `stage` of step n:
//   ybar_j = -P[(-i ky/k^2) DFT(rho_u) + (i kx/k^2) DFT(rho_v)] - nu k^2 kbar_j,
// the transposed RK4 combination, the observation source at step n (on
// stage 1), and the inverse column transforms of a, b of the next kbar.
// grid (Kc, B).
template <int N, int V = 0>
__global__ void __launch_bounds__(Geo<N, V>::THREADS) k_adj_cols(Dev d, int n, int stage, int flags) {
  using G = Geo<N, V>;
  extern __shared__ double2 sm[];
  double* T = reinterpret_cast<double*>(sm);
  double2 *a = sm + FoldInfo<N, V>::PADDED / 2, *Tu = a + 2 * N, *Tv = Tu + G::PMAX;
  const int kx = blockIdx.x, bm = blockIdx.y;
  const MemberWindow mw = member_window(d, bm);
  if (n < mw.start) return;
  load_fold<N, V>(T, d.fold);
  load_column<N, G::THREADS, 2>(a, d.Mn + ((size_t)bm * G::Kc + kx) * 2 * N);
  // the epilogue's inputs for this thread's modes (before the column
  // transforms where registers allow, as in k_fwd_cols)
  constexpr int MT = (G::Kr + G::THREADS - 1) / G::THREADS;
  double2 kbv[MT], lbv[MT], sumv[MT];
  Sym4 g[MT];
  double nk2[MT];
  auto load_inputs = [&](int t) {
    const int rr = threadIdx.x + t * G::THREADS;
    if (rr < G::Kr) {
      const size_t idx = cidx<N>(bm, rr, kx);
      kbv[t] = d.KB[idx];
      lbv[t] = d.LamBar[idx];
      sumv[t] = stage < 4 ? d.Sum[idx] : make_double2(0.0, 0.0);
      g[t] = d.symA[kx * G::Kr + rr];
      nk2[t] = mw.nu * d.k2[kx * G::Kr + rr];
    }
  };
  if constexpr (G::PREFETCH) {
#pragma unroll
    for (int t = 0; t < MT; ++t) load_inputs(t);
  }
  const int slot = (flags & F_SRC) ? obs_slot(d, n - mw.start) : -1;
  if (slot >= 0) probe_row_sums(d, bm, mw.P, slot, kx, Tu, Tv);
  __syncthreads();
  fft_folded<N, V, -1, 2, -1, G::K>(a, T);
  const double dt = d.dt;
  // each retained position is read and rewritten (both sequences) by one
  // thread only
#pragma unroll
  for (int t = 0; t < MT; ++t) {
    const int rr = threadIdx.x + t * G::THREADS;
    if (rr >= G::Kr) break;
    if constexpr (!G::PREFETCH) load_inputs(t);
    const int ky = ky_of_row(rr, G::K);
    const int qi = ky & (N - 1);
    const size_t idx = cidx<N>(bm, rr, kx);
    const double2 Ru = a[qi], Rv = a[N + qi];
    // t = (-i ky/k^2) Ru + (i kx/k^2) Rv (the 1/2 of the row unpack in a1, c1)
    const double2 tt = make_double2(fma(g[t].a, Ru.y, -g[t].b * Rv.y), fma(-g[t].a, Ru.x, g[t].b * Rv.x));
    const double2 kb = kbv[t], lb = lbv[t];
    double2 yb;
    yb.x = -fma(nk2[t], kb.x, tt.x);
    yb.y = -fma(nk2[t], kb.y, tt.y);
    double2 nk;
    if (stage == 4) {
      d.Sum[idx] = yb;
      nk = make_double2(fma(d.dt3, lb.x, dt * yb.x), fma(d.dt3, lb.y, dt * yb.y));
    } else if (stage == 3) {
      d.Sum[idx] = cadd(sumv[t], yb);
      nk = make_double2(fma(d.dt3, lb.x, d.dt2 * yb.x), fma(d.dt3, lb.y, d.dt2 * yb.y));
    } else if (stage == 2) {
      d.Sum[idx] = cadd(sumv[t], yb);
      nk = make_double2(fma(d.dt6, lb.x, d.dt2 * yb.x), fma(d.dt6, lb.y, d.dt2 * yb.y));
    } else {
      const double2 sum = cadd(sumv[t], yb);
      double2 lam = cadd(lb, sum);
      if (slot >= 0) lam = cadd(lam, probe_source(d, mw.P, kx, ky, Tu, Tv));
      d.LamBar[idx] = lam;
      nk = cscale(lam, d.dt6);
    }
    d.KB[idx] = nk;
    put_adjoint_columns<N>(a, qi, g[t], nk);
  }
  if (stage == 1 && n == mw.start) return;  // the member's first step: lambda_0 stays in LamBar
  zero_outside<N>(a, 2);
  __syncthreads();
  fft_folded<N, V, +1, 2, G::K>(a, T);
  store_mixed2<N, V>(d, a, bm, kx);
}

// Control multipliers m(k) = |k| W(k)^{1/2} on the retained set (0 at k = 0),
// per member.  grid (ceil(Kr*Kc/256), B), block 256.
template <int N, int V = 0>
__global__ void k_make_mult(double* __restrict__ mult, const int* __restrict__ kind, const double* __restrict__ param,
                            const double* __restrict__ table, const double* __restrict__ nu) {
  using G = Geo<N, V>;
  const int bm = blockIdx.y;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < G::Kr * G::Kc; i += gridDim.x * blockDim.x) {
    const int kx = i / G::Kr, r = i - kx * G::Kr;
    const int ky = ky_of_row(r, G::K);
    const double k2 = (double)(kx * kx + ky * ky);
    const double k = sqrt(k2);
    double W;
    const double a = param[bm];
    switch (kind[bm]) {
      case 0: W = 1.0; break;
      case 1: W = exp(-a * k); break;
      case 2: W = pow(k, -2.0 * a); break;
      case 3: W = exp(-nu[bm] * a * k2); break;
      default: W = table[((size_t)bm * N + (ky & (N - 1))) * G::NH + kx]; break;
    }
    mult[(size_t)bm * G::Kr * G::Kc + i] = (kx == 0 && ky == 0) ? 0.0 : k * sqrt(W);
  }
}

}  // namespace da
