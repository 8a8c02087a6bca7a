// ops.h -- per-grid-size table of kernel launchers (one translation unit per
// size instantiates the templates of kernels.cuh).
#pragma once
#include <cuda_runtime.h>

#include "kernels.cuh"

namespace da {

struct Ops {
  int n, K, Kc, Kr;
  int variant;                      // plan variant (fft.cuh)
  int threads;                      // CTA width of the pass kernels
  int fold_doubles;                 // entries of the folded twiddle table
  double flops_inverse;             // nominal flops of one band-limited inverse transform
  double flops_forward;             // ... and forward transform (band_transform_flops)
  void (*fold_table)(double* out);  // fills it on the host
  cudaError_t (*setup)();
  void (*r2c_rows)(const Dev&, const double* in, cudaStream_t);
  void (*c2r_rows)(const Dev&, double* out, cudaStream_t);
  void (*spec_to_mixed)(const Dev&, const double2* src, int mode, cudaStream_t);
  void (*compact_to_half)(const Dev&, const double2* src, double2* out, cudaStream_t);
  void (*half_to_compact)(const Dev&, const double2* in, double2* dst, cudaStream_t);
  void (*ctrl_cols)(const Dev&, int flags, cudaStream_t);
  void (*fwd_rows)(const Dev&, int n, int stage, int flags, cudaStream_t);
  void (*fwd_cols)(const Dev&, int n, int stage, int flags, cudaStream_t);
  void (*state_cols)(const Dev&, cudaStream_t);
  void (*adj_init)(const Dev&, int mode, cudaStream_t);
  void (*adj_rows)(const Dev&, int n, int stage, cudaStream_t);
  void (*adj_cols)(const Dev&, int n, int stage, int flags, cudaStream_t);
  void (*make_mult)(const Dev&, double* mult, const int* kind, const double* param, const double* table, const double* nu,
                    cudaStream_t);
};

const Ops* ops_n16_v0();
const Ops* ops_n32_v0();
const Ops* ops_n32_v1();
const Ops* ops_n64_v0();
const Ops* ops_n64_v1();
const Ops* ops_n64_v2();
const Ops* ops_n128_v0();
const Ops* ops_n128_v1();
const Ops* ops_n128_v2();
const Ops* ops_n128_v3();
const Ops* ops_n256_v0();
const Ops* ops_n256_v1();
const Ops* ops_n256_v2();
const Ops* ops_n512_v0();
const Ops* ops_n512_v1();
const Ops* ops_n512_v2();
const Ops* ops_n1024_v0();
const Ops* ops_n1024_v1();
const Ops* ops_n1024_v2();

// Launchers of plan variant v of size n (v < plan_count(n)), or nullptr.
inline const Ops* ops_for(int n, int v = 0) {
  if (v < 0 || v >= plan_count(n)) return nullptr;
  switch (n) {
    case 16: return ops_n16_v0();
    case 32: return v == 0 ? ops_n32_v0() : ops_n32_v1();
    case 64: return v == 0 ? ops_n64_v0() : v == 1 ? ops_n64_v1() : ops_n64_v2();
    case 128: return v == 0 ? ops_n128_v0() : v == 1 ? ops_n128_v1() : v == 2 ? ops_n128_v2() : ops_n128_v3();
    case 256: return v == 0 ? ops_n256_v0() : v == 1 ? ops_n256_v1() : ops_n256_v2();
    case 512: return v == 0 ? ops_n512_v0() : v == 1 ? ops_n512_v1() : ops_n512_v2();
    case 1024: return v == 0 ? ops_n1024_v0() : v == 1 ? ops_n1024_v1() : ops_n1024_v2();
    default: return nullptr;
  }
}

}  // namespace da
