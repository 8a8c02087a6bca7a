// ops.h -- per-grid-size table of kernel launchers (one translation unit per
// size instantiates the templates of kernels.cuh).
#pragma once
#include <cuda_runtime.h>

#include "kernels.cuh"

namespace da {

struct Ops {
  int n, K, Kc, Kr;
  int fold_doubles;                 // entries of the folded twiddle table
  void (*fold_table)(double* out);  // fills it on the host
  cudaError_t (*setup)();
  void (*r2c_rows)(const Dev&, const double* in, cudaStream_t);
  void (*c2r_rows)(const Dev&, double* out, cudaStream_t);
  void (*spec_to_mixed)(const Dev&, const double2* src, int mode, cudaStream_t);
  void (*compact_to_half)(const Dev&, const double2* src, double2* out, cudaStream_t);
  void (*half_to_compact)(const Dev&, const double2* in, double2* dst, cudaStream_t);
  void (*ctrl_cols)(const Dev&, int flags, cudaStream_t);
  void (*fwd_rows)(const Dev&, int n, int stage, int flags, cudaStream_t);
  void (*fwd_cols)(const Dev&, int stage, int flags, cudaStream_t);
  void (*state_cols)(const Dev&, cudaStream_t);
  void (*adj_init)(const Dev&, int mode, cudaStream_t);
  void (*adj_rows)(const Dev&, int n, int stage, cudaStream_t);
  void (*adj_cols)(const Dev&, int n, int stage, int flags, cudaStream_t);
  void (*make_mult)(const Dev&, double* mult, const int* kind, const double* param, const double* table, double nu,
                    cudaStream_t);
};

const Ops* ops_n16();
const Ops* ops_n32();
const Ops* ops_n64();
const Ops* ops_n128();
const Ops* ops_n256();
const Ops* ops_n512();
const Ops* ops_n1024();

inline const Ops* ops_for(int n) {
  switch (n) {
    case 16: return ops_n16();
    case 32: return ops_n32();
    case 64: return ops_n64();
    case 128: return ops_n128();
    case 256: return ops_n256();
    case 512: return ops_n512();
    case 1024: return ops_n1024();
    default: return nullptr;
  }
}

}  // namespace da
