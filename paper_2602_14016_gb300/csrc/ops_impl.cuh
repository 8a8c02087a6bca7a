// ops_impl.cuh -- launch configurations of the pass kernels for one N.
#pragma once
#include "ops.h"

namespace da {

template <int N, int V>
Ops make_ops() {
  using G = Geo<N, V>;
  Ops o{};
  o.n = N;
  o.K = G::K;
  o.Kc = G::Kc;
  o.Kr = G::Kr;
  o.variant = V;
  o.threads = G::THREADS;
  o.fold_doubles = FoldInfo<N, V>::DOUBLES;
  o.flops_inverse = band_transform_flops<N, V, G::K>(true);
  o.flops_forward = band_transform_flops<N, V, G::K>(false);
  o.fold_table = [](double* out) { fold_table<N, V>(out); };
  o.setup = []() -> cudaError_t {
    const int s = (int)G::SMEM;
    cudaError_t e = cudaSuccess;
    auto set = [&](const void* f) {
      if (e == cudaSuccess) e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, s);
    };
    set((const void*)k_r2c_rows<N, V>);
    set((const void*)k_c2r_rows<N, V>);
    set((const void*)k_spec_to_mixed<N, V>);
    set((const void*)k_ctrl_cols<N, V>);
    set((const void*)k_fwd_rows<N, V>);
    set((const void*)k_fwd_cols<N, V>);
    set((const void*)k_state_cols<N, V>);
    set((const void*)k_adj_init<N, V>);
    set((const void*)k_adj_rows<N, V>);
    set((const void*)k_adj_cols<N, V>);
    return e;
  };
  o.r2c_rows = [](const Dev& d, const double* in, cudaStream_t st) {
    k_r2c_rows<N, V><<<dim3(N / 2, d.B), G::THREADS, G::SMEM, st>>>(d, in);
  };
  o.c2r_rows = [](const Dev& d, double* out, cudaStream_t st) {
    k_c2r_rows<N, V><<<dim3(N / 2, d.B), G::THREADS, G::SMEM, st>>>(d, out);
  };
  o.spec_to_mixed = [](const Dev& d, const double2* src, int mode, cudaStream_t st) {
    k_spec_to_mixed<N, V><<<dim3(G::Kc, d.B), G::THREADS, G::SMEM, st>>>(d, src, mode);
  };
  o.compact_to_half = [](const Dev& d, const double2* src, double2* out, cudaStream_t st) {
    k_compact_to_half<N, V><<<dim3((N * G::NH + 255) / 256, d.B), 256, 0, st>>>(src, out);
  };
  o.half_to_compact = [](const Dev& d, const double2* in, double2* dst, cudaStream_t st) {
    k_half_to_compact<N, V><<<dim3((G::Kr * G::Kc + 255) / 256, d.B), 256, 0, st>>>(in, dst);
  };
  o.ctrl_cols = [](const Dev& d, int flags, cudaStream_t st) {
    k_ctrl_cols<N, V><<<dim3(G::Kc, d.B), G::THREADS, G::SMEM, st>>>(d, flags);
  };
  o.fwd_rows = [](const Dev& d, int n, int stage, int flags, cudaStream_t st) {
    k_fwd_rows<N, V><<<dim3(N / 2, d.B), G::THREADS, G::SMEM, st>>>(d, n, stage, flags);
  };
  o.fwd_cols = [](const Dev& d, int n, int stage, int flags, cudaStream_t st) {
    k_fwd_cols<N, V><<<dim3(G::Kc, d.B), G::THREADS, G::SMEM, st>>>(d, n, stage, flags);
  };
  o.state_cols = [](const Dev& d, cudaStream_t st) {
    k_state_cols<N, V><<<dim3(G::Kc, d.B), G::THREADS, G::SMEM, st>>>(d);
  };
  o.adj_init = [](const Dev& d, int mode, cudaStream_t st) {
    k_adj_init<N, V><<<dim3(G::Kc, d.B), G::THREADS, G::SMEM, st>>>(d, mode);
  };
  o.adj_rows = [](const Dev& d, int n, int stage, cudaStream_t st) {
    k_adj_rows<N, V><<<dim3(N / 2, d.B), G::THREADS, G::SMEM, st>>>(d, n, stage);
  };
  o.adj_cols = [](const Dev& d, int n, int stage, int flags, cudaStream_t st) {
    k_adj_cols<N, V><<<dim3(G::Kc, d.B), G::THREADS, G::SMEM, st>>>(d, n, stage, flags);
  };
  o.make_mult = [](const Dev& d, double* mult, const int* kind, const double* param, const double* table, const double* nu,
                   cudaStream_t st) {
    k_make_mult<N, V><<<dim3((G::Kr * G::Kc + 255) / 256, d.B), 256, 0, st>>>(mult, kind, param, table, nu);
  };
  return o;
}

}  // namespace da

#define DA_INSTANTIATE(NN, VV)                  \
  namespace da {                                \
  const Ops* ops_n##NN##_v##VV() {              \
    static const Ops o = make_ops<NN, VV>();    \
    return &o;                                  \
  }                                             \
  }
