// ctx.h -- the context behind the C ABI of include/da.h and the host
// helpers shared by the files that implement it (da_api.cu: creation,
// forward, cost and gradient, adjoint variants; plans.cu: FFT plan variants
// and the autotuner; lbfgs.cu: the optimiser).  Internal: nothing here is
// part of the ABI.
#pragma once
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <string>
#include <vector>

#include "../../include/da.h"
#include "ops.h"

using da::Dev;
using da::Ops;

struct da_ctx {
  int device = 0;
  int n = 0, nsteps = 0, ckpt = 0, B = 1;
  double dt = 0, nu = 0;
  da_forcing force{};
  da_obs_operator obs{};
  int nt = 0, P = 0;
  // ragged batches (da_set_member): per-member windows, end-aligned in each
  // evaluation's window of eval_steps steps (the longest live member's)
  bool ragged = false;
  std::vector<int> m_nsteps, m_px, m_force;
  std::vector<double> m_nu;
  int eval_steps = 0;
  int* d_mstart = nullptr;   // device tables read by the kernels (Dev)
  int* d_mnt = nullptr;
  int* d_mpx = nullptr;
  int* d_mforce = nullptr;
  double* d_mnu = nullptr;
  int* d_kind = nullptr;     // member kernels, for re-making the multiplier
  double *d_param = nullptr, *d_table = nullptr;
  std::vector<int> h_kind;
  std::vector<double> h_param;
  const Ops* ops = nullptr;
  Dev dev{};
  std::vector<void*> allocs;
  unsigned long long bytes = 0;
  unsigned long long launches = 0;
  bool have_obs = false;
  bool have_adj = false;
  bool have_fwd = false;  // a stored forward (stage fields / checkpoints) is valid
  int nckpt = 0;          // checkpoints held (ckpt > 0)
  double2* ckpt_buf = nullptr;
  double sobolev = 0.0;   // lambda of the regularisation term of Eq. (4)
  // shell lists of the adjoint spectra (built on the first da_adjoint_spectra)
  int nshell = 0;
  int *shell_off = nullptr, *shell_mode = nullptr;
  double *shell_wgt = nullptr, *shell_scratch = nullptr;
  double2* w0 = nullptr;  // compact initial state kept for that term
  std::string err;
  // optimiser buffers (allocated on the first da_assimilate; blas.cuh)
  double* lb_V = nullptr;      // vector banks [5 + 2 (mem + 1)][B][n^2]
  double* lb_scal = nullptr;   // device scalars [B][SC_COUNT]
  double* lb_J = nullptr;      // costs [B]
  int* lb_iargs = nullptr;     // argument tables of the vector kernels
  double* lb_dargs = nullptr;
  double* lb_host = nullptr;   // pinned mirror of lb_scal and lb_J
  int mem = 0;
  // optimiser state per member (lbfgs.cu), freed by free_optimiser
  void* lb_state = nullptr;
  // CUDA-graph replay of da_cost_grad (captured per evaluation window)
  bool use_graph = false;
  struct CapturedEval {
    int steps;                    // the evaluation window it was captured for
    cudaGraphExec_t exec;
    unsigned long long launches;  // kernel nodes in it
  };
  std::vector<CapturedEval> cg_cache;  // newest last, at most kMaxCapturedEvals
  cudaStream_t gstream = nullptr;
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  double *sbuf = nullptr, *gbuf = nullptr;
  // CUDA-graph replay of da_adjoint_spectra (captured per save_every and outputs)
  cudaGraphExec_t sp_exec = nullptr;
  unsigned long long sp_launches = 0;
  int sp_key = -1;
  double *sp_lbuf = nullptr, *sp_member = nullptr, *sp_mean = nullptr;
  // event timing of one kernel class
  int timed_class = 0;
  std::vector<cudaEvent_t> ev;
  size_t ev_used = 0;
};

// Captured evaluations kept per context: one per evaluation window that a
// ragged batch's live members produce (a window is the longest live horizon).
constexpr size_t kMaxCapturedEvals = 16;

// Drops every captured evaluation (their kernel arguments or launch sequence
// changed).
inline void drop_graphs(da_ctx* c) {
  for (auto& g : c->cg_cache) cudaGraphExecDestroy(g.exec);
  c->cg_cache.clear();
}

// Message of the last failed da_create (no context to hold it).
extern std::string g_create_error;

#define DA_TRY_CUDA(ctx, call)                                                                    \
  do {                                                                                            \
    cudaError_t e_ = (call);                                                                      \
    if (e_ != cudaSuccess) return fail((ctx), DA_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

inline da_status fail(da_ctx* c, da_status s, const std::string& msg) {
  if (c)
    c->err = msg;
  else
    g_create_error = msg;
  return s;
}

inline da_status check_launch(da_ctx* c, unsigned long long nlaunch = 1) {
  c->launches += nlaunch;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(c, DA_ECUDA, std::string("kernel launch: ") + cudaGetErrorString(e));
  return DA_OK;
}

// Brackets one launch of kernel class `cls` with events when that class is timed.
struct Timed {
  da_ctx* c;
  bool on;
  cudaStream_t st;
  Timed(da_ctx* c_, int cls, cudaStream_t s) : c(c_), on(c_->timed_class == cls), st(s) {
    if (!on) return;
    if (c->ev_used + 2 > c->ev.size()) {
      for (int i = 0; i < 256; ++i) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) {
          on = false;
          return;
        }
        c->ev.push_back(e);
      }
    }
    cudaEventRecord(c->ev[c->ev_used], st);
  }
  ~Timed() {
    if (!on) return;
    cudaEventRecord(c->ev[c->ev_used + 1], st);
    c->ev_used += 2;
  }
};

template <typename T>
da_status dalloc(da_ctx* c, T** p, size_t count) {
  *p = nullptr;
  if (count == 0) return DA_OK;
  void* v = nullptr;
  cudaError_t e = cudaMalloc(&v, count * sizeof(T));
  if (e != cudaSuccess) {
    cudaGetLastError();
    char buf[160];
    snprintf(buf, sizeof buf, "cudaMalloc of %.3f GB failed: %s", count * sizeof(T) / 1e9, cudaGetErrorString(e));
    return fail(c, DA_ENOMEM, buf);
  }
#ifdef DA_POISON_ALLOCATIONS
  // debugging builds: every fresh allocation holds NaNs (0xff bytes), so a
  // read of device memory that nothing wrote shows up as NaN in the results
  cudaMemset(v, 0xff, count * sizeof(T));
#endif
  c->allocs.push_back(v);
  c->bytes += count * sizeof(T);
  *p = static_cast<T*>(v);
  return DA_OK;
}

// Whether global step k of the evaluation window can be an observation step
// of some member (every member's window is a whole number of observation
// intervals and ends with the evaluation's, so its observation steps fall on
// multiples of obs.every; the kernels find each member's slot).
inline bool obs_step_host(const da_ctx* c, int k) { return k % c->obs.every == 0; }

// Sets the evaluation window for the members marked in `live` (all members
// with a non-empty window if live is NULL): eval_steps = the longest live
// window, each live member end-aligned in it, the others idle; uploads the
// start table of a ragged batch on stream st.  Homogeneous contexts always
// evaluate every member over the context's window.
da_status set_eval_window(da_ctx* c, const std::vector<char>* live, cudaStream_t st);

// Cost and gradient of the members marked in `live` (lbfgs.cu's evaluations).
da_status cost_grad_members(da_ctx* c, const double* s, double* J, double* grad_s, const std::vector<char>* live,
                            cudaStream_t st);

// Frees the optimiser state of lbfgs.cu (da_destroy).
void free_optimiser(da_ctx* c);

// Plan variant the autotuner chose for (n, batch) in this process, or 0
// (plans.cu).
int cached_plan(int n, int B);
