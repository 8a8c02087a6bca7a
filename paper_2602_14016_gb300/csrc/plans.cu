// plans.cu -- FFT plan variants of the pass kernels and the autotuner
// (da_plan_count, da_get_plan, da_set_plan, da_autotune of include/da.h).
#include <map>
#include <mutex>
#include <utility>

#include "ctx.h"

// Plan variant chosen by the autotuner per (grid size, batch), for the
// contexts created afterwards in this process.
static std::mutex g_plan_mu;
static std::map<std::pair<int, int>, int> g_plan_choice;

int cached_plan(int n, int B) {
  std::lock_guard<std::mutex> lock(g_plan_mu);
  auto it = g_plan_choice.find({n, B});
  return it == g_plan_choice.end() ? 0 : it->second;
}

// Switches the context's pass kernels to plan variant v: launchers, folded
// twiddle table, shared-memory attributes.  A captured graph holds the old
// kernels and is dropped; a stored forward trajectory is invalidated.
static da_status set_plan(da_ctx* c, int v) {
  const Ops* o = da::ops_for(c->n, v);
  if (!o) return fail(c, DA_EINVAL, "plan variant out of range (da_plan_count)");
  if (o == c->ops) return DA_OK;
  std::vector<double> fold(o->fold_doubles);
  o->fold_table(fold.data());
  DA_TRY_CUDA(c, cudaMemcpy((void*)c->dev.fold, fold.data(), fold.size() * sizeof(double), cudaMemcpyHostToDevice));
  DA_TRY_CUDA(c, o->setup());
  c->ops = o;
  drop_graphs(c);
  if (c->sp_exec) {
    cudaGraphExecDestroy(c->sp_exec);
    c->sp_exec = nullptr;
    c->sp_key = -1;
  }
  c->have_fwd = false;
  return DA_OK;
}

extern "C" int da_plan_count(int n) { return da::ops_for(n) ? da::plan_count(n) : 0; }

extern "C" int da_get_plan(const da_ctx* c) { return c ? c->ops->variant : -1; }

extern "C" da_status da_plan_flops(int n, int variant, double* inverse, double* forward) {
  const Ops* o = da::ops_for(n, variant);
  if (!o) return fail(nullptr, DA_EINVAL, "unsupported size or plan variant (da_plan_count)");
  if (!inverse || !forward) return fail(nullptr, DA_EINVAL, "inverse and forward must not be NULL");
  *inverse = o->flops_inverse;
  *forward = o->flops_forward;
  return DA_OK;
}

extern "C" da_status da_set_plan(da_ctx* c, int variant) {
  if (!c) return fail(c, DA_EINVAL, "ctx must not be NULL");
  // the folded table and the launchers change under any work in flight
  DA_TRY_CUDA(c, cudaDeviceSynchronize());
  return set_plan(c, variant);
}

// Zeroes the working state that the tuning passes run over.
static da_status clear_state(da_ctx* c, cudaStream_t st) {
  const Dev& d = c->dev;
  const size_t comp = (size_t)c->B * c->ops->Kr * c->ops->Kc * sizeof(double2);
  const size_t mixed = (size_t)c->B * 2 * c->n * c->ops->Kc * sizeof(double2);
  for (void* p : {(void*)d.W, (void*)d.Acc, (void*)d.Y, (void*)d.KB, (void*)d.LamBar, (void*)d.Sum})
    DA_TRY_CUDA(c, cudaMemsetAsync(p, 0, comp, st));
  DA_TRY_CUDA(c, cudaMemsetAsync(d.Mx, 0, mixed, st));
  DA_TRY_CUDA(c, cudaMemsetAsync(d.Mn, 0, mixed, st));
  return DA_OK;
}

// `steps` RK steps of the pass kernels (forward, and the adjoint when the
// context stores stage fields) over whatever the working buffers hold.
static da_status tuning_steps(da_ctx* c, int steps, cudaStream_t st) {
  const Ops* o = c->ops;
  c->dev.seg0 = 0;
  Dev d = c->dev;
  d.ragged = 0;  // every member works, whatever windows a ragged batch holds
  const bool store = d.traj != nullptr;
  for (int i = 0; i < steps; ++i) {
    const int k = store ? i % d.traj_steps : 0;
    for (int j = 1; j <= 4; ++j) {
      o->fwd_rows(d, k, j, store ? da::F_STORE : 0, st);
      o->fwd_cols(d, k, j, 0, st);
    }
    if (store)
      for (int j = 4; j >= 1; --j) {
        o->adj_rows(d, k, j, st);
        o->adj_cols(d, k, j, 0, st);
      }
    da_status r = check_launch(c, store ? 16 : 8);
    if (r) return r;
  }
  return DA_OK;
}

extern "C" da_status da_autotune(da_ctx* c, int steps, int* chosen, double* ms_per_step) {
  if (!c) return fail(c, DA_EINVAL, "ctx must not be NULL");
  if (steps < 1) return fail(c, DA_EINVAL, "steps must be >= 1");
  // the tuning passes overwrite the working state: let every evaluation in
  // flight on any stream finish first
  DA_TRY_CUDA(c, cudaDeviceSynchronize());
  // the device is idle now; the tuning runs on the legacy default stream
  // (creating a stream of its own here was measured to leave later
  // evaluations in the process about 1 % slower)
  cudaStream_t st = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  da_status r = DA_OK;
  int best = 0;
  float best_ms = 0.f;
  auto cuda = [&](cudaError_t e, const char* what) {
    if (r == DA_OK && e != cudaSuccess) r = fail(c, DA_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
  };
  cuda(cudaEventCreate(&e0), "event");
  cuda(cudaEventCreate(&e1), "event");
  for (int v = 0; r == DA_OK && v < da::plan_count(c->n); ++v) {
    if ((r = set_plan(c, v))) break;
    if ((r = clear_state(c, st))) break;
    if ((r = tuning_steps(c, 1, st))) break;  // warm-up
    cuda(cudaEventRecord(e0, st), "event record");
    if (r || (r = tuning_steps(c, steps, st))) break;
    cuda(cudaEventRecord(e1, st), "event record");
    cuda(cudaEventSynchronize(e1), "event synchronize");
    float ms = 0.f;
    cuda(cudaEventElapsedTime(&ms, e0, e1), "event elapsed time");
    if (r) break;
    ms /= steps;
    if (ms_per_step) ms_per_step[v] = ms;
    if (v == 0 || ms < best_ms) {
      best = v;
      best_ms = ms;
    }
  }
  if (r == DA_OK) r = set_plan(c, best);
  if (r == DA_OK) r = clear_state(c, st);
  if (r == DA_OK) cuda(cudaStreamSynchronize(st), "stream synchronize");
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (r) return r;
  {
    std::lock_guard<std::mutex> lock(g_plan_mu);
    g_plan_choice[{c->n, c->B}] = best;
  }
  c->have_fwd = false;
  if (chosen) *chosen = best;
  return DA_OK;
}
