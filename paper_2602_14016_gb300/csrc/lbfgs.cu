// lbfgs.cu -- the optimiser of include/da.h: da_assimilate and the stepwise
// da_lbfgs_* calls.  L-BFGS on the control (Sec. II.C: L-BFGS on the
// transformed control in the Euclidean metric), with the cost and gradient
// of da_cost_grad and the strong-Wolfe line search of linesearch.h; vector
// operations run in the kernels of blas.cuh.
#include <algorithm>

#include "blas.cuh"
#include "ctx.h"
#include "linesearch.h"

// ---------------------------------------------------------------------------
// Every member slot of a batch has its own optimiser state.  A member is
// started on a control (da_lbfgs_start); each step (da_lbfgs_iterate) then
// advances every running member to and through one shared cost-gradient
// evaluation: members whose last trial was accepted get their pair tested,
// members that need a search direction get it (the two-loop recursion, one
// launch for all of them) and a line search started, and one evaluation then
// serves every searching member's trial and every newly started member's
// first point.  Members at different points of their iterations share each
// evaluation, and no member waits for another's line search; a member that
// is not evaluated is left out (in a ragged batch its CTAs return at once)
// or, in a homogeneous batch, re-evaluates its accepted point, which changes
// nothing.  A member's own sequence of operations does not depend on when it
// joined or who else is in the batch, so its results do not either.  Each
// member keeps a ring of memory+1 vector slots for its (s, y) pairs, so a new
// pair can be formed and tested before the oldest one is dropped.
//
// The vectors and every scalar the recursion needs stay on the device: the
// two-loop recursion is one launch, and the host reads scalars only where
// its own decisions need them -- s.y, y.y and |g| after an accepted step
// (pair and convergence tests), g.d after the recursion (descent test and
// line-search start), and the cost and phi'(stp) after each evaluation.
// da_assimilate is: start every member, steps until all have finished.
// ---------------------------------------------------------------------------

namespace {

constexpr int kMaxMemory = 64;  // pairs; the recursion keeps its alphas in shared memory

enum Phase { IDLE = 0, STARTED = 1, ITERATING = 2, FINISHED = 3 };
// where a started or iterating member is within its iteration
enum Sub { FIRST_EVAL, FIRST_NORM, NEED_DIR, SEARCHING, ACCEPTED };

struct Member {
  int phase = IDLE;
  int sub = FIRST_EVAL;
  da::MoreThuente ls;
  int state = 0;            // 0 running, 1 converged, 2 line-search failure, 3 diverged
  int max_iter = 0;
  int k = 0;                // iterations begun
  int iters = 0;            // iterations that accepted a step
  int pending = -1;         // slot of a pair accepted by the last step, tested in the next
  double c1 = 1e-4, c2 = 0.9, gtol = 1e-10;
  int max_ls = 20;
  std::vector<int> pairs;   // slot indices, oldest first (at most `memory`)
  std::vector<double> rho;  // 1 / (s . y) per pair
  double f = 0, gnorm = 0, g0norm = 0;
  std::vector<double> hist;  // the cost at the start and after each accepted iteration
};

struct OptState {
  int m = 0;  // memory (pairs), fixed per context
  std::vector<Member> mb;
};

OptState& state_of(da_ctx* c) { return *static_cast<OptState*>(c->lb_state); }

// Per-call argument tables of the vector kernels, staged on the host and
// copied to the context's argument buffers (pageable host memory: the copy
// returns once the runtime has staged the bytes, so the tables can be
// rewritten right after).
struct Args {
  da_ctx* c;
  cudaStream_t st;
  int B, m;
  std::vector<int> ints;     // mask [B], cnt [B], aslot [B], pslot [B][m]
  std::vector<double> dbls;  // stp [B], prho [B][m]

  Args(da_ctx* c_, cudaStream_t s, int B_, int m_) : c(c_), st(s), B(B_), m(m_) {
    ints.assign((size_t)3 * B + (size_t)B * m, 0);
    dbls.assign((size_t)B + (size_t)B * m, 0.0);
  }
  int* mask() { return ints.data(); }
  int* cnt() { return ints.data() + B; }
  int* aslot() { return ints.data() + 2 * B; }
  int* pslot() { return ints.data() + 3 * B; }
  double* stp() { return dbls.data(); }
  double* prho() { return dbls.data() + B; }

  da::LbfgsArgs dev() const {
    da::LbfgsArgs a{};
    a.V = c->lb_V;
    a.len = (size_t)c->n * c->n;
    a.B = B;
    a.slots = m + 1;
    a.mem = m;
    a.scal = c->lb_scal;
    a.mask = c->lb_iargs;
    a.cnt = c->lb_iargs + B;
    a.aslot = c->lb_iargs + 2 * B;
    a.pslot = c->lb_iargs + 3 * B;
    a.stp = c->lb_dargs;
    a.prho = c->lb_dargs + B;
    return a;
  }
  da_status upload() {
    DA_TRY_CUDA(c, cudaMemcpyAsync(c->lb_iargs, ints.data(), ints.size() * sizeof(int), cudaMemcpyHostToDevice, st));
    DA_TRY_CUDA(c, cudaMemcpyAsync(c->lb_dargs, dbls.data(), dbls.size() * sizeof(double), cudaMemcpyHostToDevice, st));
    return DA_OK;
  }
};

// Waits for the stream and returns the device scalars and costs in the
// context's pinned mirror: lb_host[b * SC_COUNT + k], costs after them.
da_status read_scalars(da_ctx* c, cudaStream_t st) {
  const int B = c->B;
  DA_TRY_CUDA(c, cudaMemcpyAsync(c->lb_host, c->lb_scal, (size_t)B * da::SC_COUNT * sizeof(double),
                                 cudaMemcpyDeviceToHost, st));
  DA_TRY_CUDA(c, cudaMemcpyAsync(c->lb_host + (size_t)B * da::SC_COUNT, c->lb_J, B * sizeof(double),
                                 cudaMemcpyDeviceToHost, st));
  DA_TRY_CUDA(c, cudaStreamSynchronize(st));
  return DA_OK;
}

da_status alloc_optimiser(da_ctx* c, int m) {
  if (c->mem == m) return DA_OK;
  if (c->mem) return fail(c, DA_EINVAL, "memory must stay the same across calls on one context");
  const size_t B = c->B, len = (size_t)c->n * c->n, slots = m + 1;
  da_status r = DA_OK;
  auto A = [&](da_status x) {
    if (r == DA_OK) r = x;
  };
  A(dalloc(c, &c->lb_V, (da::BANK_S0 + 2 * slots) * B * len));
  A(dalloc(c, &c->lb_scal, B * da::SC_COUNT));
  A(dalloc(c, &c->lb_J, B));
  A(dalloc(c, &c->lb_iargs, 3 * B + B * m));
  A(dalloc(c, &c->lb_dargs, B + B * m));
  if (r) return r;
  void* h = nullptr;
  if (cudaMallocHost(&h, B * (da::SC_COUNT + 1) * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    return fail(c, DA_ENOMEM, "pinned host buffer of the optimiser");
  }
  c->lb_host = static_cast<double*>(h);
  auto* S = new OptState();
  S->m = m;
  S->mb.resize(c->B);
  c->lb_state = S;
  c->mem = m;
  return DA_OK;
}

da_lbfgs_opts resolve(const da_lbfgs_opts* opts) {
  da_lbfgs_opts o{10, 1e-4, 0.9, 1e-10, 20};
  if (opts) {
    if (opts->memory > 0) o.memory = opts->memory;
    if (opts->c1 > 0) o.c1 = opts->c1;
    if (opts->c2 > 0) o.c2 = opts->c2;
    if (opts->gtol_rel > 0) o.gtol_rel = opts->gtol_rel;
    if (opts->max_ls_evals > 0) o.max_ls_evals = opts->max_ls_evals;
  }
  return o;
}

// Common checks of the calls that evaluate; allocates the optimiser.
da_status prepare(da_ctx* c, const da_lbfgs_opts& o) {
  if (!c->have_obs) return fail(c, DA_EINVAL, "no observations: call da_set_observations first");
  if (!c->dev.traj) return fail(c, DA_EINVAL, "context was created forward-only (ckpt_every < 0)");
  if (o.memory > kMaxMemory) return fail(c, DA_EINVAL, "memory must be at most 64 pairs");
  return alloc_optimiser(c, o.memory);
}

void start_member(Member& M, int max_iter, const da_lbfgs_opts& o) {
  M = Member();
  M.phase = STARTED;
  M.sub = FIRST_EVAL;
  M.max_iter = max_iter;
  M.c1 = o.c1;
  M.c2 = o.c2;
  M.gtol = o.gtol_rel;
  M.max_ls = o.max_ls_evals;
}

// One step: pair tests and first norms, new directions, then one shared
// evaluation and its results.
da_status lbfgs_step(da_ctx* c, cudaStream_t st) {
  OptState& S = state_of(c);
  const int B = c->B, m = S.m, slots = m + 1;
  const size_t len = (size_t)c->n * c->n;
  std::vector<Member>& mb = S.mb;
  Args A(c, st, B, m);
  const da::LbfgsArgs dv = A.dev();
  double* XT = c->lb_V + (size_t)da::BANK_XT * B * len;
  double* GT = c->lb_V + (size_t)da::BANK_GT * B * len;
  const double* hs = c->lb_host;
  const double* hJ = c->lb_host + (size_t)B * da::SC_COUNT;
  auto sc = [&](int b, int k) { return hs[(size_t)b * da::SC_COUNT + k]; };
  auto running = [&](const Member& M) { return M.phase == STARTED || M.phase == ITERATING; };
  const dim3 ew((unsigned)((len + 4095) / 4096), B);  // element-wise kernels: 4096 elements per CTA
  da_status r;

  // 1. |g| after a first evaluation; the pair test and |g| after an accepted step
  bool need_norm = false;
  for (const Member& M : mb) need_norm |= running(M) && (M.sub == FIRST_NORM || M.sub == ACCEPTED);
  if (need_norm) {
    da::k_gnorm2<<<B, da::kBlasThreads, 0, st>>>(dv);
    if ((r = check_launch(c))) return r;
    if ((r = read_scalars(c, st))) return r;
    for (int b = 0; b < B; ++b) {
      Member& M = mb[b];
      if (!running(M)) continue;
      if (M.sub == FIRST_NORM) {
        M.g0norm = M.gnorm = std::sqrt(sc(b, da::SC_GG));
        M.phase = ITERATING;
        M.sub = NEED_DIR;
        if (!std::isfinite(M.f) || !std::isfinite(M.gnorm)) {
          M.state = 3;
          M.phase = FINISHED;
        }
      } else if (M.sub == ACCEPTED) {
        const double sy = sc(b, da::SC_SY), yy = sc(b, da::SC_YY);
        if (sy > 1e-16 * yy) {
          if ((int)M.pairs.size() == m) {
            M.pairs.erase(M.pairs.begin());
            M.rho.erase(M.rho.begin());
          }
          M.pairs.push_back(M.pending);
          M.rho.push_back(1.0 / sy);
        }
        M.pending = -1;
        M.gnorm = std::sqrt(sc(b, da::SC_GG));
        M.sub = NEED_DIR;
        if (M.state != 0) M.phase = FINISHED;  // the line search failed after accepting a lower cost
      }
    }
  }

  // 2. new iterations: convergence and budget tests, then d = -H g by the
  // two-loop recursion (one launch for all of them) and the line-search start
  std::vector<char> dir(B, 0);
  bool any_dir = false;
  for (int b = 0; b < B; ++b) {
    Member& M = mb[b];
    if (M.phase != ITERATING || M.sub != NEED_DIR) continue;
    if (M.state == 0 && M.gnorm <= M.gtol * M.g0norm) M.state = 1;
    if (M.state != 0 || M.k >= M.max_iter) {
      M.phase = FINISHED;
      continue;
    }
    dir[b] = 1;
    any_dir = true;
  }
  if (any_dir) {
    for (int b = 0; b < B; ++b) {
      A.mask()[b] = dir[b];
      const int cnt = dir[b] ? (int)mb[b].pairs.size() : 0;
      A.cnt()[b] = cnt;
      for (int j = 0; j < cnt; ++j) {
        A.pslot()[(size_t)b * m + j] = mb[b].pairs[j];
        A.prho()[(size_t)b * m + j] = mb[b].rho[j];
      }
    }
    if ((r = A.upload())) return r;
    da::k_two_loop<<<B, da::kBlasThreads, 0, st>>>(dv);
    if ((r = check_launch(c))) return r;
    if ((r = read_scalars(c, st))) return r;
    std::vector<double> gd(B, 0.0);
    bool reset = false;
    for (int b = 0; b < B; ++b) {
      A.mask()[b] = 0;
      if (!dir[b]) continue;
      gd[b] = sc(b, da::SC_GD);
      if (!(gd[b] < 0.0)) {  // not a descent direction: restart from -g
        mb[b].pairs.clear();
        mb[b].rho.clear();
        gd[b] = -mb[b].gnorm * mb[b].gnorm;
        A.mask()[b] = 1;
        reset = true;
      }
    }
    if (reset) {
      if ((r = A.upload())) return r;
      da::k_neg_grad<<<ew, 256, 0, st>>>(dv);
      if ((r = check_launch(c))) return r;
    }
    for (int b = 0; b < B; ++b) {
      if (!dir[b]) continue;
      Member& M = mb[b];
      const double s0 = M.k == 0 ? std::min(1.0, 1.0 / M.gnorm) : 1.0;
      M.ls.start(M.f, gd[b], s0, M.c1, M.c2, 1e-10, 1e-20, 1e20, M.max_ls);
      M.sub = SEARCHING;
      ++M.k;
    }
  }

  // 3. one shared evaluation: the searching members' trials, xt = x + stp d,
  // and the first points of the newly started members, xt = x
  std::vector<char> live(B, 0), searching(B, 0), fresh(B, 0);
  bool any_live = false, any_fresh = false;
  for (int b = 0; b < B; ++b) {
    const Member& M = mb[b];
    searching[b] = M.phase == ITERATING && M.sub == SEARCHING;
    fresh[b] = M.phase == STARTED && M.sub == FIRST_EVAL;
    live[b] = searching[b] || fresh[b];
    any_live |= live[b] != 0;
    any_fresh |= fresh[b] != 0;
    A.mask()[b] = searching[b];
    A.stp()[b] = searching[b] ? M.ls.stp() : 0.0;
  }
  if (!any_live) return DA_OK;
  if ((r = A.upload())) return r;
  da::k_trial<<<ew, 256, 0, st>>>(dv);
  if ((r = check_launch(c))) return r;
  if ((r = cost_grad_members(c, XT, c->lb_J, GT, &live, st))) return r;
  da::k_dot_gt_d<<<B, da::kBlasThreads, 0, st>>>(dv);
  if ((r = check_launch(c))) return r;
  if (any_fresh) {  // g = gt for the members just evaluated for the first time
    for (int b = 0; b < B; ++b) A.mask()[b] = fresh[b];
    if ((r = A.upload())) return r;
    da::k_take_gradient<<<ew, 256, 0, st>>>(dv);
    if ((r = check_launch(c))) return r;
  }
  if ((r = read_scalars(c, st))) return r;

  // 4. results
  bool accept_any = false;
  for (int b = 0; b < B; ++b) A.mask()[b] = 0;
  for (int b = 0; b < B; ++b) {
    Member& M = mb[b];
    if (fresh[b]) {
      M.f = hJ[b];
      M.hist.assign(1, hJ[b]);
      M.sub = FIRST_NORM;
      continue;
    }
    if (!searching[b]) continue;
    const double ft = hJ[b], dg = sc(b, da::SC_DG);
    if (!std::isfinite(ft) || !std::isfinite(dg)) {
      M.state = 3;
      M.phase = FINISHED;
      continue;
    }
    const int act = M.ls.step(ft, dg);
    if (act == da::MoreThuente::EVALUATE) continue;
    const bool ok = act == da::MoreThuente::CONVERGED;
    if (!ok) M.state = 2;
    if (ok || ft < M.f) {
      // accept: the new pair goes to a free slot, s = xt - x, y = gt - g
      int freeslot = 0;
      for (int t = 0; t < slots; ++t)
        if (std::find(M.pairs.begin(), M.pairs.end(), t) == M.pairs.end()) {
          freeslot = t;
          break;
        }
      M.pending = freeslot;
      A.mask()[b] = 1;
      A.aslot()[b] = freeslot;
      accept_any = true;
      M.f = ft;
      M.iters = M.k;
      M.hist.push_back(ft);
      M.sub = ACCEPTED;
    } else {
      M.phase = FINISHED;
    }
  }
  if (accept_any) {
    if ((r = A.upload())) return r;
    da::k_accept<<<B, da::kBlasThreads, 0, st>>>(dv);
    if ((r = check_launch(c))) return r;
  }
  return DA_OK;
}

da_status member_status(const Member& M) {
  return M.state == 3 ? DA_EDIVERGED : M.state == 2 ? DA_ENOTCONV : DA_OK;
}

}  // namespace

void free_optimiser(da_ctx* c) {
  delete static_cast<OptState*>(c->lb_state);
  c->lb_state = nullptr;
}

extern "C" da_status da_lbfgs_start(da_ctx* c, int member, const double* s0, int max_iter,
                                    const da_lbfgs_opts* opts, void* stream) {
  if (!c || !s0 || max_iter < 0) return fail(c, DA_EINVAL, "bad arguments");
  if (member < 0 || member >= c->B) return fail(c, DA_EINVAL, "member out of range");
  const da_lbfgs_opts o = resolve(opts);
  da_status r = prepare(c, o);
  if (r) return r;
  const size_t len = (size_t)c->n * c->n;
  double* X = c->lb_V + ((size_t)da::BANK_X * c->B + member) * len;
  DA_TRY_CUDA(c, cudaMemcpyAsync(X, s0, len * sizeof(double), cudaMemcpyDeviceToDevice, (cudaStream_t)stream));
  start_member(state_of(c).mb[member], max_iter, o);
  return DA_OK;
}

extern "C" da_status da_lbfgs_iterate(da_ctx* c, int* running, void* stream) {
  if (!c) return fail(c, DA_EINVAL, "ctx must not be NULL");
  if (!c->lb_state) {
    if (running) *running = 0;
    return DA_OK;
  }
  da_status r = lbfgs_step(c, (cudaStream_t)stream);
  if (r) return r;
  if (running) {
    int n = 0;
    for (const Member& M : state_of(c).mb) n += M.phase == STARTED || M.phase == ITERATING;
    *running = n;
  }
  return DA_OK;
}

extern "C" da_status da_lbfgs_member(da_ctx* c, int member, da_lbfgs_report* out, double* J_hist, int hist_len,
                                     double* s, void* stream) {
  if (!c || !out) return fail(c, DA_EINVAL, "ctx and out must not be NULL");
  if (member < 0 || member >= c->B) return fail(c, DA_EINVAL, "member out of range");
  *out = da_lbfgs_report{};
  if (!c->lb_state) return DA_OK;
  const Member& M = state_of(c).mb[member];
  out->phase = M.phase;
  out->status = member_status(M);
  out->iters = M.iters;
  out->J0 = M.hist.empty() ? 0.0 : M.hist.front();
  out->J = M.f;
  if (J_hist)
    for (int i = 0; i < hist_len; ++i) J_hist[i] = i < (int)M.hist.size() ? M.hist[i] : M.f;
  if (s) {
    const size_t len = (size_t)c->n * c->n;
    const double* X = c->lb_V + ((size_t)da::BANK_X * c->B + member) * len;
    DA_TRY_CUDA(c, cudaMemcpyAsync(s, X, len * sizeof(double), cudaMemcpyDeviceToDevice, (cudaStream_t)stream));
  }
  return DA_OK;
}

extern "C" da_status da_lbfgs_release(da_ctx* c, int member) {
  if (!c) return fail(c, DA_EINVAL, "ctx must not be NULL");
  if (member < 0 || member >= c->B) return fail(c, DA_EINVAL, "member out of range");
  if (c->lb_state) state_of(c).mb[member] = Member();
  return DA_OK;
}

extern "C" da_status da_assimilate(da_ctx* c, double* s, int max_iter, const da_lbfgs_opts* opts, double* J_hist,
                                   int* iters_done, int* member_status_out, void* stream) {
  if (!c || !s || !J_hist || !iters_done || max_iter < 0) return fail(c, DA_EINVAL, "bad arguments");
  const da_lbfgs_opts o = resolve(opts);
  da_status r = prepare(c, o);
  if (r) return r;
  cudaStream_t st = (cudaStream_t)stream;
  const int B = c->B;
  const size_t len = (size_t)c->n * c->n;
  double* X = c->lb_V + (size_t)da::BANK_X * B * len;
  DA_TRY_CUDA(c, cudaMemcpyAsync(X, s, B * len * sizeof(double), cudaMemcpyDeviceToDevice, st));
  OptState& S = state_of(c);
  for (int b = 0; b < B; ++b) start_member(S.mb[b], max_iter, o);
  for (;;) {
    bool running = false;
    for (const Member& M : S.mb) running |= M.phase == STARTED || M.phase == ITERATING;
    if (!running) break;
    if ((r = lbfgs_step(c, st))) return r;
  }
  bool diverged = false, failed = false;
  std::string who;
  for (int b = 0; b < B; ++b) {
    const Member& M = S.mb[b];
    iters_done[b] = M.iters;
    for (int it = 0; it <= max_iter; ++it)
      J_hist[(size_t)b * (max_iter + 1) + it] = it < (int)M.hist.size() ? M.hist[it] : M.f;
    const da_status ms = member_status(M);
    if (member_status_out) member_status_out[b] = ms;
    diverged |= ms == DA_EDIVERGED;
    failed |= ms == DA_ENOTCONV;
    if (ms != DA_OK) who += (who.empty() ? "" : ", ") + std::to_string(b);
  }
  DA_TRY_CUDA(c, cudaMemcpyAsync(s, X, B * len * sizeof(double), cudaMemcpyDeviceToDevice, st));
  DA_TRY_CUDA(c, cudaStreamSynchronize(st));
  if (diverged) return fail(c, DA_EDIVERGED, "non-finite cost or gradient (members with a non-OK status: " + who + ")");
  if (failed) return fail(c, DA_ENOTCONV, "line search failed, step-size collapse (members " + who + ")");
  return DA_OK;
}
