// lbfgs.cu -- da_assimilate of include/da.h: L-BFGS on the control, with
// the cost and gradient of da_cost_grad and the strong-Wolfe line search of
// linesearch.h; vector operations run in the kernels of blas.cuh.
#include <algorithm>

#include "blas.cuh"
#include "ctx.h"
#include "linesearch.h"

// ---------------------------------------------------------------------------
// L-BFGS driver (Sec. II.C: L-BFGS on the transformed control in the
// Euclidean metric).  Members advance in lockstep: every cost-gradient
// evaluation serves all members, and a member that is not searching
// re-evaluates its accepted point, which changes nothing.  Each member keeps
// a ring of memory+1 vector slots for its (s, y) pairs, so a new pair can be
// formed and tested before the oldest one is dropped.
//
// The vectors and every scalar the recursion needs stay on the device: the
// two-loop recursion is one launch, and the host reads scalars only where
// its own decisions need them -- g.d after the recursion (descent test and
// line-search start), the cost and phi'(stp) after each trial evaluation,
// and s.y, y.y and |g| once per iteration (pair test, convergence test).
// ---------------------------------------------------------------------------

namespace {

constexpr int kMaxMemory = 64;  // pairs; the recursion keeps its alphas in shared memory

struct Member {
  std::vector<int> pairs;   // slot indices, oldest first (at most `memory`)
  std::vector<double> rho;  // 1 / (s . y) per pair
  double f = 0, gnorm = 0, g0norm = 0;
  int state = 0;            // 0 active, 1 converged, 2 line-search failure, 3 diverged
  int iters = 0;
  int pending = -1;         // slot of a pair accepted in this iteration, tested at its end
};

// Per-call argument tables of the vector kernels, staged on the host and
// copied to the context's argument buffers (pageable host memory: the copy
// returns once the runtime has staged the bytes, so the tables can be
// rewritten right after).
struct Args {
  da_ctx* c;
  cudaStream_t st;
  int B, m;
  std::vector<int> ints;        // mask [B], cnt [B], aslot [B], pslot [B][m]
  std::vector<double> dbls;     // stp [B], prho [B][m]

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
  c->mem = m;
  return DA_OK;
}

}  // namespace

extern "C" da_status da_assimilate(da_ctx* c, double* s, int max_iter, const da_lbfgs_opts* opts, double* J_hist,
                                   int* iters_done, int* member_status, void* stream) {
  if (!c || !s || !J_hist || !iters_done || max_iter < 0) return fail(c, DA_EINVAL, "bad arguments");
  if (!c->have_obs) return fail(c, DA_EINVAL, "no observations: call da_set_observations first");
  if (!c->dev.traj) return fail(c, DA_EINVAL, "context was created forward-only (ckpt_every < 0)");
  cudaStream_t st = (cudaStream_t)stream;
  da_lbfgs_opts o{10, 1e-4, 0.9, 1e-10, 20};
  if (opts) {
    if (opts->memory > 0) o.memory = opts->memory;
    if (opts->c1 > 0) o.c1 = opts->c1;
    if (opts->c2 > 0) o.c2 = opts->c2;
    if (opts->gtol_rel > 0) o.gtol_rel = opts->gtol_rel;
    if (opts->max_ls_evals > 0) o.max_ls_evals = opts->max_ls_evals;
  }
  if (o.memory > kMaxMemory) return fail(c, DA_EINVAL, "memory must be at most 64 pairs");
  const int B = c->B, m = o.memory, slots = m + 1;
  const size_t len = (size_t)c->n * c->n;
  da_status r = DA_OK;
  if (c->mem != m) {
    if (c->mem) return fail(c, DA_EINVAL, "memory must stay the same across calls on one context");
    if ((r = alloc_optimiser(c, m))) return r;
  }
  Args A(c, st, B, m);
  const da::LbfgsArgs dv = A.dev();
  double* X = c->lb_V + (size_t)da::BANK_X * B * len;
  double* G = c->lb_V + (size_t)da::BANK_G * B * len;
  double* XT = c->lb_V + (size_t)da::BANK_XT * B * len;
  double* GT = c->lb_V + (size_t)da::BANK_GT * B * len;
  const double* hs = c->lb_host;                       // [B][SC_COUNT]
  const double* hJ = c->lb_host + (size_t)B * da::SC_COUNT;  // [B]
  auto sc = [&](int b, int k) { return hs[(size_t)b * da::SC_COUNT + k]; };
  const dim3 ew((unsigned)((len + 4095) / 4096), B);  // element-wise kernels: 4096 elements per CTA
  std::vector<Member> mb(B);

  DA_TRY_CUDA(c, cudaMemcpyAsync(X, s, B * len * sizeof(double), cudaMemcpyDeviceToDevice, st));
  if ((r = da_cost_grad(c, X, c->lb_J, G, st))) return r;
  da::k_gnorm2<<<B, da::kBlasThreads, 0, st>>>(dv);
  if ((r = check_launch(c))) return r;
  if ((r = read_scalars(c, st))) return r;
  for (int b = 0; b < B; ++b) {
    mb[b].f = hJ[b];
    mb[b].g0norm = mb[b].gnorm = std::sqrt(sc(b, da::SC_GG));
    if (!std::isfinite(hJ[b]) || !std::isfinite(sc(b, da::SC_GG))) mb[b].state = 3;
    J_hist[(size_t)b * (max_iter + 1)] = hJ[b];
  }

  for (int it = 0; it < max_iter; ++it) {
    bool any = false;
    for (int b = 0; b < B; ++b) {
      if (mb[b].state == 0 && mb[b].gnorm <= o.gtol_rel * mb[b].g0norm) mb[b].state = 1;
      any |= mb[b].state == 0;
    }
    if (!any) break;
    auto active = [&](int b) { return mb[b].state == 0; };

    // d = -H g by the two-loop recursion, one launch for every active member
    for (int b = 0; b < B; ++b) {
      A.mask()[b] = active(b);
      const int cnt = active(b) ? (int)mb[b].pairs.size() : 0;
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
      if (!active(b)) continue;
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

    // line search, all searching members together
    std::vector<da::MoreThuente> ls(B);
    std::vector<int> searching(B, 0);
    for (int b = 0; b < B; ++b) {
      if (!active(b)) continue;
      const double s0 = it == 0 ? std::min(1.0, 1.0 / mb[b].gnorm) : 1.0;
      ls[b].start(mb[b].f, gd[b], s0, o.c1, o.c2, 1e-10, 1e-20, 1e20, o.max_ls_evals);
      searching[b] = 1;
    }
    for (;;) {
      bool anys = false;
      for (int b = 0; b < B; ++b) anys |= searching[b] != 0;
      if (!anys) break;
      // xt = x + stp d for searching members, x otherwise
      for (int b = 0; b < B; ++b) {
        A.mask()[b] = searching[b];
        A.stp()[b] = searching[b] ? ls[b].stp() : 0.0;
      }
      if ((r = A.upload())) return r;
      da::k_trial<<<ew, 256, 0, st>>>(dv);
      if ((r = check_launch(c))) return r;
      if ((r = da_cost_grad(c, XT, c->lb_J, GT, st))) return r;
      da::k_dot_gt_d<<<B, da::kBlasThreads, 0, st>>>(dv);
      if ((r = check_launch(c))) return r;
      if ((r = read_scalars(c, st))) return r;
      bool accept_any = false;
      for (int b = 0; b < B; ++b) A.mask()[b] = 0;
      for (int b = 0; b < B; ++b) {
        if (!searching[b]) continue;
        const double ft = hJ[b], dg = sc(b, da::SC_DG);
        if (!std::isfinite(ft) || !std::isfinite(dg)) {
          searching[b] = 0;
          mb[b].state = 3;
          continue;
        }
        const int act = ls[b].step(ft, dg);
        if (act == da::MoreThuente::EVALUATE) continue;
        searching[b] = 0;
        const bool ok = act == da::MoreThuente::CONVERGED;
        if (ok || ft < mb[b].f) {
          // accept: the new pair goes to a free slot, s = xt - x, y = gt - g
          int freeslot = 0;
          for (int t = 0; t < slots; ++t)
            if (std::find(mb[b].pairs.begin(), mb[b].pairs.end(), t) == mb[b].pairs.end()) {
              freeslot = t;
              break;
            }
          mb[b].pending = freeslot;
          A.mask()[b] = 1;
          A.aslot()[b] = freeslot;
          accept_any = true;
          mb[b].f = ft;
          mb[b].iters = it + 1;
          J_hist[(size_t)b * (max_iter + 1) + it + 1] = ft;
        }
        if (!ok) mb[b].state = 2;
      }
      if (accept_any) {
        if ((r = A.upload())) return r;
        da::k_accept<<<B, da::kBlasThreads, 0, st>>>(dv);
        if ((r = check_launch(c))) return r;
      }
    }
    // end of the iteration: pair tests and gradient norms
    da::k_gnorm2<<<B, da::kBlasThreads, 0, st>>>(dv);
    if ((r = check_launch(c))) return r;
    if ((r = read_scalars(c, st))) return r;
    for (int b = 0; b < B; ++b) {
      if (mb[b].pending >= 0) {
        const double sy = sc(b, da::SC_SY), yy = sc(b, da::SC_YY);
        if (sy > 1e-16 * yy) {
          if ((int)mb[b].pairs.size() == m) {
            mb[b].pairs.erase(mb[b].pairs.begin());
            mb[b].rho.erase(mb[b].rho.begin());
          }
          mb[b].pairs.push_back(mb[b].pending);
          mb[b].rho.push_back(1.0 / sy);
        }
        mb[b].pending = -1;
      }
      mb[b].gnorm = std::sqrt(sc(b, da::SC_GG));
    }
  }
  bool diverged = false, failed = false;
  std::string who;
  for (int b = 0; b < B; ++b) {
    iters_done[b] = mb[b].iters;
    for (int it = mb[b].iters + 1; it <= max_iter; ++it) J_hist[(size_t)b * (max_iter + 1) + it] = mb[b].f;
    const da_status ms = mb[b].state == 3 ? DA_EDIVERGED : mb[b].state == 2 ? DA_ENOTCONV : DA_OK;
    if (member_status) member_status[b] = ms;
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
