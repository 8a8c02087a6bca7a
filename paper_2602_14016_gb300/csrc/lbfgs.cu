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
// ---------------------------------------------------------------------------

namespace {

struct Vec {
  da_ctx* c;
  cudaStream_t st;
  size_t len;

  // out[b] = a_b . x_b (NULL pointer: 0)
  da_status dot(const std::vector<const double*>& a, const std::vector<const double*>& x, std::vector<double>& out) {
    const int B = c->B;
    std::vector<const double*> ptrs(2 * B);
    for (int b = 0; b < B; ++b) {
      ptrs[b] = a[b];
      ptrs[B + b] = x[b];
    }
    DA_TRY_CUDA(c, cudaMemcpyAsync(c->ptrs, ptrs.data(), 2 * B * sizeof(void*), cudaMemcpyHostToDevice, st));
    const int chunks = da::dot_chunks(len);
    da::k_dot_partial<<<dim3(chunks, B), 256, 0, st>>>((const double* const*)c->ptrs,
                                                        (const double* const*)c->ptrs + B, c->part, len);
    da::k_dot_final<<<B, 256, 0, st>>>(c->part, c->dots, chunks);
    da_status r = check_launch(c, 2);
    if (r) return r;
    out.assign(B, 0.0);
    DA_TRY_CUDA(c, cudaMemcpyAsync(out.data(), c->dots, B * sizeof(double), cudaMemcpyDeviceToHost, st));
    DA_TRY_CUDA(c, cudaStreamSynchronize(st));
    return DA_OK;
  }

  // y_b = alpha_b x_b + beta_b y_b (NULL pointer: member untouched)
  da_status axpby(const std::vector<double>& alpha, const std::vector<const double*>& x,
                  const std::vector<double>& beta, const std::vector<double*>& y) {
    const int B = c->B;
    std::vector<const void*> ptrs(2 * B);
    std::vector<double> ab(2 * B);
    for (int b = 0; b < B; ++b) {
      ptrs[b] = x[b];
      ptrs[B + b] = y[b];
      ab[b] = alpha[b];
      ab[B + b] = beta[b];
    }
    DA_TRY_CUDA(c, cudaMemcpyAsync(c->ptrs, ptrs.data(), 2 * B * sizeof(void*), cudaMemcpyHostToDevice, st));
    DA_TRY_CUDA(c, cudaMemcpyAsync(c->scal, ab.data(), 2 * B * sizeof(double), cudaMemcpyHostToDevice, st));
    da::k_axpby<<<dim3((unsigned)((len + 1023) / 1024), B), 256, 0, st>>>(
        (const double* const*)c->ptrs, (double* const*)c->ptrs + B, c->scal, c->scal + B, len);
    da_status r = check_launch(c);
    if (r) return r;
    DA_TRY_CUDA(c, cudaStreamSynchronize(st));  // host arrays must outlive the copies
    return DA_OK;
  }

  double* member(double* base, int b) const { return base + (size_t)b * len; }
};

struct Member {
  std::vector<int> pairs;    // slot indices, oldest first (at most `memory`)
  std::vector<double> rho;   // 1 / (s . y) per pair
  double f = 0, gnorm = 0, g0norm = 0;
  int state = 0;             // 0 active, 1 converged, 2 line-search failure, 3 diverged
  int iters = 0;
};

}  // namespace

extern "C" da_status da_assimilate(da_ctx* c, double* s, int max_iter, const da_lbfgs_opts* opts, double* J_hist,
                                   int* iters_done, void* stream) {
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
  const int B = c->B, m = o.memory, slots = m + 1;
  const size_t len = (size_t)c->n * c->n;
  da_status r = DA_OK;
  if (c->mem != m) {
    if (c->mem) return fail(c, DA_EINVAL, "memory must stay the same across calls on one context");
    auto A = [&](da_status x) {
      if (r == DA_OK) r = x;
    };
    A(dalloc(c, &c->x, B * len));
    A(dalloc(c, &c->g, B * len));
    A(dalloc(c, &c->d, B * len));
    A(dalloc(c, &c->xt, B * len));
    A(dalloc(c, &c->gt, B * len));
    A(dalloc(c, &c->S, (size_t)slots * B * len));
    A(dalloc(c, &c->Y, (size_t)slots * B * len));
    A(dalloc(c, &c->part, (size_t)B * da::dot_chunks(len)));
    A(dalloc(c, &c->dots, (size_t)B));
    A(dalloc(c, &c->scal, (size_t)2 * B));
    A(dalloc<void*>(c, &c->ptrs, (size_t)2 * B));
    if (r) return r;
    c->mem = m;
  }
  Vec V{c, st, len};
  auto Sslot = [&](int slot, int b) { return c->S + ((size_t)slot * B + b) * len; };
  auto Yslot = [&](int slot, int b) { return c->Y + ((size_t)slot * B + b) * len; };
  const std::vector<double> zeros(B, 0.0), ones(B, 1.0);
  std::vector<Member> mb(B);
  std::vector<double> f(B), tmp;
  std::vector<const double*> pa(B), pb(B);
  std::vector<double*> py(B);

  DA_TRY_CUDA(c, cudaMemcpyAsync(c->x, s, B * len * sizeof(double), cudaMemcpyDeviceToDevice, st));
  if ((r = da_cost_grad(c, c->x, f.data(), c->g, st))) return r;
  for (int b = 0; b < B; ++b) pa[b] = V.member(c->g, b);
  if ((r = V.dot(pa, pa, tmp))) return r;
  for (int b = 0; b < B; ++b) {
    mb[b].f = f[b];
    mb[b].g0norm = mb[b].gnorm = std::sqrt(tmp[b]);
    if (!std::isfinite(f[b]) || !std::isfinite(tmp[b])) mb[b].state = 3;
    J_hist[(size_t)b * (max_iter + 1)] = f[b];
  }

  for (int it = 0; it < max_iter; ++it) {
    bool any = false;
    for (int b = 0; b < B; ++b) {
      if (mb[b].state == 0 && mb[b].gnorm <= o.gtol_rel * mb[b].g0norm) mb[b].state = 1;
      any |= mb[b].state == 0;
    }
    if (!any) break;
    auto active = [&](int b) { return mb[b].state == 0; };

    // d = -H g by the two-loop recursion (d carries -q)
    for (int b = 0; b < B; ++b) {
      pa[b] = active(b) ? V.member(c->g, b) : nullptr;
      py[b] = active(b) ? V.member(c->d, b) : nullptr;
    }
    std::vector<double> minus(B, -1.0);
    if ((r = V.axpby(minus, pa, zeros, py))) return r;
    int hmax = 0;
    for (int b = 0; b < B; ++b)
      if (active(b)) hmax = std::max(hmax, (int)mb[b].pairs.size());
    std::vector<std::vector<double>> alpha(B, std::vector<double>(hmax, 0.0));
    for (int h = 0; h < hmax; ++h) {  // newest to oldest
      for (int b = 0; b < B; ++b) {
        const int cnt = (int)mb[b].pairs.size();
        const bool use = active(b) && h < cnt;
        pa[b] = use ? Sslot(mb[b].pairs[cnt - 1 - h], b) : nullptr;
        pb[b] = use ? V.member(c->d, b) : nullptr;
      }
      if ((r = V.dot(pa, pb, tmp))) return r;
      std::vector<double> al(B, 0.0);
      for (int b = 0; b < B; ++b) {
        const int cnt = (int)mb[b].pairs.size();
        const bool use = active(b) && h < cnt;
        if (use) al[b] = alpha[b][h] = -mb[b].rho[cnt - 1 - h] * tmp[b];  // rho s.q
        pa[b] = use ? Yslot(mb[b].pairs[cnt - 1 - h], b) : nullptr;
        py[b] = use ? V.member(c->d, b) : nullptr;
      }
      if ((r = V.axpby(al, pa, ones, py))) return r;  // q -= alpha y
    }
    if (hmax > 0) {  // H0 = (s.y / y.y) I from the newest pair
      for (int b = 0; b < B; ++b) {
        const bool use = active(b) && !mb[b].pairs.empty();
        pa[b] = use ? Yslot(mb[b].pairs.back(), b) : nullptr;
      }
      if ((r = V.dot(pa, pa, tmp))) return r;
      std::vector<double> gam(B, 1.0);
      for (int b = 0; b < B; ++b) {
        const bool use = active(b) && !mb[b].pairs.empty();
        if (use) gam[b] = 1.0 / (mb[b].rho.back() * tmp[b]);
        pa[b] = use ? V.member(c->d, b) : nullptr;
        py[b] = use ? V.member(c->d, b) : nullptr;
      }
      if ((r = V.axpby(zeros, pa, gam, py))) return r;
    }
    for (int h = hmax - 1; h >= 0; --h) {  // oldest to newest
      for (int b = 0; b < B; ++b) {
        const int cnt = (int)mb[b].pairs.size();
        const bool use = active(b) && h < cnt;
        pa[b] = use ? Yslot(mb[b].pairs[cnt - 1 - h], b) : nullptr;
        pb[b] = use ? V.member(c->d, b) : nullptr;
      }
      if ((r = V.dot(pa, pb, tmp))) return r;
      std::vector<double> al(B, 0.0);
      for (int b = 0; b < B; ++b) {
        const int cnt = (int)mb[b].pairs.size();
        const bool use = active(b) && h < cnt;
        if (use) al[b] = -(alpha[b][h] - (-mb[b].rho[cnt - 1 - h] * tmp[b]));  // r += (alpha - beta) s
        pa[b] = use ? Sslot(mb[b].pairs[cnt - 1 - h], b) : nullptr;
        py[b] = use ? V.member(c->d, b) : nullptr;
      }
      if ((r = V.axpby(al, pa, ones, py))) return r;
    }
    for (int b = 0; b < B; ++b) {
      pa[b] = active(b) ? V.member(c->g, b) : nullptr;
      pb[b] = active(b) ? V.member(c->d, b) : nullptr;
    }
    std::vector<double> gd;
    if ((r = V.dot(pa, pb, gd))) return r;
    {
      std::vector<double> al(B, 0.0);
      bool reset = false;
      for (int b = 0; b < B; ++b) {
        pa[b] = nullptr;
        py[b] = nullptr;
        if (active(b) && !(gd[b] < 0.0)) {  // not a descent direction: restart from -g
          mb[b].pairs.clear();
          mb[b].rho.clear();
          al[b] = -1.0;
          pa[b] = V.member(c->g, b);
          py[b] = V.member(c->d, b);
          gd[b] = -mb[b].gnorm * mb[b].gnorm;
          reset = true;
        }
      }
      if (reset && (r = V.axpby(al, pa, zeros, py))) return r;
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
    std::vector<double> ft(B), dg;
    for (;;) {
      bool anys = false;
      for (int b = 0; b < B; ++b) anys |= searching[b] != 0;
      if (!anys) break;
      // xt = x + stp d for searching members, x otherwise
      DA_TRY_CUDA(c, cudaMemcpyAsync(c->xt, c->x, B * len * sizeof(double), cudaMemcpyDeviceToDevice, st));
      std::vector<double> al(B, 0.0);
      for (int b = 0; b < B; ++b) {
        al[b] = searching[b] ? ls[b].stp() : 0.0;
        pa[b] = searching[b] ? V.member(c->d, b) : nullptr;
        py[b] = searching[b] ? V.member(c->xt, b) : nullptr;
      }
      if ((r = V.axpby(al, pa, ones, py))) return r;
      if ((r = da_cost_grad(c, c->xt, ft.data(), c->gt, st))) return r;
      for (int b = 0; b < B; ++b) {
        pa[b] = searching[b] ? V.member(c->gt, b) : nullptr;
        pb[b] = searching[b] ? V.member(c->d, b) : nullptr;
      }
      if ((r = V.dot(pa, pb, dg))) return r;
      for (int b = 0; b < B; ++b) {
        if (!searching[b]) continue;
        if (!std::isfinite(ft[b]) || !std::isfinite(dg[b])) {
          searching[b] = 0;
          mb[b].state = 3;
          continue;
        }
        const int act = ls[b].step(ft[b], dg[b]);
        if (act == da::MoreThuente::EVALUATE) continue;
        searching[b] = 0;
        const bool ok = act == da::MoreThuente::CONVERGED;
        if (ok || ft[b] < mb[b].f) {
          // accept: new pair in a free slot, s = xt - x, y = gt - g
          int freeslot = 0;
          for (int t = 0; t < slots; ++t)
            if (std::find(mb[b].pairs.begin(), mb[b].pairs.end(), t) == mb[b].pairs.end()) {
              freeslot = t;
              break;
            }
          double* Sd = Sslot(freeslot, b);
          double* Yd = Yslot(freeslot, b);
          DA_TRY_CUDA(c, cudaMemcpyAsync(Sd, V.member(c->xt, b), len * sizeof(double), cudaMemcpyDeviceToDevice, st));
          DA_TRY_CUDA(c, cudaMemcpyAsync(Yd, V.member(c->gt, b), len * sizeof(double), cudaMemcpyDeviceToDevice, st));
          std::vector<double> neg(B, 0.0);
          std::vector<const double*> xs(B, nullptr);
          std::vector<double*> ys(B, nullptr);
          neg[b] = -1.0;
          xs[b] = V.member(c->x, b);
          ys[b] = Sd;
          if ((r = V.axpby(neg, xs, ones, ys))) return r;
          xs[b] = V.member(c->g, b);
          ys[b] = Yd;
          if ((r = V.axpby(neg, xs, ones, ys))) return r;
          std::vector<const double*> sa(B, nullptr), ya(B, nullptr);
          sa[b] = Sd;
          ya[b] = Yd;
          std::vector<double> sy, yy;
          if ((r = V.dot(sa, ya, sy))) return r;
          if ((r = V.dot(ya, ya, yy))) return r;
          if (sy[b] > 1e-16 * yy[b]) {
            if ((int)mb[b].pairs.size() == m) {
              mb[b].pairs.erase(mb[b].pairs.begin());
              mb[b].rho.erase(mb[b].rho.begin());
            }
            mb[b].pairs.push_back(freeslot);
            mb[b].rho.push_back(1.0 / sy[b]);
          }
          DA_TRY_CUDA(c, cudaMemcpyAsync(V.member(c->x, b), V.member(c->xt, b), len * sizeof(double),
                                         cudaMemcpyDeviceToDevice, st));
          DA_TRY_CUDA(c, cudaMemcpyAsync(V.member(c->g, b), V.member(c->gt, b), len * sizeof(double),
                                         cudaMemcpyDeviceToDevice, st));
          mb[b].f = ft[b];
          mb[b].iters = it + 1;
          J_hist[(size_t)b * (max_iter + 1) + it + 1] = ft[b];
        }
        if (!ok) mb[b].state = 2;
      }
    }
    for (int b = 0; b < B; ++b) pa[b] = V.member(c->g, b);
    if ((r = V.dot(pa, pa, tmp))) return r;
    for (int b = 0; b < B; ++b) mb[b].gnorm = std::sqrt(tmp[b]);
  }
  bool diverged = false, failed = false;
  for (int b = 0; b < B; ++b) {
    iters_done[b] = mb[b].iters;
    for (int it = mb[b].iters + 1; it <= max_iter; ++it) J_hist[(size_t)b * (max_iter + 1) + it] = mb[b].f;
    diverged |= mb[b].state == 3;
    failed |= mb[b].state == 2;
  }
  DA_TRY_CUDA(c, cudaMemcpyAsync(s, c->x, B * len * sizeof(double), cudaMemcpyDeviceToDevice, st));
  DA_TRY_CUDA(c, cudaStreamSynchronize(st));
  if (diverged) return fail(c, DA_EDIVERGED, "non-finite cost or gradient");
  if (failed) return fail(c, DA_ENOTCONV, "line search failed (step-size collapse)");
  return DA_OK;
}
