// da_api.cu -- the C ABI of include/da.h: context creation and
// validation, buffers, and the launch sequences of the forward solve, the
// adjoint sweep and their variants (cost and gradient, vector-Jacobian
// product, terminal adjoint, shell spectra).  The FFT plan variants and the
// autotuner are in plans.cu, the optimiser in lbfgs.cu.  All arithmetic of
// the path runs in the kernels of kernels.cuh; this file only orders
// launches and moves scalars.
#include <algorithm>
#include <cstring>

#include "ctx.h"

std::string g_create_error;

// exp(-2 pi i t / m), t < m, rounded from long double.
static std::vector<double2> roots_of_unity(int m) {
  std::vector<double2> w(m);
  const long double pi = 3.141592653589793238462643383279502884L;
  for (int t = 0; t < m; ++t) {
    long double a = -2.0L * pi * (long double)t / (long double)m;
    w[t] = make_double2((double)cosl(a), (double)sinl(a));
  }
  return w;
}

extern "C" da_status da_create(da_ctx** out, const da_grid* grid, double nu, const da_forcing* forcing,
                               const da_obs_operator* obs, const da_kernel* kernels) {
  if (!out) return fail(nullptr, DA_EINVAL, "out is NULL");
  *out = nullptr;
  if (!grid || !obs || !kernels) return fail(nullptr, DA_EINVAL, "grid, obs and kernels must not be NULL");
  const int n = grid->n;
  if (!da::ops_for(n)) return fail(nullptr, DA_EINVAL, "n must be a power of two in [16, 1024]");
  const Ops* ops = da::ops_for(n, grid->batch >= 1 ? cached_plan(n, grid->batch) : 0);
  if (grid->L != 0.0 && std::fabs(grid->L - 2.0 * M_PI) > 1e-12) return fail(nullptr, DA_EINVAL, "L must be 2 pi");
  if (!(grid->dt > 0.0) || !std::isfinite(grid->dt)) return fail(nullptr, DA_EINVAL, "dt must be positive");
  if (grid->nsteps < 1) return fail(nullptr, DA_EINVAL, "nsteps must be >= 1");
  if (grid->batch < 1) return fail(nullptr, DA_EINVAL, "batch must be >= 1");
  if (grid->ckpt_every < -1) return fail(nullptr, DA_EINVAL, "ckpt_every must be -1 (no store), 0 (all steps) or a checkpoint interval");
  if (!(nu >= 0.0) || !std::isfinite(nu)) return fail(nullptr, DA_EINVAL, "nu must be >= 0");
  da_forcing f{DA_FORCE_NONE, 0.0, 0};
  if (forcing) f = *forcing;
  if (f.kind != DA_FORCE_NONE && f.kind != DA_FORCE_KOLMOGOROV) return fail(nullptr, DA_EINVAL, "unknown forcing kind");
  if (f.kind == DA_FORCE_KOLMOGOROV && (f.nf < 1 || f.nf > ops->K))
    return fail(nullptr, DA_EINVAL, "forcing wavenumber must be in [1, floor((n-1)/3)]");
  if (obs->px != obs->py) return fail(nullptr, DA_EINVAL, "px must equal py");
  if (obs->px < 1 || obs->px > da::Geo<16>::PMAX || n % obs->px) return fail(nullptr, DA_EINVAL, "px must divide n and be <= 64");
  if (obs->every < 1 || grid->nsteps % obs->every) return fail(nullptr, DA_EINVAL, "obs.every must divide nsteps");
  for (int b = 0; b < grid->batch; ++b) {
    const da_kernel& k = kernels[b];
    if (k.kind < DA_KERNEL_IDENTITY || k.kind > DA_KERNEL_TABLE) return fail(nullptr, DA_EINVAL, "unknown kernel kind");
    if (k.kind == DA_KERNEL_TABLE && !k.table) return fail(nullptr, DA_EINVAL, "table kernel needs a table");
    if (!std::isfinite(k.param)) return fail(nullptr, DA_EINVAL, "kernel parameter must be finite");
  }

  da_ctx* c = new da_ctx();
  cudaGetDevice(&c->device);
  c->n = n;
  c->nsteps = grid->nsteps;
  c->ckpt = grid->ckpt_every;
  c->B = grid->batch;
  c->dt = grid->dt;
  c->nu = nu;
  c->force = f;
  c->obs = *obs;
  c->P = obs->px;
  c->nt = grid->nsteps / obs->every + (obs->include_t0 ? 1 : 0);
  c->ops = ops;

  Dev& d = c->dev;
  d.B = c->B;
  d.nsteps = c->nsteps;
  d.every = obs->every;
  d.include_t0 = obs->include_t0 ? 1 : 0;
  d.px = c->P;
  d.nt = c->nt;
  d.dt = c->dt;
  d.dt2 = c->dt / 2.0;
  d.dt3 = c->dt / 3.0;
  d.dt6 = c->dt / 6.0;
  d.nu = nu;
  d.force = f.kind == DA_FORCE_KOLMOGOROV;
  d.amp = f.amp;
  d.nf = f.nf;
  d.ragged = 0;
  d.obs_stride = (size_t)c->nt * c->P * c->P * 2;
  c->eval_steps = c->nsteps;
  c->m_nsteps.assign(c->B, c->nsteps);
  c->m_px.assign(c->B, c->P);
  c->m_nu.assign(c->B, nu);
  c->m_force.assign(c->B, d.force);

  const size_t B = c->B, N = n, comp = B * ops->Kr * ops->Kc, P2 = (size_t)c->P * c->P;
  da_status s = DA_OK;
  auto A = [&](da_status st) {
    if (s == DA_OK) s = st;
  };
  A(dalloc(c, &d.W, comp));
  A(dalloc(c, &d.Acc, comp));
  A(dalloc(c, &d.Y, comp));
  A(dalloc(c, &d.KB, comp));
  A(dalloc(c, &d.LamBar, comp));
  A(dalloc(c, &d.Sum, comp));
  A(dalloc(c, &d.Mx, B * 2 * N * ops->Kc));
  A(dalloc(c, &d.Mn, B * 2 * N * ops->Kc));
  A(dalloc(c, &d.obs, B * c->nt * P2 * 2));
  A(dalloc(c, (double**)&d.mobs, B * c->nt * P2 * 2));
  A(dalloc(c, &d.res, B * c->nt * P2 * 2));
  A(dalloc(c, &d.J, B));
  A(dalloc(c, (double**)&d.mult, comp));
  size_t fold_max = 0;  // room for the folded table of any plan variant
  for (int v = 0; v < da::plan_count(n); ++v) fold_max = std::max(fold_max, (size_t)da::ops_for(n, v)->fold_doubles);
  A(dalloc(c, (double**)&d.fold, fold_max));
  A(dalloc(c, (double2**)&d.twP, (size_t)64));
  A(dalloc(c, (da::Sym4**)&d.symF, comp / B));
  A(dalloc(c, (da::Sym4**)&d.symA, comp / B));
  A(dalloc(c, (double**)&d.k2, comp / B));
  A(dalloc(c, &c->d_mstart, B));
  A(dalloc(c, &c->d_mnt, B));
  A(dalloc(c, &c->d_mpx, B));
  A(dalloc(c, &c->d_mforce, B));
  A(dalloc(c, &c->d_mnu, B));
  d.mstart = c->d_mstart;
  d.mnt = c->d_mnt;
  d.mpx = c->d_mpx;
  d.mforce = c->d_mforce;
  d.mnu = c->d_mnu;
  // stage-field store: the whole window, or one checkpoint segment
  if (c->ckpt == 0) {
    d.traj_steps = c->nsteps;
  } else if (c->ckpt > 0) {
    d.traj_steps = std::min(c->ckpt, c->nsteps);
    c->nckpt = (c->nsteps + c->ckpt - 1) / c->ckpt;
    A(dalloc(c, &c->ckpt_buf, (size_t)c->nckpt * comp));
  }
  if (c->ckpt >= 0) A(dalloc(c, &d.traj, B * (size_t)d.traj_steps * 8 * N * N));
  A(dalloc(c, &c->d_kind, B));
  A(dalloc(c, &c->d_param, B));
  bool any_table = false;
  for (int b = 0; b < c->B; ++b) any_table |= kernels[b].kind == DA_KERNEL_TABLE;
  if (any_table) A(dalloc(c, &c->d_table, B * N * (N / 2 + 1)));
  int* d_kind = c->d_kind;
  double *d_param = c->d_param, *d_table = c->d_table;
  if (s != DA_OK) {
    g_create_error = c->err;
    da_destroy(c);
    return s;
  }
  // constant tables: folded twiddles of the FFT plan, twiddles of the probe
  // lattice
  std::vector<double> fold(ops->fold_doubles);
  ops->fold_table(fold.data());
  std::vector<double2> twP = roots_of_unity(64);
  std::vector<int>& kind = c->h_kind;
  std::vector<double>& param = c->h_param;
  kind.resize(B);
  param.resize(B);
  for (size_t b = 0; b < B; ++b) {
    kind[b] = kernels[b].kind;
    param[b] = kernels[b].param;
  }
  cudaError_t e = cudaMemcpy((void*)d.fold, fold.data(), fold.size() * sizeof(double), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy((void*)d.twP, twP.data(), 64 * sizeof(double2), cudaMemcpyHostToDevice);
  // per-mode symbols of the column passes, column-major [Kc][Kr]
  const int K = ops->K, Kr = ops->Kr, Kc = ops->Kc;
  std::vector<da::Sym4> symF((size_t)Kr * Kc), symA((size_t)Kr * Kc);
  std::vector<double> k2tab((size_t)Kr * Kc);
  const double s2 = 1.0 / ((double)n * n);
  for (int kx = 0; kx < Kc; ++kx)
    for (int r = 0; r < Kr; ++r) {
      const int ky = r <= K ? r : r - Kr;
      const double k2 = (double)(kx * kx + ky * ky);
      const double ik2 = k2 > 0.0 ? 1.0 / k2 : 0.0;
      const size_t i = (size_t)kx * Kr + r;
      symF[i] = {ky * ik2 * s2, kx * ik2 * s2, 0.5 * (ky * ky - kx * kx), -0.5 * kx * ky};
      symA[i] = {0.5 * ky * ik2, 0.5 * kx * ik2, -2.0 * kx * ky * s2, (double)(ky * ky - kx * kx) * s2};
      k2tab[i] = k2;
    }
  if (e == cudaSuccess) e = cudaMemcpy((void*)d.symF, symF.data(), symF.size() * sizeof(da::Sym4), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy((void*)d.symA, symA.data(), symA.size() * sizeof(da::Sym4), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy((void*)d.k2, k2tab.data(), k2tab.size() * sizeof(double), cudaMemcpyHostToDevice);
  {
    const std::vector<int> zeros(B, 0), nts(B, c->nt), pxs(B, c->P), forces(B, d.force);
    const std::vector<double> nus(B, nu);
    if (e == cudaSuccess) e = cudaMemcpy(c->d_mstart, zeros.data(), B * sizeof(int), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(c->d_mnt, nts.data(), B * sizeof(int), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(c->d_mpx, pxs.data(), B * sizeof(int), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(c->d_mforce, forces.data(), B * sizeof(int), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(c->d_mnu, nus.data(), B * sizeof(double), cudaMemcpyHostToDevice);
  }
  if (e == cudaSuccess) e = cudaMemcpy(d_kind, kind.data(), B * sizeof(int), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(d_param, param.data(), B * sizeof(double), cudaMemcpyHostToDevice);
  for (size_t b = 0; b < B && e == cudaSuccess; ++b)
    if (kernels[b].kind == DA_KERNEL_TABLE)
      e = cudaMemcpy(d_table + b * N * (N / 2 + 1), kernels[b].table, N * (N / 2 + 1) * sizeof(double),
                     cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(d.obs, 0, B * c->nt * P2 * 2 * sizeof(double));
  if (e == cudaSuccess) e = ops->setup();
  if (e != cudaSuccess) {
    g_create_error = std::string("setup: ") + cudaGetErrorString(e);
    da_destroy(c);
    return DA_ECUDA;
  }
  // the multiplier on a stream of its own, waited for alone (a device-wide
  // wait would also disturb other threads' work, e.g. a graph capture)
  cudaStream_t mk = nullptr;
  e = cudaStreamCreateWithFlags(&mk, cudaStreamNonBlocking);
  if (e == cudaSuccess) {
    ops->make_mult(d, (double*)d.mult, d_kind, d_param, d_table, c->d_mnu, mk);
    c->launches++;
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(mk);
    cudaStreamDestroy(mk);
  }
  std::vector<double> mult(comp);
  if (e == cudaSuccess) e = cudaMemcpy(mult.data(), d.mult, comp * sizeof(double), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) {
    g_create_error = std::string("kernel table: ") + cudaGetErrorString(e);
    da_destroy(c);
    return DA_ECUDA;
  }
  for (double m : mult)
    if (!std::isfinite(m) || m < 0.0) {
      g_create_error = "kernel W is not finite and non-negative on the retained set";
      da_destroy(c);
      return DA_EINVAL;
    }
  *out = c;
  return DA_OK;
}

extern "C" da_status da_time_kernels(da_ctx* c, int kernel_class) {
  if (!c || kernel_class < 0 || kernel_class > 4) return fail(c, DA_EINVAL, "kernel_class must be in [0, 4]");
  c->timed_class = kernel_class;  // while on, da_cost_grad launches directly, not by graph
  c->ev_used = 0;
  return DA_OK;
}

extern "C" da_status da_kernel_time(da_ctx* c, double* total_ms, unsigned long long* launches) {
  if (!c || !total_ms || !launches) return fail(c, DA_EINVAL, "arguments must not be NULL");
  double tot = 0.0;
  if (c->ev_used) DA_TRY_CUDA(c, cudaEventSynchronize(c->ev[c->ev_used - 1]));
  for (size_t i = 0; i + 1 < c->ev_used; i += 2) {
    float ms = 0.f;
    DA_TRY_CUDA(c, cudaEventElapsedTime(&ms, c->ev[i], c->ev[i + 1]));
    tot += ms;
  }
  *total_ms = tot;
  *launches = c->ev_used / 2;
  c->ev_used = 0;
  return DA_OK;
}

extern "C" void da_destroy(da_ctx* c) {
  if (!c) return;
  free_optimiser(c);
  drop_graphs(c);
  if (c->sp_exec) cudaGraphExecDestroy(c->sp_exec);
  if (c->ev_in) cudaEventDestroy(c->ev_in);
  if (c->ev_out) cudaEventDestroy(c->ev_out);
  if (c->gstream) cudaStreamDestroy(c->gstream);
  for (cudaEvent_t e : c->ev) cudaEventDestroy(e);
  for (void* p : c->allocs) cudaFree(p);
  if (c->lb_host) cudaFreeHost(c->lb_host);
  delete c;
}

extern "C" const char* da_last_error(const da_ctx* c) { return c ? c->err.c_str() : g_create_error.c_str(); }
extern "C" int da_num_obs_times(const da_ctx* c) { return c ? c->nt : 0; }
extern "C" unsigned long long da_device_bytes(const da_ctx* c) { return c ? c->bytes : 0; }
extern "C" unsigned long long da_launch_count(const da_ctx* c) { return c ? c->launches : 0; }

extern "C" da_status da_set_sobolev(da_ctx* c, double lambda) {
  if (!c || !std::isfinite(lambda) || lambda < 0.0) return fail(c, DA_EINVAL, "lambda must be finite and >= 0");
  if (lambda != 0.0 && !c->w0) {
    da_status r = dalloc(c, &c->w0, (size_t)c->B * c->ops->Kr * c->ops->Kc);
    if (r) return r;
  }
  c->sobolev = lambda;
  drop_graphs(c);  // the captured sequences depend on the regularisation
  return DA_OK;
}

extern "C" da_status da_set_observations(da_ctx* c, const double* m, void* stream) {
  if (!c || !m) return fail(c, DA_EINVAL, "ctx and m must not be NULL");
  const size_t bytes = (size_t)c->B * c->nt * c->P * c->P * 2 * sizeof(double);
  DA_TRY_CUDA(c, cudaMemcpyAsync((void*)c->dev.mobs, m, bytes, cudaMemcpyDefault, (cudaStream_t)stream));
  c->have_obs = true;
  return DA_OK;
}

// Forward window from control s.  With storage, the stage fields of every
// step (ckpt == 0) or the state every ckpt steps plus the stage fields of the
// last segment (ckpt > 0) are kept for the adjoint.  gather: fill the model
// observations.
static da_status run_forward(da_ctx* c, const double* s, bool gather, cudaStream_t st) {
  const Ops* o = c->ops;
  Dev& d = c->dev;
  const bool store = d.traj != nullptr;
  const int E = c->eval_steps;  // the evaluation's window (all of nsteps unless a ragged batch is shorter)
  const int K = c->ckpt > 0 ? c->ckpt : E;
  const int last0 = ((E - 1) / K) * K;  // first step of the last segment
  const size_t comp = (size_t)c->B * o->Kr * o->Kc;
  c->have_fwd = false;
  o->r2c_rows(d, s, st);
  o->ctrl_cols(d, 0, st);
  da_status r = check_launch(c, 2);
  if (r) return r;
  if (c->w0) DA_TRY_CUDA(c, cudaMemcpyAsync(c->w0, d.W, comp * sizeof(double2), cudaMemcpyDeviceToDevice, st));
  d.seg0 = last0;
  if (c->ckpt == 0) d.seg0 = 0;
  for (int k = 0; k < E; ++k) {
    if (c->ckpt > 0 && store && k % K == 0)
      DA_TRY_CUDA(c, cudaMemcpyAsync(c->ckpt_buf + (size_t)(k / K) * comp, d.W, comp * sizeof(double2),
                                     cudaMemcpyDeviceToDevice, st));
    const int obs_flag = (gather && obs_step_host(c, k)) ? da::F_OBS : 0;
    const int store_flag = (store && k >= d.seg0) ? da::F_STORE : 0;
    for (int j = 1; j <= 4; ++j) {
      {
        Timed t(c, 1, st);
        o->fwd_rows(d, k, j, store_flag | (j == 1 ? obs_flag : 0), st);
      }
      Timed t(c, 2, st);
      o->fwd_cols(d, k, j, 0, st);
    }
    if ((r = check_launch(c, 8))) return r;
  }
  if (gather && obs_step_host(c, E)) {
    o->fwd_rows(d, E, 1, da::F_OBS_ONLY, st);
    if ((r = check_launch(c))) return r;
  }
  c->have_fwd = store;
  return DA_OK;
}

// Where the adjoint sweep records shell spectra (every `every` steps of
// backward time, slot (nsteps - k)/every).
struct SpectraOut {
  int every = 0;
  double* member = nullptr;  // [B][nsave][nshell]
  double* mean = nullptr;    // [nsave][nshell]
  double* scratch = nullptr; // [B][nshell]
};

static da_status record_spectra(da_ctx* c, const SpectraOut* sp, int k, cudaStream_t st) {
  if (!sp || sp->every <= 0 || (c->nsteps - k) % sp->every) return DA_OK;
  const int slot = (c->nsteps - k) / sp->every;
  const int nsave = c->nsteps / sp->every + 1;
  const int nmodes = c->ops->Kr * c->ops->Kc;
  if (sp->member) {
    da::k_shell_member<<<dim3(c->nshell, c->B), 128, 0, st>>>(c->dev.LamBar, c->shell_off, c->shell_mode,
                                                              c->shell_wgt, nmodes, sp->scratch, c->nshell);
    da_status r = check_launch(c);
    if (r) return r;
    // scratch [B][nshell] -> member[b][slot][:]
    DA_TRY_CUDA(c, cudaMemcpy2DAsync(sp->member + (size_t)slot * c->nshell, (size_t)nsave * c->nshell * sizeof(double),
                                     sp->scratch, (size_t)c->nshell * sizeof(double), c->nshell * sizeof(double), c->B,
                                     cudaMemcpyDeviceToDevice, st));
  }
  if (sp->mean) {
    da::k_shell_mean<<<c->nshell, 128, 0, st>>>(c->dev.LamBar, c->B, c->shell_off, c->shell_mode, c->shell_wgt,
                                                 nmodes, sp->mean + (size_t)slot * c->nshell);
    da_status r = check_launch(c);
    if (r) return r;
  }
  return DA_OK;
}

// Backward sweep from the state in LamBar/KB/Mx (set by adj_init), segment by
// segment from the last.  With checkpoints, every segment but the last is
// first recomputed from its checkpoint (bitwise the same stage fields as the
// first pass), then the inverse column transforms of the adjoint fields of
// kbar, which the forward recompute overwrote, are redone.
static da_status run_adjoint(da_ctx* c, bool sources, cudaStream_t st, const SpectraOut* sp = nullptr) {
  const Ops* o = c->ops;
  Dev& d = c->dev;
  const int E = c->eval_steps;
  const int K = c->ckpt > 0 ? c->ckpt : E;
  const int nseg = (E + K - 1) / K;
  const size_t comp = (size_t)c->B * o->Kr * o->Kc;
  da_status r;
  for (int seg = nseg - 1; seg >= 0; --seg) {
    const int k0 = seg * K, k1 = std::min(k0 + K, E);
    if (seg != nseg - 1) {
      DA_TRY_CUDA(c, cudaMemcpyAsync(d.W, c->ckpt_buf + (size_t)seg * comp, comp * sizeof(double2),
                                     cudaMemcpyDeviceToDevice, st));
      d.seg0 = k0;
      o->state_cols(d, st);
      if ((r = check_launch(c))) return r;
      for (int k = k0; k < k1; ++k) {
        for (int j = 1; j <= 4; ++j) {
          {
            Timed t(c, 1, st);
            o->fwd_rows(d, k, j, da::F_STORE, st);
          }
          Timed t(c, 2, st);
          o->fwd_cols(d, k, j, 0, st);
        }
        if ((r = check_launch(c, 8))) return r;
      }
      o->adj_init(d, da::INIT_RESUME, st);
      if ((r = check_launch(c))) return r;
    }
    d.seg0 = k0;
    for (int k = k1 - 1; k >= k0; --k) {
      for (int j = 4; j >= 1; --j) {
        const int flags = (j == 1 && sources && obs_step_host(c, k)) ? da::F_SRC : 0;
        {
          Timed t(c, 3, st);
          o->adj_rows(d, k, j, st);
        }
        Timed t(c, 4, st);
        o->adj_cols(d, k, j, flags, st);
      }
      if ((r = check_launch(c, 8))) return r;
      if ((r = record_spectra(c, sp, k, st))) return r;
    }
  }
  // the stored segment is now the first one; a later vjp must rerun the forward
  c->have_fwd = c->ckpt == 0;
  return DA_OK;
}

static da_status copy_scalars_out(da_ctx* c, double* J, cudaStream_t st) {
  if (!J) return DA_OK;
  cudaPointerAttributes at{};
  cudaError_t e = cudaPointerGetAttributes(&at, J);
  if (e != cudaSuccess) {
    cudaGetLastError();
    at.type = cudaMemoryTypeUnregistered;
  }
  const bool dev = at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
  DA_TRY_CUDA(c, cudaMemcpyAsync(J, c->dev.J, c->B * sizeof(double), cudaMemcpyDefault, st));
  if (!dev) DA_TRY_CUDA(c, cudaStreamSynchronize(st));
  return DA_OK;
}

static da_status gradient_out(da_ctx* c, double* grad_s, cudaStream_t st) {
  if (!grad_s) return DA_OK;
  c->ops->spec_to_mixed(c->dev, c->dev.LamBar, da::M_CTRL, st);
  c->ops->c2r_rows(c->dev, grad_s, st);
  return check_launch(c, 2);
}

da_status set_eval_window(da_ctx* c, const std::vector<char>* live, cudaStream_t st) {
  if (!c->ragged) {
    c->eval_steps = c->nsteps;
    c->dev.nsteps = c->nsteps;
    return DA_OK;
  }
  int E = 0;
  for (int b = 0; b < c->B; ++b)
    if ((!live || (*live)[b]) && c->m_nsteps[b] > 0) E = std::max(E, c->m_nsteps[b]);
  if (E == 0) E = c->obs.every;  // nothing live: a minimal window over idle members
  std::vector<int> start(c->B);
  for (int b = 0; b < c->B; ++b) {
    const bool on = (!live || (*live)[b]) && c->m_nsteps[b] > 0;
    start[b] = on ? E - c->m_nsteps[b] : E + 1;  // idle: later than the window's last step
  }
  DA_TRY_CUDA(c, cudaMemcpyAsync(c->d_mstart, start.data(), c->B * sizeof(int), cudaMemcpyHostToDevice, st));
  c->eval_steps = E;
  c->dev.nsteps = E;
  return DA_OK;
}

extern "C" da_status da_set_member(da_ctx* c, int member, const da_member_window* w, const da_kernel* kernel,
                                   const double* m, void* stream) {
  if (!c || !w) return fail(c, DA_EINVAL, "ctx and w must not be NULL");
  if (member < 0 || member >= c->B) return fail(c, DA_EINVAL, "member out of range");
  if (w->nsteps < 0 || w->nsteps > c->nsteps || w->nsteps % c->obs.every)
    return fail(c, DA_EINVAL, "member nsteps must be a multiple of obs.every in [0, the context's nsteps]");
  if (w->nsteps > 0) {
    if (w->px < 1 || w->px > c->P || c->n % w->px)
      return fail(c, DA_EINVAL, "member px must divide n and be at most the context's px");
    if (!(w->nu >= 0.0) || !std::isfinite(w->nu)) return fail(c, DA_EINVAL, "member nu must be finite and >= 0");
    if (w->forcing != 0 && w->forcing != 1) return fail(c, DA_EINVAL, "member forcing must be 0 or 1");
    if (w->forcing && !c->dev.force) return fail(c, DA_EINVAL, "member forcing needs a context created with forcing");
    if (!kernel) return fail(c, DA_EINVAL, "kernel must not be NULL");
    if (kernel->kind < DA_KERNEL_IDENTITY || kernel->kind > DA_KERNEL_TABLE || !std::isfinite(kernel->param))
      return fail(c, DA_EINVAL, "unknown kernel kind or non-finite parameter");
    if (kernel->kind == DA_KERNEL_TABLE && !kernel->table) return fail(c, DA_EINVAL, "table kernel needs a table");
    if (!m) return fail(c, DA_EINVAL, "observations must not be NULL");
  }
  cudaStream_t st = (cudaStream_t)stream;
  const int n = c->n;
  const int nt = w->nsteps > 0 ? w->nsteps / c->obs.every + (c->obs.include_t0 ? 1 : 0) : 0;
  // work in flight may read the member's tables, multiplier and data
  DA_TRY_CUDA(c, cudaStreamSynchronize(st));
  if (w->nsteps > 0) {
    if (kernel->kind == DA_KERNEL_TABLE) {
      if (!c->d_table) {
        da_status r = dalloc(c, &c->d_table, (size_t)c->B * n * (n / 2 + 1));
        if (r) return r;
      }
      DA_TRY_CUDA(c, cudaMemcpy(c->d_table + (size_t)member * n * (n / 2 + 1), kernel->table,
                                (size_t)n * (n / 2 + 1) * sizeof(double), cudaMemcpyHostToDevice));
    }
    const int kind = kernel->kind;
    const double param = kernel->param;
    DA_TRY_CUDA(c, cudaMemcpy(c->d_kind + member, &kind, sizeof(int), cudaMemcpyHostToDevice));
    DA_TRY_CUDA(c, cudaMemcpy(c->d_param + member, &param, sizeof(double), cudaMemcpyHostToDevice));
    // the multiplier of every member with its kernel and viscosity; this
    // member's must be finite and non-negative on the retained set
    DA_TRY_CUDA(c, cudaMemcpy(c->d_mnu + member, &w->nu, sizeof(double), cudaMemcpyHostToDevice));
    c->ops->make_mult(c->dev, (double*)c->dev.mult, c->d_kind, c->d_param, c->d_table, c->d_mnu, 0);
    da_status r = check_launch(c);
    if (r) return r;
    const size_t nm = (size_t)c->ops->Kr * c->ops->Kc;
    std::vector<double> mult(nm);
    DA_TRY_CUDA(c, cudaMemcpy(mult.data(), c->dev.mult + member * nm, nm * sizeof(double), cudaMemcpyDeviceToHost));
    for (double v : mult)
      if (!std::isfinite(v) || v < 0.0) {
        c->m_nsteps[member] = 0;  // the slot stays idle
        return fail(c, DA_EINVAL, "kernel W is not finite and non-negative on the retained set");
      }
    c->h_kind[member] = kind;
    c->h_param[member] = param;
    const size_t cnt = (size_t)nt * w->px * w->px * 2;
    DA_TRY_CUDA(c, cudaMemcpyAsync((void*)(c->dev.mobs + member * c->dev.obs_stride), m, cnt * sizeof(double),
                                   cudaMemcpyDefault, st));
    c->m_px[member] = w->px;
    c->m_nu[member] = w->nu;
    c->m_force[member] = w->forcing;
  }
  c->m_nsteps[member] = w->nsteps;
  const int px = c->m_px[member], force = c->m_force[member];
  const double nu = c->m_nu[member];
  DA_TRY_CUDA(c, cudaMemcpy(c->d_mnt + member, &nt, sizeof(int), cudaMemcpyHostToDevice));
  DA_TRY_CUDA(c, cudaMemcpy(c->d_mpx + member, &px, sizeof(int), cudaMemcpyHostToDevice));
  DA_TRY_CUDA(c, cudaMemcpy(c->d_mforce + member, &force, sizeof(int), cudaMemcpyHostToDevice));
  DA_TRY_CUDA(c, cudaMemcpy(c->d_mnu + member, &nu, sizeof(double), cudaMemcpyHostToDevice));
  if (!c->ragged) {
    drop_graphs(c);  // captured sequences hold the homogeneous kernel arguments
    c->ragged = true;
    c->dev.ragged = 1;
    c->have_obs = true;  // the other members keep the observations they had (or zeros)
  }

  c->have_fwd = false;
  return DA_OK;
}

extern "C" da_status da_forward(da_ctx* c, const double* s, double* omegaT, double* obs, void* stream) {
  if (!c || !s) return fail(c, DA_EINVAL, "ctx and s must not be NULL");
  cudaStream_t st = (cudaStream_t)stream;
  da_status r = set_eval_window(c, nullptr, st);
  if (r) return r;
  r = run_forward(c, s, obs != nullptr, st);
  if (r) return r;
  if (omegaT) {
    c->ops->compact_to_half(c->dev, c->dev.W, (double2*)omegaT, st);
    if ((r = check_launch(c))) return r;
  }
  if (obs)
    DA_TRY_CUDA(c, cudaMemcpyAsync(obs, c->dev.obs, (size_t)c->B * c->nt * c->P * c->P * 2 * sizeof(double),
                                   cudaMemcpyDefault, st));
  return DA_OK;
}

// The launch sequence of one cost-and-gradient evaluation, on stream st.
static da_status enqueue_cost_grad(da_ctx* c, const double* s, double* grad_s, cudaStream_t st) {
  da_status r = run_forward(c, s, true, st);
  if (r) return r;
  da::k_residual<<<c->B, 256, 0, st>>>(c->dev);
  if (c->sobolev != 0.0) {
    da::k_sobolev_cost<<<c->B, 256, 0, st>>>(c->dev.J, c->w0, c->sobolev, c->n, c->ops->Kr, c->ops->Kc);
    if ((r = check_launch(c))) return r;
  }
  c->ops->adj_init(c->dev, da::INIT_SRC, st);
  if ((r = check_launch(c, 2))) return r;
  if ((r = run_adjoint(c, true, st))) return r;
  if (c->sobolev != 0.0) {
    const int count = c->B * c->ops->Kr * c->ops->Kc;
    da::k_sobolev_grad<<<(count + 255) / 256, 256, 0, st>>>(c->dev.LamBar, c->w0, c->sobolev, count);
    if ((r = check_launch(c))) return r;
  }
  return gradient_out(c, grad_s, st);
}

extern "C" da_status da_set_graphs(da_ctx* c, int enable) {
  if (!c) return fail(c, DA_EINVAL, "ctx must not be NULL");
  if (!enable) {
    c->use_graph = false;
    return DA_OK;
  }
  if (!c->gstream) {
    const size_t len = (size_t)c->B * c->n * c->n;
    da_status r = dalloc(c, &c->sbuf, len);
    if (!r) r = dalloc(c, &c->gbuf, len);
    if (r) return r;
    DA_TRY_CUDA(c, cudaStreamCreateWithFlags(&c->gstream, cudaStreamNonBlocking));
    DA_TRY_CUDA(c, cudaEventCreateWithFlags(&c->ev_in, cudaEventDisableTiming));
    DA_TRY_CUDA(c, cudaEventCreateWithFlags(&c->ev_out, cudaEventDisableTiming));
  }
  c->use_graph = true;
  return DA_OK;
}

extern "C" da_status da_cost_grad(da_ctx* c, const double* s, double* J, double* grad_s, void* stream) {
  if (!c || !s) return fail(c, DA_EINVAL, "ctx and s must not be NULL");
  if (!c->have_obs) return fail(c, DA_EINVAL, "no observations: call da_set_observations first");
  if (!c->dev.traj) return fail(c, DA_EINVAL, "context was created forward-only (ckpt_every < 0)");
  return cost_grad_members(c, s, J, grad_s, nullptr, (cudaStream_t)stream);
}

da_status cost_grad_members(da_ctx* c, const double* s, double* J, double* grad_s, const std::vector<char>* live,
                            cudaStream_t st) {
  da_status r = set_eval_window(c, live, st);
  if (r) return r;
  if (c->use_graph && c->timed_class == 0) {
    // one captured sequence per evaluation window (its launch count)
    const size_t bytes = (size_t)c->B * c->n * c->n * sizeof(double);
    DA_TRY_CUDA(c, cudaMemcpyAsync(c->sbuf, s, bytes, cudaMemcpyDeviceToDevice, st));
    DA_TRY_CUDA(c, cudaEventRecord(c->ev_in, st));
    DA_TRY_CUDA(c, cudaStreamWaitEvent(c->gstream, c->ev_in, 0));
    da_ctx::CapturedEval* ce = nullptr;
    for (auto& g : c->cg_cache)
      if (g.steps == c->eval_steps) ce = &g;
    bool direct = false;
    if (!ce) {
      cudaGraph_t g = nullptr;
      cudaGraphExec_t ex = nullptr;
      const unsigned long long l0 = c->launches;
      DA_TRY_CUDA(c, cudaStreamBeginCapture(c->gstream, cudaStreamCaptureModeThreadLocal));
      r = enqueue_cost_grad(c, c->sbuf, c->gbuf, c->gstream);
      cudaError_t e = cudaStreamEndCapture(c->gstream, &g);
      if (r || e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        c->launches = l0;
        // Another thread's device-wide synchronisation (a cudaFree, say)
        // invalidates a capture in flight: nothing of it ran, so this
        // evaluation runs by direct launches instead, and a later call
        // captures again.
        if (e != cudaErrorStreamCaptureInvalidated && (r != DA_ECUDA || e == cudaSuccess))
          return r ? r : fail(c, DA_ECUDA, std::string("graph capture: ") + cudaGetErrorString(e));
        direct = true;
      } else {
        e = cudaGraphInstantiate(&ex, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) return fail(c, DA_ECUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
        if (c->cg_cache.size() >= kMaxCapturedEvals) {  // evict the oldest
          cudaGraphExecDestroy(c->cg_cache.front().exec);
          c->cg_cache.erase(c->cg_cache.begin());
        }
        c->cg_cache.push_back({c->eval_steps, ex, c->launches - l0});
        c->launches = l0;
        ce = &c->cg_cache.back();
      }
    }
    if (direct) {
      if ((r = enqueue_cost_grad(c, c->sbuf, c->gbuf, c->gstream))) return r;
    } else {
      DA_TRY_CUDA(c, cudaGraphLaunch(ce->exec, c->gstream));
      c->launches += ce->launches;
    }
    c->have_fwd = c->ckpt == 0;
    DA_TRY_CUDA(c, cudaEventRecord(c->ev_out, c->gstream));
    DA_TRY_CUDA(c, cudaStreamWaitEvent(st, c->ev_out, 0));
    if (grad_s) DA_TRY_CUDA(c, cudaMemcpyAsync(grad_s, c->gbuf, bytes, cudaMemcpyDeviceToDevice, st));
  } else {
    if ((r = enqueue_cost_grad(c, s, grad_s, st))) return r;
  }
  c->have_adj = true;
  return copy_scalars_out(c, J, st);
}

extern "C" da_status da_adjoint_terminal(da_ctx* c, const double* s, const double* lamT, double* grad_s, void* stream) {
  if (!c || !s || !lamT) return fail(c, DA_EINVAL, "ctx, s and lamT must not be NULL");
  if (!c->dev.traj) return fail(c, DA_EINVAL, "context was created forward-only (ckpt_every < 0)");
  cudaStream_t st = (cudaStream_t)stream;
  da_status r = set_eval_window(c, nullptr, st);
  if (r) return r;
  r = run_forward(c, s, false, st);
  if (r) return r;
  c->ops->half_to_compact(c->dev, (const double2*)lamT, c->dev.LamBar, st);
  c->ops->adj_init(c->dev, da::INIT_LAMBAR, st);
  if ((r = check_launch(c, 2))) return r;
  if ((r = run_adjoint(c, false, st))) return r;
  c->have_adj = true;
  return gradient_out(c, grad_s, st);
}

extern "C" da_status da_vjp(da_ctx* c, const double* dobs, const double* dwT, double* grad_s, void* stream) {
  if (!c) return fail(c, DA_EINVAL, "ctx must not be NULL");
  if (!c->have_fwd) return fail(c, DA_EINVAL, "da_vjp needs a stored forward: call da_forward on this context first");
  cudaStream_t st = (cudaStream_t)stream;
  const size_t nobs = (size_t)c->B * c->nt * c->P * c->P * 2;
  if (dobs)
    DA_TRY_CUDA(c, cudaMemcpyAsync(c->dev.res, dobs, nobs * sizeof(double), cudaMemcpyDefault, st));
  if (dwT) {
    c->ops->half_to_compact(c->dev, (const double2*)dwT, c->dev.LamBar, st);
    da_status r = check_launch(c);
    if (r) return r;
  }
  c->ops->adj_init(c->dev, (dwT ? da::INIT_LAMBAR : 0) | (dobs ? da::INIT_SRC : 0), st);
  da_status r = check_launch(c);
  if (r) return r;
  if ((r = run_adjoint(c, dobs != nullptr, st))) return r;
  c->have_adj = true;
  return gradient_out(c, grad_s, st);
}

// Mode lists per shell k <= |k| < k+1 over the compact set, with weights
// (1 or 2) k^2 / (2 N^4) turning |lambda_hat|^2 into the shell energy of
// the adjoint velocity.
static da_status build_shells(da_ctx* c) {
  if (c->nshell) return DA_OK;
  const int K = c->ops->K, Kc = c->ops->Kc, Kr = c->ops->Kr;
  const int nshell = (int)std::floor(std::sqrt(2.0) * K) + 1;
  std::vector<std::vector<int>> modes(nshell);
  std::vector<std::vector<double>> wgts(nshell);
  const double n4 = std::pow((double)c->n, 4);
  for (int r = 0; r < Kr; ++r)
    for (int kx = 0; kx < Kc; ++kx) {
      const int ky = r <= K ? r : r - Kr;
      const double k2 = (double)kx * kx + (double)ky * ky;
      if (k2 == 0.0) continue;
      const int sh = (int)std::floor(std::sqrt(k2));
      modes[sh].push_back(kx * Kr + r);  // compact arrays are column-major
      wgts[sh].push_back((kx == 0 ? 1.0 : 2.0) * k2 / (2.0 * n4));
    }
  std::vector<int> off(nshell + 1, 0), mode;
  std::vector<double> wgt;
  for (int sh = 0; sh < nshell; ++sh) {
    off[sh + 1] = off[sh] + (int)modes[sh].size();
    mode.insert(mode.end(), modes[sh].begin(), modes[sh].end());
    wgt.insert(wgt.end(), wgts[sh].begin(), wgts[sh].end());
  }
  da_status r = DA_OK;
  auto A = [&](da_status x) {
    if (r == DA_OK) r = x;
  };
  A(dalloc(c, &c->shell_off, off.size()));
  A(dalloc(c, &c->shell_mode, mode.size()));
  A(dalloc(c, &c->shell_wgt, wgt.size()));
  if (r) return r;
  DA_TRY_CUDA(c, cudaMemcpy(c->shell_off, off.data(), off.size() * sizeof(int), cudaMemcpyHostToDevice));
  DA_TRY_CUDA(c, cudaMemcpy(c->shell_mode, mode.data(), mode.size() * sizeof(int), cudaMemcpyHostToDevice));
  DA_TRY_CUDA(c, cudaMemcpy(c->shell_wgt, wgt.data(), wgt.size() * sizeof(double), cudaMemcpyHostToDevice));
  c->nshell = nshell;
  return DA_OK;
}

extern "C" int da_num_shells(const da_ctx* c) { return c ? (int)std::floor(std::sqrt(2.0) * c->ops->K) + 1 : 0; }

// The launch sequence of da_adjoint_spectra on stream st (buffers set up).
static da_status enqueue_spectra(da_ctx* c, const double* s, const double* lamT, const SpectraOut& sp,
                                 cudaStream_t st) {
  da_status r = run_forward(c, s, false, st);
  if (r) return r;
  c->ops->half_to_compact(c->dev, (const double2*)lamT, c->dev.LamBar, st);
  c->ops->adj_init(c->dev, da::INIT_LAMBAR, st);
  if ((r = check_launch(c, 2))) return r;
  if ((r = record_spectra(c, &sp, c->nsteps, st))) return r;
  return run_adjoint(c, false, st, &sp);
}

extern "C" da_status da_adjoint_spectra(da_ctx* c, const double* s, const double* lamT, int save_every,
                                        double* member, double* mean, void* stream) {
  if (!c || !s || !lamT) return fail(c, DA_EINVAL, "ctx, s and lamT must not be NULL");
  if (save_every < 1 || c->nsteps % save_every) return fail(c, DA_EINVAL, "save_every must divide nsteps");
  if (!c->dev.traj) return fail(c, DA_EINVAL, "context was created forward-only (ckpt_every < 0)");
  if (c->ragged) return fail(c, DA_EINVAL, "adjoint spectra need every member on the context's window");
  da_status r = build_shells(c);
  if (r) return r;
  cudaStream_t st = (cudaStream_t)stream;
  if (member && !c->shell_scratch) {
    if ((r = dalloc(c, &c->shell_scratch, (size_t)c->B * c->nshell))) return r;
  }
  SpectraOut sp;
  sp.every = save_every;
  sp.scratch = c->shell_scratch;
  if (!(c->use_graph && c->timed_class == 0)) {
    sp.member = member;
    sp.mean = mean;
    if ((r = enqueue_spectra(c, s, lamT, sp, st))) return r;
    c->have_adj = true;
    return DA_OK;
  }
  // graph replay: inputs copied into and outputs out of internal buffers,
  // the sequence captured once per (save_every, outputs asked for)
  const int nsave = c->nsteps / save_every + 1;
  const int key = save_every * 4 + (member ? 2 : 0) + (mean ? 1 : 0);
  const size_t sbytes = (size_t)c->B * c->n * c->n * sizeof(double);
  const size_t lbytes = (size_t)c->B * c->n * (c->n / 2 + 1) * 2 * sizeof(double);
  if (!c->sp_lbuf && (r = dalloc(c, &c->sp_lbuf, lbytes / sizeof(double)))) return r;
  if (c->sp_key != key) {
    if (c->sp_exec) cudaGraphExecDestroy(c->sp_exec);
    c->sp_exec = nullptr;
    c->sp_member = c->sp_mean = nullptr;
    if (member && (r = dalloc(c, &c->sp_member, (size_t)c->B * nsave * c->nshell))) return r;
    if (mean && (r = dalloc(c, &c->sp_mean, (size_t)nsave * c->nshell))) return r;
    c->sp_key = key;
  }
  sp.member = c->sp_member;
  sp.mean = c->sp_mean;
  DA_TRY_CUDA(c, cudaMemcpyAsync(c->sbuf, s, sbytes, cudaMemcpyDeviceToDevice, st));
  DA_TRY_CUDA(c, cudaMemcpyAsync(c->sp_lbuf, lamT, lbytes, cudaMemcpyDeviceToDevice, st));
  DA_TRY_CUDA(c, cudaEventRecord(c->ev_in, st));
  DA_TRY_CUDA(c, cudaStreamWaitEvent(c->gstream, c->ev_in, 0));
  if (!c->sp_exec) {
    cudaGraph_t g = nullptr;
    const unsigned long long l0 = c->launches;
    DA_TRY_CUDA(c, cudaStreamBeginCapture(c->gstream, cudaStreamCaptureModeThreadLocal));
    r = enqueue_spectra(c, c->sbuf, c->sp_lbuf, sp, c->gstream);
    cudaError_t e = cudaStreamEndCapture(c->gstream, &g);
    if (r) {
      if (g) cudaGraphDestroy(g);
      return r;
    }
    if (e != cudaSuccess) return fail(c, DA_ECUDA, std::string("graph capture: ") + cudaGetErrorString(e));
    e = cudaGraphInstantiate(&c->sp_exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
      c->sp_exec = nullptr;
      return fail(c, DA_ECUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
    }
    c->sp_launches = c->launches - l0;
    c->launches = l0;
  }
  DA_TRY_CUDA(c, cudaGraphLaunch(c->sp_exec, c->gstream));
  c->launches += c->sp_launches;
  c->have_fwd = c->ckpt == 0;
  DA_TRY_CUDA(c, cudaEventRecord(c->ev_out, c->gstream));
  DA_TRY_CUDA(c, cudaStreamWaitEvent(st, c->ev_out, 0));
  if (member)
    DA_TRY_CUDA(c, cudaMemcpyAsync(member, c->sp_member, (size_t)c->B * nsave * c->nshell * sizeof(double),
                                   cudaMemcpyDeviceToDevice, st));
  if (mean)
    DA_TRY_CUDA(c, cudaMemcpyAsync(mean, c->sp_mean, (size_t)nsave * c->nshell * sizeof(double),
                                   cudaMemcpyDeviceToDevice, st));
  c->have_adj = true;
  return DA_OK;
}

extern "C" da_status da_last_adjoint(da_ctx* c, double* lam0, double* filtered, void* stream) {
  if (!c) return fail(c, DA_EINVAL, "ctx must not be NULL");
  if (!c->have_adj) return fail(c, DA_EINVAL, "no adjoint has been run on this context");
  cudaStream_t st = (cudaStream_t)stream;
  if (lam0) c->ops->compact_to_half(c->dev, c->dev.LamBar, (double2*)lam0, st);
  if (filtered) {
    c->ops->spec_to_mixed(c->dev, c->dev.LamBar, da::M_FILTERED, st);
    c->ops->c2r_rows(c->dev, filtered, st);
  }
  return check_launch(c, (lam0 ? 1 : 0) + (filtered ? 2 : 0));
}

extern "C" da_status da_omega_from_control(da_ctx* c, const double* s, double* omega0, void* stream) {
  if (!c || !s || !omega0) return fail(c, DA_EINVAL, "arguments must not be NULL");
  cudaStream_t st = (cudaStream_t)stream;
  c->ops->r2c_rows(c->dev, s, st);
  c->ops->ctrl_cols(c->dev, da::F_NO_NEXT, st);
  c->ops->compact_to_half(c->dev, c->dev.W, (double2*)omega0, st);
  return check_launch(c, 3);
}

extern "C" da_status da_control_from_omega(da_ctx* c, const double* omega0, double* s, void* stream) {
  if (!c || !s || !omega0) return fail(c, DA_EINVAL, "arguments must not be NULL");
  cudaStream_t st = (cudaStream_t)stream;
  c->ops->half_to_compact(c->dev, (const double2*)omega0, c->dev.Y, st);
  c->ops->spec_to_mixed(c->dev, c->dev.Y, da::M_INV_CTRL, st);
  c->ops->c2r_rows(c->dev, s, st);
  return check_launch(c, 3);
}
