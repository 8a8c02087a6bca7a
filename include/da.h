/*
 * da.h -- C ABI of the GB300 cost-and-gradient library for preconditioned
 * adjoint data assimilation of 2D incompressible Navier-Stokes turbulence
 * (vorticity form, periodic box [0, 2pi)^2, FP64 throughout).
 *
 * What it computes (Ke, You & Wang, "Preconditioned Adjoint Data
 * Assimilation for Two-Dimensional Decaying and Forced Turbulence"):
 *   - forward model: Eq. (1), or Eq. (24) with Kolmogorov forcing, in
 *     vorticity form, Fourier pseudo-spectral in space (2/3-rule square
 *     truncation |kx|,|ky| <= floor((n-1)/3)), classical RK4 in time;
 *   - cost: Eq. (2)-(3), J = 1/2 sum over probes x_i and observation times
 *     t_j of |u(x_i, t_j) - m_ij|^2, velocity sampled at lattice nodes;
 *   - gradient: the exact discrete adjoint of that scheme (Eq. 11-12 as
 *     their discrete counterparts), run backward against the stored forward
 *     stage fields, with the observation mismatch injected at each
 *     observation step;
 *   - preconditioner: the control is s = G^{-1/2} c (Eq. 18-19), c the
 *     scalar field with c_hat = w_hat/|k| (which carries the norm of the
 *     initial velocity), so w0_hat = |k| W(k)^{1/2} s_hat and
 *     grad_s J = IDFT(|k| W^{1/2} DFT(grad_{w0} J)); W = G_hat is the
 *     Fourier kernel of the G-inner product (Eq. 13, 16; kernel families of
 *     Sec. III.B).
 *
 * Conventions
 *   Physical fields: double [n][n], row-major [iy][ix], x_j = 2 pi j / n.
 *   Spectral fields: complex double interleaved (re, im), half spectrum
 *     [n][n/2+1] indexed [q][p] with kx = p, ky = q (q < n/2) or q - n;
 *     forward transforms are unnormalised, inverse carry 1/n^2.
 *   A gradient is the Euclidean gradient over grid values; its spectral form
 *     is the DFT of that grid field.
 *   Batches: a context holds `batch` independent members that share the
 *     grid, physics and probe geometry; each member has its own kernel W,
 *     observations, control and results.  Member b's arrays follow member
 *     b-1's contiguously.
 *   Memory: every array argument is a DEVICE pointer owned by the caller
 *     unless stated otherwise; the context owns only its internal buffers
 *     (trajectory of stage fields, work arrays, observations, tables).
 *   Streams: `stream` is a cudaStream_t passed as void*; all work is
 *     enqueued on it.  One context must not be used from two streams at once.
 *   Errors: every call returns a da_status and never aborts; da_last_error
 *     gives the message of the last failure on that context.
 */
#ifndef DA_GB300_H
#define DA_GB300_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct da_ctx da_ctx;

typedef enum {
  DA_OK = 0,
  DA_EINVAL = 1,     /* invalid argument or unsupported size */
  DA_ENOMEM = 2,     /* device allocation failed (trajectory too large, ...) */
  DA_ECUDA = 3,      /* a CUDA call failed; context state is undefined */
  DA_ETIMEOUT = 4,   /* reserved: a bounded device wait gave up (no call of this version
                        waits on the device) */
  DA_EDIVERGED = 5,  /* non-finite cost or gradient */
  DA_ENOTCONV = 6    /* the optimiser stopped on a line-search failure */
} da_status;

/* Grid and time window.  n: points per side, a power of two in [16, 1024].
 * L: domain side, must be 2 pi (0 means 2 pi).  dt, nsteps: RK4 step and
 * count.  ckpt_every: 0 stores every stage field of every step for the
 * adjoint (the default; 64 n^2 bytes per step per member: u, v of the four
 * RK stages); K > 0 keeps the
 * state every K steps and the stage fields of one K-step segment, and the
 * adjoint recomputes each segment from its checkpoint (one extra forward
 * solve; results are bitwise those of full storage); -1 keeps nothing
 * (forward only).  batch: members per context (>= 1). */
typedef struct {
  int n;
  double L;
  double dt;
  int nsteps;
  int ckpt_every;
  int batch;
} da_grid;

typedef enum { DA_FORCE_NONE = 0, DA_FORCE_KOLMOGOROV = 1 } da_force_kind;

/* Body force f = (amp sin(nf y), 0) of Eq. (24); vorticity source
 * -amp nf cos(nf y).  Requires 1 <= nf <= floor((n-1)/3). */
typedef struct {
  da_force_kind kind;
  double amp;
  int nf;
} da_forcing;

/* Pointwise velocity probes of Eq. (3) on a uniform lattice: probe
 * i = r*px + q sits on node (iy, ix) = (r n/py, q n/px).  px must equal py
 * and divide n.  Observation times are steps j*every, j = 1..nsteps/every
 * (every must divide nsteps), plus step 0 if include_t0. */
typedef struct {
  int px, py;
  int every;
  int include_t0;
} da_obs_operator;

typedef enum {
  DA_KERNEL_IDENTITY = 0, /* W = 1: the standard adjoint in the velocity metric */
  DA_KERNEL_EXP_ABS = 1,  /* W = exp(-param |k|) */
  DA_KERNEL_FRAC = 2,     /* W = |k|^(-2 param): fractional integral, Sec. III.B G_p */
  DA_KERNEL_EXP_SQ = 3,   /* W = exp(-nu param k^2): heat kernel, Sec. III.B G_e */
  DA_KERNEL_TABLE = 4     /* W from `table`: HOST pointer to [n][n/2+1] doubles */
} da_kernel_kind;

typedef struct {
  da_kernel_kind kind;
  double param;
  const double* table;
} da_kernel;

/* L-BFGS settings of da_assimilate (the paper names L-BFGS, Sec. II.C,
 * without settings).  Zero fields take the defaults in brackets. */
typedef struct {
  int memory;        /* history pairs [10] */
  double c1, c2;     /* strong Wolfe constants [1e-4, 0.9] */
  double gtol_rel;   /* stop when |g| <= gtol_rel |g0| [1e-10] */
  int max_ls_evals;  /* cost-gradient evaluations per line search [20] */
} da_lbfgs_opts;

/* Create a context for a batch of assimilation windows of the model of
 * Eq. (1) (Eq. 24 with Kolmogorov forcing), the probes and times of Eq. (3)
 * and one preconditioning kernel W per member (Sec. II.C, III.B).
 * `kernels` points to grid->batch descriptors (one per member).  Allocates
 * the device buffers of the forward solve, the stored trajectory and the
 * adjoint sweep, so that da_forward, da_cost_grad, da_vjp,
 * da_adjoint_terminal, the control maps and da_last_adjoint allocate
 * nothing; da_assimilate, da_set_sobolev, da_set_graphs and
 * da_adjoint_spectra allocate their own buffers on first use (stated at
 * each).  Returns DA_EINVAL for unsupported sizes or a kernel whose W is not
 * finite and non-negative on the retained set (message via
 * da_last_error(NULL)), DA_ENOMEM if a device allocation (usually the
 * trajectory, 64 n^2 bytes per step per member) fails; on failure *out is
 * NULL and nothing stays allocated. */
da_status da_create(da_ctx** out, const da_grid* grid, double nu, const da_forcing* forcing,
                    const da_obs_operator* obs, const da_kernel* kernels);

/* Sobolev regularisation of Eq. (4): da_cost_grad and da_assimilate add
 * lambda/2 sum_grid |grad u0|^2 (= lambda/2 sum_grid w0^2 for the
 * divergence-free initial field) to J and its gradient to grad_s.
 * lambda >= 0; 0 (the default) turns it off.  Allocates one compact
 * spectrum per member on the first non-zero lambda. */
da_status da_set_sobolev(da_ctx* ctx, double lambda);

/* Observations m_ij of Eq. (3): DEVICE (or host) pointer
 * [batch][nt][px*py][2] (u, v per probe) with nt = da_num_obs_times(ctx);
 * copied into the context on `stream` (the caller's buffer may be reused once
 * the stream has passed the copy). */
da_status da_set_observations(da_ctx* ctx, const double* m, void* stream);

/* Forward solve of Eq. (1)/(24) over the window from the initial vorticity
 * w0_hat = P |k| W^{1/2} DFT(s) (Eq. 18-19).  s: DEVICE [batch][n][n];
 * omegaT (nullable): DEVICE [batch][n][n/2+1] complex, the final vorticity
 * half spectrum; obs (nullable): DEVICE [batch][nt][px*py][2], the model
 * velocities at the probes and times of Eq. (3).  Keeps the trajectory for
 * da_vjp when the context stores one. */
da_status da_forward(da_ctx* ctx, const double* s, double* omegaT, double* obs, void* stream);

/* Cost J of Eq. (2)-(3) and its gradient with respect to the control,
 * grad_s J = IDFT(P |k| W^{1/2} DFT(grad_{w0} J)) (Eq. 19), grad_{w0} J from
 * the discrete adjoint of the forward scheme (Eq. 11-12).  s: DEVICE
 * [batch][n][n]; J: [batch], HOST or DEVICE pointer (a host pointer makes
 * the call wait for the stream); grad_s: DEVICE [batch][n][n] (nullable).
 * Uses the observations of da_set_observations (DA_EINVAL without them). */
da_status da_cost_grad(da_ctx* ctx, const double* s, double* J, double* grad_s, void* stream);

/* Vector-Jacobian product of the last da_forward on this context (which
 * must have kept its trajectory, ckpt_every >= 0): the gradient with
 * respect to the control s of <dobs, obs(s)> + <dwT, omega_T(s)>, i.e. the
 * adjoint of Eq. (11) driven by arbitrary cotangents.  dobs: DEVICE
 * [batch][nt][px*py][2] cotangent of the model observations (nullable);
 * dwT: DEVICE [batch][n][n/2+1] complex, the DFT of the cotangent of the
 * final vorticity grid values (nullable); grad_s: DEVICE [batch][n][n]
 * (nullable).  da_cost_grad is the case dobs = obs - m, dwT = NULL.  With
 * checkpoints, a second da_vjp needs a new da_forward. */
da_status da_vjp(da_ctx* ctx, const double* dobs, const double* dwT, double* grad_s, void* stream);

/* enable != 0: da_cost_grad (and so da_assimilate) and da_adjoint_spectra
 * capture their whole launch sequence into a CUDA graph on the first call
 * (da_adjoint_spectra: the first call per save_every and choice of outputs)
 * and replay it afterwards on an internal stream, ordered after and before
 * the caller's stream by events; inputs are copied into and outputs out of
 * internal buffers.  For small grids this removes the per-launch host cost.  The
 * capture is redone after da_set_sobolev; kernel timing (da_time_kernels)
 * bypasses the graph.  The first call must not itself be inside a capture.
 * The first enabling call allocates the two internal buffers (2 batch n^2
 * doubles), a stream and two events. */
da_status da_set_graphs(da_ctx* ctx, int enable);

/* FFT plan variants (no counterpart in the paper, whose solver is not
 * FFT-based on GPUs): each grid size n has da_plan_count(n) variants of the
 * radix schedule and CTA width of the pass kernels (0 if n is not a
 * supported size).  All variants compute the same transforms; results
 * differ only by rounding.  A context starts on variant 0, or on the variant
 * da_autotune last chose in this process for the same n and batch. */
int da_plan_count(int n);

/* The context's current plan variant (-1 for a NULL ctx). */
int da_get_plan(const da_ctx* ctx);

/* Switches to plan variant `variant` (DA_EINVAL if out of range).  Waits
 * for all work on the device first (cudaDeviceSynchronize), since work in
 * flight may use the context's twiddle table.  Drops a captured graph and
 * any stored forward trajectory (call da_forward or da_cost_grad again
 * before da_vjp). */
da_status da_set_plan(da_ctx* ctx, int variant);

/* Autotuner: for each plan variant of the context's n, runs one warm-up and
 * `steps` timed RK steps of the forward and (when stage fields are stored)
 * adjoint pass kernels over the context's own batch, on zeroed working
 * buffers, timed with CUDA events; switches the context to the fastest and
 * records the choice for later contexts of the same n and batch in this
 * process.  chosen (nullable): HOST int, the variant taken; ms_per_step
 * (nullable): HOST double[da_plan_count(n)], the measured milliseconds per
 * step of each variant.  Synchronous (it first waits for all work on the
 * device, then runs on the legacy default stream); it overwrites the context's state and
 * stored trajectory, so call it before the evaluations (observations set by
 * da_set_observations are kept).  DA_EINVAL for steps < 1. */
da_status da_autotune(da_ctx* ctx, int steps, int* chosen, double* ms_per_step);

/* Nominal flops of one band-limited transform of n points as the pass
 * kernels run it under plan variant `variant` (Sec. II.B: the 2/3 rule keeps
 * |kx|, |ky| <= K = (n-1)/3): 5 n log2 n less the operations they skip,
 * namely the additions of the first stage that a zero input of the gap
 * K < q < n - K would enter (inverse transforms, whose inputs are zero
 * there) and the last-stage outputs in the gap (forward transforms, read
 * back only on the band).  A skip counts only where it holds for all 32
 * lanes of a warp.  inverse, forward: HOST double, one value each.  Host
 * only, no device work; DA_EINVAL (message via da_last_error(NULL)) for an
 * unsupported size or variant or a NULL pointer. */
da_status da_plan_flops(int n, int variant, double* inverse, double* forward);

/* Optional extra outputs of the last da_cost_grad / da_adjoint_terminal on
 * this context: lam0 [batch][n][n/2+1] complex, the DFT of grad_{w0} J
 * (the physical adjoint at t = 0, Eq. 12); filtered [batch][n][n] the
 * gradient in the G-metric, IDFT(|k| W DFT(grad_{w0} J)) (Eq. 17 in the
 * scalar representation).  Either may be NULL. */
da_status da_last_adjoint(da_ctx* ctx, double* lam0, double* filtered, void* stream);

/* Adjoint of the window driven by a terminal field only (the adjoint
 * Green's function runs of Sec. IV): lamT [batch][n][n/2+1] complex is the
 * DFT of a gradient with respect to the final vorticity; returns grad_s
 * [batch][n][n] (nullable).  Observations are not used. */
da_status da_adjoint_terminal(da_ctx* ctx, const double* s, const double* lamT, double* grad_s, void* stream);

/* Adjoint statistics of Sec. IV: the adjoint driven by the terminal field
 * lamT (as da_adjoint_terminal) with, every save_every steps of backward
 * time tau = (nsteps - k) dt (slot (nsteps - k)/save_every, from tau = 0 to
 * the initial time), the energy per wavenumber shell k <= |k| < k+1 of the
 * adjoint velocity u_dagger = (d lambda/dy, -d lambda/dx):
 * E(k) = 1/2 sum over the shell of |u_dagger_hat|^2 with normalised Fourier
 * coefficients (the shell sum of Eq. 20).  member: DEVICE
 * [batch][nsteps/save_every + 1][nshell] per member (nullable); mean: DEVICE
 * [nsteps/save_every + 1][nshell] of the ensemble-mean adjoint over the
 * batch (nullable).  nshell = da_num_shells(ctx).  Reductions run in a fixed
 * order.  save_every must divide nsteps.  The first call allocates the shell
 * lists (one int and one double per retained mode) and, with `member`, a
 * [batch][nshell] scratch. */
da_status da_adjoint_spectra(da_ctx* ctx, const double* s, const double* lamT, int save_every, double* member,
                             double* mean, void* stream);

/* Number of wavenumber shells of da_adjoint_spectra: floor(sqrt(2) K) + 1. */
int da_num_shells(const da_ctx* ctx);

/* L-BFGS on the transformed control (Sec. II.C, Eq. 18-19: the paper's
 * optimiser, run in the Euclidean metric of s) for up to max_iter
 * iterations, each member independently; the members of the batch advance in
 * lockstep and share every cost-and-gradient evaluation.
 *   s: DEVICE [batch][n][n], in: first guesses; out: each member's last
 *     accepted control (its first guess if it never accepted a step).
 *   J_hist: HOST [batch][max_iter+1], the cost at the start and after every
 *     iteration (entries past a member's last iteration repeat its final cost).
 *   iters_done: HOST [batch], iterations each member completed.
 *   member_status: HOST [batch] (nullable), per member DA_OK (converged or
 *     max_iter reached), DA_ENOTCONV (line-search failure: the step-size
 *     collapse of Sec. III.C-D) or DA_EDIVERGED (non-finite cost or
 *     gradient); one member's failure leaves the others' results intact.
 * Returns DA_EDIVERGED if some member diverged, else DA_ENOTCONV if some
 * member's line search failed, else DA_OK; DA_EINVAL for bad arguments or
 * opts->memory > 64.  opts may be NULL.  The first call on a context
 * allocates the optimiser's device buffers ((2 memory + 7) n^2 doubles per
 * member) and a small pinned host buffer.  The call waits for `stream` (the
 * line search decides on the host): one host read per trial evaluation and
 * two per iteration. */
da_status da_assimilate(da_ctx* ctx, double* s, int max_iter, const da_lbfgs_opts* opts, double* J_hist,
                        int* iters_done, int* member_status, void* stream);

/* Ragged batches.  A member slot can hold its own assimilation window
 * (Eq. 1-3 with its own horizon, probe lattice, viscosity and forcing switch;
 * grid, dt and obs.every stay the context's), so that jobs of one grid size
 * share every launch.  In each evaluation the windows are end-aligned: the
 * evaluation runs the longest live window, and a member with a shorter one
 * starts later and ends with it; a member whose window is empty is idle (its
 * launches return at once; its cost is 0, its gradient 0).  A member's
 * results are those of a batch-1 context with its window on the same plan
 * variant (the kernels do the same arithmetic for it).
 *   nsteps: 0 (idle) or a multiple of obs.every, at most the context's
 *     nsteps (which sizes the trajectory);
 *   px: divides n, at most the context's px (which sizes the observation
 *     buffers);
 *   nu >= 0; forcing: 0 or 1 (the context's Kolmogorov forcing, which the
 *     context must have been created with). */
typedef struct {
  int nsteps;
  int px;
  double nu;
  int forcing;
} da_member_window;

/* Gives member slot `member` its window, kernel and observations m (DEVICE
 * or host pointer, [nt][px*px][2] with nt = nsteps/every (+1 with
 * include_t0)); with w->nsteps == 0 the slot becomes idle and kernel and m
 * are not read.  Waits for `stream`, recomputes the multiplier |k| W^{1/2}
 * (DA_EINVAL, slot left idle, if it is not finite and non-negative on the
 * retained set), copies m on `stream`; drops a captured graph.  From the
 * first call on, the context is a ragged batch: the other members keep the
 * context's window until they are set.  da_adjoint_spectra needs a
 * homogeneous batch. */
da_status da_set_member(da_ctx* ctx, int member, const da_member_window* w, const da_kernel* kernel,
                        const double* m, void* stream);

/* Stepwise L-BFGS over the member slots (Sec. II.C), for loops that start and
 * retire members between evaluations: da_assimilate is da_lbfgs_start on
 * every member, then da_lbfgs_iterate until none runs.  A member's iterates
 * do not depend on when it started or on the other members. */
typedef struct {
  int phase;   /* 0 idle, 1 started (first evaluation pending), 2 iterating, 3 finished */
  int status;  /* DA_OK, DA_ENOTCONV (line-search failure) or DA_EDIVERGED */
  int iters;   /* iterations that accepted a step */
  double J0;   /* cost at the start (after its first evaluation) */
  double J;    /* cost at the current control */
} da_lbfgs_report;

/* (Re)starts member `member` at control s0 (DEVICE [n][n], copied on
 * `stream`) with an iteration budget max_iter and the settings opts (NULL:
 * defaults; memory must be the same for every member and call on a context).
 * The first call allocates the optimiser's buffers (see da_assimilate). */
da_status da_lbfgs_start(da_ctx* ctx, int member, const double* s0, int max_iter, const da_lbfgs_opts* opts,
                         void* stream);

/* One step: advances every running member to and through one shared
 * cost-and-gradient evaluation -- members whose last trial was accepted get
 * their (s, y) pair tested, members starting an iteration get their search
 * direction (the two-loop recursion) and line search, and one evaluation
 * serves every searching member's trial and every newly started member's
 * first point.  Members at different points of their iterations share the
 * evaluation; none waits for another's line search.  A member finishes when
 * it converges (|g| <= gtol_rel |g0|), spends its budget, its line search
 * fails or its cost turns non-finite.  running (HOST, nullable): members
 * still started or iterating.  Waits for `stream` (the line search decides
 * on the host). */
da_status da_lbfgs_iterate(da_ctx* ctx, int* running, void* stream);

/* Report of member `member` (HOST out); J_hist (HOST, nullable, hist_len
 * entries): the cost at the start and after every iteration, padded with the
 * current cost; s (DEVICE [n][n], nullable): its current control, copied on
 * `stream`. */
da_status da_lbfgs_member(da_ctx* ctx, int member, da_lbfgs_report* out, double* J_hist, int hist_len, double* s,
                          void* stream);

/* Returns member slot `member`'s optimiser to idle (its window is unchanged:
 * da_set_member with nsteps 0 idles the evaluations too). */
da_status da_lbfgs_release(da_ctx* ctx, int member);

/* Control maps of the change of variables of Eq. (18)-(19), one kernel per
 * member: omega0 DEVICE [batch][n][n/2+1] complex (half spectrum) <-> s
 * DEVICE [batch][n][n].  da_omega_from_control writes
 * w0_hat = P |k| W^{1/2} DFT(s) (zero mean, zero outside the retained set);
 * da_control_from_omega is its right inverse on the retained set,
 * s = IDFT(w0_hat / (|k| W^{1/2})) there and 0 elsewhere (modes where the
 * multiplier underflows to 0 map to 0). */
da_status da_omega_from_control(da_ctx* ctx, const double* s, double* omega0, void* stream);
da_status da_control_from_omega(da_ctx* ctx, const double* omega0, double* s, void* stream);

/* Control map s -> w0_hat of da_omega_from_control for ONE member, without
 * a context and without allocating device memory.  The paper has no
 * counterpart: this entry point exists for callers that cannot call
 * cudaMalloc, such as code inside a host framework that owns all device
 * memory through its own pool, or a serving loop that must not allocate
 * (or take the implicit synchronisation an allocation may bring) once it is
 * running.  Its scratch is a file-scope static device array sized for
 * n <= 256 (a 256 x 86 complex mixed field plus a 256-entry twiddle table,
 * about 356 KB, held on every GPU that loads the library until exit).
 *   n: 16, 32, 64, 128 or 256 (larger n: DA_EINVAL); nu: viscosity (used by
 *   the heat kernel); kernel: identity, exp_abs, frac or exp_sq (a table
 *   kernel: DA_EINVAL); s: DEVICE [n][n] double; omega0: DEVICE
 *   [n][n/2+1] complex (every entry is written); message (nullable)
 *   receives a static string describing a failure.
 * The first call on a device sets that device up (it looks up the arrays'
 * device addresses and copies the twiddles, synchronously); make that first
 * call before any stream capture.  Every call shares the scratch: calls
 * that can overlap on the GPU (other streams, other threads) race and must
 * be serialised by the caller.  Each call writes every scratch entry it
 * later reads, so no state carries over between calls. */
da_status da_omega_from_control_static(int n, double nu, const da_kernel* kernel, const double* s, double* omega0,
                                       void* stream, const char** message);

/* FP64 throughput probe, a measurement utility (the paper has no
 * counterpart): the pass kernels are bound by FP64 arithmetic, and this
 * probe measures the pipe's issue rate that bounds them.  Runs 8 independent
 * dependency chains per thread of one operation -- kind 0: DFMA with a
 * register multiplicand and a constant addend; 1: DFMA with three register
 * operands; 2: DADD; 3: DMUL -- on 4 CTAs of 256 threads per SM, iters x 32
 * operations per thread, after a short warm-up launch, timed with CUDA
 * events on `stream`.  gflops (HOST, required): FP64 flop/s / 1e9 (a DFMA
 * counts 2); ops_per_clk_per_sm (HOST, nullable): operations per SM clock
 * per SM; sm_mhz (HOST, nullable): the SM clock the probe ran at (clock64
 * over %globaltimer on one thread).  Synchronous; allocates and frees a
 * small device buffer (DA_ENOMEM if it cannot).  DA_EINVAL for kind outside
 * [0, 3] or iters < 1. */
da_status da_fp64_probe(int kind, int iters, double* gflops, double* ops_per_clk_per_sm, double* sm_mhz,
                        void* stream);

/* Number of observation times of the context (nt). */
int da_num_obs_times(const da_ctx* ctx);

/* Device bytes held by the context. */
unsigned long long da_device_bytes(const da_ctx* ctx);

/* Number of kernel launches the context has issued so far. */
unsigned long long da_launch_count(const da_ctx* ctx);

/* Event timing of one class of pass kernels, for roofline reports:
 * kernel_class 0 off, 1 forward row pass, 2 forward column pass, 3 adjoint
 * row pass, 4 adjoint column pass.  While on, every launch of that class is
 * bracketed by two CUDA events on the launch stream. */
da_status da_time_kernels(da_ctx* ctx, int kernel_class);

/* Total device time (ms) and launch count of the timed class since the last
 * call; waits for the last recorded event. */
da_status da_kernel_time(da_ctx* ctx, double* total_ms, unsigned long long* launches);

/* Message of the last failure on ctx (NULL: the last failed da_create). */
const char* da_last_error(const da_ctx* ctx);

/* Free every device buffer of ctx; waits for no stream. */
void da_destroy(da_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif
