/*
 * da_oracle.c -- plain, slow, FP64 CPU oracle for the cost-and-gradient
 * evaluation of preconditioned adjoint data assimilation for 2D incompressible
 * Navier-Stokes in vorticity form on the periodic box [0, 2pi)^2.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py may load, call or link this code.
 * It shares no code with the CUDA path: its FFT, operators, adjoint and
 * control map are written here independently, as plain loops that follow the
 * definitions, with no blocking, fusion, pruning or reordering.
 *
 * Discretisation (the paper's own solver is a different scheme, Sec. III;
 * this is the vorticity-form pseudo-spectral reading):
 *   grid      x_j = 2*pi*j/n on both axes, arrays [iy][ix], ix fastest;
 *   spectrum  w_hat[q][p] = sum_{iy,ix} w[iy][ix] exp(-i(kx x + ky y)),
 *             half spectrum p = kx = 0..n/2, q = 0..n-1 with ky = q (q < n/2)
 *             or q - n; inverse carries 1/n^2;
 *   Biot-Savart  u = d(psi)/dy, v = -d(psi)/dx, w = dv/dx - du/dy,
 *             so u_hat = i ky w_hat / k^2, v_hat = -i kx w_hat / k^2;
 *   dealias   the 2/3 rule as a square truncation: mode kept iff
 *             |kx| <= K and |ky| <= K, K = floor((n-1)/3).
 *
 * Every inner product is the Euclidean sum over grid values.
 *
 * Parity status: every exported function is pinned by tests under tests/
 * (brute-force DFT, closed-form single modes, Taylor-Green decay, laminar
 * Kolmogorov fixed point, conservation, dot-product tests, finite
 * differences).
 */
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cplx;

/* Problem definition shared with the Python side through ctypes.  Field order
 * is fixed; oracle/__init__.py mirrors it. */
typedef struct {
  int n;           /* grid points per side (power of two) */
  int nsteps;      /* RK4 steps in the window */
  double dt;       /* time step */
  double nu;       /* kinematic viscosity, 1/Re */
  int force_kind;  /* 0: none; 1: Kolmogorov f = (amp sin(nf y), 0) */
  double amp;
  int nf;
  int px;          /* probes per side: lattice nodes (r n/px, q n/px) */
  int every;       /* observation interval in steps */
  int include_t0;  /* 1: also observe the initial state */
  int kernel_kind; /* 0 identity, 1 exp(-a|k|), 2 |k|^(-2a), 3 exp(-nu a k^2), 4 table */
  double kparam;   /* the kernel parameter a */
  const double* ktable; /* kind 4: W per half-spectrum mode, [n][n/2+1] */
  double sobolev;  /* lambda of the regularisation term of Eq. (4); 0: none */
} orc_cfg;

/* ------------------------------------------------------------------------ */
/* Index helpers                                                             */
/* ------------------------------------------------------------------------ */

static int nh(int n) { return n / 2 + 1; }
static int ky_of(int q, int n) { return q < n / 2 ? q : q - n; }
static int kcut(int n) { return (n - 1) / 3; }

/* Retained set of the 2/3 rule. */
static int in_R(int kx, int ky, int n) {
  int K = kcut(n);
  return abs(kx) <= K && abs(ky) <= K;
}

static void* xalloc(size_t bytes) {
  void* p = calloc(1, bytes ? bytes : 1);
  if (!p) abort();
  return p;
}

/* ------------------------------------------------------------------------ */
/* Transforms                                                                */
/* ------------------------------------------------------------------------ */

/* In-place iterative radix-2 complex FFT of length m (power of two),
 * X[k] = sum_j x[j] exp(sign * 2 pi i j k / m), no scaling. */
static void fft_inplace(cplx* x, int m, int sign) {
  for (int i = 1, j = 0; i < m; ++i) { /* bit-reversal permutation */
    int bit = m >> 1;
    for (; j & bit; bit >>= 1) j ^= bit;
    j ^= bit;
    if (i < j) {
      cplx t = x[i];
      x[i] = x[j];
      x[j] = t;
    }
  }
  for (int len = 2; len <= m; len <<= 1) {
    for (int i = 0; i < m; i += len) {
      for (int j = 0; j < len / 2; ++j) {
        double ang = sign * 2.0 * M_PI * (double)j / (double)len;
        cplx w = cos(ang) + I * sin(ang);
        cplx a = x[i + j];
        cplx b = x[i + j + len / 2] * w;
        x[i + j] = a + b;
        x[i + j + len / 2] = a - b;
      }
    }
  }
}

/* Strided 1D transform through a contiguous scratch copy. */
static void fft_strided(cplx* x, int m, int stride, int sign, cplx* tmp) {
  for (int j = 0; j < m; ++j) tmp[j] = x[(size_t)j * stride];
  fft_inplace(tmp, m, sign);
  for (int j = 0; j < m; ++j) x[(size_t)j * stride] = tmp[j];
}

/* Full complex 2D transform of an n x n array: rows (along x), then columns. */
static void fft2_full(cplx* a, int n, int sign) {
  cplx* tmp = xalloc(sizeof(cplx) * n);
  for (int iy = 0; iy < n; ++iy) fft_strided(a + (size_t)iy * n, n, 1, sign, tmp);
  for (int ix = 0; ix < n; ++ix) fft_strided(a + ix, n, n, sign, tmp);
  free(tmp);
}

/* Real field -> half spectrum (unnormalised forward DFT). */
static void r2c(const double* f, cplx* h, int n) {
  cplx* a = xalloc(sizeof(cplx) * n * n);
  for (int i = 0; i < n * n; ++i) a[i] = f[i];
  fft2_full(a, n, -1);
  for (int q = 0; q < n; ++q)
    for (int p = 0; p < nh(n); ++p) h[q * nh(n) + p] = a[q * n + p];
  free(a);
}

/* Half spectrum -> real field: extend by Hermitian symmetry
 * F(-k) = conj(F(k)), inverse DFT, keep the real part, scale by 1/n^2. */
static void c2r(const cplx* h, double* f, int n) {
  cplx* a = xalloc(sizeof(cplx) * n * n);
  for (int q = 0; q < n; ++q)
    for (int p = 0; p < n; ++p) {
      if (p <= n / 2)
        a[q * n + p] = h[q * nh(n) + p];
      else
        a[q * n + p] = conj(h[((n - q) % n) * nh(n) + (n - p)]);
    }
  fft2_full(a, n, +1);
  for (int i = 0; i < n * n; ++i) f[i] = creal(a[i]) / ((double)n * n);
  free(a);
}

/* ------------------------------------------------------------------------ */
/* Spectral multipliers                                                      */
/* ------------------------------------------------------------------------ */

/* Multiply a half spectrum by a symbol sym(kx, ky) and by the 2/3-rule mask. */
typedef cplx (*symbol_fn)(int kx, int ky);

static cplx sym_u(int kx, int ky) { /* u from w: i ky / k^2 */
  double k2 = (double)kx * kx + (double)ky * ky;
  return k2 > 0 ? I * ky / k2 : 0;
}
static cplx sym_v(int kx, int ky) { /* v from w: -i kx / k^2 */
  double k2 = (double)kx * kx + (double)ky * ky;
  return k2 > 0 ? -I * kx / k2 : 0;
}
static cplx sym_dx(int kx, int ky) { (void)ky; return I * kx; }
static cplx sym_dy(int kx, int ky) { (void)kx; return I * ky; }

/* out = P sym(k) in, optionally with the conjugate symbol (the transpose of
 * the operator with respect to the Euclidean inner product on real fields). */
static void apply_sym(const cplx* in, cplx* out, int n, symbol_fn sym, int transpose) {
  for (int q = 0; q < n; ++q)
    for (int p = 0; p < nh(n); ++p) {
      int kx = p, ky = ky_of(q, n);
      cplx s = (in_R(kx, ky, n)) ? sym(kx, ky) : 0;
      if (transpose) s = conj(s);
      out[q * nh(n) + p] = s * in[q * nh(n) + p];
    }
}

static void mask_R(cplx* h, int n) {
  for (int q = 0; q < n; ++q)
    for (int p = 0; p < nh(n); ++p)
      if (!in_R(p, ky_of(q, n), n)) h[q * nh(n) + p] = 0;
}

/* Physical field of sym(k) w_hat. */
static void physical_of(const cplx* w, double* f, int n, symbol_fn sym, cplx* scratch) {
  apply_sym(w, scratch, n, sym, 0);
  c2r(scratch, f, n);
}

/* Forcing term of the vorticity equation: curl (amp sin(nf y), 0) =
 * -amp nf cos(nf y), whose DFT is -amp nf n^2/2 at (kx, ky) = (0, +-nf). */
static void add_forcing(const orc_cfg* c, cplx* F, double scale) {
  if (c->force_kind != 1) return;
  int n = c->n;
  double v = -c->amp * c->nf * (double)n * n / 2.0;
  if (!in_R(0, c->nf, n)) return;
  F[(c->nf % n) * nh(n)] += scale * v;
  F[((n - c->nf) % n) * nh(n)] += scale * v;
}

/* ------------------------------------------------------------------------ */
/* Right-hand side of the vorticity equation and its linearisations          */
/* ------------------------------------------------------------------------ */

/* The four physical fields the advection term needs at state w. */
typedef struct { double *u, *v, *wx, *wy; } velgrad;

static velgrad velgrad_alloc(int n) {
  velgrad g;
  g.u = xalloc(sizeof(double) * n * n);
  g.v = xalloc(sizeof(double) * n * n);
  g.wx = xalloc(sizeof(double) * n * n);
  g.wy = xalloc(sizeof(double) * n * n);
  return g;
}
static void velgrad_free(velgrad* g) { free(g->u); free(g->v); free(g->wx); free(g->wy); }

static void velgrad_of(const cplx* w, int n, velgrad* g, cplx* scratch) {
  physical_of(w, g->u, n, sym_u, scratch);
  physical_of(w, g->v, n, sym_v, scratch);
  physical_of(w, g->wx, n, sym_dx, scratch);
  physical_of(w, g->wy, n, sym_dy, scratch);
}

/* F(w) = -P DFT(u dw/dx + v dw/dy) - nu k^2 w + f_hat: the vorticity form of
 * Eq. (1) (decaying) or Eq. (24) (Kolmogorov forcing), pseudo-spectral with
 * the nonlinear product formed on the grid and projected onto the retained
 * set. */
void orc_rhs(const orc_cfg* c, const double* w_in, double* F_out) {
  int n = c->n, nn = n * nh(n);
  const cplx* w = (const cplx*)w_in;
  cplx* F = (cplx*)F_out;
  cplx* scratch = xalloc(sizeof(cplx) * nn);
  double* nl = xalloc(sizeof(double) * n * n);
  velgrad g = velgrad_alloc(n);
  velgrad_of(w, n, &g, scratch);
  for (int i = 0; i < n * n; ++i) nl[i] = g.u[i] * g.wx[i] + g.v[i] * g.wy[i];
  r2c(nl, scratch, n);
  for (int q = 0; q < n; ++q)
    for (int p = 0; p < nh(n); ++p) {
      int kx = p, ky = ky_of(q, n);
      double k2 = (double)kx * kx + (double)ky * ky;
      int i = q * nh(n) + p;
      F[i] = in_R(kx, ky, n) ? (-scratch[i] - c->nu * k2 * w[i]) : 0;
    }
  add_forcing(c, F, 1.0);
  velgrad_free(&g);
  free(nl);
  free(scratch);
}

/* Tangent-linear RHS: dF = J_F(y) dy
 *   = -P DFT( (U dy) y_x + (V dy) y_y + u (Dx dy) + v (Dy dy) ) - nu k^2 dy,
 * the linearisation of the advection term, cf. the variation Eq. (7). */
void orc_rhs_tlm(const orc_cfg* c, const double* y_in, const double* dy_in, double* out) {
  int n = c->n, nn = n * nh(n);
  const cplx* dy = (const cplx*)dy_in;
  cplx* o = (cplx*)out;
  cplx* scratch = xalloc(sizeof(cplx) * nn);
  double* nl = xalloc(sizeof(double) * n * n);
  velgrad g = velgrad_alloc(n), d = velgrad_alloc(n);
  velgrad_of((const cplx*)y_in, n, &g, scratch);
  velgrad_of(dy, n, &d, scratch);
  for (int i = 0; i < n * n; ++i)
    nl[i] = d.u[i] * g.wx[i] + d.v[i] * g.wy[i] + g.u[i] * d.wx[i] + g.v[i] * d.wy[i];
  r2c(nl, scratch, n);
  for (int q = 0; q < n; ++q)
    for (int p = 0; p < nh(n); ++p) {
      int kx = p, ky = ky_of(q, n);
      double k2 = (double)kx * kx + (double)ky * ky;
      int i = q * nh(n) + p;
      o[i] = in_R(kx, ky, n) ? (-scratch[i] - c->nu * k2 * dy[i]) : 0;
    }
  velgrad_free(&g);
  velgrad_free(&d);
  free(nl);
  free(scratch);
}

/* Transposed RHS Jacobian, the discrete counterpart of the adjoint operator
 * of Eq. (11).  mu is a Euclidean gradient with respect to the grid values
 * of the vorticity, held as its DFT.  Transposing each factor of orc_rhs_tlm
 * (pointwise products are symmetric; a Fourier multiplier's transpose has the
 * conjugate symbol; P and the viscous term are symmetric):
 *   J_F^T mu = P[ -U^T(y_x m) - V^T(y_y m) - Dx^T(u m) - Dy^T(v m) ] - nu k^2 mu,
 *   m = IDFT(P mu). */
void orc_rhs_adj(const orc_cfg* c, const double* y_in, const double* mu_in, double* out) {
  int n = c->n, nn = n * nh(n);
  const cplx* mu = (const cplx*)mu_in;
  cplx* o = (cplx*)out;
  cplx* scratch = xalloc(sizeof(cplx) * nn);
  cplx* acc = xalloc(sizeof(cplx) * nn);
  cplx* term = xalloc(sizeof(cplx) * nn);
  double* m = xalloc(sizeof(double) * n * n);
  double* prod = xalloc(sizeof(double) * n * n);
  velgrad g = velgrad_alloc(n);
  velgrad_of((const cplx*)y_in, n, &g, scratch);
  memcpy(scratch, mu, sizeof(cplx) * nn);
  mask_R(scratch, n);
  c2r(scratch, m, n);

  /* each of the four transposed products: DFT of (field * m), then the
   * conjugate symbol of the operator that produced the field */
  const double* fields[4] = {g.wx, g.wy, g.u, g.v};
  symbol_fn syms[4] = {sym_u, sym_v, sym_dx, sym_dy};
  for (int t = 0; t < 4; ++t) {
    for (int i = 0; i < n * n; ++i) prod[i] = fields[t][i] * m[i];
    r2c(prod, scratch, n);
    apply_sym(scratch, term, n, syms[t], 1);
    for (int i = 0; i < nn; ++i) acc[i] -= term[i];
  }
  for (int q = 0; q < n; ++q)
    for (int p = 0; p < nh(n); ++p) {
      int kx = p, ky = ky_of(q, n);
      double k2 = (double)kx * kx + (double)ky * ky;
      int i = q * nh(n) + p;
      o[i] = in_R(kx, ky, n) ? (acc[i] - c->nu * k2 * mu[i]) : 0;
    }
  velgrad_free(&g);
  free(prod);
  free(m);
  free(term);
  free(acc);
  free(scratch);
}

/* ------------------------------------------------------------------------ */
/* Classical RK4 step, its tangent and its transpose                         */
/* ------------------------------------------------------------------------ */

static void axpy_c(cplx* out, const cplx* x, double a, const cplx* y, int nn) {
  for (int i = 0; i < nn; ++i) out[i] = x[i] + a * y[i];
}

/* One classical fourth-order Runge-Kutta step of dw/dt = F(w). */
void orc_step(const orc_cfg* c, const double* w_in, double* w_out) {
  int nn = c->n * nh(c->n);
  double dt = c->dt;
  const cplx* w = (const cplx*)w_in;
  cplx *k1 = xalloc(sizeof(cplx) * nn), *k2 = xalloc(sizeof(cplx) * nn);
  cplx *k3 = xalloc(sizeof(cplx) * nn), *k4 = xalloc(sizeof(cplx) * nn);
  cplx* y = xalloc(sizeof(cplx) * nn);
  orc_rhs(c, (const double*)w, (double*)k1);
  axpy_c(y, w, dt / 2, k1, nn);
  orc_rhs(c, (const double*)y, (double*)k2);
  axpy_c(y, w, dt / 2, k2, nn);
  orc_rhs(c, (const double*)y, (double*)k3);
  axpy_c(y, w, dt, k3, nn);
  orc_rhs(c, (const double*)y, (double*)k4);
  cplx* o = (cplx*)w_out;
  for (int i = 0; i < nn; ++i) o[i] = w[i] + dt / 6.0 * (k1[i] + 2.0 * k2[i] + 2.0 * k3[i] + k4[i]);
  free(k1); free(k2); free(k3); free(k4); free(y);
}

/* The four stage states y1..y4 of the RK4 step from w (y1 = w). */
static void stage_states(const orc_cfg* c, const cplx* w, cplx* ys[4]) {
  int nn = c->n * nh(c->n);
  double dt = c->dt;
  cplx* k = xalloc(sizeof(cplx) * nn);
  memcpy(ys[0], w, sizeof(cplx) * nn);
  orc_rhs(c, (const double*)ys[0], (double*)k);
  axpy_c(ys[1], w, dt / 2, k, nn);
  orc_rhs(c, (const double*)ys[1], (double*)k);
  axpy_c(ys[2], w, dt / 2, k, nn);
  orc_rhs(c, (const double*)ys[2], (double*)k);
  axpy_c(ys[3], w, dt, k, nn);
  free(k);
}

/* Tangent of one RK4 step: returns the step of w in w_out and of dw in dw_out. */
void orc_step_tlm(const orc_cfg* c, const double* w_in, const double* dw_in, double* w_out, double* dw_out) {
  int nn = c->n * nh(c->n);
  double dt = c->dt;
  const cplx* dw = (const cplx*)dw_in;
  cplx* ys[4];
  for (int j = 0; j < 4; ++j) ys[j] = xalloc(sizeof(cplx) * nn);
  stage_states(c, (const cplx*)w_in, ys);
  cplx* dk[4];
  for (int j = 0; j < 4; ++j) dk[j] = xalloc(sizeof(cplx) * nn);
  cplx* dy = xalloc(sizeof(cplx) * nn);
  orc_rhs_tlm(c, (double*)ys[0], dw_in, (double*)dk[0]);
  axpy_c(dy, dw, dt / 2, dk[0], nn);
  orc_rhs_tlm(c, (double*)ys[1], (double*)dy, (double*)dk[1]);
  axpy_c(dy, dw, dt / 2, dk[1], nn);
  orc_rhs_tlm(c, (double*)ys[2], (double*)dy, (double*)dk[2]);
  axpy_c(dy, dw, dt, dk[2], nn);
  orc_rhs_tlm(c, (double*)ys[3], (double*)dy, (double*)dk[3]);
  cplx* o = (cplx*)dw_out;
  for (int i = 0; i < nn; ++i) o[i] = dw[i] + dt / 6.0 * (dk[0][i] + 2.0 * dk[1][i] + 2.0 * dk[2][i] + dk[3][i]);
  if (w_out) orc_step(c, w_in, w_out);
  for (int j = 0; j < 4; ++j) { free(ys[j]); free(dk[j]); }
  free(dy);
}

/* Transpose of one RK4 step linearised at w: reverse sweep through the
 * stages.  With lb = lambda_{n+1}:
 *   kb4 = dt/6 lb,             yb4 = J4^T kb4
 *   kb3 = dt/3 lb + dt   yb4,  yb3 = J3^T kb3
 *   kb2 = dt/3 lb + dt/2 yb3,  yb2 = J2^T kb2
 *   kb1 = dt/6 lb + dt/2 yb2,  yb1 = J1^T kb1
 *   lambda_n = lb + yb1 + yb2 + yb3 + yb4. */
void orc_step_adj(const orc_cfg* c, const double* w_in, const double* lam_in, double* lam_out) {
  int nn = c->n * nh(c->n);
  double dt = c->dt;
  const cplx* lb = (const cplx*)lam_in;
  cplx* ys[4];
  for (int j = 0; j < 4; ++j) ys[j] = xalloc(sizeof(cplx) * nn);
  stage_states(c, (const cplx*)w_in, ys);
  cplx* kb = xalloc(sizeof(cplx) * nn);
  cplx* yb = xalloc(sizeof(cplx) * nn);
  cplx* sum = xalloc(sizeof(cplx) * nn);
  const double a_lb[4] = {dt / 6, dt / 3, dt / 3, dt / 6};  /* stages 4,3,2,1 */
  const double a_yb[4] = {0, dt, dt / 2, dt / 2};
  for (int s = 0; s < 4; ++s) {
    int j = 3 - s; /* stage index 4,3,2,1 -> 3,2,1,0 */
    for (int i = 0; i < nn; ++i) kb[i] = a_lb[s] * lb[i] + a_yb[s] * yb[i];
    orc_rhs_adj(c, (double*)ys[j], (double*)kb, (double*)yb);
    for (int i = 0; i < nn; ++i) sum[i] += yb[i];
  }
  cplx* o = (cplx*)lam_out;
  for (int i = 0; i < nn; ++i) o[i] = lb[i] + sum[i];
  for (int j = 0; j < 4; ++j) free(ys[j]);
  free(kb); free(yb); free(sum);
}

/* ------------------------------------------------------------------------ */
/* Observation operator (Eq. 3): velocity at lattice probes                  */
/* ------------------------------------------------------------------------ */

/* out[i][0..1] = (u, v) at probe i = r*px + q, node (iy, ix) = (r n/px, q n/px). */
void orc_observe(const orc_cfg* c, const double* w_in, double* out) {
  int n = c->n, P = c->px, st = n / c->px;
  cplx* scratch = xalloc(sizeof(cplx) * n * nh(n));
  double* u = xalloc(sizeof(double) * n * n);
  double* v = xalloc(sizeof(double) * n * n);
  physical_of((const cplx*)w_in, u, n, sym_u, scratch);
  physical_of((const cplx*)w_in, v, n, sym_v, scratch);
  for (int r = 0; r < P; ++r)
    for (int q = 0; q < P; ++q) {
      int node = (r * st) * n + q * st;
      out[2 * (r * P + q) + 0] = u[node];
      out[2 * (r * P + q) + 1] = v[node];
    }
  free(u); free(v); free(scratch);
}

/* Transpose of the observation operator: H^T r = U^T S^T r_u + V^T S^T r_v,
 * S^T the scatter of probe values onto an otherwise zero grid; returned as a
 * DFT on the retained set.  This is the source term M^T(M(u) - m) of Eq. (11). */
void orc_observe_adj(const orc_cfg* c, const double* r, double* out) {
  int n = c->n, P = c->px, st = n / c->px, nn = n * nh(n);
  double* gu = xalloc(sizeof(double) * n * n);
  double* gv = xalloc(sizeof(double) * n * n);
  for (int rr = 0; rr < P; ++rr)
    for (int q = 0; q < P; ++q) {
      int node = (rr * st) * n + q * st;
      gu[node] = r[2 * (rr * P + q) + 0];
      gv[node] = r[2 * (rr * P + q) + 1];
    }
  cplx* hu = xalloc(sizeof(cplx) * nn);
  cplx* hv = xalloc(sizeof(cplx) * nn);
  cplx* t = xalloc(sizeof(cplx) * nn);
  r2c(gu, hu, n);
  r2c(gv, hv, n);
  cplx* o = (cplx*)out;
  apply_sym(hu, o, n, sym_u, 1);
  apply_sym(hv, t, n, sym_v, 1);
  for (int i = 0; i < nn; ++i) o[i] += t[i];
  free(gu); free(gv); free(hu); free(hv); free(t);
}

/* ------------------------------------------------------------------------ */
/* Preconditioner: control map s -> w0 and gradient map (Sec. II.C, III.B)   */
/* ------------------------------------------------------------------------ */

/* W(|k|) = G_hat, the Fourier multiplier of the G-inner product (Eq. 13, 16):
 * kind 1 exp(-a|k|), kind 2 the fractional integral |k|^(-2a) (Sec. III.B's
 * G_p with alpha = a), kind 3 the heat kernel exp(-nu a k^2) (Sec. III.B's G_e
 * with beta = a), kind 4 a per-mode table. */
static double kernel_W(const orc_cfg* c, int kx, int ky, int q, int p) {
  double k2 = (double)kx * kx + (double)ky * ky;
  double k = sqrt(k2);
  switch (c->kernel_kind) {
    case 0: return 1.0;
    case 1: return exp(-c->kparam * k);
    case 2: return pow(k, -2.0 * c->kparam);
    case 3: return exp(-c->nu * c->kparam * k2);
    case 4: return c->ktable[q * nh(c->n) + p];
    default: return NAN;
  }
}

/* Multiplier m(k) = P |k| W^{1/2} (zero at k = 0).  The control s is the
 * half-sharpened scalar representation of the initial velocity: the scalar c
 * with c_hat = w_hat/|k| carries the same Euclidean norm as u (|u_hat|^2 +
 * |v_hat|^2 = |w_hat|^2/k^2), and s = G^{-1/2} c as in Eq. (18)-(19). */
static double control_mult(const orc_cfg* c, int q, int p) {
  int n = c->n, kx = p, ky = ky_of(q, n);
  if (!in_R(kx, ky, n) || (kx == 0 && ky == 0)) return 0.0;
  double k = sqrt((double)kx * kx + (double)ky * ky);
  return k * sqrt(kernel_W(c, kx, ky, q, p));
}

/* w0_hat = m(k) DFT(s). */
void orc_omega_from_control(const orc_cfg* c, const double* s, double* w0_out) {
  int n = c->n;
  cplx* w0 = (cplx*)w0_out;
  r2c(s, w0, n);
  for (int q = 0; q < n; ++q)
    for (int p = 0; p < nh(n); ++p) w0[q * nh(n) + p] *= control_mult(c, q, p);
}

/* Right inverse of the control map on the retained set: s = IDFT(w0_hat/m). */
void orc_control_from_omega(const orc_cfg* c, const double* w0_in, double* s) {
  int n = c->n, nn = n * nh(n);
  const cplx* w0 = (const cplx*)w0_in;
  cplx* h = xalloc(sizeof(cplx) * nn);
  for (int q = 0; q < n; ++q)
    for (int p = 0; p < nh(n); ++p) {
      double m = control_mult(c, q, p);
      h[q * nh(n) + p] = m != 0.0 ? w0[q * nh(n) + p] / m : 0;
    }
  c2r(h, s, n);
  free(h);
}

/* Gradient in the control: the map s -> w0 is the symmetric operator
 * IDFT m DFT (m real and even), so grad_s J = IDFT(m lambda0_hat), which is
 * G^{1/2} applied to the physical adjoint, Eq. (19). */
void orc_gradient_map(const orc_cfg* c, const double* lam0_in, double* g_s) {
  int n = c->n, nn = n * nh(n);
  const cplx* lam0 = (const cplx*)lam0_in;
  cplx* h = xalloc(sizeof(cplx) * nn);
  for (int q = 0; q < n; ++q)
    for (int p = 0; p < nh(n); ++p) h[q * nh(n) + p] = control_mult(c, q, p) * lam0[q * nh(n) + p];
  c2r(h, g_s, n);
  free(h);
}

/* ------------------------------------------------------------------------ */
/* Window: forward solve, cost (Eq. 2-3) and gradient (Eq. 11-12, 19)        */
/* ------------------------------------------------------------------------ */

/* Observation slot of step k, or -1: steps j*every (j >= 1), and step 0 when
 * include_t0 is set. */
static int obs_slot(const orc_cfg* c, int k) {
  if (k == 0) return c->include_t0 ? 0 : -1;
  if (k % c->every) return -1;
  return k / c->every - 1 + (c->include_t0 ? 1 : 0);
}

int orc_num_obs_times(const orc_cfg* c) { return c->nsteps / c->every + (c->include_t0 ? 1 : 0); }

/* Forward solve from control s: final state wT (half spectrum, may be NULL),
 * model observations obs [nt][px*px][2] (may be NULL), and, if traj is not
 * NULL, the state at every step [nsteps+1][n][n/2+1]. */
void orc_forward(const orc_cfg* c, const double* s, double* wT, double* obs, double* traj) {
  int n = c->n, nn = n * nh(n), P2 = c->px * c->px;
  cplx* w = xalloc(sizeof(cplx) * nn);
  cplx* w2 = xalloc(sizeof(cplx) * nn);
  orc_omega_from_control(c, s, (double*)w);
  for (int k = 0; k <= c->nsteps; ++k) {
    if (traj) memcpy(traj + (size_t)2 * nn * k, w, sizeof(cplx) * nn);
    int slot = obs_slot(c, k);
    if (slot >= 0 && obs) orc_observe(c, (double*)w, obs + (size_t)2 * P2 * slot);
    if (k == c->nsteps) break;
    orc_step(c, (double*)w, (double*)w2);
    memcpy(w, w2, sizeof(cplx) * nn);
  }
  if (wT) memcpy(wT, w, sizeof(cplx) * nn);
  free(w);
  free(w2);
}

/* Regularisation term of Eq. (4), lambda/2 sum over the grid of |grad u0|^2
 * (sums over grid nodes replace the integral, as for every inner product
 * here), with u0 the Biot-Savart velocity of w0: the four derivative fields
 * du/dx, du/dy, dv/dx, dv/dy are formed spectrally and squared on the grid. */
double orc_sobolev_term(const orc_cfg* c, const double* w0_in) {
  int n = c->n, nn = n * nh(n);
  const cplx* w0 = (const cplx*)w0_in;
  cplx* t1 = xalloc(sizeof(cplx) * nn);
  cplx* t2 = xalloc(sizeof(cplx) * nn);
  double* f = xalloc(sizeof(double) * n * n);
  symbol_fn vel[2] = {sym_u, sym_v}, der[2] = {sym_dx, sym_dy};
  double sum = 0.0;
  for (int a = 0; a < 2; ++a)
    for (int b = 0; b < 2; ++b) {
      apply_sym(w0, t1, n, vel[a], 0);
      apply_sym(t1, t2, n, der[b], 0);
      c2r(t2, f, n);
      for (int i = 0; i < n * n; ++i) sum += f[i] * f[i];
    }
  free(t1); free(t2); free(f);
  return 0.5 * c->sobolev * sum;
}

/* Gradient of the regularisation term with respect to the grid values of w0,
 * as a DFT: lambda sum_{a,b} V_a^T D_b^T D_b V_a w0 (each factor transposed),
 * accumulated into lam. */
static void sobolev_gradient(const orc_cfg* c, const cplx* w0, cplx* lam) {
  int n = c->n, nn = n * nh(n);
  cplx* t1 = xalloc(sizeof(cplx) * nn);
  cplx* t2 = xalloc(sizeof(cplx) * nn);
  symbol_fn vel[2] = {sym_u, sym_v}, der[2] = {sym_dx, sym_dy};
  for (int a = 0; a < 2; ++a)
    for (int b = 0; b < 2; ++b) {
      apply_sym(w0, t1, n, vel[a], 0);
      apply_sym(t1, t2, n, der[b], 0);
      apply_sym(t2, t1, n, der[b], 1);
      apply_sym(t1, t2, n, vel[a], 1);
      for (int i = 0; i < nn; ++i) lam[i] += c->sobolev * t2[i];
    }
  free(t1); free(t2);
}

/* Cost J = 1/2 sum_j sum_i |u(x_i, t_j) - m_ij|^2 (Eq. 2-3) and its gradient
 * with respect to the control s.  The adjoint runs backward from
 * lambda_{nsteps} = H^T r_{nsteps} (terminal condition zero plus the source
 * at the last observation), adding H^T r at every observation step.
 * lam0 (may be NULL) receives the DFT of grad_{w0} J. */
void orc_cost_grad(const orc_cfg* c, const double* s, const double* m, double* J, double* g_s, double* lam0) {
  int n = c->n, nn = n * nh(n), P2 = c->px * c->px, nt = orc_num_obs_times(c);
  double* traj = xalloc(sizeof(double) * 2 * (size_t)nn * (c->nsteps + 1));
  double* obs = xalloc(sizeof(double) * 2 * (size_t)P2 * nt);
  orc_forward(c, s, NULL, obs, traj);
  double* r = xalloc(sizeof(double) * 2 * (size_t)P2 * nt);
  double Jv = 0;
  for (int i = 0; i < 2 * P2 * nt; ++i) {
    r[i] = obs[i] - m[i];
    Jv += 0.5 * r[i] * r[i];
  }
  if (c->sobolev != 0.0) Jv += orc_sobolev_term(c, traj);
  *J = Jv;
  cplx* lam = xalloc(sizeof(cplx) * nn);
  cplx* lam2 = xalloc(sizeof(cplx) * nn);
  cplx* src = xalloc(sizeof(cplx) * nn);
  for (int k = c->nsteps; k >= 0; --k) {
    if (k < c->nsteps) {
      orc_step_adj(c, traj + (size_t)2 * nn * k, (double*)lam, (double*)lam2);
      memcpy(lam, lam2, sizeof(cplx) * nn);
    }
    int slot = obs_slot(c, k);
    if (slot >= 0) {
      orc_observe_adj(c, r + (size_t)2 * P2 * slot, (double*)src);
      for (int i = 0; i < nn; ++i) lam[i] += src[i];
    }
  }
  if (c->sobolev != 0.0) sobolev_gradient(c, (const cplx*)traj, lam);
  if (lam0) memcpy(lam0, lam, sizeof(cplx) * nn);
  if (g_s) orc_gradient_map(c, (double*)lam, g_s);
  free(traj); free(obs); free(r); free(lam); free(lam2); free(src);
}

/* Tangent-linear model of the window: dwT = d wT / ds applied to ds. */
void orc_forward_tlm(const orc_cfg* c, const double* s, const double* ds, double* dwT) {
  int nn = c->n * nh(c->n);
  cplx *w = xalloc(sizeof(cplx) * nn), *dw = xalloc(sizeof(cplx) * nn);
  cplx *w2 = xalloc(sizeof(cplx) * nn), *dw2 = xalloc(sizeof(cplx) * nn);
  orc_omega_from_control(c, s, (double*)w);
  orc_omega_from_control(c, ds, (double*)dw);
  for (int k = 0; k < c->nsteps; ++k) {
    orc_step_tlm(c, (double*)w, (double*)dw, (double*)w2, (double*)dw2);
    memcpy(w, w2, sizeof(cplx) * nn);
    memcpy(dw, dw2, sizeof(cplx) * nn);
  }
  memcpy(dwT, dw, sizeof(cplx) * nn);
  free(w); free(dw); free(w2); free(dw2);
}

/* Adjoint of the window driven only by a terminal field: given lamT (the DFT
 * of a gradient with respect to the final vorticity), returns lam0 (may be
 * NULL) and the control gradient g_s (may be NULL).  This is the adjoint
 * Green's-function run of Sec. IV with a general terminal field. */
void orc_adjoint_terminal(const orc_cfg* c, const double* s, const double* lamT, double* lam0, double* g_s) {
  int nn = c->n * nh(c->n);
  double* traj = xalloc(sizeof(double) * 2 * (size_t)nn * (c->nsteps + 1));
  orc_forward(c, s, NULL, NULL, traj);
  cplx* lam = xalloc(sizeof(cplx) * nn);
  cplx* lam2 = xalloc(sizeof(cplx) * nn);
  memcpy(lam, lamT, sizeof(cplx) * nn);
  mask_R(lam, c->n);
  for (int k = c->nsteps - 1; k >= 0; --k) {
    orc_step_adj(c, traj + (size_t)2 * nn * k, (double*)lam, (double*)lam2);
    memcpy(lam, lam2, sizeof(cplx) * nn);
  }
  if (lam0) memcpy(lam0, lam, sizeof(cplx) * nn);
  if (g_s) orc_gradient_map(c, (double*)lam, g_s);
  free(traj); free(lam); free(lam2);
}

/* ------------------------------------------------------------------------ */
/* Exposed transforms (for the pins)                                         */
/* ------------------------------------------------------------------------ */

void orc_fft1d(double* x, int m, int sign) { fft_inplace((cplx*)x, m, sign); }
void orc_r2c(const double* f, double* h, int n) { r2c(f, (cplx*)h, n); }
void orc_c2r(const double* h, double* f, int n) { c2r((const cplx*)h, f, n); }
