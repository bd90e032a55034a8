/*
 * fiber_oracle.c -- plain, slow, FP64 CPU oracle for the fiber-based
 * monodomain split step (Maier 2021, "Scalable Biophysical Simulations of the
 * Neuromuscular System").
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  It shares no code,
 * header, table or constant with the CUDA library; it reads plain arrays that
 * the seeded workload generator draws.
 *
 * What it computes, in the thesis's order and notation:
 *   * Hodgkin-Huxley subcellular model (sec:subcelullar_model,
 *     eq:subcellular_model_helper3/4/5, eq:subcellular): state y = (V, m, h, n),
 *     C_m dV/dt = -I_ion(V, y) + I_stim,
 *     I_ion = gNa m^3 h (V - ENa) + gK n^4 (V - EK) + gL (V - EL),
 *     dg/dt = alpha_g (1 - g) - beta_g g  (the printed "+ beta_n n" is a sign
 *     typo; the generated-code fragment in sec:code_generation uses "-").
 *     Rates: the HH 1952 squid-axon rates cited by the thesis, written in the
 *     depolarisation u = V - Vrest (the thesis prints alpha_m in V with
 *     Vrest = -75 mV: -0.1 (V + 50) / (exp(-(V + 50)/10) - 1)).
 *   * Monodomain equation on each 1D fiber (eq:monodomain) with homogeneous
 *     Neumann ends (eq:monodomain_bc1); diffusion prefactor
 *     c = sigma_eff / (Am Cm).
 *   * Linear finite elements with mass lumping (sec:discretization_diffusion,
 *     eq:diffusion_matrices, sec:mass_lumping): stiffness K = -(1/h)[1 -2 1]
 *     (end rows -(1/h)[-1 1]), lumped mass h (h/2 at the two end nodes).
 *   * Crank-Nicolson in the lumped form eq:lumping_crank_nicolson_2:
 *     (I - dt/2 M^-1 K) u+ = (I + dt/2 M^-1 K) u, solved by the Thomas
 *     algorithm (sec:improved_parallel_solver_for_fiber_based).
 *   * Heun's method eq:heun on the full state (V, m, h, n).
 *   * Optionally the thesis's approximated exponential exp*(x) =
 *     (1 + x/1024)^1024 (eq:apx-e-function) in place of every exp of the rates.
 *   * Implicit Euler in the lumped form eq:lumping_implicit_euler_2:
 *     (I - dt M^-1 K) u+ = u (selectable instead of CN).
 *   * Strang splitting eq:monodomain_strang: diffusion dt/2, reaction dt,
 *     diffusion dt/2, with the reaction sub-cycled in Heun steps of dt_0d and
 *     each diffusion half in CN steps of dt_1d.  Selectable instead: Godunov
 *     splitting eq:monodomain_godunov (diffusion dt, reaction dt), and the
 *     orderings of the splitting figures (reaction dt/2, diffusion dt,
 *     reaction dt/2; reaction dt, diffusion dt).
 *   * Stimulus (sec:stimulation_times_callbacks): current injection of
 *     stim_amplitude at the junction node and its neighbours (3 nodes),
 *     switched on for stim_duration after each firing time of the fiber's
 *     motor unit.
 *
 * Readings where the thesis is silent or garbled are listed in the project's
 * design notes: exact-rest leak reversal, stimulus window in whole Heun
 * substeps (k_f = round-half-even(t_f / dt_0d)), overlapping pulses OR-ed,
 * Heun stages holding I_stim of the substep start, Strang order 1D/0D/1D.
 *
 * Build: cc -O2 -fPIC -shared fiber_oracle.c -lm -lpthread (no -ffast-math).
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
  double Cm, gNa, gK, gL, ENa, EK, EL, Vrest; /* EL NaN: derive exact rest */
  double sigma_eff, Am, h;
  double dt_split, dt_0d, dt_1d;
  double stim_amplitude, stim_duration;
  int32_t stim_half_width;
  int32_t splitting; /* 0: Strang 1D(dt/2), 0D(dt), 1D(dt/2)   (eq:monodomain_strang, L1 = diffusion)
                        1: Godunov 1D(dt), 0D(dt)              (eq:monodomain_godunov, L1 = diffusion)
                        2: Strang 0D(dt/2), 1D(dt), 0D(dt/2)   (fig:strang_splitting)
                        3: Godunov 0D(dt), 1D(dt)              (fig:godunov_splitting) */
  int32_t diffusion; /* 0: Crank-Nicolson (eq:lumping_crank_nicolson_2)
                        1: implicit Euler (eq:lumping_implicit_euler_2) */
  int32_t exp_approx; /* 1: every exponential of the rates is exp*(x) = (1 + x/1024)^1024
                         (eq:apx-e-function) */
} orc_params;

enum { ORC_OK = 0, ORC_EINVAL = 1, ORC_ENOMEM = 2 };

/* ------------------------------------------------------------------------ */
/* Hodgkin-Huxley rates (HH 1952, shifted so that u = V - Vrest).            */
/* ------------------------------------------------------------------------ */

/* x / (1 - exp(-x/k)): the alpha_m / alpha_n shape; its removable
 * singularity at x = 0 has the limit k.  expm1 keeps it accurate near 0. */
static double vtrap(double x, double k) {
  if (x == 0.0) return k;
  return x / (-expm1(-x / k));
}

/* exp*(x) = (1 + x/1024)^1024, evaluated as one addition and ten squarings
 * (eq:apx-e-function). */
double orc_exp_star(double x) {
  double y = 1.0 + x / 1024.0;
  for (int i = 0; i < 10; ++i) y = y * y;
  return y;
}

/* x / (1 - exp*(-x/k)), the same shape with exp* (limit k at x = 0). */
static double vtrap_star(double x, double k) {
  if (x == 0.0) return k;
  return x / (1.0 - orc_exp_star(-x / k));
}

/* out = {alpha_m, beta_m, alpha_h, beta_h, alpha_n, beta_n} in 1/ms at V. */
void orc_hh_rates(const orc_params* p, double V, double out[6]) {
  const double u = V - p->Vrest;
  if (p->exp_approx) {
    /* the same formulas with each exponential replaced by exp* */
    out[0] = 0.1 * vtrap_star(u - 25.0, 10.0);
    out[1] = 4.0 * orc_exp_star(-u / 18.0);
    out[2] = 0.07 * orc_exp_star(-u / 20.0);
    out[3] = 1.0 / (1.0 + orc_exp_star((30.0 - u) / 10.0));
    out[4] = 0.01 * vtrap_star(u - 10.0, 10.0);
    out[5] = 0.125 * orc_exp_star(-u / 80.0);
    return;
  }
  out[0] = 0.1 * vtrap(u - 25.0, 10.0);          /* alpha_m */
  out[1] = 4.0 * exp(-u / 18.0);                 /* beta_m  */
  out[2] = 0.07 * exp(-u / 20.0);                /* alpha_h */
  out[3] = 1.0 / (1.0 + exp((30.0 - u) / 10.0)); /* beta_h  */
  out[4] = 0.01 * vtrap(u - 10.0, 10.0);         /* alpha_n */
  out[5] = 0.125 * exp(-u / 80.0);               /* beta_n  */
}

/* Steady-state gates g_inf = alpha / (alpha + beta) at V (n_inf = alpha tau). */
void orc_gates_inf(const orc_params* p, double V, double g[3]) {
  double r[6];
  orc_hh_rates(p, V, r);
  g[0] = r[0] / (r[0] + r[1]);
  g[1] = r[2] / (r[2] + r[3]);
  g[2] = r[4] / (r[4] + r[5]);
}

/* Leak reversal that makes (Vrest, m_inf, h_inf, n_inf) an exact fixed
 * point: I_ion(Vrest) = 0 solved for EL. */
double orc_leak_reversal_exact(const orc_params* p) {
  double g[3];
  orc_gates_inf(p, p->Vrest, g);
  const double m = g[0], hh = g[1], n = g[2];
  const double ina = p->gNa * m * m * m * hh * (p->Vrest - p->ENa);
  const double ik = p->gK * n * n * n * n * (p->Vrest - p->EK);
  return p->Vrest + (ina + ik) / p->gL;
}

static double leak_reversal(const orc_params* p) {
  return isnan(p->EL) ? orc_leak_reversal_exact(p) : p->EL;
}

/* Right-hand side of the subcellular model: dy/dt at y = (V, m, h, n) with
 * the stimulus current density istim (uA/cm^2) injected. */
void orc_hh_rhs(const orc_params* p, double EL, const double y[4], double istim, double dy[4]) {
  double r[6];
  orc_hh_rates(p, y[0], r);
  const double V = y[0], m = y[1], hh = y[2], n = y[3];
  const double iion = p->gNa * m * m * m * hh * (V - p->ENa) + p->gK * n * n * n * n * (V - p->EK) +
                      p->gL * (V - EL);
  dy[0] = (-iion + istim) / p->Cm;
  dy[1] = r[0] * (1.0 - m) - r[1] * m;
  dy[2] = r[2] * (1.0 - hh) - r[3] * hh;
  dy[3] = r[4] * (1.0 - n) - r[5] * n;
}

/* One Heun step (eq:heun) of width dt, istim held over both stages. */
void orc_heun_step(const orc_params* p, double EL, double y[4], double istim, double dt) {
  double f0[4], y1[4], f1[4];
  orc_hh_rhs(p, EL, y, istim, f0);
  for (int i = 0; i < 4; ++i) y1[i] = y[i] + dt * f0[i];
  orc_hh_rhs(p, EL, y1, istim, f1);
  for (int i = 0; i < 4; ++i) y[i] = y[i] + 0.5 * dt * (f0[i] + f1[i]);
}

/* ------------------------------------------------------------------------ */
/* Tridiagonal systems                                                        */
/* ------------------------------------------------------------------------ */

/* Thomas algorithm for a_i x_{i-1} + b_i x_i + c_i x_{i+1} = d_i, i = 0..n-1
 * (a_0 and c_{n-1} ignored).  Forward elimination then back substitution.
 * work: n doubles.  Returns ORC_EINVAL on a zero pivot. */
int orc_thomas(int n, const double* a, const double* b, const double* c, const double* d, double* x,
               double* work) {
  if (n <= 0) return ORC_OK;
  double piv = b[0];
  if (piv == 0.0) return ORC_EINVAL;
  work[0] = (n > 1) ? c[0] / piv : 0.0;
  x[0] = d[0] / piv;
  for (int i = 1; i < n; ++i) {
    piv = b[i] - a[i] * work[i - 1];
    if (piv == 0.0) return ORC_EINVAL;
    work[i] = (i < n - 1) ? c[i] / piv : 0.0;
    x[i] = (d[i] - a[i] * x[i - 1]) / piv;
  }
  for (int i = n - 2; i >= 0; --i) x[i] -= work[i] * x[i + 1];
  return ORC_OK;
}

/* Rows of the lumped CN system for one fiber of n nodes and one CN step of
 * width dt: (I - dt/2 L) V+ = (I + dt/2 L) V with L = c M_L^-1 K.  With
 * r = c dt / h^2, interior rows of L are (c/h^2)[1 -2 1], end rows
 * (c/h^2)[-2 2] (lumped end mass h/2).  Fills the LHS bands a, b, cc and the
 * RHS d from V.  n == 1: no diffusion (identity). */
static void cn_rows(int n, double r, const double* V, double* a, double* b, double* cc, double* d) {
  if (n == 1) {
    a[0] = 0.0; b[0] = 1.0; cc[0] = 0.0; d[0] = V[0];
    return;
  }
  for (int i = 0; i < n; ++i) {
    if (i == 0) {
      a[i] = 0.0; b[i] = 1.0 + r; cc[i] = -r;
      d[i] = (1.0 - r) * V[0] + r * V[1];
    } else if (i == n - 1) {
      a[i] = -r; b[i] = 1.0 + r; cc[i] = 0.0;
      d[i] = r * V[n - 2] + (1.0 - r) * V[n - 1];
    } else {
      a[i] = -0.5 * r; b[i] = 1.0 + r; cc[i] = -0.5 * r;
      d[i] = 0.5 * r * V[i - 1] + (1.0 - r) * V[i] + 0.5 * r * V[i + 1];
    }
  }
}

/* Rows of the lumped implicit-Euler system (eq:lumping_implicit_euler_2):
 * (I - dt L) V+ = V with the same L as cn_rows: with q = c dt / h^2, interior
 * rows (-q, 1 + 2q, -q), end rows (1 + 2q, -2q). */
static void ie_rows(int n, double q, const double* V, double* a, double* b, double* cc, double* d) {
  for (int i = 0; i < n; ++i) {
    d[i] = V[i];
    if (n == 1) {
      a[i] = 0.0; b[i] = 1.0; cc[i] = 0.0;
    } else if (i == 0) {
      a[i] = 0.0; b[i] = 1.0 + 2.0 * q; cc[i] = -2.0 * q;
    } else if (i == n - 1) {
      a[i] = -2.0 * q; b[i] = 1.0 + 2.0 * q; cc[i] = 0.0;
    } else {
      a[i] = -q; b[i] = 1.0 + 2.0 * q; cc[i] = -q;
    }
  }
}

/* Diffusion prefactor c = sigma_eff / (Am Cm) (eq:monodomain). */
static double diffusion_c(const orc_params* p) { return p->sigma_eff / (p->Am * p->Cm); }

/* Exported for tests: the CN matrix bands and RHS of one step of width dt. */
int orc_cn_system(const orc_params* p, int n, double dt, const double* V, double* a, double* b, double* c,
                  double* d) {
  if (n < 1) return ORC_EINVAL;
  cn_rows(n, diffusion_c(p) * dt / (p->h * p->h), V, a, b, c, d);
  return ORC_OK;
}

/* One implicit-Euler step of width dt on V (in place).  work: 5n doubles. */
int orc_ie_step(const orc_params* p, int n, double dt, double* V, double* work) {
  if (n < 1) return ORC_EINVAL;
  double *a = work, *b = work + n, *c = work + 2 * n, *d = work + 3 * n, *w = work + 4 * n;
  ie_rows(n, diffusion_c(p) * dt / (p->h * p->h), V, a, b, c, d);
  return orc_thomas(n, a, b, c, d, V, w);
}

/* One CN step of width dt on V (in place).  work: 5n doubles. */
int orc_cn_step(const orc_params* p, int n, double dt, double* V, double* work) {
  if (n < 1) return ORC_EINVAL;
  double *a = work, *b = work + n, *c = work + 2 * n, *d = work + 3 * n, *w = work + 4 * n;
  cn_rows(n, diffusion_c(p) * dt / (p->h * p->h), V, a, b, c, d);
  return orc_thomas(n, a, b, c, d, V, w);
}

/* ------------------------------------------------------------------------ */
/* Stimulus schedule                                                          */
/* ------------------------------------------------------------------------ */

/* Whole substeps of width dt_0d in an interval (round half to even). */
static int64_t substeps_of(double t_ms, double dt0) { return (int64_t)nearbyint(t_ms / dt0); }

/* Is the fiber's MU pulse on during Heun substep k (start t = k dt_0d)?  On
 * iff some firing f has k_f <= k < k_f + P.  fire_k sorted ascending. */
static int stim_on(const int64_t* fire_k, int64_t n_fire, int64_t P, int64_t k) {
  for (int64_t f = 0; f < n_fire; ++f) {
    if (fire_k[f] > k) break;
    if (k < fire_k[f] + P) return 1;
  }
  return 0;
}

/* ------------------------------------------------------------------------ */
/* One fiber, many split steps                                                */
/* ------------------------------------------------------------------------ */

typedef struct {
  int64_t n_sub;  /* Heun substeps per split step */
  int64_t n_cn;   /* CN steps per diffusion half */
  double dt0, dt1;
  int64_t P;      /* pulse length in substeps */
  double EL;
} orc_derived;

static int derive(const orc_params* p, orc_derived* o) {
  if (!(p->dt_split > 0.0) || !(p->dt_0d > 0.0) || !(p->dt_1d > 0.0) || !(p->h > 0.0) || !(p->Cm > 0.0) ||
      !(p->Am > 0.0) || p->stim_half_width < 0 || p->splitting < 0 || p->splitting > 3 || p->diffusion < 0 ||
      p->diffusion > 1)
    return ORC_EINVAL;
  /* Heun substeps per split step, and diffusion steps per diffusion phase:
   * half a split step (Strang 1D-0D-1D) or a whole one (the others). */
  const double q0 = p->dt_split / p->dt_0d;
  const double q1 = (p->splitting == 0 ? 0.5 : 1.0) * p->dt_split / p->dt_1d;
  o->n_sub = (int64_t)nearbyint(q0);
  o->n_cn = (int64_t)nearbyint(q1);
  if (o->n_sub < 1 || o->n_cn < 1 || fabs(q0 - (double)o->n_sub) > 1e-9 * q0 ||
      fabs(q1 - (double)o->n_cn) > 1e-9 * q1)
    return ORC_EINVAL;
  o->dt0 = p->dt_0d;
  o->dt1 = p->dt_1d;
  o->P = substeps_of(p->stim_duration, p->dt_0d);
  o->EL = leak_reversal(p);
  if (p->splitting == 2 && (o->n_sub % 2) != 0) return ORC_EINVAL; /* dt/2 in whole substeps */
  return ORC_OK;
}

/* Runs split steps step0 .. step0+n_steps-1 on one fiber of n nodes.
 * state: V, m, h, nn (each n doubles), in/out.
 * fire_ms: the fiber's MU firing times (ms), sorted ascending.
 * Every sample_every steps (if > 0 and samples != NULL) V is appended to
 * samples (row-major, n per row).  work: 5n doubles; fire_k: n_fire int64. */
static int fiber_run(const orc_params* p, const orc_derived* o, int n, int junction, const double* fire_ms,
                     int64_t n_fire, double* V, double* m, double* hh, double* nn, int64_t step0,
                     int64_t n_steps, int64_t sample_every, double* samples, int64_t sample_stride,
                     double* work, int64_t* fire_k) {
  for (int64_t f = 0; f < n_fire; ++f) fire_k[f] = substeps_of(fire_ms[f], o->dt0);
  const int lo = junction - p->stim_half_width < 0 ? 0 : junction - p->stim_half_width;
  const int hi = junction + p->stim_half_width > n - 1 ? n - 1 : junction + p->stim_half_width;
  int64_t row = 0;
  for (int64_t s = 0; s < n_steps; ++s) {
    const int64_t step = step0 + s;
    /* reaction: Heun substeps k0 <= k < k1 of this split step at every node */
#define ORC_REACT(k0, k1)                                                          \
    for (int64_t k = (k0); k < (k1); ++k) {                                        \
      const int64_t kk = step * o->n_sub + k;                                      \
      const int on = stim_on(fire_k, n_fire, o->P, kk);                            \
      for (int i = 0; i < n; ++i) {                                                \
        double y[4] = {V[i], m[i], hh[i], nn[i]};                                  \
        const double istim = (on && i >= lo && i <= hi) ? p->stim_amplitude : 0.0; \
        orc_heun_step(p, o->EL, y, istim, o->dt0);                                 \
        V[i] = y[0]; m[i] = y[1]; hh[i] = y[2]; nn[i] = y[3];                      \
      }                                                                            \
    }
    /* diffusion: n_cn steps of dt_1d with the selected method */
#define ORC_DIFFUSE()                                                                          \
    for (int64_t c = 0; c < o->n_cn; ++c)                                                      \
      if ((p->diffusion == 1 ? orc_ie_step(p, n, o->dt1, V, work)                              \
                             : orc_cn_step(p, n, o->dt1, V, work)) != ORC_OK) return ORC_EINVAL;
    if (p->splitting == 0) {        /* 1D(dt/2), 0D(dt), 1D(dt/2) */
      ORC_DIFFUSE()
      ORC_REACT(0, o->n_sub)
      ORC_DIFFUSE()
    } else if (p->splitting == 1) { /* 1D(dt), 0D(dt) */
      ORC_DIFFUSE()
      ORC_REACT(0, o->n_sub)
    } else if (p->splitting == 2) { /* 0D(dt/2), 1D(dt), 0D(dt/2) */
      ORC_REACT(0, o->n_sub / 2)
      ORC_DIFFUSE()
      ORC_REACT(o->n_sub / 2, o->n_sub)
    } else {                        /* 0D(dt), 1D(dt) */
      ORC_REACT(0, o->n_sub)
      ORC_DIFFUSE()
    }
#undef ORC_DIFFUSE
#undef ORC_REACT
    if (samples && sample_every > 0 && ((s + 1) % sample_every) == 0) {
      memcpy(samples + row * sample_stride, V, sizeof(double) * (size_t)n);
      ++row;
    }
  }
  return ORC_OK;
}

/* Initial state of a bundle in the ragged layout: V = vm0 (or Vrest), gates
 * at their steady state at Vrest.  state: 4 * total doubles (V | m | h | n). */
int orc_init_state(const orc_params* p, int64_t total, const float* vm0, double* state) {
  double g[3];
  orc_gates_inf(p, p->Vrest, g);
  for (int64_t i = 0; i < total; ++i) {
    state[i] = vm0 ? (double)vm0[i] : p->Vrest;
    state[total + i] = g[0];
    state[2 * total + i] = g[1];
    state[3 * total + i] = g[2];
  }
  return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Many fibers on host threads (fibers are independent: eq:discretized_fibers) */
/* ------------------------------------------------------------------------ */

typedef struct {
  const orc_params* p;
  const orc_derived* o;
  int32_t n_fibers;
  const int32_t *n_nodes, *mu_of_fiber, *junction;
  int32_t n_mu;
  const int64_t* mu_offsets;
  const double* fire_ms;
  const int64_t* off; /* ragged offsets, n_fibers + 1 */
  int64_t total;
  double* state;
  int64_t step0, n_steps, sample_every;
  double* samples; /* n_rows x total */
  pthread_mutex_t lock;
  int32_t next;
  int status;
} orc_job;

static void* worker(void* arg) {
  orc_job* J = (orc_job*)arg;
  int64_t max_n = 1, max_fire = 1;
  for (int32_t f = 0; f < J->n_fibers; ++f)
    if (J->n_nodes[f] > max_n) max_n = J->n_nodes[f];
  for (int32_t k = 0; k < J->n_mu; ++k)
    if (J->mu_offsets[k + 1] - J->mu_offsets[k] > max_fire) max_fire = J->mu_offsets[k + 1] - J->mu_offsets[k];
  double* work = (double*)malloc(sizeof(double) * 5 * (size_t)max_n);
  int64_t* fire_k = (int64_t*)malloc(sizeof(int64_t) * (size_t)max_fire);
  if (!work || !fire_k) {
    pthread_mutex_lock(&J->lock);
    J->status = ORC_ENOMEM;
    pthread_mutex_unlock(&J->lock);
    free(work);
    free(fire_k);
    return NULL;
  }
  for (;;) {
    pthread_mutex_lock(&J->lock);
    const int32_t f = J->next++;
    const int bad = J->status != ORC_OK;
    pthread_mutex_unlock(&J->lock);
    if (f >= J->n_fibers || bad) break;
    const int64_t o = J->off[f];
    const int mu = J->mu_of_fiber[f];
    const double* fire = J->fire_ms;
    int64_t nf = 0;
    if (mu >= 0 && mu < J->n_mu) {
      fire = J->fire_ms + J->mu_offsets[mu];
      nf = J->mu_offsets[mu + 1] - J->mu_offsets[mu];
    }
    const int64_t T = J->total;
    int st = fiber_run(J->p, J->o, J->n_nodes[f], J->junction[f], fire, nf, J->state + o, J->state + T + o,
                       J->state + 2 * T + o, J->state + 3 * T + o, J->step0, J->n_steps, J->sample_every,
                       J->samples ? J->samples + o : NULL, T, work, fire_k);
    if (st != ORC_OK) {
      pthread_mutex_lock(&J->lock);
      J->status = st;
      pthread_mutex_unlock(&J->lock);
    }
  }
  free(work);
  free(fire_k);
  return NULL;
}

/* Runs split steps [step0, step0 + n_steps) on every fiber of a bundle.
 * state: 4 * total doubles in the ragged layout (V | m | h | n), in/out.
 * samples (nullable): (n_steps / sample_every) rows of total doubles (V).
 * n_threads <= 0: one thread.  Returns ORC_OK / ORC_EINVAL / ORC_ENOMEM. */
int orc_run_fibers(const orc_params* p, int32_t n_fibers, const int32_t* n_nodes, const int32_t* mu_of_fiber,
                   const int32_t* junction, int32_t n_mu, const int64_t* mu_offsets, const double* fire_ms,
                   double* state, int64_t step0, int64_t n_steps, int64_t sample_every, double* samples,
                   int32_t n_threads) {
  orc_derived o;
  if (derive(p, &o) != ORC_OK || n_fibers < 0 || n_mu < 0 || n_steps < 0 || step0 < 0) return ORC_EINVAL;
  int64_t* off = (int64_t*)malloc(sizeof(int64_t) * ((size_t)n_fibers + 1));
  if (!off) return ORC_ENOMEM;
  off[0] = 0;
  for (int32_t f = 0; f < n_fibers; ++f) {
    if (n_nodes[f] < 1 || junction[f] < 0 || junction[f] >= n_nodes[f]) {
      free(off);
      return ORC_EINVAL;
    }
    off[f + 1] = off[f] + n_nodes[f];
  }
  orc_job J;
  memset(&J, 0, sizeof(J));
  J.p = p; J.o = &o; J.n_fibers = n_fibers; J.n_nodes = n_nodes; J.mu_of_fiber = mu_of_fiber;
  J.junction = junction; J.n_mu = n_mu; J.mu_offsets = mu_offsets; J.fire_ms = fire_ms; J.off = off;
  J.total = off[n_fibers]; J.state = state; J.step0 = step0; J.n_steps = n_steps;
  J.sample_every = sample_every; J.samples = samples; J.next = 0; J.status = ORC_OK;
  pthread_mutex_init(&J.lock, NULL);
  int nt = n_threads < 1 ? 1 : n_threads;
  if (nt > n_fibers && n_fibers > 0) nt = n_fibers;
  if (nt <= 1) {
    worker(&J);
  } else {
    pthread_t* th = (pthread_t*)malloc(sizeof(pthread_t) * (size_t)nt);
    int started = 0;
    if (th)
      for (; started < nt; ++started)
        if (pthread_create(&th[started], NULL, worker, &J) != 0) break;
    if (started == 0) worker(&J);
    for (int i = 0; i < started; ++i) pthread_join(th[i], NULL);
    free(th);
  }
  pthread_mutex_destroy(&J.lock);
  free(off);
  return J.status;
}
