// Hodgkin-Huxley device arithmetic shared by the split-step kernel and the
// surrogate kernels (sec:subcelullar_model; HH 1952 rates in the
// depolarisation u = V - Vrest).
#pragma once

#include "fibers_internal.h"

namespace fib {
namespace {

// ---------------------------------------------------------------------------
// Hodgkin-Huxley right-hand side (HH 1952 rates in u = V - Vrest)
// ---------------------------------------------------------------------------

__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

__device__ __forceinline__ float rcp_approx(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// log2(e) multiples used to turn exp(x) into 2^(x log2 e).
constexpr float kLog2e = 1.4426950408889634f;
constexpr float kE25 = 12.182493960703473f;  // e^2.5
constexpr float kE30 = 20.085536923187668f;  // e^3
constexpr float kE10 = 2.718281828459045f;   // e^1

// Removable singularities.  alpha_m = z_m / (e^z_m - 1) with z_m = (25 - u)/10
// and alpha_n = z_n' / (e^(10 z_n') - 1) with z_n' = (10 - u)/100 have finite
// limits at z = 0, where the direct quotient loses accuracy (cancellation in
// e^z - 1) and is 0/0 at the point itself.  Within |z_m| < 0.01 (|z_n'| <
// 0.001) the first two terms of the Bernoulli series z/(e^z - 1) = 1 - z/2 +
// z^2/12 - ... replace it.  The dropped terms stay below 8.3e-6 relative in
// the window, under the direct form's own error at the window's edge (about
// 3e-5 relative, shrinking as 1/|z| outside it), so the pair bounds the
// error of the rate by 3e-5 everywhere with one FMA for the series.  Both
// forms choose per node with a branch-free select.
//
// Signs: the code carries nz = -z, -alpha_m, -alpha_n, -beta_h, -(dm/dt) and
// -(dn/dt), so that every subtraction becomes an FMA with a constant of the
// right sign or a plain subtraction, and the packed FP32x2 form (which has no
// negate modifier) needs no extra instruction.  Both forms execute the same
// operations.
__device__ __forceinline__ bool near_singular(float nzm, float nzn) {
  return fabsf(nzm) < 0.01f || fabsf(nzn) < 0.001f;
}
// -(1 - z/2) with z = -nzm
__device__ __forceinline__ float nam_series(float nzm) { return fmaf(nzm, -0.5f, -1.0f); }
// -(0.1 - z/2) with z = -nzn
__device__ __forceinline__ float nan_series(float nzn) { return fmaf(nzn, -0.5f, -0.1f); }

// Right-hand side of the HH model at one node.  With E = exp(-u/10):
//   alpha_m = 0.1 (25-u)/(exp((25-u)/10) - 1)   exp((25-u)/10) = e^2.5 E
//   beta_m  = 4 exp(-u/18)
//   alpha_h = 0.07 exp(-u/20)
//   beta_h  = 1/(exp((30-u)/10) + 1)             exp((30-u)/10) = e^3 E
//   alpha_n = 0.01 (10-u)/(exp((10-u)/10) - 1)   exp((10-u)/10) = e E
//   beta_n  = 0.125 exp(-u/80)
//   dg/dt   = alpha_g - (alpha_g + beta_g) g
//   du/dt   = gNa m^3 h (uNa - u) + gK n^4 (uK - u) + gL (uL - u) + stim
//           = (gNa uNa m^3 h + gK uK n^4 + gL uL + stim) - u (gNa m^3 h + gK n^4 + gL)
// (conductances divided by Cm).  Returns du/dt, -dm/dt, dh/dt, -dn/dt.
// `gl_ul` is gL uL + stim.
struct Deriv {
  float u, m, h, n;
};

// The thesis's approximated exponential exp*(x) = (1 + x/1024)^1024
// (eq:apx-e-function): one FMA (x/1024 is exact) and ten squarings, all on
// the FP32 pipe instead of the special-function unit.
__device__ __forceinline__ float exp_star(float x) {
  float y = fmaf(x, 1.0f / 1024.0f, 1.0f);
#pragma unroll
  for (int i = 0; i < 10; ++i) y = y * y;
  return y;
}

// The exponential terms of the rates.  Exact form: one ex2 gives
// E = e^(-u/10) and the three /10 rates reuse it through e^2.5, e and e^3.
// EXPAPX: each exponential of the rate formulas becomes its own exp*, since
// exp* is not multiplicative.  Returns the quotient denominators
// e^((25-u)/10) - 1, e^((10-u)/10) - 1, -e^((30-u)/10) - 1 and the scaled
// exponentials beta_m, alpha_h, beta_n.
struct RateExps {
  float dm, dn, dh, bm, ah, bn;
};

template <bool EXPAPX>
__device__ __forceinline__ RateExps rate_exps(float u, float nzm, float nzn) {
  RateExps r;
  if (EXPAPX) {
    r.dm = exp_star(-nzm) - 1.0f;                              // (25 - u)/10 = -nzm
    r.dn = exp_star(fmaf(u, -0.1f, 1.0f)) - 1.0f;              // (10 - u)/10
    r.dh = fmaf(exp_star(fmaf(u, -0.1f, 3.0f)), -1.0f, -1.0f);
    r.bm = 4.0f * exp_star(u * (-1.0f / 18.0f));
    r.ah = 0.07f * exp_star(u * (-1.0f / 20.0f));
    r.bn = 0.125f * exp_star(u * (-1.0f / 80.0f));
  } else {
    const float E = ex2_approx(u * (-kLog2e / 10.0f));
    r.bm = ex2_approx(fmaf(u, -kLog2e / 18.0f, 2.0f));                    // 4 e^(-u/18)
    r.ah = ex2_approx(fmaf(u, -kLog2e / 20.0f, -3.8365012677171206f));    // 0.07 e^(-u/20)
    r.bn = ex2_approx(fmaf(u, -kLog2e / 80.0f, -3.0f));                   // 0.125 e^(-u/80)
    r.dm = fmaf(kE25, E, -1.0f);
    r.dn = fmaf(kE10, E, -1.0f);
    r.dh = fmaf(-kE30, E, -1.0f);
  }
  return r;
}

template <bool EXPAPX = false>
__device__ __forceinline__ Deriv hh_rhs(float u, float m, float h, float n, float gl_ul, const HHConst& c) {
  const float nzm = fmaf(u, 0.1f, -2.5f);    // -(25 - u) / 10
  const float nzn = fmaf(u, 0.01f, -0.1f);   // -(10 - u) / 100
  const RateExps x = rate_exps<EXPAPX>(u, nzm, nzn);
  const float bm = x.bm, ah = x.ah, bn = x.bn;
  // branch-free (a branch would split the unrolled node loop into blocks
  // the scheduler cannot interleave)
  const float nam = fabsf(nzm) < 0.01f ? nam_series(nzm) : nzm * rcp_approx(x.dm);
  const float nan_ = fabsf(nzn) < 0.001f ? nan_series(nzn) : nzn * rcp_approx(x.dn);
  const float nbh = rcp_approx(x.dh);
  Deriv d;
  d.m = fmaf(bm - nam, m, nam);     // (am + bm) m - am
  d.h = fmaf(nbh - ah, h, ah);      // ah - (ah + bh) h
  d.n = fmaf(bn - nan_, n, nan_);   // (an + bn) n - an
  const float A = (m * m) * (m * h);
  float B = n * n;
  B = B * B;
  const float t = fmaf(A, c.gNa_uNa, fmaf(B, c.gK_uK, gl_ul));
  const float nS = fmaf(A, -c.gNa, fmaf(B, -c.gK, -c.gL));
  d.u = fmaf(u, nS, t);
  return d;
}

// One Heun substep (eq:heun) of every node a thread holds.  STIM: the
// thread owns at least one junction node and the pulse is on; `mask` has
// bit j set for stimulated nodes.  The gate arrays hold g - (c.m0, c.h0,
// c.n0): the right-hand sides and the predictor use absolute gates, the
// corrector accumulates into the deviations.
template <int K, bool STIM, bool EXPAPX = false>
__device__ __forceinline__ void heun_nodes(float (&u)[K], float (&m)[K], float (&h)[K], float (&n)[K],
                                           const HHConst& c, uint32_t mask) {
  const float dt = c.dt0, hdt = 0.5f * c.dt0;
#pragma unroll
  for (int j = 0; j < K; ++j) {
    const float s = (STIM && ((mask >> j) & 1u)) ? c.gL_uL + c.stim : c.gL_uL;
    const float ma = m[j] + c.m0, ha = h[j] + c.h0, na = n[j] + c.n0;
    const Deriv f0 = hh_rhs<EXPAPX>(u[j], ma, ha, na, s, c);
    const float u1 = fmaf(dt, f0.u, u[j]);
    const float m1 = fmaf(-dt, f0.m, ma);
    const float h1 = fmaf(dt, f0.h, ha);
    const float n1 = fmaf(-dt, f0.n, na);
    // y + dt/2 (f0 + f1) as (y + dt/2 f0) + dt/2 f1: y is then dead once
    // the predictor is formed
    u[j] = fmaf(hdt, f0.u, u[j]);
    m[j] = fmaf(-hdt, f0.m, m[j]);
    h[j] = fmaf(hdt, f0.h, h[j]);
    n[j] = fmaf(-hdt, f0.n, n[j]);
    const Deriv f1 = hh_rhs<EXPAPX>(u1, m1, h1, n1, s, c);
    u[j] = fmaf(hdt, f1.u, u[j]);
    m[j] = fmaf(-hdt, f1.m, m[j]);
    h[j] = fmaf(hdt, f1.h, h[j]);
    n[j] = fmaf(-hdt, f1.n, n[j]);
  }
}

}  // namespace
}  // namespace fib
