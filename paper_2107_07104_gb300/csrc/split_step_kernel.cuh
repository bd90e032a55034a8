// Fused split-step kernel for many independent 1D fibers (sm_103a), as a
// template shared by the translation units that instantiate it
// (split_step.cu: exact exponentials; split_step_expapx.cu: exp*).
//
// One launch advances every fiber by n_steps split steps (eq:monodomain_strang):
//   diffusion half (Crank-Nicolson, eq:lumping_crank_nicolson_2) ->
//   reaction over dt_split in Heun substeps (eq:heun) of the Hodgkin-Huxley
//   model (sec:subcelullar_model) with motor-unit stimulus
//   (sec:stimulation_times_callbacks) -> diffusion half.
// The same kernel runs the other orderings (Godunov, eq:monodomain_godunov;
// the 0D-1D-0D order of the splitting figures) as reaction substeps
// [0, k_split), diffusion, substeps [k_split, n_sub), diffusion, with either
// phase possibly empty, and implicit-Euler diffusion
// (eq:lumping_implicit_euler_2) in place of Crank-Nicolson.
// Fibers never interact (eq:discretized_fibers), so each fiber is owned by a
// group of whole warps of one CTA for the entire launch:
//   * thread p of a fiber holds nodes [pK, pK + K) of V, m, h, n in registers
//     across all steps and substeps of the launch; HBM is touched once per
//     launch to load and once to store the state;
//   * the reaction step is node-local, K independent nodes per thread;
//   * the tridiagonal CN solve is partitioned: Thomas elimination inside each
//     thread's chunk, then cyclic reduction over the chunks with the
//     boundary values exchanged through shared memory under a named barrier
//     of the fiber's warps only (coefficients: solver_tables.cpp).
// The state is kept as u = V - Vrest (the Hodgkin-Huxley depolarisation), so
// the common resting value is 0 and FP32 keeps full relative precision there.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "fibers_internal.h"
#include "hh_device.cuh"

namespace fib {
namespace {

// Hodgkin-Huxley right-hand side: hh_device.cuh

// ---------------------------------------------------------------------------
// The same substep on node pairs with Blackwell's packed FP32x2 arithmetic
// (fma/add/mul.rn.f32x2: two IEEE round-to-nearest FP32 operations per
// instruction, bit-identical to the scalar ones).  The special functions
// (ex2, rcp) and the singularity selects stay per node.
// ---------------------------------------------------------------------------

struct F2 {
  unsigned long long v;
};

__device__ __forceinline__ F2 mk2(float a, float b) {
  F2 r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r.v) : "f"(a), "f"(b));
  return r;
}
__device__ __forceinline__ void un2(F2 x, float& a, float& b) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(x.v));
}
__device__ __forceinline__ F2 sp2(float a) { return mk2(a, a); }
__device__ __forceinline__ F2 fma2(F2 a, F2 b, F2 c) {
  F2 d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d.v) : "l"(a.v), "l"(b.v), "l"(c.v));
  return d;
}
__device__ __forceinline__ F2 mul2(F2 a, F2 b) {
  F2 d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d.v) : "l"(a.v), "l"(b.v));
  return d;
}
__device__ __forceinline__ F2 add2(F2 a, F2 b) {
  F2 d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d.v) : "l"(a.v), "l"(b.v));
  return d;
}
__device__ __forceinline__ F2 ex2_2(F2 x) {
  float a, b;
  un2(x, a, b);
  return mk2(ex2_approx(a), ex2_approx(b));
}
__device__ __forceinline__ F2 rcp_2(F2 x) {
  float a, b;
  un2(x, a, b);
  return mk2(rcp_approx(a), rcp_approx(b));
}

__device__ __forceinline__ F2 sub2(F2 a, F2 b) {
  F2 d;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d.v) : "l"(a.v), "l"(b.v));
  return d;
}

struct Deriv2 {
  F2 u, m, h, n;
};

// exp* on a pair: the scalar exp_star's operations, packed.
__device__ __forceinline__ F2 exp_star2(F2 x) {
  F2 y = fma2(x, sp2(1.0f / 1024.0f), sp2(1.0f));
#pragma unroll
  for (int i = 0; i < 10; ++i) y = mul2(y, y);
  return y;
}

// hh_rhs on a node pair: the same operations in the same order as the
// scalar hh_rhs, so both forms give identical bits.
template <bool EXPAPX>
__device__ __forceinline__ Deriv2 hh_rhs2(F2 u, F2 m, F2 h, F2 n, F2 gl_ul, const HHConst& c) {
  const F2 nzm = fma2(u, sp2(0.1f), sp2(-2.5f));
  const F2 nzn = fma2(u, sp2(0.01f), sp2(-0.1f));
  F2 bm, ah, bn, dm, dn, dh;
  if (EXPAPX) {
    dm = add2(exp_star2(fma2(u, sp2(-0.1f), sp2(2.5f))), sp2(-1.0f));
    dn = add2(exp_star2(fma2(u, sp2(-0.1f), sp2(1.0f))), sp2(-1.0f));
    dh = fma2(exp_star2(fma2(u, sp2(-0.1f), sp2(3.0f))), sp2(-1.0f), sp2(-1.0f));
    bm = mul2(sp2(4.0f), exp_star2(mul2(u, sp2(-1.0f / 18.0f))));
    ah = mul2(sp2(0.07f), exp_star2(mul2(u, sp2(-1.0f / 20.0f))));
    bn = mul2(sp2(0.125f), exp_star2(mul2(u, sp2(-1.0f / 80.0f))));
  } else {
    const F2 E = ex2_2(mul2(u, sp2(-kLog2e / 10.0f)));
    bm = ex2_2(fma2(u, sp2(-kLog2e / 18.0f), sp2(2.0f)));
    ah = ex2_2(fma2(u, sp2(-kLog2e / 20.0f), sp2(-3.8365012677171206f)));
    bn = ex2_2(fma2(u, sp2(-kLog2e / 80.0f), sp2(-3.0f)));
    dm = fma2(sp2(kE25), E, sp2(-1.0f));
    dn = fma2(sp2(kE10), E, sp2(-1.0f));
    dh = fma2(sp2(-kE30), E, sp2(-1.0f));
  }
  F2 nam = mul2(nzm, rcp_2(dm));
  F2 nan_ = mul2(nzn, rcp_2(dn));
  const F2 nbh = rcp_2(dh);
  {
    // removable singularities: per-node selects, as in the scalar form (a
    // warp vote and branch here split the unrolled pair loop into blocks
    // the scheduler cannot interleave, which costs more than the selects)
    float zm0, zm1, zn0, zn1, a0, a1, b0, b1;
    un2(nzm, zm0, zm1);
    un2(nzn, zn0, zn1);
    un2(nam, a0, a1);
    un2(nan_, b0, b1);
    if (fabsf(zm0) < 0.01f) a0 = nam_series(zm0);
    if (fabsf(zm1) < 0.01f) a1 = nam_series(zm1);
    if (fabsf(zn0) < 0.001f) b0 = nan_series(zn0);
    if (fabsf(zn1) < 0.001f) b1 = nan_series(zn1);
    nam = mk2(a0, a1);
    nan_ = mk2(b0, b1);
  }
  Deriv2 d;
  d.m = fma2(sub2(bm, nam), m, nam);
  d.h = fma2(sub2(nbh, ah), h, ah);
  d.n = fma2(sub2(bn, nan_), n, nan_);
  const F2 A = mul2(mul2(m, m), mul2(m, h));
  F2 B = mul2(n, n);
  B = mul2(B, B);
  const F2 t = fma2(A, sp2(c.gNa_uNa), fma2(B, sp2(c.gK_uK), gl_ul));
  const F2 nS = fma2(A, sp2(-c.gNa), fma2(B, sp2(-c.gK), sp2(-c.gL)));
  d.u = fma2(u, nS, t);
  return d;
}

// y + s * f on a pair, with the step s a constant
__device__ __forceinline__ F2 step2(float s, F2 f, F2 y) {
  return fma2(sp2(s), f, y);
}

// One Heun substep (eq:heun) of every node a thread holds, on node pairs;
// y + dt/2 (f0 + f1) is formed as (y + dt/2 f0) + dt/2 f1 like the scalar
// form, so the two give identical bits.  Gates are held as deviations from
// rest (see heun_nodes).
template <int K, bool STIM, bool EXPAPX>
__device__ __forceinline__ void heun_nodes_packed(float (&u)[K], float (&m)[K], float (&h)[K], float (&n)[K],
                                                  const HHConst& c, uint32_t mask) {
  const float dt = c.dt0, hdt = 0.5f * c.dt0;
#pragma unroll
  for (int j = 0; j < K; j += 2) {
    const float s0 = (STIM && ((mask >> j) & 1u)) ? c.gL_uL + c.stim : c.gL_uL;
    const float s1 = (STIM && ((mask >> (j + 1)) & 1u)) ? c.gL_uL + c.stim : c.gL_uL;
    const F2 st = mk2(s0, s1);
    const F2 y_u = mk2(u[j], u[j + 1]), y_m = mk2(m[j], m[j + 1]);
    const F2 y_h = mk2(h[j], h[j + 1]), y_n = mk2(n[j], n[j + 1]);
    // absolute gates for the right-hand sides and the predictor
    const F2 a_m = add2(y_m, sp2(c.m0)), a_h = add2(y_h, sp2(c.h0)), a_n = add2(y_n, sp2(c.n0));
    const Deriv2 f0 = hh_rhs2<EXPAPX>(y_u, a_m, a_h, a_n, st, c);
    const F2 v_u = step2(dt, f0.u, y_u), v_m = step2(-dt, f0.m, a_m);
    const F2 v_h = step2(dt, f0.h, a_h), v_n = step2(-dt, f0.n, a_n);
    const F2 p_u = step2(hdt, f0.u, y_u), p_m = step2(-hdt, f0.m, y_m);
    const F2 p_h = step2(hdt, f0.h, y_h), p_n = step2(-hdt, f0.n, y_n);
    const Deriv2 f1 = hh_rhs2<EXPAPX>(v_u, v_m, v_h, v_n, st, c);
    un2(step2(hdt, f1.u, p_u), u[j], u[j + 1]);
    un2(step2(-hdt, f1.m, p_m), m[j], m[j + 1]);
    un2(step2(hdt, f1.h, p_h), h[j], h[j + 1]);
    un2(step2(-hdt, f1.n, p_n), n[j], n[j + 1]);
  }
}

// ---------------------------------------------------------------------------
// Crank-Nicolson half step: partitioned tridiagonal solve
// ---------------------------------------------------------------------------

__device__ __forceinline__ void fiber_barrier(int id, int count) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}

template <typename R>
struct Exchange {  // per-CTA shared buffers, one element per thread
  R* first;
  R* last;
  R* D;
  R* E;
  R* y;
  R* r2;  // 2 x blockDim, double-buffered PCR values
};

// Per-thread reduced-system coefficients, kept in shared memory (one column
// per thread, row k at cf[k * kStride]) rather than in registers.  The
// exchange buffers and this table use the fixed stride kStride (the largest
// CTA) rather than blockDim.x, so every shared-memory address in the solve is
// the thread's own offset plus an immediate.
enum { kInvB = 0, kAb, kCb, kC0, kKE, kKD, kKDn, kPKE, kPKD, kPKDn, kNumCoef };
constexpr int kStride = 32 * kMaxWarpsPerCta;

// Row coefficients of a chunk in shared memory, coefficient-major: the K
// values of coefficient c (kF1 .. kBt, the host tables' per-row order) at
// set[c * K .. c * K + K), so four rows come in one 16-byte load (K is a
// multiple of 4 and every set starts on a 16-byte boundary).
enum { kF1 = 0, kF2, kG, kAp, kBt };

__device__ __forceinline__ void load4(const float* p, float (&v)[4]) {
  const float4 q = *reinterpret_cast<const float4*>(p);
  v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
}
__device__ __forceinline__ void load4(const double* p, double (&v)[4]) {
  const double2 q0 = *reinterpret_cast<const double2*>(p), q1 = *reinterpret_cast<const double2*>(p + 2);
  v[0] = q0.x; v[1] = q0.y; v[2] = q1.x; v[3] = q1.y;
}

// Stages one row set from the host tables' row-major order (row j,
// coefficient c at j * kCoefPerRow + c) into the coefficient-major order
// above; threads t0, t0 + stride, ... share the work.
template <int K, typename R>
__device__ __forceinline__ void stage_set(R* dst, const R* src, int t0, int stride) {
  for (int i = t0; i < K * kCoefPerRow; i += stride) {
    const int j = i / kCoefPerRow, c = i - j * kCoefPerRow;
    dst[c * K + j] = src[i];
  }
}

template <int K, typename R>
struct SolveCtx {
  const R* set;  // row coefficients of this thread's chunk (shared memory, coefficient-major)
  const R* rec;  // this thread's reduced-system record (global memory)
  const R* cf;   // this thread's column of the coefficient table (shared memory)
  R r;           // c dt_1d / h^2 (0 for single-node fibers)
  int p, Tw, tid, nreal, bar_id, levels;
  bool edge;     // chunk holds the fiber's last row or padding
  bool ie;       // implicit Euler: right-hand side is u itself
};

// CS: stride of the coefficient table and of the PCR buffers (kStride, or
// the solving threads' count in a kernel that gives the solve fewer threads).
template <int K, typename R, int CS = kStride>
__device__ __forceinline__ void cn_solve(float (&u)[K], const SolveCtx<K, R>& s, const Exchange<R>& x) {
  R d[K];
  if (s.ie) {
    // implicit Euler (eq:lumping_implicit_euler_2): (I - dt L) u+ = u; the
    // tables hold the left-hand side for 2 c dt / h^2, which is the same
    // matrix (uniform per fiber, so the barrier below is skipped by all of
    // a fiber's threads together)
#pragma unroll
    for (int j = 0; j < K; ++j) d[j] = (!s.edge || j < s.nreal) ? (R)u[j] : (R)0;
  } else {
  // neighbour values for the right-hand side (I + dt/2 L) u
  x.first[s.tid] = (R)u[0];
  x.last[s.tid] = (R)u[K - 1];
  fiber_barrier(s.bar_id, s.Tw);
  const R left = (s.p > 0) ? x.last[s.tid - 1] : (R)u[1];  // row 0: ghost u(-1) = u(1)
  const R right = (s.p + 1 < s.Tw) ? x.first[s.tid + 1] : (R)0;
  const R a0 = (R)1 - s.r, hr = (R)0.5 * s.r;
  if (!s.edge) {
#pragma unroll
    for (int j = 0; j < K; ++j) {
      const R um = (j == 0) ? left : (R)u[j - 1];
      const R up = (j == K - 1) ? right : (R)u[j + 1];
      d[j] = a0 * (R)u[j] + hr * (um + up);
    }
  } else {
#pragma unroll
    for (int j = 0; j < K; ++j) {
      const R um = (j == 0) ? left : (R)u[j - 1];
      R up = (j == K - 1) ? right : (R)u[j + 1];
      if (j == s.nreal - 1) up = um;  // last row: ghost u(N) = u(N-2)
      d[j] = (j < s.nreal) ? a0 * (R)u[j] + hr * (um + up) : (R)0;
    }
  }
  }
  // forward elimination inside the chunk (row coefficients four rows at a
  // time, one vector load per coefficient)
  {
    R f1[4], f2[4];
#pragma unroll
    for (int j = 1; j < K; ++j) {
      if (j == 1 || (j & 3) == 0) {
        load4(s.set + kF1 * K + (j & ~3), f1);
        load4(s.set + kF2 * K + (j & ~3), f2);
      }
      d[j] = (j == 1) ? d[1] * f1[1] : d[j] * f1[j & 3] - f2[j & 3] * d[j - 1];
    }
  }
  // back substitution towards the chunk's first row
  {
    R g[4];
#pragma unroll
    for (int j = K - 3; j >= 1; --j) {
      if (j == K - 3 || (j & 3) == 3) load4(s.set + kG * K + (j & ~3), g);
      d[j] = d[j] - g[j & 3] * d[j + 1];
    }
  }
  const R D = d[0] - s.cf[kC0 * CS] * d[1];
  const R E = d[K - 1];
  R y, ym;
  if (s.levels == 0) {
    // The reduced system is already decoupled: y_p needs D of the next
    // chunk, and this thread forms y_(p-1) itself from the previous chunk's
    // D and E with the same expression that thread evaluates, so one
    // exchange serves both.  Implicit Euler has no exchange barrier before
    // this point, so it waits here until every thread of the fiber has read
    // the previous solve's D and E.
    if (s.ie) fiber_barrier(s.bar_id, s.Tw);
    x.D[s.tid] = D;
    x.E[s.tid] = E;
    fiber_barrier(s.bar_id, s.Tw);
    const R Dn = (s.p + 1 < s.Tw) ? x.D[s.tid + 1] : (R)0;
    y = E * s.cf[kKE * CS] - s.cf[kKD * CS] * D - s.cf[kKDn * CS] * Dn;
    ym = (R)0;
    if (s.p > 0) {
      const R Dp = x.D[s.tid - 1], Ep = x.E[s.tid - 1];
      ym = Ep * s.cf[kPKE * CS] - s.cf[kPKD * CS] * Dp - s.cf[kPKDn * CS] * D;
    }
  } else {
    x.D[s.tid] = D;
    fiber_barrier(s.bar_id, s.Tw);
    const R Dn = (s.p + 1 < s.Tw) ? x.D[s.tid + 1] : (R)0;
    R rr = E * s.cf[kKE * CS] - s.cf[kKD * CS] * D - s.cf[kKDn * CS] * Dn;
    // parallel cyclic reduction over the chunks' last unknowns
    for (int l = 0, st = 1; l < s.levels; ++l, st <<= 1) {
      R* buf = x.r2 + (l & 1) * CS;
      buf[s.tid] = rr;
      fiber_barrier(s.bar_id, s.Tw);
      const R rm = (s.p - st >= 0) ? buf[s.tid - st] : (R)0;
      const R rp = (s.p + st < s.Tw) ? buf[s.tid + st] : (R)0;
      const R* lv = s.rec + kRecBase + kRecPerLevel * l;
      rr = rr * lv[0] - lv[1] * rm - lv[2] * rp;
    }
    y = rr;
    x.y[s.tid] = y;
    fiber_barrier(s.bar_id, s.Tw);
    ym = (s.p > 0) ? x.y[s.tid - 1] : (R)0;
  }
  const R xs = D * s.cf[kInvB * CS] - s.cf[kAb * CS] * ym - s.cf[kCb * CS] * y;
  u[0] = (float)xs;
  u[K - 1] = (float)y;
  {
    R ap[4], bt[4];
#pragma unroll
    for (int j = 1; j < K - 1; ++j) {
      if (j == 1 || (j & 3) == 0) {
        load4(s.set + kAp * K + (j & ~3), ap);
        load4(s.set + kBt * K + (j & ~3), bt);
      }
      u[j] = (float)(d[j] - ap[j & 3] * xs - bt[j & 3] * y);
    }
  }
}

// ---------------------------------------------------------------------------
// Surrogate mode: the list of nodes for the network pass
// ---------------------------------------------------------------------------

// Does a node take the plain HH step?  Outside the network's training
// envelope, or inside the quiet box around rest (where the exact step keeps
// rest an exact fixed point).
__device__ __forceinline__ bool sur_plain(const StepArgs& a, const float (&raw)[5]) {
  bool outside = false, quiet = true;
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    outside = outside || !(raw[k] >= a.sur_env_lo[k] && raw[k] <= a.sur_env_hi[k]);
    quiet = quiet && raw[k] >= a.sur_quiet_lo[k] && raw[k] <= a.sur_quiet_hi[k];
  }
  return outside || quiet;
}

// Lists this thread's network nodes (state before the reaction, stimulus
// fraction of the split step) with one atomic per warp.
template <int K>
__device__ __forceinline__ void list_network_nodes(const StepArgs& a, const float (&u)[K], const float (&m)[K],
                                                   const float (&h)[K], const float (&n)[K], uint32_t mask,
                                                   int64_t cur, int64_t fend, int64_t stp, int nreal,
                                                   int64_t base) {
  float sfrac = 0.0f;
  if (mask) {  // substeps of this split step with the pulse on (a private copy of the cursor)
    int on = 0;
    for (int k = 0; k < a.n_sub; ++k) {
      const int64_t kk = stp * a.n_sub + k;
      while (cur < fend && a.fire_k[cur] + a.pulse <= kk) ++cur;
      on += (cur < fend) && (a.fire_k[cur] <= kk);
    }
    sfrac = (float)on * a.inv_n_sub;
  }
  uint32_t netm = 0;
#pragma unroll
  for (int j = 0; j < K; ++j) {
    const float raw[5] = {u[j], m[j] + a.hh.m0, h[j] + a.hh.h0, n[j] + a.hh.n0, ((mask >> j) & 1u) ? sfrac : 0.0f};
    if (j < nreal && !sur_plain(a, raw)) netm |= 1u << j;
  }
  const int cnt = __popc(netm);
  if (!__any_sync(0xffffffffu, cnt > 0)) return;
  const int lane = threadIdx.x & 31;
  int incl = cnt;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, incl, d);
    if (lane >= d) incl += y;
  }
  unsigned int first = 0;
  if (lane == 31) first = atomicAdd(a.sur_count + (stp & 1), (unsigned int)incl);
  first = __shfl_sync(0xffffffffu, first, 31);
  const unsigned int warp_total = (unsigned int)__shfl_sync(0xffffffffu, incl, 31);
  // A node is listed at most once per step, so the list cannot outgrow
  // sur_cap unless its counter was left stale; then nothing is stored and
  // the host reports the overflow.
  if ((unsigned long long)first + warp_total > (unsigned long long)a.sur_cap) {
    if (lane == 31) atomicOr(a.flag, 2);
    return;
  }
  unsigned int pos = first + (unsigned int)(incl - cnt);
  float* L = a.sur_list + (stp & 1) * 6 * a.sur_cap;
#pragma unroll
  for (int j = 0; j < K; ++j)
    if ((netm >> j) & 1u) {
      L[pos] = __int_as_float((int)(base + j));
      L[a.sur_cap + pos] = u[j];
      L[2 * a.sur_cap + pos] = m[j] + a.hh.m0;  // absolute gates: the network's inputs
      L[3 * a.sur_cap + pos] = h[j] + a.hh.h0;
      L[4 * a.sur_cap + pos] = n[j] + a.hh.n0;
      L[5 * a.sur_cap + pos] = ((mask >> j) & 1u) ? sfrac : 0.0f;
      ++pos;
    }
}

// ---------------------------------------------------------------------------
// The split-step kernel
// ---------------------------------------------------------------------------

// MINB: CTAs of up to 256 threads that must fit on one SM at once; it sets
// the register budget (2: up to 128 registers per thread, 3: up to 85).
// ADAPT: adaptive computation (sec:adaptive_computation_for_fiber_based):
// a fiber in equilibrium with no pulse due skips a whole launch.  Only the
// adaptive instantiations carry its code.
// SUR: surrogate mode's split step (one per launch).  Before the reaction,
// nodes that the network handles are listed with their state; the plain
// reaction then runs on every node, and the network pass overwrites the
// listed ones.
template <int K, typename R, bool PACKED, int MINB, bool EXPAPX, bool ADAPT, bool SUR>
__global__ void __launch_bounds__(32 * kMaxWarpsPerCta, MINB)
    split_step_kernel(const StepArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int B = blockDim.x;
  const int tid = threadIdx.x;
  const int warp = tid >> 5;
  const int set_len = K * kCoefPerRow;
  R* s_rows = reinterpret_cast<R*>(smem_raw);  // interior set + one last set per CTA fiber
  Exchange<R> x;
  x.first = s_rows + (1 + kMaxFibersPerCta) * set_len;
  x.last = x.first + kStride;
  x.D = x.last + kStride;
  x.E = x.D + kStride;
  x.y = x.E + kStride;
  x.r2 = x.y + kStride;
  R* s_coef = x.r2 + 2 * kStride;  // kNumCoef x kStride
  float* s_keep = reinterpret_cast<float*>(s_coef + kNumCoef * kStride);  // ADAPT: 4 K x B state copy
  int* s_eq = reinterpret_cast<int*>(s_keep + (ADAPT ? 4 * K * B : 0));  // ADAPT: one per warp

  const WarpMap wm = a.warps[(int64_t)blockIdx.x * a.W + warp];
  const R* g_rows = static_cast<const R*>(a.rows);
  stage_set<K>(s_rows, g_rows, tid, B);
  FiberDesc fd;
  if (wm.fiber >= 0) {
    fd = a.fibers[wm.fiber];
    if (warp == wm.first_warp) stage_set<K>(s_rows + (1 + wm.slot) * set_len, g_rows + fd.last_set, tid & 31, 32);
  }
  __syncthreads();  // every thread of the CTA, before idle warps leave
  if (wm.fiber < 0) return;

  const int Tw = 32 * wm.n_warps;
  const int p = tid - 32 * wm.first_warp;
  const int Tf = (fd.n + K - 1) / K;
  const int nreal = min(max(fd.n - p * K, 0), K);

  SolveCtx<K, R> sc;
  sc.p = p;
  sc.Tw = Tw;
  sc.tid = tid;
  sc.nreal = nreal;
  sc.bar_id = wm.slot + 1;
  sc.levels = a.n_levels;
  sc.edge = (nreal < K) || (p == Tf - 1);
  sc.set = s_rows + ((p == Tf - 1) ? (1 + wm.slot) * set_len : 0);
  sc.r = fd.n > 1 ? (R)a.r : (R)0;
  sc.ie = a.implicit_euler != 0;
  const R* g_recs = static_cast<const R*>(a.recs);
  sc.rec = g_recs + fd.rec + (int64_t)p * a.rec_stride;
  for (int k = 0; k < 7; ++k) s_coef[k * kStride + tid] = sc.rec[k];
  s_coef[kPKE * kStride + tid] = p > 0 ? sc.rec[4 - a.rec_stride] : (R)0;
  s_coef[kPKD * kStride + tid] = p > 0 ? sc.rec[5 - a.rec_stride] : (R)0;
  s_coef[kPKDn * kStride + tid] = p > 0 ? sc.rec[6 - a.rec_stride] : (R)0;
  sc.cf = s_coef + tid;  // own column: read back only by this thread

  // load this thread's K nodes (vectorised: slot and K are multiples of 4);
  // a launch without the reaction phase (diffusion only) touches u alone
  const bool gates = ADAPT || (a.phases & 2) != 0;
  float u[K], m[K], h[K], n[K];
  const int64_t base = fd.slot + (int64_t)p * K;
#pragma unroll
  for (int j = 0; j < K; j += 4) {
    const float4 vu = *reinterpret_cast<const float4*>(a.u + base + j);
    u[j] = vu.x; u[j + 1] = vu.y; u[j + 2] = vu.z; u[j + 3] = vu.w;
    float4 vm = make_float4(0.f, 0.f, 0.f, 0.f), vh = vm, vn = vm;
    if (gates) {
      vm = *reinterpret_cast<const float4*>(a.m + base + j);
      vh = *reinterpret_cast<const float4*>(a.h + base + j);
      vn = *reinterpret_cast<const float4*>(a.n + base + j);
    }
    m[j] = vm.x; m[j + 1] = vm.y; m[j + 2] = vm.z; m[j + 3] = vm.w;
    h[j] = vh.x; h[j + 1] = vh.y; h[j + 2] = vh.z; h[j + 3] = vh.w;
    n[j] = vn.x; n[j + 1] = vn.y; n[j + 2] = vn.z; n[j + 3] = vn.w;
  }

  const int64_t step0 = *a.step_base + a.step_offset;
  if (ADAPT) {
    // Adaptive computation (sec:adaptive_computation_for_fiber_based): a
    // fiber that was in equilibrium at the end of its last launch and whose
    // motor unit has no pulse overlapping this launch is skipped whole.  The
    // decision depends only on per-fiber data, so all its warps agree.
    bool pulse_due = false;
    if (fd.mu >= 0 && fd.mu < a.n_mu) {
      const int64_t k0 = step0 * a.n_sub, k1 = k0 + (int64_t)a.n_steps * a.n_sub;
      int64_t lo_f = a.mu_off[fd.mu], hi_f = a.mu_off[fd.mu + 1];
      const int64_t end = hi_f;
      while (lo_f < hi_f) {
        const int64_t mid = (lo_f + hi_f) >> 1;
        if (a.fire_k[mid] + a.pulse <= k0) lo_f = mid + 1;
        else hi_f = mid;
      }
      pulse_due = lo_f < end && a.fire_k[lo_f] < k1;
    }
    if (a.quiet[wm.fiber] && !pulse_due) {
      if (p == 0) atomicAdd(a.skipped, (unsigned long long)a.n_steps);
      return;  // every thread of this fiber leaves here, before any fiber barrier
    }
  }

  // stimulated nodes of this thread and the MU firing cursor; fk caches
  // fire_k[cur] (INT64_MAX past the end), so a substep's stimulus test reads
  // global memory only when the cursor moves past an ended pulse
  uint32_t mask = 0;
  int64_t cur = 0, fend = 0, fk = INT64_MAX;
  if (fd.mu >= 0 && fd.mu < a.n_mu) {
    const int lo = max(fd.junction - a.hw, 0), hi = min(fd.junction + a.hw, fd.n - 1);
#pragma unroll
    for (int j = 0; j < K; ++j) {
      const int i = p * K + j;
      if (i >= lo && i <= hi) mask |= 1u << j;
    }
    if (mask) {
      // first firing whose pulse has not ended at the launch's first substep
      int64_t lo_f = a.mu_off[fd.mu];
      int64_t hi_f = a.mu_off[fd.mu + 1];
      fend = hi_f;
      const int64_t k0 = step0 * a.n_sub;
      while (lo_f < hi_f) {
        const int64_t mid = (lo_f + hi_f) >> 1;
        if (a.fire_k[mid] + a.pulse <= k0) lo_f = mid + 1;
        else hi_f = mid;
      }
      cur = lo_f;
      if (cur < fend) fk = a.fire_k[cur];
    }
  }

  const int first_half = a.phases & 1, reaction = a.phases & 2, second_half = a.phases & 4;
  for (int s = 0; s < a.n_steps; ++s) {
    const int64_t stp = step0 + s;
    if (ADAPT && s == a.n_steps - 1) {
#pragma unroll
      for (int j = 0; j < K; ++j) {
        s_keep[(0 * K + j) * B + tid] = u[j];
        s_keep[(1 * K + j) * B + tid] = m[j];
        s_keep[(2 * K + j) * B + tid] = h[j];
        s_keep[(3 * K + j) * B + tid] = n[j];
      }
    }
    // segment 0: substeps [0, k_split) then the first diffusion phase;
    // segment 1: substeps [k_split, n_sub)
    for (int seg = 0; seg < 2; ++seg) {
      const int kb = seg ? a.k_split : 0, ke = seg ? a.n_sub : a.k_split;
      if (SUR && seg == 1 && reaction) list_network_nodes<K>(a, u, m, h, n, mask, cur, fend, stp, nreal, base);
      for (int k = kb; reaction && k < ke; ++k) {
        bool on = false;
        if (mask) {
          const int64_t kk = stp * a.n_sub + k;
          while (fk != INT64_MAX && fk + a.pulse <= kk) {
            ++cur;
            fk = cur < fend ? a.fire_k[cur] : INT64_MAX;
          }
          on = fk <= kk;
        }
        if (PACKED) {
          if (on) heun_nodes_packed<K, true, EXPAPX>(u, m, h, n, a.hh, mask);
          else heun_nodes_packed<K, false, EXPAPX>(u, m, h, n, a.hh, mask);
        } else {
          if (on) heun_nodes<K, true, EXPAPX>(u, m, h, n, a.hh, mask);
          else heun_nodes<K, false, EXPAPX>(u, m, h, n, a.hh, mask);
        }
      }
      if (seg == 0 && first_half)
        for (int c = 0; c < a.n_cn; ++c) cn_solve<K, R>(u, sc, x);
    }
    if (second_half)
      for (int c = 0; c < a.n_cn2; ++c) cn_solve<K, R>(u, sc, x);
  }

  if (ADAPT) {
    // equilibrium test over the launch's last split step: every component of
    // every real node changed by at most eq_tol relative (V taken absolute)
    bool eq = true;
#pragma unroll
    for (int j = 0; j < K; ++j) {
      if (j < nreal) {
        const float Vo = s_keep[(0 * K + j) * B + tid] + a.vrest, Vn = u[j] + a.vrest;
        // gates are held as deviations from rest: differences are the same,
        // the relative scale is the absolute gate
        const float mo = s_keep[(1 * K + j) * B + tid], ho = s_keep[(2 * K + j) * B + tid];
        const float no = s_keep[(3 * K + j) * B + tid];
        eq = eq && fabsf(Vn - Vo) <= a.eq_tol * fabsf(Vo) && fabsf(m[j] - mo) <= a.eq_tol * fabsf(mo + a.hh.m0) &&
             fabsf(h[j] - ho) <= a.eq_tol * fabsf(ho + a.hh.h0) && fabsf(n[j] - no) <= a.eq_tol * fabsf(no + a.hh.n0);
      }
    }
    const bool warp_eq = __all_sync(0xffffffffu, eq);
    if ((tid & 31) == 0) s_eq[(tid >> 5)] = warp_eq ? 1 : 0;
    fiber_barrier(sc.bar_id, Tw);
    if (p == 0) {
      int all = 1;
      for (int w = 0; w < wm.n_warps; ++w) all &= s_eq[wm.first_warp + w];
      a.quiet[wm.fiber] = (uint8_t)all;
    }
  }

  bool finite = true;
#pragma unroll
  for (int j = 0; j < K; ++j)
    finite = finite && isfinite(u[j]) && isfinite(m[j]) && isfinite(h[j]) && isfinite(n[j]);
  if (!finite) atomicOr(a.flag, 1);
#pragma unroll
  for (int j = 0; j < K; j += 4) {
    *reinterpret_cast<float4*>(a.u + base + j) = make_float4(u[j], u[j + 1], u[j + 2], u[j + 3]);
    if (gates) {
      *reinterpret_cast<float4*>(a.m + base + j) = make_float4(m[j], m[j + 1], m[j + 2], m[j + 3]);
      *reinterpret_cast<float4*>(a.h + base + j) = make_float4(h[j], h[j + 1], h[j + 2], h[j + 3]);
      *reinterpret_cast<float4*>(a.n + base + j) = make_float4(n[j], n[j + 1], n[j + 2], n[j + 3]);
    }
  }
}

template <int K, typename R, bool PACKED, int MINB, bool EXPAPX, bool ADAPT, bool SUR>
int launch_one(const StepArgs& a, int n_ctas, void* stream) {
  const size_t smem = split_step_smem_bytes(K, sizeof(R) == 8, a.W, ADAPT);
  if (smem > 48 * 1024) {  // opt in to more than the default dynamic shared memory
    const cudaError_t e = cudaFuncSetAttribute(split_step_kernel<K, R, PACKED, MINB, EXPAPX, ADAPT, SUR>,
                                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return (int)e;
  }
  split_step_kernel<K, R, PACKED, MINB, EXPAPX, ADAPT, SUR>
      <<<n_ctas, 32 * a.W, smem, static_cast<cudaStream_t>(stream)>>>(a);
  return (int)cudaGetLastError();
}

template <int K, typename R, bool EXPAPX, bool ADAPT, bool SUR>
int launch_k(const StepArgs& a, int n_ctas, void* stream) {
  if (sizeof(R) == 8) return launch_one<K, R, false, 2, EXPAPX, ADAPT, SUR>(a, n_ctas, stream);  // FP64 solve
  if (a.occ == 4)
    return a.packed ? launch_one<K, R, true, 4, EXPAPX, ADAPT, SUR>(a, n_ctas, stream)
                    : launch_one<K, R, false, 4, EXPAPX, ADAPT, SUR>(a, n_ctas, stream);
  if (a.occ == 3)
    return a.packed ? launch_one<K, R, true, 3, EXPAPX, ADAPT, SUR>(a, n_ctas, stream)
                    : launch_one<K, R, false, 3, EXPAPX, ADAPT, SUR>(a, n_ctas, stream);
  return a.packed ? launch_one<K, R, true, 2, EXPAPX, ADAPT, SUR>(a, n_ctas, stream)
                  : launch_one<K, R, false, 2, EXPAPX, ADAPT, SUR>(a, n_ctas, stream);
}

// Dispatch on K for one (R, EXPAPX, ADAPT, SUR) family of instantiations.
template <typename R, bool EXPAPX, bool ADAPT, bool SUR = false>
int launch_family(int K, const StepArgs& a, int n_ctas, void* stream) {
  switch (K) {
    case 4: return launch_k<4, R, EXPAPX, ADAPT, SUR>(a, n_ctas, stream);
    case 8: return launch_k<8, R, EXPAPX, ADAPT, SUR>(a, n_ctas, stream);
    case 12: return launch_k<12, R, EXPAPX, ADAPT, SUR>(a, n_ctas, stream);
    case 16: return launch_k<16, R, EXPAPX, ADAPT, SUR>(a, n_ctas, stream);
    default: return (int)cudaErrorInvalidValue;
  }
}

}  // namespace
}  // namespace fib
