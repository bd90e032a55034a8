// Split step with dedicated reaction and diffusion warps (plain FP32,
// Strang 1D-0D-1D with Crank-Nicolson: eq:monodomain_strang,
// eq:lumping_crank_nicolson_2, eq:heun), for fibers of at most kWsSlot
// nodes.
//
// The fused kernel (split_step_kernel.cuh) gives every warp of a fiber both
// the reaction and the diffusion solve.  The solve couples the fiber's
// warps, so each of its exchanges waits at a fiber barrier for the slowest
// warp, and the warps of a fiber drift apart over the long reaction phase.
// Here the two jobs go to different warps of one CTA, which owns two fibers
// whose state lives in shared memory for a whole launch:
//   * kWsReactWarps reaction warps (kWsKR nodes per lane) run the Heun
//     substeps of one fiber while
//   * the diffusion warps (kWsKC nodes per lane) run the two Crank-Nicolson
//     halves between that fiber's reactions on the other fiber,
// so the fibers alternate: reaction(A) | solve(B), reaction(B) | solve(A).
// The roles hand fibers over through shared-memory mbarriers: a reaction
// warp waits only until the diffusion warps have released the fiber it is
// about to integrate (one slot earlier), never for the other reaction
// warps.  Every wait is bounded; a wait that gives up sets bit 2 of the
// error flag, and the kernel finishes with its state unreliable instead of
// hanging.  Results equal the fused kernel's up to rounding order
// (the same reaction arithmetic; the solve at kWsKC nodes per thread).
#include "split_step_kernel.cuh"
#include "split_step_ws.h"

namespace fib {
namespace {

constexpr int kWsThreads = 32 * kWsWarps;
constexpr int kWsSpin = 1 << 20;  // try_wait rounds before a wait gives up
// The diffusion warps' coefficient table and exchange buffers hold one
// column per diffusion thread.
constexpr int kWsCS = kWsCnThreads;

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(smem_addr(bar))
               : "memory");
}
// Waits for the phase of the given parity to complete; gives up after a
// bounded number of rounds (then sets bit 2 of *flag and every later wait
// of this thread returns at once).
__device__ __forceinline__ void mbar_wait(uint64_t* bar, uint32_t parity, int32_t* flag, bool& abort) {
  if (abort) return;
  const uint32_t addr = smem_addr(bar);
  for (int i = 0; i < kWsSpin; ++i) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(addr), "r"(parity)
        : "memory");
    if (done) return;
  }
  atomicOr(flag, 4);
  abort = true;
}

// Stimulus state of one reaction lane for one fiber (see the fused kernel).
struct Stim {
  uint32_t mask;
  int64_t cur, fend, fk;
};

template <int KR>
__device__ __forceinline__ Stim stim_init(const StepArgs& a, const FiberDesc& fd, int first_node, int64_t step0) {
  Stim s{0u, 0, 0, INT64_MAX};
  if (fd.mu < 0 || fd.mu >= a.n_mu) return s;
  const int lo = max(fd.junction - a.hw, 0), hi = min(fd.junction + a.hw, fd.n - 1);
#pragma unroll
  for (int j = 0; j < KR; ++j) {
    const int i = first_node + j;
    if (i >= lo && i <= hi) s.mask |= 1u << j;
  }
  if (!s.mask) return s;
  int64_t lo_f = a.mu_off[fd.mu], hi_f = a.mu_off[fd.mu + 1];
  s.fend = hi_f;
  const int64_t k0 = step0 * a.n_sub;
  while (lo_f < hi_f) {
    const int64_t mid = (lo_f + hi_f) >> 1;
    if (a.fire_k[mid] + a.pulse <= k0) lo_f = mid + 1;
    else hi_f = mid;
  }
  s.cur = lo_f;
  if (s.cur < s.fend) s.fk = a.fire_k[s.cur];
  return s;
}

// One split step's reaction (n_sub Heun substeps, eq:heun, with the motor
// unit's stimulus) on the KR nodes of one lane, read from and written back
// to a fiber's state in shared memory (u, m, h, n rows kWsSlot apart).
template <int KR>
__device__ __forceinline__ void react_lane(const StepArgs& a, float* base, Stim& z, int64_t stp) {
  float u[KR], m[KR], h[KR], n[KR];
#pragma unroll
  for (int j = 0; j < KR; j += 4) {
    const float4 vu = *reinterpret_cast<const float4*>(base + j);
    const float4 vm = *reinterpret_cast<const float4*>(base + kWsSlot + j);
    const float4 vh = *reinterpret_cast<const float4*>(base + 2 * kWsSlot + j);
    const float4 vn = *reinterpret_cast<const float4*>(base + 3 * kWsSlot + j);
    u[j] = vu.x; u[j + 1] = vu.y; u[j + 2] = vu.z; u[j + 3] = vu.w;
    m[j] = vm.x; m[j + 1] = vm.y; m[j + 2] = vm.z; m[j + 3] = vm.w;
    h[j] = vh.x; h[j + 1] = vh.y; h[j + 2] = vh.z; h[j + 3] = vh.w;
    n[j] = vn.x; n[j + 1] = vn.y; n[j + 2] = vn.z; n[j + 3] = vn.w;
  }
  for (int k = 0; k < a.n_sub; ++k) {
    bool on = false;
    if (z.mask) {
      const int64_t kk = stp * a.n_sub + k;
      while (z.fk != INT64_MAX && z.fk + a.pulse <= kk) {
        ++z.cur;
        z.fk = z.cur < z.fend ? a.fire_k[z.cur] : INT64_MAX;
      }
      on = z.fk <= kk;
    }
    if (on) heun_nodes_packed<KR, true, false>(u, m, h, n, a.hh, z.mask);
    else heun_nodes_packed<KR, false, false>(u, m, h, n, a.hh, z.mask);
  }
#pragma unroll
  for (int j = 0; j < KR; j += 4) {
    *reinterpret_cast<float4*>(base + j) = make_float4(u[j], u[j + 1], u[j + 2], u[j + 3]);
    *reinterpret_cast<float4*>(base + kWsSlot + j) = make_float4(m[j], m[j + 1], m[j + 2], m[j + 3]);
    *reinterpret_cast<float4*>(base + 2 * kWsSlot + j) = make_float4(h[j], h[j + 1], h[j + 2], h[j + 3]);
    *reinterpret_cast<float4*>(base + 3 * kWsSlot + j) = make_float4(n[j], n[j + 1], n[j + 2], n[j + 3]);
  }
}

// count Crank-Nicolson solves of one fiber's u row (kWsKC nodes per
// thread, chunk p), in and out of shared memory.
__device__ __forceinline__ void solve_chunk(float* ub, const SolveCtx<kWsKC, float>& sc, const Exchange<float>& x,
                                            int count) {
  float u[kWsKC];
#pragma unroll
  for (int j = 0; j < kWsKC; j += 4) {
    const float4 v = *reinterpret_cast<const float4*>(ub + j);
    u[j] = v.x; u[j + 1] = v.y; u[j + 2] = v.z; u[j + 3] = v.w;
  }
  for (int c = 0; c < count; ++c) cn_solve<kWsKC, float, kWsCS>(u, sc, x);
#pragma unroll
  for (int j = 0; j < kWsKC; j += 4)
    *reinterpret_cast<float4*>(ub + j) = make_float4(u[j], u[j + 1], u[j + 2], u[j + 3]);
}

__global__ void __launch_bounds__(kWsThreads, kWsMinBlocks) split_step_ws_kernel(const StepArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  // layout: state of 2 fibers (u m h n x kWsSlot each), solve tables and
  // exchange buffers of the diffusion warps, 4 mbarriers
  float* st = reinterpret_cast<float*>(smem_raw);                         // [2][4][kWsSlot]
  float* s_rows = st + 2 * 4 * kWsSlot;                                   // [interior | last A | last B] sets
  constexpr int set_len = kWsKC * kCoefPerRow;
  float* s_coef = s_rows + 3 * set_len;                                   // [2][kNumCoef][kWsCS]
  Exchange<float> x;
  x.first = s_coef + 2 * kNumCoef * kWsCS;
  x.last = x.first + kWsCS;
  x.D = x.last + kWsCS;
  x.E = x.D + kWsCS;
  x.y = x.E + kWsCS;
  x.r2 = x.y + kWsCS;
  uint64_t* bars = reinterpret_cast<uint64_t*>(x.r2 + 2 * kWsCS);       // ready_R[2], ready_C[2]

  const int tid = threadIdx.x;
  const int64_t f0 = 2 * (int64_t)blockIdx.x;
  const int64_t left = (int64_t)a.n_fib - f0;
  const int nf = left < 2 ? (int)left : 2;  // fibers of this CTA (1 or 2)
  FiberDesc fd[2];
#pragma unroll
  for (int q = 0; q < 2; ++q) fd[q] = a.fibers[f0 + (q < nf ? q : 0)];

  // load the state (gates as deviations from rest), tables, barriers
  for (int q = 0; q < nf; ++q) {
    for (int v = 0; v < 4; ++v) {
      const float* src = v == 0 ? a.u : v == 1 ? a.m : v == 2 ? a.h : a.n;
      const float4* g = reinterpret_cast<const float4*>(src + fd[q].slot);
      float4* s4 = reinterpret_cast<float4*>(st + (q * 4 + v) * kWsSlot);
      for (int i = tid; i < kWsSlot / 4; i += kWsThreads) s4[i] = g[i];
    }
  }
  const float* g_rows = static_cast<const float*>(a.rows);
  stage_set<kWsKC>(s_rows, g_rows, tid, kWsThreads);
  for (int q = 0; q < 2; ++q) stage_set<kWsKC>(s_rows + (1 + q) * set_len, g_rows + fd[q].last_set, tid, kWsThreads);
  const float* g_recs = static_cast<const float*>(a.recs);
  if (tid < 2 * kWsCnThreads) {
    const int q = tid / kWsCnThreads, p = tid % kWsCnThreads;
    const float* rec = g_recs + fd[q].rec + (int64_t)p * a.rec_stride;
    float* cf = s_coef + q * kNumCoef * kWsCS;
    for (int k = 0; k < 7; ++k) cf[k * kWsCS + p] = rec[k];
    cf[kPKE * kWsCS + p] = p > 0 ? rec[4 - a.rec_stride] : 0.0f;
    cf[kPKD * kWsCS + p] = p > 0 ? rec[5 - a.rec_stride] : 0.0f;
    cf[kPKDn * kWsCS + p] = p > 0 ? rec[6 - a.rec_stride] : 0.0f;
  }
  if (tid == 0) {
    mbar_init(&bars[0], kWsCnThreads);  // ready_R[A]: the diffusion warps released fiber A
    mbar_init(&bars[1], kWsCnThreads);  // ready_R[B]
    mbar_init(&bars[2], 32 * kWsReactWarps);  // ready_C[A]: the reaction warps released fiber A
    mbar_init(&bars[3], 32 * kWsReactWarps);  // ready_C[B]
  }
  __syncthreads();

  const int64_t step0 = *a.step_base + a.step_offset;
  const int S = a.n_steps;
  bool abort = false;
  const int warp = tid >> 5;
  if (warp < kWsReactWarps) {
    // ---- reaction warps: kWsKR nodes per lane, fibers A, B alternately ----
    const int q0 = tid;  // nodes [kWsKR q0, kWsKR q0 + kWsKR)
    Stim sm[2];
#pragma unroll
    for (int q = 0; q < 2; ++q) sm[q] = stim_init<kWsKR>(a, fd[q], kWsKR * q0, step0);
    for (int s = 0; s < S; ++s) {
      const int64_t stp = step0 + s;
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        mbar_wait(&bars[q], (uint32_t)(s & 1), a.flag, abort);
        if (q < nf) {
          float* base = st + q * 4 * kWsSlot + kWsKR * q0;
          react_lane<kWsKR>(a, base, sm[q], stp);
        }
        mbar_arrive(&bars[2 + q]);
      }
    }
  } else {
    // ---- diffusion warps: the Crank-Nicolson halves between reactions ----
    const int p = tid - 32 * kWsReactWarps;  // chunk [kWsKC p, kWsKC p + kWsKC)
    SolveCtx<kWsKC, float> sc[2];
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const int Tf = (fd[q].n + kWsKC - 1) / kWsKC;
      const int nreal = min(max(fd[q].n - p * kWsKC, 0), kWsKC);
      sc[q].p = p;
      sc[q].Tw = kWsCnThreads;
      sc[q].tid = p;
      sc[q].nreal = nreal;
      sc[q].bar_id = 1;  // the diffusion warps' own named barrier
      sc[q].levels = a.n_levels;
      sc[q].edge = (nreal < kWsKC) || (p == Tf - 1);
      sc[q].set = s_rows + ((p == Tf - 1) ? (1 + q) * set_len : 0);
      sc[q].r = fd[q].n > 1 ? (float)a.r : 0.0f;
      sc[q].ie = false;
      sc[q].rec = g_recs + fd[q].rec + (int64_t)p * a.rec_stride;
      sc[q].cf = s_coef + q * kNumCoef * kWsCS + p;
    }
    for (int s = 0; s <= S; ++s) {
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        // before step s: the second half of step s - 1 (after its reaction)
        // and the first half of step s
        if (s > 0) mbar_wait(&bars[2 + q], (uint32_t)((s - 1) & 1), a.flag, abort);
        const int count = (s > 0 ? a.n_cn : 0) + (s < S ? a.n_cn : 0);
        if (q < nf) solve_chunk(st + q * 4 * kWsSlot + kWsKC * p, sc[q], x, count);  // uniform over the warps
        if (s < S) mbar_arrive(&bars[q]);
      }
    }
  }
  __syncthreads();

  // store the state and test it
  bool finite = true;
  for (int q = 0; q < nf; ++q) {
    for (int v = 0; v < 4; ++v) {
      float* dst = v == 0 ? a.u : v == 1 ? a.m : v == 2 ? a.h : a.n;
      float4* g = reinterpret_cast<float4*>(dst + fd[q].slot);
      const float4* s4 = reinterpret_cast<const float4*>(st + (q * 4 + v) * kWsSlot);
      for (int i = tid; i < kWsSlot / 4; i += kWsThreads) {
        const float4 w = s4[i];
        finite = finite && isfinite(w.x) && isfinite(w.y) && isfinite(w.z) && isfinite(w.w);
        g[i] = w;
      }
    }
  }
  if (!finite) atomicOr(a.flag, 1);
}

// ---------------------------------------------------------------------------
// Wide shape: one CTA of 1024 threads per SM holds 8 fibers, two sets of 4.
// 24 reaction warps (8 nodes per lane: four packed pairs, as in the fused
// kernel) integrate one set while 8 diffusion warps, in two groups of 4 (12
// nodes per lane, one fiber per group at a time), run the other set's two
// half-steps.  Registers move from the diffusion warpgroups (40 per thread)
// to the reaction warpgroups (72) with setmaxnreg: 6 x 128 x 72 + 2 x 128 x 40
// = 65536 = 1024 x 64, exactly the registers the CTA is launched with.
// ---------------------------------------------------------------------------
constexpr int kW8Set = 4;                    // fibers per set
constexpr int kW8Fibers = 2 * kW8Set;        // fibers per CTA
constexpr int kW8RWarps = 24;
constexpr int kW8KR = 8;
constexpr int kW8Groups = 2;                 // diffusion groups, kWsCnThreads threads each
constexpr int kW8CWarps = kW8Groups * kWsCnThreads / 32;
constexpr int kW8Threads = 32 * (kW8RWarps + kW8CWarps);
constexpr int kW8RPerFiber = kWsSlot / kW8KR;  // reaction threads per fiber
constexpr int kW8RegLaunch = 64, kW8RegR = 72, kW8RegC = 40;
static_assert(kW8Threads == 1024, "one CTA of 1024 threads");
static_assert(32 * kW8RWarps * kW8KR == kW8Set * kWsSlot, "reaction warps cover a set");
static_assert(kW8Set == 2 * kW8Groups, "each diffusion group solves two fibers of a set");
static_assert(kW8RWarps % 4 == 0 && kW8CWarps % 4 == 0, "each role is whole warpgroups");
static_assert((kW8RWarps / 4) * 128 * kW8RegR + (kW8CWarps / 4) * 128 * kW8RegC == kW8Threads * kW8RegLaunch,
              "the register split adds up to the registers of the launch");

__device__ __forceinline__ void regs_to_reaction() { asm volatile("setmaxnreg.inc.sync.aligned.u32 72;" ::: "memory"); }
__device__ __forceinline__ void regs_from_diffusion() { asm volatile("setmaxnreg.dec.sync.aligned.u32 40;" ::: "memory"); }
static_assert(kW8RegR == 72 && kW8RegC == 40, "the setmaxnreg immediates above");

// Stores the CTA's fibers from shared memory (thread t of kW8Threads) and
// reports non-finite values.
__device__ __forceinline__ void ws8_store(const StepArgs& a, const float* st, int64_t f0, int nf, int t) {
  bool finite = true;
  for (int q = 0; q < nf; ++q) {
    const int64_t slot = a.fibers[f0 + q].slot;
    for (int v = 0; v < 4; ++v) {
      float* dst = v == 0 ? a.u : v == 1 ? a.m : v == 2 ? a.h : a.n;
      float4* g = reinterpret_cast<float4*>(dst + slot);
      const float4* s4 = reinterpret_cast<const float4*>(st + (q * 4 + v) * kWsSlot);
      for (int i = t; i < kWsSlot / 4; i += kW8Threads) {
        const float4 w = s4[i];
        finite = finite && isfinite(w.x) && isfinite(w.y) && isfinite(w.z) && isfinite(w.w);
        g[i] = w;
      }
    }
  }
  if (!finite) atomicOr(a.flag, 1);
}

__global__ void __launch_bounds__(kW8Threads, 1) split_step_ws8_kernel(const StepArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  // layout: state of 8 fibers, row sets (interior + one per fiber), each
  // diffusion group's coefficient column table and exchange buffers, 4
  // mbarriers
  float* st = reinterpret_cast<float*>(smem_raw);                       // [8][4][kWsSlot]
  constexpr int set_len = kWsKC * kCoefPerRow;
  float* s_rows = st + kW8Fibers * 4 * kWsSlot;
  float* s_coef = s_rows + (1 + kW8Fibers) * set_len;                   // [group][kNumCoef][kWsCS]
  float* s_x = s_coef + kW8Groups * kNumCoef * kWsCS;                   // [group][7][kWsCS]
  uint64_t* bars = reinterpret_cast<uint64_t*>(s_x + kW8Groups * 7 * kWsCS);  // released[2], reacted[2]

  const int tid = threadIdx.x;
  const int64_t f0 = (int64_t)kW8Fibers * blockIdx.x;
  const int64_t left = (int64_t)a.n_fib - f0;
  const int nf = left < kW8Fibers ? (int)left : kW8Fibers;  // fibers of this CTA (1..8)

  for (int q = 0; q < nf; ++q) {
    const int64_t slot = a.fibers[f0 + q].slot;
    for (int v = 0; v < 4; ++v) {
      const float* src = v == 0 ? a.u : v == 1 ? a.m : v == 2 ? a.h : a.n;
      const float4* g = reinterpret_cast<const float4*>(src + slot);
      float4* s4 = reinterpret_cast<float4*>(st + (q * 4 + v) * kWsSlot);
      for (int i = tid; i < kWsSlot / 4; i += kW8Threads) s4[i] = g[i];
    }
  }
  const float* g_rows = static_cast<const float*>(a.rows);
  stage_set<kWsKC>(s_rows, g_rows, tid, kW8Threads);
  for (int q = 0; q < nf; ++q)
    stage_set<kWsKC>(s_rows + (1 + q) * set_len, g_rows + a.fibers[f0 + q].last_set, tid, kW8Threads);
  if (tid == 0) {
    mbar_init(&bars[0], kW8Groups * kWsCnThreads);  // released[set 0]: the diffusion groups are done with it
    mbar_init(&bars[1], kW8Groups * kWsCnThreads);  // released[set 1]
    mbar_init(&bars[2], 32 * kW8RWarps);            // reacted[set 0]: the reaction warps are done with it
    mbar_init(&bars[3], 32 * kW8RWarps);            // reacted[set 1]
  }
  __syncthreads();

  const int64_t step0 = *a.step_base + a.step_offset;
  const int S = a.n_steps;
  bool abort = false;
  if ((tid >> 5) < kW8RWarps) {
    // ---- reaction warps: 8 nodes per lane, sets 0 and 1 alternately ----
    regs_to_reaction();
    const int fi = tid / kW8RPerFiber;                  // fiber within a set
    const int node0 = (tid - fi * kW8RPerFiber) * kW8KR;
    Stim sm[2];
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const int fc = q * kW8Set + fi;
      sm[q] = Stim{0u, 0, 0, INT64_MAX};
      if (fc < nf) sm[q] = stim_init<kW8KR>(a, a.fibers[f0 + fc], node0, step0);
    }
    for (int s = 0; s < S; ++s) {
      const int64_t stp = step0 + s;
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        mbar_wait(&bars[q], (uint32_t)(s & 1), a.flag, abort);
        const int fc = q * kW8Set + fi;
        if (fc < nf) {
          float* base = st + fc * 4 * kWsSlot + node0;
          react_lane<kW8KR>(a, base, sm[q], stp);
        }
        mbar_arrive(&bars[2 + q]);
      }
    }
    fiber_barrier(0, kW8Threads);
    ws8_store(a, st, f0, nf, tid);
  } else {
    // ---- diffusion groups: group g solves fibers 2g, 2g + 1 of a set ----
    regs_from_diffusion();
    const int c = tid - 32 * kW8RWarps;
    const int g = c / kWsCnThreads;
    const int p = c - g * kWsCnThreads;  // chunk [kWsKC p, kWsKC p + kWsKC)
    float* cfb = s_coef + g * kNumCoef * kWsCS;
    float* xb = s_x + g * 7 * kWsCS;
    Exchange<float> x;
    x.first = xb;
    x.last = xb + kWsCS;
    x.D = xb + 2 * kWsCS;
    x.E = xb + 3 * kWsCS;
    x.y = xb + 4 * kWsCS;
    x.r2 = xb + 5 * kWsCS;
    const float* g_recs = static_cast<const float*>(a.recs);
    for (int s = 0; s <= S; ++s) {
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        if (s > 0) mbar_wait(&bars[2 + q], (uint32_t)((s - 1) & 1), a.flag, abort);
        // the second half of step s - 1 and the first half of step s
        const int count = (s > 0 ? a.n_cn : 0) + (s < S ? a.n_cn : 0);
        for (int k = 0; k < 2; ++k) {
          const int fc = q * kW8Set + 2 * g + k;
          if (fc >= nf) continue;  // the same for every thread of the group
          const FiberDesc fd = a.fibers[f0 + fc];
          const float* rec = g_recs + fd.rec + (int64_t)p * a.rec_stride;
          // this thread's coefficient column (read back by this thread only)
          for (int e = 0; e < 7; ++e) cfb[e * kWsCS + p] = rec[e];
          cfb[kPKE * kWsCS + p] = p > 0 ? rec[4 - a.rec_stride] : 0.0f;
          cfb[kPKD * kWsCS + p] = p > 0 ? rec[5 - a.rec_stride] : 0.0f;
          cfb[kPKDn * kWsCS + p] = p > 0 ? rec[6 - a.rec_stride] : 0.0f;
          SolveCtx<kWsKC, float> sc;
          const int Tf = (fd.n + kWsKC - 1) / kWsKC;
          sc.p = p;
          sc.Tw = kWsCnThreads;
          sc.tid = p;
          sc.nreal = min(max(fd.n - p * kWsKC, 0), kWsKC);
          sc.bar_id = 1 + g;
          sc.levels = a.n_levels;
          sc.edge = (sc.nreal < kWsKC) || (p == Tf - 1);
          sc.set = s_rows + ((p == Tf - 1) ? (1 + fc) * set_len : 0);
          sc.r = fd.n > 1 ? (float)a.r : 0.0f;
          sc.ie = false;
          sc.rec = rec;
          sc.cf = cfb + p;
          solve_chunk(st + fc * 4 * kWsSlot + kWsKC * p, sc, x, count);
        }
        if (s < S) mbar_arrive(&bars[q]);
      }
    }
    fiber_barrier(0, kW8Threads);
    ws8_store(a, st, f0, nf, tid);
  }
}

}  // namespace

size_t split_step_ws_smem_bytes() {
  return 4 * ((size_t)2 * 4 * kWsSlot + 3 * kWsKC * kCoefPerRow + 2 * kNumCoef * kWsCS + 7 * kWsCS) +
         4 * sizeof(uint64_t) + 16;
}

size_t split_step_ws8_smem_bytes() {
  return 4 * ((size_t)kW8Fibers * 4 * kWsSlot + (1 + kW8Fibers) * kWsKC * kCoefPerRow +
              (size_t)kW8Groups * (kNumCoef + 7) * kWsCS) +
         4 * sizeof(uint64_t) + 16;
}

int split_step_ws8_fibers_per_cta() { return kW8Fibers; }
int split_step_ws8_warps() { return kW8Threads / 32; }

int launch_split_step_ws8(const StepArgs& a, int n_ctas, void* stream) {
  if (n_ctas <= 0 || a.n_steps <= 0) return 0;
  // The register split is exact only if the kernel is launched with
  // kW8RegLaunch registers per thread; with fewer, the reaction warpgroups'
  // setmaxnreg.inc could never be satisfied, so refuse to launch.
  cudaFuncAttributes fa;
  cudaError_t e = cudaFuncGetAttributes(&fa, split_step_ws8_kernel);
  if (e != cudaSuccess) return (int)e;
  if (fa.numRegs != kW8RegLaunch) return (int)cudaErrorInvalidConfiguration;
  const size_t smem = split_step_ws8_smem_bytes();
  e = cudaFuncSetAttribute(split_step_ws8_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return (int)e;
  split_step_ws8_kernel<<<n_ctas, kW8Threads, smem, static_cast<cudaStream_t>(stream)>>>(a);
  return (int)cudaGetLastError();
}

int launch_split_step_ws(const StepArgs& a, int n_ctas, void* stream) {
  if (n_ctas <= 0 || a.n_steps <= 0) return 0;
  const size_t smem = split_step_ws_smem_bytes();
  cudaError_t e = cudaFuncSetAttribute(split_step_ws_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return (int)e;
  split_step_ws_kernel<<<n_ctas, kWsThreads, smem, static_cast<cudaStream_t>(stream)>>>(a);
  return (int)cudaGetLastError();
}

}  // namespace fib
