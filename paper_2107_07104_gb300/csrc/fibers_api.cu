// Host implementation of the C ABI in include/fibers.h.
//
// The context owns the device-resident state of all fibers in a padded
// structure-of-arrays layout (u = V - Vrest, m, h, n), the fiber/CTA maps of
// the split-step kernel, the tridiagonal-solve tables, the stimulus tables,
// and an optional captured CUDA graph of a block of split steps.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "fibers.h"
#include "fibers_internal.h"
#include "split_step_ws.h"
#include "surrogate_internal.h"

#include <cuda_bf16.h>

using namespace fib;

struct fib_ctx {
  fib_params p{};
  double EL = 0.0;
  double m0 = 0.0, h0 = 0.0, n0 = 0.0;  // rest gates
  int64_t n_sub = 0, n_cn = 0, pulse = 0;
  double r = 0.0;

  int32_t n_fibers = 0;
  std::vector<int32_t> n_nodes, mu, junction;
  std::vector<int64_t> coff;  // ragged offsets
  int64_t total = 0;
  int32_t max_n = 0;

  cudaStream_t stream = nullptr;
  cudaStream_t cap_stream = nullptr;
  int device = 0;
  fib_tuning tune{};

  // layout-dependent device data
  int K = 0, W = 0, n_ctas = 0, levels = 0, rec_stride = 0;
  int ws = 0;  // split warp roles (split_step_ws.cu): 0 fused kernel, 2 two-fiber shape, 3 eight-fiber shape
  int64_t slots_total = 0;
  float* d_state = nullptr;  // 4 * slots_total
  FiberDesc* d_fibers = nullptr;
  WarpMap* d_warps = nullptr;
  void* d_rows = nullptr;
  void* d_recs = nullptr;

  // stimulus
  int32_t n_mu = 0;
  int64_t* d_mu_off = nullptr;
  int64_t* d_fire_k = nullptr;

  int64_t* d_step = nullptr;
  int32_t* d_flag = nullptr;
  uint8_t* d_quiet = nullptr;               // adaptive: per-fiber equilibrium flag
  unsigned long long* d_skipped = nullptr;  // adaptive: fiber-steps skipped
  int64_t next_step = 0;
  int64_t launches = 0;

  float* d_stage = nullptr;  // compact staging (read/write of host buffers)
  size_t stage_elems = 0;

  // read_vm_async: a copy stream, two staging buffers with their status
  // words, and the events that order them against the steps
  cudaStream_t copy_stream = nullptr;
  float* d_async[2] = {nullptr, nullptr};
  int32_t* d_async_flag = nullptr;  // [2]
  int32_t* h_async_flag = nullptr;  // [2], page-locked
  cudaEvent_t ev_gathered[2] = {nullptr, nullptr};
  cudaEvent_t ev_copied[2] = {nullptr, nullptr};
  int64_t async_issued = 0;
  bool async_ready = false;

  cudaGraphExec_t graph = nullptr;
  int64_t graph_launches = 0;

  // reaction-step surrogate (FIB_MODE_SURROGATE)
  float* d_sur_list = nullptr;          // surrogate: network-node lists (2 parities x 6 x slots_total)
  unsigned int* d_sur_count = nullptr;  // surrogate: their lengths [2]
  uint16_t* d_sur_wts = nullptr;     // bf16 weight images
  float* d_sur_bias = nullptr;
  unsigned long long* d_fallback = nullptr;
  bool sur_loaded = false;
  float in_mu[kIn] = {}, in_inv_sigma[kIn] = {}, out_mu[kOut] = {}, out_sigma[kOut] = {};
  float env_lo[kIn] = {}, env_hi[kIn] = {};
  float quiet_lo[kIn] = {}, quiet_hi[kIn] = {};

  std::string err;
};

// Surrogate mode's split steps (defined below), enqueued on stream s.
fib_status surrogate_steps(fib_ctx* c, cudaStream_t s, int64_t n);

namespace {

thread_local std::string g_create_error;

fib_status fail(fib_ctx* c, fib_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  if (c) c->err = buf;
  else g_create_error = buf;
  return s;
}

#define CU(ctx, call)                                                                       \
  do {                                                                                      \
    cudaError_t e_ = (call);                                                                \
    if (e_ != cudaSuccess)                                                                  \
      return fail(ctx, e_ == cudaErrorMemoryAllocation ? FIB_ENOMEM : FIB_ECUDA, "%s: %s (%s:%d)", \
                  #call, cudaGetErrorString(e_), __FILE__, __LINE__);                       \
  } while (0)

template <typename T>
void dfree(T*& p) {
  if (p) cudaFree((void*)p);
  p = nullptr;
}

// ---- model constants (double precision, host) ----------------------------

// exp*(x) = (1 + x/1024)^1024 (eq:apx-e-function), or exp(x).
double rate_exp(double x, bool apx) {
  if (!apx) return std::exp(x);
  double y = 1.0 + x / 1024.0;
  for (int i = 0; i < 10; ++i) y *= y;
  return y;
}

// x / (1 - exp(-x/k)) with its limit k at x = 0.
double vtrap(double x, double k, bool apx) {
  if (x == 0.0) return k;
  return apx ? x / (1.0 - rate_exp(-x / k, true)) : x / (-std::expm1(-x / k));
}

// Steady-state gates at depolarisation u, with exact or approximated exponentials.
void rest_gates(double u, double* m, double* h, double* n, bool apx) {
  const double am = 0.1 * vtrap(u - 25.0, 10.0, apx), bm = 4.0 * rate_exp(-u / 18.0, apx);
  const double ah = 0.07 * rate_exp(-u / 20.0, apx), bh = 1.0 / (1.0 + rate_exp((30.0 - u) / 10.0, apx));
  const double an = 0.01 * vtrap(u - 10.0, 10.0, apx), bn = 0.125 * rate_exp(-u / 80.0, apx);
  *m = am / (am + bm);
  *h = ah / (ah + bh);
  *n = an / (an + bn);
}

bool finite_pos(double v) { return std::isfinite(v) && v > 0.0; }

// Length of one diffusion phase: half a split step for Strang 1D-0D-1D, a
// whole one for the other orderings.
double diffusion_phase(const fib_params* p) {
  return (p->splitting == FIB_SPLIT_STRANG_1D0D1D ? 0.5 : 1.0) * p->dt_split;
}

fib_status validate(const fib_params* p) {
  if (!p) return fail(nullptr, FIB_EINVAL, "params is NULL");
  const double vals[] = {p->Cm, p->Am, p->h, p->dt_split, p->dt_0d, p->dt_1d, p->sigma_eff};
  for (double v : vals)
    if (!finite_pos(v)) return fail(nullptr, FIB_EINVAL, "Cm, Am, h, dt_split, dt_0d, dt_1d, sigma_eff must be > 0");
  const double fin[] = {p->gNa, p->gK, p->gL, p->ENa, p->EK, p->Vrest, p->stim_amplitude, p->stim_duration};
  for (double v : fin)
    if (!std::isfinite(v)) return fail(nullptr, FIB_EINVAL, "non-finite model parameter");
  if (p->gNa < 0 || p->gK < 0 || p->gL < 0 || p->stim_duration < 0)
    return fail(nullptr, FIB_EINVAL, "conductances and stim_duration must be >= 0");
  if (std::isnan(p->EL) && !(p->gL > 0))
    return fail(nullptr, FIB_EINVAL, "EL = NaN (derive exact rest) needs gL > 0");
  if (!std::isnan(p->EL) && !std::isfinite(p->EL)) return fail(nullptr, FIB_EINVAL, "EL must be finite or NaN");
  if (p->stim_half_width < 0 || p->stim_half_width > 8)
    return fail(nullptr, FIB_EINVAL, "stim_half_width must be in [0, 8]");
  if (p->mode != FIB_MODE_FP32 && p->mode != FIB_MODE_FP64_THOMAS && p->mode != FIB_MODE_SURROGATE)
    return fail(nullptr, FIB_EINVAL, "unknown mode %d", p->mode);
  if ((p->flags & ~(FIB_FLAG_ADAPTIVE | FIB_FLAG_EXP_APPROX)) != 0 || p->reserved != 0)
    return fail(nullptr, FIB_EINVAL, "unknown flags or nonzero reserved field");
  if ((p->flags & FIB_FLAG_EXP_APPROX) && p->mode != FIB_MODE_FP32)
    return fail(nullptr, FIB_EINVAL, "the exp* approximation runs in FIB_MODE_FP32 only");
  if ((p->flags & FIB_FLAG_ADAPTIVE) && p->mode == FIB_MODE_SURROGATE)
    return fail(nullptr, FIB_EINVAL, "adaptive computation is not available in surrogate mode");
  if (p->splitting < FIB_SPLIT_STRANG_1D0D1D || p->splitting > FIB_SPLIT_GODUNOV_0D1D)
    return fail(nullptr, FIB_EINVAL, "unknown splitting %d", p->splitting);
  if (p->diffusion != FIB_DIFFUSION_CRANK_NICOLSON && p->diffusion != FIB_DIFFUSION_IMPLICIT_EULER)
    return fail(nullptr, FIB_EINVAL, "unknown diffusion method %d", p->diffusion);
  if (p->mode == FIB_MODE_SURROGATE &&
      (p->splitting != FIB_SPLIT_STRANG_1D0D1D || p->diffusion != FIB_DIFFUSION_CRANK_NICOLSON))
    return fail(nullptr, FIB_EINVAL, "surrogate mode runs only Strang 1D-0D-1D with Crank-Nicolson");
  const double q0 = p->dt_split / p->dt_0d, q1 = diffusion_phase(p) / p->dt_1d;
  const double r0 = std::nearbyint(q0), r1 = std::nearbyint(q1);
  if (r0 < 1 || r1 < 1 || std::fabs(q0 - r0) > 1e-9 * q0 || std::fabs(q1 - r1) > 1e-9 * q1)
    return fail(nullptr, FIB_EINVAL, "dt_split/dt_0d and the diffusion phase over dt_1d must be whole numbers >= 1");
  if (r0 > 1000 || r1 > 1000) return fail(nullptr, FIB_EINVAL, "too many substeps per split step");
  if (p->splitting == FIB_SPLIT_STRANG_0D1D0D && ((int64_t)r0 % 2) != 0)
    return fail(nullptr, FIB_EINVAL, "0D-1D-0D Strang needs an even number of Heun substeps per split step");
  return FIB_OK;
}

// ---- layout ---------------------------------------------------------------

// Warps a fiber of n nodes needs at K nodes per thread (64-bit, so that no
// int32 length can wrap it below the limit checks).
int warps_for(int32_t n, int K) {
  const int64_t T = ((int64_t)n + K - 1) / K;
  return (int)std::min<int64_t>((T + 31) / 32, INT32_MAX);
}

// Nodes per thread when the caller leaves it open.  The plain FP32 step
// (exact or exp* exponentials) runs fastest at K = 12 on GB300 (packed pairs,
// 8-warp CTAs, the 80-register budget: 0.893 ms per split step on the
// 67,600-fiber bundle against 0.927 at K = 8); the surrogate step (one split
// step per launch) and adaptive computation measured faster at K = 8, as
// does the FP64 solve's register budget.  Longer fibers take the K that
// fits them with the fewest padded nodes.
int auto_K(const std::vector<int32_t>& n_nodes, bool plain_fp32) {
  int max_n = 0;
  for (int32_t n : n_nodes) max_n = std::max(max_n, n);
  const int first = plain_fp32 ? 12 : 8;
  if (warps_for(max_n, first) <= kMaxWarpsPerCta) return first;
  int best = 16;
  int64_t best_pad = -1;
  for (int K : {12, 16}) {
    int64_t pad = 0;
    bool ok = true;
    for (int32_t n : n_nodes) {
      const int w = warps_for(n, K);
      if (w > kMaxWarpsPerCta) ok = false;
      pad += (int64_t)32 * w * K;
    }
    if (ok && (best_pad < 0 || pad < best_pad)) {
      best = K;
      best_pad = pad;
    }
  }
  return best;
}

int auto_W(int w_max) { return w_max * std::max(1, kMaxWarpsPerCta / w_max); }

// Whether the automatic shape uses split warp roles where they apply.
constexpr bool kWsAuto = false;
constexpr int kWsAutoShape = 2;

void free_layout(fib_ctx* c) {
  if (c->graph) cudaGraphExecDestroy(c->graph);
  c->graph = nullptr;
  dfree(c->d_state);
  dfree(c->d_fibers);
  dfree(c->d_warps);
  dfree(c->d_rows);
  dfree(c->d_recs);
  dfree(c->d_sur_list);
  dfree(c->d_sur_count);
}

// Can the split-role kernel run this context?  Plain FP32, no flags,
// Strang 1D-0D-1D with Crank-Nicolson, every fiber within its slot.
bool ws_eligible(const fib_ctx* c) {
  return c->p.mode == FIB_MODE_FP32 && c->p.flags == 0 && c->p.splitting == FIB_SPLIT_STRANG_1D0D1D &&
         c->p.diffusion == FIB_DIFFUSION_CRANK_NICOLSON && c->n_fibers > 0 && c->max_n <= kWsSlot;
}

// Layout of the split-role kernel: slots of kWsSlot nodes, two fibers per
// CTA, solver tables for kWsKC nodes per diffusion thread.
fib_status build_layout_ws(fib_ctx* c, const fib_tuning& t, int shape) {
  constexpr int KC = kWsKC;
  std::map<int32_t, int> cls;
  std::vector<int32_t> lens, tw;
  for (int32_t n : c->n_nodes)
    if (!cls.count(n)) {
      cls[n] = (int)lens.size();
      lens.push_back(n);
      tw.push_back(kWsCnThreads);
    }
  SolverTables tab;
  if (!build_solver_tables(KC, c->r, lens, tw, false, &tab))
    return fail(c, FIB_EINVAL, "tridiagonal tables: zero pivot (r = %g)", c->r);
  std::vector<FiberDesc> fd(c->n_fibers);
  for (int32_t f = 0; f < c->n_fibers; ++f) {
    const int ci = cls[c->n_nodes[f]];
    fd[f].slot = (int64_t)f * kWsSlot;
    fd[f].coff = c->coff[f];
    fd[f].rec = tab.class_rec[ci];
    fd[f].n = c->n_nodes[f];
    fd[f].junction = c->junction[f];
    fd[f].mu = c->mu[f];
    fd[f].last_set = (int32_t)tab.class_last[ci];
    fd[f].slot_len = kWsSlot;
    fd[f].pad = 0;
  }
  const int64_t slot = (int64_t)c->n_fibers * kWsSlot;
  free_layout(c);
  const bool wide = shape == 3;
  const int per_cta = wide ? split_step_ws8_fibers_per_cta() : 2;
  c->ws = shape;
  c->K = KC;
  c->W = wide ? split_step_ws8_warps() : kWsWarps;
  c->n_ctas = (c->n_fibers + per_cta - 1) / per_cta;
  c->levels = tab.levels;
  c->rec_stride = tab.rec_stride;
  c->slots_total = slot;
  c->tune.nodes_per_thread = 0;
  c->tune.warps_per_cta = c->W;
  c->tune.steps_per_launch = t.steps_per_launch ? t.steps_per_launch : 100;
  c->tune.graph_steps = t.graph_steps;
  c->tune.reaction_pairs = 2;
  c->tune.ctas_per_sm = wide ? 1 : kWsMinBlocks;
  c->tune.warp_roles = shape;
  CU(c, cudaMalloc(&c->d_state, sizeof(float) * 4 * (size_t)slot));
  CU(c, cudaMalloc(&c->d_fibers, sizeof(FiberDesc) * fd.size()));
  CU(c, cudaMalloc(&c->d_warps, sizeof(WarpMap)));
  CU(c, cudaMalloc(&c->d_rows, 4 * tab.rows.size()));
  CU(c, cudaMalloc(&c->d_recs, 4 * std::max<size_t>(tab.recs.size(), 1)));
  CU(c, cudaMemcpy(c->d_fibers, fd.data(), sizeof(FiberDesc) * fd.size(), cudaMemcpyHostToDevice));
  std::vector<float> rf(tab.rows.begin(), tab.rows.end()), cf(tab.recs.begin(), tab.recs.end());
  CU(c, cudaMemcpy(c->d_rows, rf.data(), 4 * rf.size(), cudaMemcpyHostToDevice));
  if (!cf.empty()) CU(c, cudaMemcpy(c->d_recs, cf.data(), 4 * cf.size(), cudaMemcpyHostToDevice));
  return FIB_OK;
}

// Builds the padded layout, CTA packing and solver tables for tuning t.
// Allocates (uninitialised) state; the caller fills it.
fib_status build_layout(fib_ctx* c, const fib_tuning& t) {
  if (t.warp_roles < 0 || t.warp_roles > 3) return fail(c, FIB_EINVAL, "warp_roles must be 0, 1, 2 or 3");
  if (t.warp_roles >= 2 && !ws_eligible(c))
    return fail(c, FIB_EINVAL,
                "split warp roles need FIB_MODE_FP32 with no flags, Strang 1D-0D-1D, Crank-Nicolson and fibers of "
                "at most %d nodes", kWsSlot);
  if (t.steps_per_launch < 0 || t.graph_steps < 0) return fail(c, FIB_EINVAL, "negative steps in tuning");
  if (t.warp_roles >= 2) return build_layout_ws(c, t, t.warp_roles);
  if (t.warp_roles == 0 && kWsAuto && t.nodes_per_thread == 0 && ws_eligible(c)) return build_layout_ws(c, t, kWsAutoShape);
  const bool plain_fp32 = c->p.mode == FIB_MODE_FP32 && !(c->p.flags & FIB_FLAG_ADAPTIVE);
  int K = t.nodes_per_thread ? t.nodes_per_thread : auto_K(c->n_nodes, plain_fp32);
  if (K != 4 && K != 8 && K != 12 && K != 16) return fail(c, FIB_EINVAL, "nodes_per_thread must be 4, 8, 12 or 16");
  int w_max = 1;
  for (int32_t n : c->n_nodes) w_max = std::max(w_max, warps_for(n, K));
  if (w_max > kMaxWarpsPerCta)
    return fail(c, FIB_EINVAL, "a fiber of %d nodes needs %d warps at %d nodes per thread (max %d warps)", c->max_n,
                w_max, K, kMaxWarpsPerCta);
  int W = t.warps_per_cta ? t.warps_per_cta : auto_W(w_max);
  if (W < 1 || W > kMaxWarpsPerCta) return fail(c, FIB_EINVAL, "warps_per_cta must be in [1, %d]", kMaxWarpsPerCta);
  if (W < w_max) return fail(c, FIB_EINVAL, "warps_per_cta %d < %d warps needed by the longest fiber", W, w_max);
  if (t.steps_per_launch < 0 || t.graph_steps < 0) return fail(c, FIB_EINVAL, "negative steps in tuning");
  if (t.reaction_pairs < 0 || t.reaction_pairs > 2) return fail(c, FIB_EINVAL, "reaction_pairs must be 0, 1 or 2");
  if (t.ctas_per_sm != 0 && (t.ctas_per_sm < 2 || t.ctas_per_sm > 4))
    return fail(c, FIB_EINVAL, "ctas_per_sm must be 0, 2, 3 or 4");

  // length classes
  std::map<int32_t, int> cls;
  std::vector<int32_t> lens, tw;
  for (int32_t n : c->n_nodes)
    if (!cls.count(n)) {
      cls[n] = (int)lens.size();
      lens.push_back(n);
      tw.push_back(32 * warps_for(n, K));
    }
  SolverTables tab;
  const bool fp64_tables = c->p.mode == FIB_MODE_FP64_THOMAS;
  if (!lens.empty() && !build_solver_tables(K, c->r, lens, tw, fp64_tables, &tab))
    return fail(c, FIB_EINVAL, "tridiagonal tables: zero pivot (r = %g)", c->r);
  if (lens.empty()) {  // keep valid (unused) tables
    std::vector<int32_t> one{1}, t1{32};
    build_solver_tables(K, c->r, one, t1, fp64_tables, &tab);
  }

  // slots and packing: fibers by warp count (descending), next-fit into CTAs
  std::vector<FiberDesc> fd(c->n_fibers);
  int64_t slot = 0;
  for (int32_t f = 0; f < c->n_fibers; ++f) {
    const int w = warps_for(c->n_nodes[f], K);
    const int ci = cls[c->n_nodes[f]];
    fd[f].slot = slot;
    fd[f].coff = c->coff[f];
    fd[f].rec = tab.class_rec[ci];
    fd[f].n = c->n_nodes[f];
    fd[f].junction = c->junction[f];
    fd[f].mu = c->mu[f];
    fd[f].last_set = (int32_t)tab.class_last[ci];
    fd[f].slot_len = 32 * w * K;
    fd[f].pad = 0;
    slot += fd[f].slot_len;
  }
  std::vector<int32_t> order(c->n_fibers);
  for (int32_t f = 0; f < c->n_fibers; ++f) order[f] = f;
  std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) {
    return warps_for(c->n_nodes[a], K) > warps_for(c->n_nodes[b], K);
  });
  std::vector<WarpMap> wm;
  int used = W, nfib = kMaxFibersPerCta;  // force a new CTA for the first fiber
  int n_ctas = 0;
  for (int32_t f : order) {
    const int w = warps_for(c->n_nodes[f], K);
    if (used + w > W || nfib >= kMaxFibersPerCta) {
      ++n_ctas;
      wm.resize((size_t)n_ctas * W, WarpMap{-1, 0, 0, 0, 0});
      used = 0;
      nfib = 0;
    }
    for (int k = 0; k < w; ++k) {
      WarpMap& e = wm[(size_t)(n_ctas - 1) * W + used + k];
      e.fiber = f;
      e.first_warp = (int16_t)used;
      e.n_warps = (int16_t)w;
      e.slot = nfib;
    }
    used += w;
    ++nfib;
  }

  free_layout(c);
  c->ws = 0;
  c->tune.warp_roles = 1;
  c->K = K;
  c->W = W;
  c->n_ctas = n_ctas;
  c->levels = tab.levels;
  c->rec_stride = tab.rec_stride;
  c->slots_total = slot;
  c->tune.nodes_per_thread = K;
  c->tune.warps_per_cta = W;
  c->tune.steps_per_launch = t.steps_per_launch ? t.steps_per_launch : 100;
  c->tune.graph_steps = t.graph_steps;
  c->tune.reaction_pairs = t.reaction_pairs ? t.reaction_pairs : 2;
  c->tune.ctas_per_sm = t.ctas_per_sm ? t.ctas_per_sm : 3;

  const bool fp64 = c->p.mode == FIB_MODE_FP64_THOMAS;
  const size_t es = fp64 ? 8 : 4;
  CU(c, cudaMalloc(&c->d_state, sizeof(float) * 4 * (size_t)std::max<int64_t>(slot, 4)));
  CU(c, cudaMalloc(&c->d_fibers, sizeof(FiberDesc) * std::max<size_t>(fd.size(), 1)));
  CU(c, cudaMalloc(&c->d_warps, sizeof(WarpMap) * std::max<size_t>(wm.size(), 1)));
  CU(c, cudaMalloc(&c->d_rows, es * tab.rows.size()));
  CU(c, cudaMalloc(&c->d_recs, es * std::max<size_t>(tab.recs.size(), 1)));
  if (!fd.empty()) CU(c, cudaMemcpy(c->d_fibers, fd.data(), sizeof(FiberDesc) * fd.size(), cudaMemcpyHostToDevice));
  if (c->p.mode == FIB_MODE_SURROGATE && slot > INT32_MAX)
    return fail(c, FIB_EINVAL, "surrogate mode holds slot indices in 32 bits: %lld slots", (long long)slot);
  if (c->p.mode == FIB_MODE_SURROGATE && slot > 0) {
    CU(c, cudaMalloc(&c->d_sur_list, sizeof(float) * 12 * (size_t)slot));
    CU(c, cudaMalloc(&c->d_sur_count, 2 * sizeof(unsigned int)));
    CU(c, cudaMemset(c->d_sur_count, 0, 2 * sizeof(unsigned int)));
  }
  if (!wm.empty()) CU(c, cudaMemcpy(c->d_warps, wm.data(), sizeof(WarpMap) * wm.size(), cudaMemcpyHostToDevice));
  if (fp64) {
    CU(c, cudaMemcpy(c->d_rows, tab.rows.data(), 8 * tab.rows.size(), cudaMemcpyHostToDevice));
    if (!tab.recs.empty()) CU(c, cudaMemcpy(c->d_recs, tab.recs.data(), 8 * tab.recs.size(), cudaMemcpyHostToDevice));
  } else {
    std::vector<float> rf(tab.rows.begin(), tab.rows.end()), cf(tab.recs.begin(), tab.recs.end());
    CU(c, cudaMemcpy(c->d_rows, rf.data(), 4 * rf.size(), cudaMemcpyHostToDevice));
    if (!cf.empty()) CU(c, cudaMemcpy(c->d_recs, cf.data(), 4 * cf.size(), cudaMemcpyHostToDevice));
  }
  return FIB_OK;
}

float* st_u(fib_ctx* c) { return c->d_state; }
float* st_m(fib_ctx* c) { return c->d_state + c->slots_total; }
float* st_h(fib_ctx* c) { return c->d_state + 2 * c->slots_total; }
float* st_n(fib_ctx* c) { return c->d_state + 3 * c->slots_total; }

fib_status ensure_stage(fib_ctx* c, size_t elems) {
  if (c->stage_elems >= elems && c->d_stage) return FIB_OK;
  dfree(c->d_stage);
  c->stage_elems = 0;
  CU(c, cudaMalloc(&c->d_stage, sizeof(float) * std::max<size_t>(elems, 1)));
  c->stage_elems = elems;
  return FIB_OK;
}

fib_status check_launch(fib_ctx* c, int e, const char* what) {
  if (e != 0) return fail(c, FIB_ECUDA, "%s launch failed: %s", what, cudaGetErrorString((cudaError_t)e));
  return FIB_OK;
}

HHConst hh_const(const fib_params& p, double EL) {
  HHConst h{};
  const double Cm = p.Cm;
  h.gNa = (float)(p.gNa / Cm);
  h.gK = (float)(p.gK / Cm);
  h.gL = (float)(p.gL / Cm);
  h.uNa = (float)(p.ENa - p.Vrest);
  h.uK = (float)(p.EK - p.Vrest);
  h.uL = (float)(EL - p.Vrest);
  h.stim = (float)(p.stim_amplitude / Cm);
  h.dt0 = (float)p.dt_0d;
  h.gNa_uNa = (float)((p.gNa / Cm) * (p.ENa - p.Vrest));
  h.gK_uK = (float)((p.gK / Cm) * (p.EK - p.Vrest));
  h.gL_uL = (float)((p.gL / Cm) * (EL - p.Vrest));
  return h;
}

double exact_leak_reversal(const fib_params& p) {
  double m0, h0, n0;
  rest_gates(0.0, &m0, &h0, &n0, (p.flags & FIB_FLAG_EXP_APPROX) != 0);
  const double ina = p.gNa * m0 * m0 * m0 * h0 * (p.Vrest - p.ENa);
  const double ik = p.gK * n0 * n0 * n0 * n0 * (p.Vrest - p.EK);
  return p.Vrest + (ina + ik) / p.gL;
}

StepArgs make_args(fib_ctx* c) {
  StepArgs a{};
  a.u = st_u(c);
  a.m = st_m(c);
  a.h = st_h(c);
  a.n = st_n(c);
  a.fibers = c->d_fibers;
  a.warps = c->d_warps;
  a.rows = c->d_rows;
  a.recs = c->d_recs;
  a.mu_off = c->d_mu_off;
  a.fire_k = c->d_fire_k;
  a.step_base = c->d_step;
  a.flag = c->d_flag;
  a.hh = hh_const(c->p, c->EL);
  a.hh.m0 = (float)c->m0;  // the state arrays hold gate deviations from rest
  a.hh.h0 = (float)c->h0;
  a.hh.n0 = (float)c->n0;
  a.r = c->r;
  a.n_sub = (int32_t)c->n_sub;
  a.n_cn = (int32_t)c->n_cn;
  switch (c->p.splitting) {
    case FIB_SPLIT_STRANG_1D0D1D: a.k_split = 0; a.n_cn2 = a.n_cn; break;
    case FIB_SPLIT_GODUNOV_1D0D: a.k_split = 0; a.n_cn2 = 0; break;
    case FIB_SPLIT_STRANG_0D1D0D: a.k_split = a.n_sub / 2; a.n_cn2 = 0; break;
    default: a.k_split = a.n_sub; a.n_cn2 = 0; break;  // FIB_SPLIT_GODUNOV_0D1D
  }
  a.implicit_euler = c->p.diffusion == FIB_DIFFUSION_IMPLICIT_EULER ? 1 : 0;
  a.exp_approx = (c->p.flags & FIB_FLAG_EXP_APPROX) ? 1 : 0;
  a.pulse = (int32_t)c->pulse;
  a.hw = c->p.stim_half_width;
  a.n_mu = c->n_mu;
  a.n_levels = c->levels;
  a.rec_stride = c->rec_stride;
  a.W = c->W;
  a.packed = c->tune.reaction_pairs == 2 ? 1 : 0;
  a.occ = c->tune.ctas_per_sm;
  a.phases = 7;
  a.adaptive = (c->p.flags & FIB_FLAG_ADAPTIVE) ? 1 : 0;
  a.quiet = c->d_quiet;
  a.skipped = c->d_skipped;
  a.eq_tol = 1e-5f;
  a.vrest = (float)c->p.Vrest;
  a.n_fib = c->n_fibers;
  return a;
}

// Enqueues split steps [next + offset0, next + offset0 + n) as launches of
// steps_per_launch, without advancing the device step counter.
fib_status enqueue_launches(fib_ctx* c, cudaStream_t s, int64_t offset0, int64_t n) {
  if (c->n_ctas == 0) return FIB_OK;
  StepArgs a = make_args(c);
  const int64_t S = c->tune.steps_per_launch;
  for (int64_t done = 0; done < n; done += S) {
    a.step_offset = offset0 + done;
    a.n_steps = (int32_t)std::min<int64_t>(S, n - done);
    const int e = c->ws == 3 ? launch_split_step_ws8(a, c->n_ctas, s)
                  : c->ws ? launch_split_step_ws(a, c->n_ctas, s)
                        : launch_split_step(c->K, c->p.mode == FIB_MODE_FP64_THOMAS, a, c->n_ctas, s);
    fib_status st = check_launch(c, e, "split step");
    if (st != FIB_OK) return st;
    ++c->launches;
  }
  return FIB_OK;
}

// Captures graph_steps split steps (and the step counter's advance) of the
// context's mode into one CUDA graph.
fib_status build_graph(fib_ctx* c) {
  const int64_t G = c->tune.graph_steps;
  CU(c, cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal));
  const int64_t before = c->launches;
  fib_status st = c->p.mode == FIB_MODE_SURROGATE ? surrogate_steps(c, c->cap_stream, G)
                                                  : enqueue_launches(c, c->cap_stream, 0, G);
  int e = st == FIB_OK ? launch_advance(c->d_step, G, c->cap_stream) : 0;
  cudaGraph_t g = nullptr;
  cudaError_t ee = cudaStreamEndCapture(c->cap_stream, &g);
  c->graph_launches = (c->launches - before) + 1;
  c->launches = before;
  if (st != FIB_OK) {
    if (g) cudaGraphDestroy(g);
    return st;
  }
  if (e != 0 || ee != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return fail(c, FIB_ECUDA, "graph capture failed: %s", cudaGetErrorString(ee != cudaSuccess ? ee : (cudaError_t)e));
  }
  cudaError_t ie = cudaGraphInstantiate(&c->graph, g, 0);
  cudaGraphDestroy(g);
  if (ie != cudaSuccess) {
    c->graph = nullptr;
    return fail(c, FIB_ECUDA, "graph instantiate failed: %s", cudaGetErrorString(ie));
  }
  return FIB_OK;
}

fib_status flag_status(fib_ctx* c, int32_t flag) {
  if (flag & 4)
    return fail(c, FIB_ETIMEOUT, "a bounded wait between the reaction and diffusion warps gave up; state unreliable");
  if (flag & 2) return fail(c, FIB_ESTATE, "surrogate network-node list overflowed; its entries were dropped");
  if (flag & 1) return fail(c, FIB_ENONFINITE, "state became non-finite (NaN/Inf)");
  return FIB_OK;
}

fib_status check_flag(fib_ctx* c) {
  int32_t flag = 0;
  CU(c, cudaMemcpy(&flag, c->d_flag, sizeof(flag), cudaMemcpyDeviceToHost));
  return flag_status(c, flag);
}

// Surrogate mode: the network-node list counters of both step parities
// start at zero.  Needed wherever the step index is set, since the network
// pass empties only the other parity's list for the next step.
fib_status reset_sur_lists(fib_ctx* c) {
  if (c->d_sur_count) CU(c, cudaMemsetAsync(c->d_sur_count, 0, 2 * sizeof(unsigned int), c->stream));
  return FIB_OK;
}

fib_status set_device(fib_ctx* c) {
  CU(c, cudaSetDevice(c->device));
  return FIB_OK;
}

// Gathers the internal state (u|m|h|n, u = V - Vrest) into dst (device,
// 4 * total) in ragged order.  Bit-exact: no arithmetic on the values.
fib_status gather_state(fib_ctx* c, float* dst) {
  const float adds[4] = {0.f, 0.f, 0.f, 0.f};
  float* src[4] = {st_u(c), st_m(c), st_h(c), st_n(c)};
  for (int k = 0; k < 4; ++k) {
    fib_status st = check_launch(c, launch_gather(c->d_fibers, c->n_fibers, src[k], dst + k * c->total, adds[k], c->stream),
                                 "gather");
    if (st != FIB_OK) return st;
    ++c->launches;
  }
  return FIB_OK;
}

// Fills the padded layout from a compact (u|m|h|n) device buffer (bit-exact).
// A replaced state is re-tested by the adaptive scheme: all fibers active.
fib_status scatter_state(fib_ctx* c, const float* src) {
  if (c->d_quiet) CU(c, cudaMemsetAsync(c->d_quiet, 0, std::max<size_t>(c->n_fibers, 1), c->stream));
  fib_status st = check_launch(c, launch_fill_layout(c->d_fibers, c->n_fibers, st_u(c), st_m(c), st_h(c), st_n(c),
                                                     nullptr, (float)c->p.Vrest, 0.0f, 0.0f, 0.0f, c->stream),
                               "fill");
  if (st != FIB_OK) return st;
  ++c->launches;
  const float adds[4] = {0.f, 0.f, 0.f, 0.f};
  float* dst[4] = {st_u(c), st_m(c), st_h(c), st_n(c)};
  for (int k = 0; k < 4; ++k) {
    st = check_launch(c, launch_scatter(c->d_fibers, c->n_fibers, src + k * c->total, dst[k], adds[k], c->stream),
                      "scatter");
    if (st != FIB_OK) return st;
    ++c->launches;
  }
  return FIB_OK;
}

// read_vm_async's copy stream, staging buffers, status words and events
// (all or nothing: free_async undoes a partial setup).
fib_status setup_async(fib_ctx* c) {
  CU(c, cudaStreamCreateWithFlags(&c->copy_stream, cudaStreamNonBlocking));
  CU(c, cudaMalloc(&c->d_async_flag, 2 * sizeof(int32_t)));
  CU(c, cudaHostAlloc(&c->h_async_flag, 2 * sizeof(int32_t), cudaHostAllocDefault));
  c->h_async_flag[0] = c->h_async_flag[1] = 0;
  for (int k = 0; k < 2; ++k) {
    CU(c, cudaEventCreateWithFlags(&c->ev_gathered[k], cudaEventDisableTiming));
    CU(c, cudaEventCreateWithFlags(&c->ev_copied[k], cudaEventDisableTiming));
    if (c->total > 0) CU(c, cudaMalloc(&c->d_async[k], sizeof(float) * (size_t)c->total));
  }
  return FIB_OK;
}

void free_async(fib_ctx* c) {
  if (c->copy_stream) {
    cudaStreamSynchronize(c->copy_stream);
    cudaStreamDestroy(c->copy_stream);
    c->copy_stream = nullptr;
  }
  for (int k = 0; k < 2; ++k) {
    dfree(c->d_async[k]);
    if (c->ev_gathered[k]) cudaEventDestroy(c->ev_gathered[k]);
    if (c->ev_copied[k]) cudaEventDestroy(c->ev_copied[k]);
    c->ev_gathered[k] = c->ev_copied[k] = nullptr;
  }
  dfree(c->d_async_flag);
  if (c->h_async_flag) cudaFreeHost(c->h_async_flag);
  c->h_async_flag = nullptr;
  c->async_ready = false;
}

}  // namespace

// Surrogate mode, per split step: one launch of the step kernel (the
// previous step's second diffusion half, this step's first, and the plain
// reaction of every node, listing the nodes the network handles), then the
// network pass over that list; after the last step, the second diffusion
// half alone.  Two diffusion halves in a row are 2 n_cn steps of one
// operator, so merging them keeps the bits.
fib_status surrogate_steps(fib_ctx* c, cudaStream_t stream, int64_t n) {
  if (c->n_ctas == 0 || n <= 0) return FIB_OK;
  StepArgs a = make_args(c);
  a.n_steps = 1;
  a.sur_list = c->d_sur_list;
  a.sur_count = c->d_sur_count;
  a.sur_cap = c->slots_total;
  for (int k = 0; k < kIn; ++k) {
    a.sur_env_lo[k] = c->env_lo[k];
    a.sur_env_hi[k] = c->env_hi[k];
    a.sur_quiet_lo[k] = c->quiet_lo[k];
    a.sur_quiet_hi[k] = c->quiet_hi[k];
  }
  a.inv_n_sub = 1.0f / (float)c->n_sub;
  SurArgs s{};
  s.u = st_u(c);
  s.m = st_m(c);
  s.h = st_h(c);
  s.n = st_n(c);
  s.list = c->d_sur_list;
  s.list_count = c->d_sur_count;
  s.list_cap = c->slots_total;
  s.step_base = c->d_step;
  s.real_nodes = c->total;
  s.wts = c->d_sur_wts;
  s.bias = c->d_sur_bias;
  s.fallback_count = c->d_fallback;
  for (int k = 0; k < kIn; ++k) {
    s.in_mu[k] = c->in_mu[k];
    s.in_inv_sigma[k] = c->in_inv_sigma[k];
  }
  for (int k = 0; k < kOut; ++k) {
    s.out_mu[k] = c->out_mu[k];
    s.out_sigma[k] = c->out_sigma[k];
  }
  s.rest[0] = 0.0f;
  s.rest[1] = (float)c->m0;
  s.rest[2] = (float)c->h0;
  s.rest[3] = (float)c->n0;
  const int32_t n_cn = (int32_t)c->n_cn;
  fib_status st = FIB_OK;
  for (int64_t i = 0; i < n; ++i) {
    a.step_offset = i;
    a.phases = 1 | 2;
    a.n_cn = i == 0 ? n_cn : 2 * n_cn;
    st = check_launch(c, launch_split_step_sur(c->K, a, c->n_ctas, stream), "surrogate step");
    if (st != FIB_OK) return st;
    s.step_offset = i;
    st = check_launch(c, launch_sur_net(s, stream), "surrogate network");
    if (st != FIB_OK) return st;
    c->launches += 2;
  }
  a.phases = 1;  // the last step's second diffusion half (u only)
  a.n_cn = n_cn;
  a.step_offset = n;
  st = check_launch(c, launch_split_step(c->K, false, a, c->n_ctas, stream), "diffusion");
  if (st != FIB_OK) return st;
  ++c->launches;
  return FIB_OK;
}

fib_status fib::ctx_view(fib_ctx* c, fib::CtxView* v) {
  if (!c) return fail(nullptr, FIB_EINVAL, "ctx is NULL");
  v->device = c->device;
  v->stream = c->stream;
  v->fibers = c->d_fibers;
  v->n_fibers = c->n_fibers;
  v->u = c->d_state;
  v->total = c->total;
  v->vrest = (float)c->p.Vrest;
  v->flag = c->d_flag;
  v->launches = &c->launches;
  v->n_nodes = c->n_nodes.data();
  v->h = c->p.h;
  return FIB_OK;
}

fib_status fib::ctx_fail(fib_ctx* c, fib_status s, const char* msg) { return fail(c, s, "%s", msg); }

// ===========================================================================
// C ABI
// ===========================================================================

extern "C" {

fib_status fibers_create(const fib_params* p, int32_t n_fibers, const int32_t* n_nodes, const int32_t* mu_of_fiber,
                         const int32_t* junction_node, const float* vm0, const fib_tuning* tuning, void* cuda_stream,
                         fib_ctx** out) {
  if (!out) return fail(nullptr, FIB_EINVAL, "out is NULL");
  *out = nullptr;
  fib_status st = validate(p);
  if (st != FIB_OK) return st;
  if (n_fibers < 0) return fail(nullptr, FIB_EINVAL, "n_fibers < 0");
  if (n_fibers > 0 && (!n_nodes || !mu_of_fiber || !junction_node))
    return fail(nullptr, FIB_EINVAL, "n_nodes, mu_of_fiber and junction_node are required");
  std::unique_ptr<fib_ctx> c(new (std::nothrow) fib_ctx());
  if (!c) return fail(nullptr, FIB_ENOMEM, "host allocation failed");
  c->p = *p;
  c->n_fibers = n_fibers;
  c->n_nodes.assign(n_nodes, n_nodes + n_fibers);
  c->mu.assign(mu_of_fiber, mu_of_fiber + n_fibers);
  c->junction.assign(junction_node, junction_node + n_fibers);
  c->coff.resize(n_fibers + 1);
  c->coff[0] = 0;
  for (int32_t f = 0; f < n_fibers; ++f) {
    if (c->n_nodes[f] < 1) return fail(nullptr, FIB_EINVAL, "fiber %d has %d nodes (need >= 1)", f, c->n_nodes[f]);
    if (c->junction[f] < 0 || c->junction[f] >= c->n_nodes[f])
      return fail(nullptr, FIB_EINVAL, "fiber %d: junction %d outside [0, %d)", f, c->junction[f], c->n_nodes[f]);
    if (c->mu[f] < -1) return fail(nullptr, FIB_EINVAL, "fiber %d: motor unit %d < -1", f, c->mu[f]);
    c->coff[f + 1] = c->coff[f] + c->n_nodes[f];
    c->max_n = std::max(c->max_n, c->n_nodes[f]);
  }
  c->total = c->coff[n_fibers];
  if (vm0)
    for (int64_t i = 0; i < c->total; ++i)
      if (!std::isfinite(vm0[i])) return fail(nullptr, FIB_EINVAL, "vm0[%lld] is not finite", (long long)i);

  // derived constants
  c->n_sub = (int64_t)std::nearbyint(p->dt_split / p->dt_0d);
  c->n_cn = (int64_t)std::nearbyint(diffusion_phase(p) / p->dt_1d);
  c->pulse = (int64_t)std::nearbyint(p->stim_duration / p->dt_0d);
  const double cdiff = p->sigma_eff / (p->Am * p->Cm);
  // The tables hold (I - r/2 L') with L' the unit-spaced [1 -2 1] stencil:
  // r = c dt_1d / h^2 gives the CN left-hand side, twice that the implicit
  // Euler one.
  c->r = (p->diffusion == FIB_DIFFUSION_IMPLICIT_EULER ? 2.0 : 1.0) * cdiff * p->dt_1d / (p->h * p->h);
  rest_gates(0.0, &c->m0, &c->h0, &c->n0, (p->flags & FIB_FLAG_EXP_APPROX) != 0);
  if (std::isnan(p->EL)) {
    const double ina = p->gNa * c->m0 * c->m0 * c->m0 * c->h0 * (p->Vrest - p->ENa);
    const double ik = p->gK * c->n0 * c->n0 * c->n0 * c->n0 * (p->Vrest - p->EK);
    c->EL = p->Vrest + (ina + ik) / p->gL;
  } else {
    c->EL = p->EL;
  }

  fib_ctx* cx = c.get();
  cudaError_t e = cudaGetDevice(&cx->device);
  if (e != cudaSuccess) return fail(nullptr, FIB_ECUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
  cx->stream = static_cast<cudaStream_t>(cuda_stream);
  // Reserve read_vm_static's staging array on this device now (a failure
  // here is not an error of this call: read_vm_static tries again).
  if (fib::prepare_static_stage(cx->device) != 0) cudaGetLastError();
  fib_tuning t = tuning ? *tuning : fib_tuning{0, 0, 0, 1000, 0, 0, 0};
  st = build_layout(cx, t);
  if (st == FIB_OK) {
    if ((e = cudaStreamCreateWithFlags(&cx->cap_stream, cudaStreamNonBlocking)) != cudaSuccess)
      st = fail(cx, FIB_ECUDA, "stream create: %s", cudaGetErrorString(e));
  }
  if (st == FIB_OK) {
    if ((e = cudaMalloc(&cx->d_step, sizeof(int64_t))) != cudaSuccess ||
        (e = cudaMalloc(&cx->d_flag, sizeof(int32_t))) != cudaSuccess ||
        (e = cudaMemset(cx->d_step, 0, sizeof(int64_t))) != cudaSuccess ||
        (e = cudaMemset(cx->d_flag, 0, sizeof(int32_t))) != cudaSuccess)
      st = fail(cx, e == cudaErrorMemoryAllocation ? FIB_ENOMEM : FIB_ECUDA, "allocation: %s", cudaGetErrorString(e));
  }
  if (st == FIB_OK && (p->flags & FIB_FLAG_ADAPTIVE)) {
    if ((e = cudaMalloc(&cx->d_quiet, std::max<size_t>(cx->n_fibers, 1))) != cudaSuccess ||
        (e = cudaMalloc(&cx->d_skipped, sizeof(unsigned long long))) != cudaSuccess ||
        (e = cudaMemset(cx->d_quiet, 0, std::max<size_t>(cx->n_fibers, 1))) != cudaSuccess ||
        (e = cudaMemset(cx->d_skipped, 0, sizeof(unsigned long long))) != cudaSuccess)
      st = fail(cx, e == cudaErrorMemoryAllocation ? FIB_ENOMEM : FIB_ECUDA, "allocation: %s", cudaGetErrorString(e));
  }
  float* d_vm0 = nullptr;
  if (st == FIB_OK && vm0 && cx->total > 0) {
    if ((e = cudaMalloc(&d_vm0, sizeof(float) * cx->total)) != cudaSuccess ||
        (e = cudaMemcpy(d_vm0, vm0, sizeof(float) * cx->total, cudaMemcpyHostToDevice)) != cudaSuccess)
      st = fail(cx, FIB_ECUDA, "vm0 upload: %s", cudaGetErrorString(e));
  }
  if (st == FIB_OK) {
    // gates start at rest: zero deviation in the state arrays
    st = check_launch(cx, launch_fill_layout(cx->d_fibers, cx->n_fibers, st_u(cx), st_m(cx), st_h(cx), st_n(cx), d_vm0,
                                             (float)p->Vrest, 0.0f, 0.0f, 0.0f, cx->stream),
                      "fill");
    ++cx->launches;
  }
  if (st == FIB_OK && (e = cudaStreamSynchronize(cx->stream)) != cudaSuccess)
    st = fail(cx, FIB_ECUDA, "init: %s", cudaGetErrorString(e));
  if (d_vm0) cudaFree(d_vm0);
  if (st != FIB_OK) {
    g_create_error = cx->err;
    fibers_destroy(c.release());
    return st;
  }
  *out = c.release();
  return FIB_OK;
}

fib_status set_stimulus_times(fib_ctx* c, int32_t n_mu, const int64_t* offsets, const double* fire_times_ms) {
  if (!c) return fail(nullptr, FIB_EINVAL, "ctx is NULL");
  if (n_mu < 0) return fail(c, FIB_EINVAL, "n_mu < 0");
  if (n_mu > 0 && !offsets) return fail(c, FIB_EINVAL, "offsets is NULL");
  std::vector<int64_t> off(offsets, offsets + (n_mu > 0 ? n_mu + 1 : 0));
  if (n_mu > 0 && off[0] != 0) return fail(c, FIB_EINVAL, "offsets[0] must be 0");
  for (int32_t k = 0; k < n_mu; ++k)
    if (off[k + 1] < off[k]) return fail(c, FIB_EINVAL, "offsets must be non-decreasing");
  const int64_t nf = n_mu > 0 ? off[n_mu] : 0;
  if (nf > 0 && !fire_times_ms) return fail(c, FIB_EINVAL, "fire_times_ms is NULL");
  for (int32_t f = 0; f < c->n_fibers; ++f)
    if (c->mu[f] >= n_mu) return fail(c, FIB_EINVAL, "fiber %d refers to motor unit %d >= n_mu %d", f, c->mu[f], n_mu);
  std::vector<int64_t> fk(std::max<int64_t>(nf, 1), 0);
  for (int32_t k = 0; k < n_mu; ++k)
    for (int64_t i = off[k]; i < off[k + 1]; ++i) {
      const double t = fire_times_ms[i];
      if (!std::isfinite(t) || t < 0) return fail(c, FIB_EINVAL, "fire time %lld is negative or not finite", (long long)i);
      if (i > off[k] && t < fire_times_ms[i - 1]) return fail(c, FIB_EINVAL, "fire times of MU %d are not ascending", k);
      const double q = t / c->p.dt_0d;
      if (q > 4.0e18) return fail(c, FIB_EINVAL, "fire time %g ms too large", t);
      fk[i] = (int64_t)std::nearbyint(q);  // round half to even (default rounding mode)
    }
  if (set_device(c) != FIB_OK) return FIB_ECUDA;
  CU(c, cudaStreamSynchronize(c->stream));
  dfree(c->d_mu_off);
  dfree(c->d_fire_k);
  c->n_mu = 0;
  if (n_mu > 0) {
    CU(c, cudaMalloc(&c->d_mu_off, sizeof(int64_t) * (n_mu + 1)));
    CU(c, cudaMalloc(&c->d_fire_k, sizeof(int64_t) * fk.size()));
    CU(c, cudaMemcpy(c->d_mu_off, off.data(), sizeof(int64_t) * (n_mu + 1), cudaMemcpyHostToDevice));
    CU(c, cudaMemcpy(c->d_fire_k, fk.data(), sizeof(int64_t) * fk.size(), cudaMemcpyHostToDevice));
  }
  c->n_mu = n_mu;
  if (c->graph) cudaGraphExecDestroy(c->graph);  // captured arguments changed
  c->graph = nullptr;
  return FIB_OK;
}

fib_status step(fib_ctx* c, int64_t n_steps) {
  if (!c) return fail(nullptr, FIB_EINVAL, "ctx is NULL");
  if (n_steps < 0) return fail(c, FIB_EINVAL, "n_steps < 0");
  if (n_steps == 0) return FIB_OK;
  if (set_device(c) != FIB_OK) return FIB_ECUDA;
  const bool sur = c->p.mode == FIB_MODE_SURROGATE;
  if (sur && !c->sur_loaded) return fail(c, FIB_ESTATE, "surrogate mode needs fibers_load_surrogate before step");
  const int64_t G = c->tune.graph_steps;
  if (G > 0 && n_steps >= G && c->n_ctas > 0) {
    if (!c->graph) {
      fib_status st = build_graph(c);
      if (st != FIB_OK) return st;
    }
    while (n_steps >= G) {
      CU(c, cudaGraphLaunch(c->graph, c->stream));
      c->launches += c->graph_launches;
      c->next_step += G;
      n_steps -= G;
    }
  }
  if (n_steps > 0) {
    fib_status st = sur ? surrogate_steps(c, c->stream, n_steps) : enqueue_launches(c, c->stream, 0, n_steps);
    if (st != FIB_OK) return st;
    st = check_launch(c, launch_advance(c->d_step, n_steps, c->stream), "advance");
    if (st != FIB_OK) return st;
    ++c->launches;
    c->next_step += n_steps;
  }
  return FIB_OK;
}

fib_status read_vm(fib_ctx* c, float* out, size_t capacity, int32_t out_is_device) {
  if (!c) return fail(nullptr, FIB_EINVAL, "ctx is NULL");
  if (capacity < (size_t)c->total) return fail(c, FIB_EINVAL, "capacity %zu < %lld nodes", capacity, (long long)c->total);
  if (c->total > 0 && !out) return fail(c, FIB_EINVAL, "out is NULL");
  if (set_device(c) != FIB_OK) return FIB_ECUDA;
  if (c->total > 0) {
    float* dst = out;
    if (!out_is_device) {
      fib_status st = ensure_stage(c, (size_t)c->total);
      if (st != FIB_OK) return st;
      dst = c->d_stage;
    }
    fib_status st = check_launch(c, launch_gather(c->d_fibers, c->n_fibers, st_u(c), dst, (float)c->p.Vrest, c->stream),
                                 "gather");
    if (st != FIB_OK) return st;
    ++c->launches;
    if (!out_is_device)
      CU(c, cudaMemcpyAsync(out, c->d_stage, sizeof(float) * c->total, cudaMemcpyDeviceToHost, c->stream));
  }
  CU(c, cudaStreamSynchronize(c->stream));
  return check_flag(c);
}

fib_status read_vm_async(fib_ctx* c, float* out, size_t capacity, int64_t* ticket) {
  if (!c) return fail(nullptr, FIB_EINVAL, "ctx is NULL");
  if (capacity < (size_t)c->total) return fail(c, FIB_EINVAL, "capacity %zu < %lld nodes", capacity, (long long)c->total);
  if (c->total > 0 && !out) return fail(c, FIB_EINVAL, "out is NULL");
  if (set_device(c) != FIB_OK) return FIB_ECUDA;
  if (!c->async_ready) {
    fib_status st = setup_async(c);
    if (st != FIB_OK) {
      free_async(c);
      return st;
    }
    c->async_ready = true;
  }
  const int k = (int)(c->async_issued & 1);
  // the staging buffer's previous copy must finish before the gather
  // overwrites it (a device-side wait: the host does not block)
  if (c->async_issued >= 2) CU(c, cudaStreamWaitEvent(c->stream, c->ev_copied[k], 0));
  CU(c, cudaMemsetAsync(c->d_async_flag + k, 0, sizeof(int32_t), c->stream));
  if (c->total > 0) {
    fib_status st = check_launch(c, launch_gather_checked(c->d_fibers, c->n_fibers, st_u(c), c->d_async[k],
                                                          (float)c->p.Vrest, c->d_flag, c->d_async_flag + k, c->stream),
                                 "gather");
    if (st != FIB_OK) return st;
    ++c->launches;
  } else {
    CU(c, cudaMemcpyAsync(c->d_async_flag + k, c->d_flag, sizeof(int32_t), cudaMemcpyDeviceToDevice, c->stream));
  }
  CU(c, cudaEventRecord(c->ev_gathered[k], c->stream));
  CU(c, cudaStreamWaitEvent(c->copy_stream, c->ev_gathered[k], 0));
  if (c->total > 0)
    CU(c, cudaMemcpyAsync(out, c->d_async[k], sizeof(float) * (size_t)c->total, cudaMemcpyDeviceToHost,
                          c->copy_stream));
  CU(c, cudaMemcpyAsync(c->h_async_flag + k, c->d_async_flag + k, sizeof(int32_t), cudaMemcpyDeviceToHost,
                        c->copy_stream));
  CU(c, cudaEventRecord(c->ev_copied[k], c->copy_stream));
  if (ticket) *ticket = c->async_issued;
  ++c->async_issued;
  return FIB_OK;
}

fib_status read_vm_wait(fib_ctx* c, int64_t ticket) {
  if (!c) return fail(nullptr, FIB_EINVAL, "ctx is NULL");
  if (ticket < 0 || ticket >= c->async_issued)
    return fail(c, FIB_EINVAL, "ticket %lld was not issued (%lld issued)", (long long)ticket, (long long)c->async_issued);
  if (set_device(c) != FIB_OK) return FIB_ECUDA;
  const int k = (int)(ticket & 1);
  CU(c, cudaEventSynchronize(c->ev_copied[k]));
  return flag_status(c, c->h_async_flag[k]);
}

fib_status fibers_read_state(fib_ctx* c, float* out, size_t capacity, int32_t out_is_device) {
  if (!c) return fail(nullptr, FIB_EINVAL, "ctx is NULL");
  const size_t need = 4 * (size_t)c->total;
  if (capacity < need) return fail(c, FIB_EINVAL, "capacity %zu < %zu", capacity, need);
  if (need > 0 && !out) return fail(c, FIB_EINVAL, "out is NULL");
  if (set_device(c) != FIB_OK) return FIB_ECUDA;
  if (need > 0) {
    float* dst = out;
    if (!out_is_device) {
      fib_status st = ensure_stage(c, need);
      if (st != FIB_OK) return st;
      dst = c->d_stage;
    }
    fib_status st = gather_state(c, dst);
    if (st != FIB_OK) return st;
    if (!out_is_device) CU(c, cudaMemcpyAsync(out, c->d_stage, sizeof(float) * need, cudaMemcpyDeviceToHost, c->stream));
  }
  CU(c, cudaStreamSynchronize(c->stream));
  return check_flag(c);
}

fib_status fibers_write_state(fib_ctx* c, const float* in, size_t count, int32_t in_is_device, int64_t step_index) {
  if (!c) return fail(nullptr, FIB_EINVAL, "ctx is NULL");
  const size_t need = 4 * (size_t)c->total;
  if (count != need) return fail(c, FIB_EINVAL, "count %zu != 4 * nodes = %zu", count, need);
  if (need > 0 && !in) return fail(c, FIB_EINVAL, "in is NULL");
  if (step_index < 0) return fail(c, FIB_EINVAL, "step_index < 0");
  if (set_device(c) != FIB_OK) return FIB_ECUDA;
  if (need > 0) {
    const float* src = in;
    if (!in_is_device) {
      fib_status st = ensure_stage(c, need);
      if (st != FIB_OK) return st;
      CU(c, cudaMemcpyAsync(c->d_stage, in, sizeof(float) * need, cudaMemcpyHostToDevice, c->stream));
      src = c->d_stage;
    }
    fib_status st = scatter_state(c, src);
    if (st != FIB_OK) return st;
  }
  CU(c, cudaMemcpyAsync(c->d_step, &step_index, sizeof(int64_t), cudaMemcpyHostToDevice, c->stream));
  CU(c, cudaMemsetAsync(c->d_flag, 0, sizeof(int32_t), c->stream));
  fib_status st = reset_sur_lists(c);
  if (st != FIB_OK) return st;
  CU(c, cudaStreamSynchronize(c->stream));
  c->next_step = step_index;
  return FIB_OK;
}

fib_status fibers_stats(fib_ctx* c, int64_t* steps_done, int64_t* fallback_nodes) {
  if (!c) return fail(nullptr, FIB_EINVAL, "ctx is NULL");
  if (set_device(c) != FIB_OK) return FIB_ECUDA;
  CU(c, cudaStreamSynchronize(c->stream));
  if (steps_done) *steps_done = c->next_step;
  if (fallback_nodes) {
    unsigned long long fb = 0;
    if (c->d_fallback) CU(c, cudaMemcpy(&fb, c->d_fallback, sizeof(fb), cudaMemcpyDeviceToHost));
    *fallback_nodes = (int64_t)fb;
  }
  return check_flag(c);
}

fib_status fibers_adaptive_stats(fib_ctx* c, int64_t* skipped) {
  if (!c || !skipped) return fail(c, FIB_EINVAL, "ctx or output is NULL");
  if (set_device(c) != FIB_OK) return FIB_ECUDA;
  CU(c, cudaStreamSynchronize(c->stream));
  unsigned long long v = 0;
  if (c->d_skipped) CU(c, cudaMemcpy(&v, c->d_skipped, sizeof(v), cudaMemcpyDeviceToHost));
  *skipped = (int64_t)v;
  return check_flag(c);
}

fib_status fibers_synchronize(fib_ctx* c) {
  if (!c) return fail(nullptr, FIB_EINVAL, "ctx is NULL");
  if (set_device(c) != FIB_OK) return FIB_ECUDA;
  CU(c, cudaStreamSynchronize(c->stream));
  if (c->copy_stream) CU(c, cudaStreamSynchronize(c->copy_stream));
  return check_flag(c);
}

fib_status fibers_get_tuning(const fib_ctx* c, fib_tuning* out) {
  if (!c || !out) return fail(nullptr, FIB_EINVAL, "ctx or out is NULL");
  *out = c->tune;
  return FIB_OK;
}

fib_status fibers_set_tuning(fib_ctx* c, const fib_tuning* t) {
  if (!c || !t) return fail(c, FIB_EINVAL, "ctx or tuning is NULL");
  if (set_device(c) != FIB_OK) return FIB_ECUDA;
  // keep the state across the re-layout: compact copy, rebuild, scatter back
  const size_t need = 4 * (size_t)c->total;
  float* keep = nullptr;
  if (need > 0) {
    CU(c, cudaMalloc(&keep, sizeof(float) * need));
    fib_status st = gather_state(c, keep);
    if (st != FIB_OK) {
      cudaFree(keep);
      return st;
    }
  }
  cudaError_t e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) {
    cudaFree(keep);
    return fail(c, FIB_ECUDA, "sync: %s", cudaGetErrorString(e));
  }
  const fib_tuning old = c->tune;
  fib_status st = build_layout(c, *t);
  if (st != FIB_OK) {
    const std::string why = c->err;
    if (build_layout(c, old) != FIB_OK) {
      cudaFree(keep);
      return fail(c, FIB_ECUDA, "tuning rejected (%s) and the old layout could not be restored", why.c_str());
    }
    c->err = why;
  }
  fib_status st2 = need > 0 ? scatter_state(c, keep) : FIB_OK;
  e = cudaStreamSynchronize(c->stream);
  cudaFree(keep);
  if (st2 != FIB_OK) return st2;
  if (e != cudaSuccess) return fail(c, FIB_ECUDA, "sync: %s", cudaGetErrorString(e));
  return st;
}

namespace {

// ---------------------------------------------------------------------------
// Autotune cache: the winning launch shape per (GPU model, method switches,
// r, substeps, length histogram), process-wide under a mutex, with a text
// file form.  The histogram is every distinct fiber length with its count;
// contexts with equal keys have identical layouts and identical work, so the
// stored shape is the one timing would choose again (up to timing noise).
// ---------------------------------------------------------------------------

struct TuneKey {
  std::string gpu;  // name, SM count and compute capability
  int32_t mode = 0, flags = 0, splitting = 0, diffusion = 0;
  int64_t n_sub = 0, n_cn = 0;
  double r = 0.0;
  std::vector<std::pair<int32_t, int64_t>> hist;  // (length, fibers), ascending length
  bool operator<(const TuneKey& o) const {
    return std::tie(gpu, mode, flags, splitting, diffusion, n_sub, n_cn, r, hist) <
           std::tie(o.gpu, o.mode, o.flags, o.splitting, o.diffusion, o.n_sub, o.n_cn, o.r, o.hist);
  }
};
struct TuneChoice {
  int32_t nodes_per_thread = 0, warps_per_cta = 0, reaction_pairs = 0, ctas_per_sm = 0, warp_roles = 0;
};
std::mutex g_tune_mu;
std::map<TuneKey, TuneChoice> g_tune_cache;

bool tune_key(const fib_ctx* c, TuneKey* k) {
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, c->device) != cudaSuccess) return false;
  char gpu[320];
  snprintf(gpu, sizeof(gpu), "%s|%d SMs|sm_%d%d", prop.name, prop.multiProcessorCount, prop.major, prop.minor);
  for (char* q = gpu; *q; ++q)
    if (*q == '\t' || *q == '\n') *q = ' ';
  k->gpu = gpu;
  k->mode = c->p.mode;
  k->flags = c->p.flags;
  k->splitting = c->p.splitting;
  k->diffusion = c->p.diffusion;
  k->n_sub = c->n_sub;
  k->n_cn = c->n_cn;
  k->r = c->r;
  std::map<int32_t, int64_t> h;
  for (int32_t n : c->n_nodes) ++h[n];
  k->hist.assign(h.begin(), h.end());
  return true;
}

// One line per entry, tab-separated fields:
//   gpu  mode flags splitting diffusion n_sub n_cn r(hex float)
//   K W pairs occ roles  n_lengths length:count ...
std::string tune_line(const TuneKey& k, const TuneChoice& v) {
  std::string s = k.gpu;
  char buf[256];
  snprintf(buf, sizeof(buf), "\t%d %d %d %d %lld %lld %a\t%d %d %d %d %d\t%zu", k.mode, k.flags, k.splitting,
           k.diffusion, (long long)k.n_sub, (long long)k.n_cn, k.r, v.nodes_per_thread, v.warps_per_cta,
           v.reaction_pairs, v.ctas_per_sm, v.warp_roles, k.hist.size());
  s += buf;
  for (const auto& e : k.hist) {
    snprintf(buf, sizeof(buf), " %d:%lld", e.first, (long long)e.second);
    s += buf;
  }
  return s;
}

bool parse_tune_line(const std::string& line, TuneKey* k, TuneChoice* v) {
  const size_t t1 = line.find('\t');
  if (t1 == std::string::npos || t1 == 0) return false;
  k->gpu = line.substr(0, t1);
  const char* q = line.c_str() + t1 + 1;
  long long n_sub = 0, n_cn = 0;
  int used = 0;
  if (sscanf(q, "%d %d %d %d %lld %lld %la%n", &k->mode, &k->flags, &k->splitting, &k->diffusion, &n_sub, &n_cn,
             &k->r, &used) != 7)
    return false;
  k->n_sub = n_sub;
  k->n_cn = n_cn;
  q += used;
  size_t n_len = 0;
  if (sscanf(q, " %d %d %d %d %d %zu%n", &v->nodes_per_thread, &v->warps_per_cta, &v->reaction_pairs,
             &v->ctas_per_sm, &v->warp_roles, &n_len, &used) != 6)
    return false;
  q += used;
  if (n_len == 0 || n_len > (1u << 24)) return false;
  k->hist.clear();
  int32_t prev = 0;
  for (size_t i = 0; i < n_len; ++i) {
    int len = 0;
    long long cnt = 0;
    if (sscanf(q, " %d:%lld%n", &len, &cnt, &used) != 2) return false;
    if (len <= prev || cnt <= 0) return false;  // ascending, positive
    k->hist.emplace_back(len, (int64_t)cnt);
    prev = len;
    q += used;
  }
  while (*q == ' ' || *q == '\r') ++q;
  return *q == 0;
}

}  // namespace

fib_status fibers_autotune(fib_ctx* c, int32_t n_trial_steps, fib_tuning* best) {
  if (!c) return fail(nullptr, FIB_EINVAL, "ctx is NULL");
  if (n_trial_steps < 1) return fail(c, FIB_EINVAL, "n_trial_steps must be >= 1");
  if (c->p.mode == FIB_MODE_SURROGATE)
    return fail(c, FIB_ENOTSUP, "autotune times the plain step kernel, which surrogate mode does not run");
  if (set_device(c) != FIB_OK) return FIB_ECUDA;
  TuneKey key;
  const bool keyed = tune_key(c, &key);
  if (keyed) {
    TuneChoice hit;
    bool found = false;
    {
      std::lock_guard<std::mutex> lock(g_tune_mu);
      auto it = g_tune_cache.find(key);
      if (it != g_tune_cache.end()) {
        hit = it->second;
        found = true;
      }
    }
    if (found) {
      // the cached shape, keeping this context's launch lengths
      const fib_tuning t{hit.nodes_per_thread, hit.warps_per_cta, c->tune.steps_per_launch, c->tune.graph_steps,
                         hit.reaction_pairs, hit.ctas_per_sm, hit.warp_roles};
      if (fibers_set_tuning(c, &t) == FIB_OK) {
        if (best) *best = c->tune;
        return FIB_OK;
      }
    }
  }
  const size_t need = 4 * (size_t)c->total;
  const int64_t step_keep = c->next_step;
  // the trial launches of adaptive mode count skipped fiber-steps; keep the
  // context's own count
  unsigned long long skipped_keep = 0;
  CU(c, cudaStreamSynchronize(c->stream));
  if (c->d_skipped) CU(c, cudaMemcpy(&skipped_keep, c->d_skipped, sizeof(skipped_keep), cudaMemcpyDeviceToHost));
  float* keep = nullptr;
  if (need > 0) {
    CU(c, cudaMalloc(&keep, sizeof(float) * need));
    fib_status st = gather_state(c, keep);
    if (st != FIB_OK) {
      cudaFree(keep);
      return st;
    }
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const fib_tuning start = c->tune;
  fib_tuning win = start;
  float win_ms = -1.0f;
  fib_status result = FIB_OK;
  std::vector<fib_tuning> cands;
  for (int K : {8, 12, 16}) {
    int w_max = 1;
    for (int32_t n : c->n_nodes) w_max = std::max(w_max, warps_for(n, K));
    if (w_max > kMaxWarpsPerCta) continue;
    std::vector<int> Ws{auto_W(w_max)};
    if (w_max * 2 <= kMaxWarpsPerCta && auto_W(w_max) != w_max) Ws.push_back(w_max);
    for (int W : Ws)
      for (int pairs : {1, 2})
        for (int occ : {2, 3, 4}) cands.push_back(fib_tuning{K, W, start.steps_per_launch, start.graph_steps, pairs, occ, 1});
  }
  // the two-fiber split-role shape; the eight-fiber one (warp_roles 3) was
  // slower on every workload measured and is left to explicit requests
  if (ws_eligible(c)) cands.push_back(fib_tuning{0, 0, start.steps_per_launch, start.graph_steps, 0, 0, 2});
  for (const fib_tuning& t : cands) {
    if (build_layout(c, t) != FIB_OK) continue;
    if (need > 0 && scatter_state(c, keep) != FIB_OK) continue;
    StepArgs a = make_args(c);
    a.step_offset = 0;
    a.n_steps = n_trial_steps;
    const bool fp64 = c->p.mode == FIB_MODE_FP64_THOMAS;
    auto launch = [&]() {
      return c->ws == 3 ? launch_split_step_ws8(a, c->n_ctas, c->stream)
             : c->ws ? launch_split_step_ws(a, c->n_ctas, c->stream)
                   : launch_split_step(c->K, fp64, a, c->n_ctas, c->stream);
    };
    // one warm-up launch, then the timed one
    launch();
    cudaEventRecord(e0, c->stream);
    int le = launch();
    cudaEventRecord(e1, c->stream);
    c->launches += 2;
    if (le != 0 || cudaEventSynchronize(e1) != cudaSuccess) continue;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (win_ms < 0 || ms < win_ms) {
      win_ms = ms;
      win = c->tune;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  // restore: chosen layout, saved state, step index, clean flag
  result = build_layout(c, win);
  if (result == FIB_OK && need > 0) result = scatter_state(c, keep);
  if (result == FIB_OK) {
    cudaMemcpyAsync(c->d_step, &step_keep, sizeof(int64_t), cudaMemcpyHostToDevice, c->stream);
    cudaMemsetAsync(c->d_flag, 0, sizeof(int32_t), c->stream);
    if (c->d_skipped)
      cudaMemcpyAsync(c->d_skipped, &skipped_keep, sizeof(skipped_keep), cudaMemcpyHostToDevice, c->stream);
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) result = fail(c, FIB_ECUDA, "autotune restore: %s", cudaGetErrorString(e));
  }
  cudaFree(keep);
  c->next_step = step_keep;
  if (best) *best = c->tune;
  if (win_ms < 0 && result == FIB_OK) result = fail(c, FIB_ECUDA, "autotune: no candidate ran");
  if (result == FIB_OK && keyed) {
    const TuneChoice v{c->tune.nodes_per_thread, c->tune.warps_per_cta, c->tune.reaction_pairs, c->tune.ctas_per_sm,
                       c->tune.warp_roles};
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_tune_cache[key] = v;
  }
  return result;
}

int64_t fibers_autotune_cache_size(void) {
  std::lock_guard<std::mutex> lock(g_tune_mu);
  return (int64_t)g_tune_cache.size();
}

fib_status fibers_autotune_cache_clear(void) {
  std::lock_guard<std::mutex> lock(g_tune_mu);
  g_tune_cache.clear();
  return FIB_OK;
}

fib_status fibers_autotune_cache_save(const char* path) {
  if (!path) return fail(nullptr, FIB_EINVAL, "path is NULL");
  std::string text = "fibers-autotune-cache 1\n";
  {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    for (const auto& e : g_tune_cache) text += tune_line(e.first, e.second) + "\n";
  }
  FILE* f = fopen(path, "w");
  if (!f) return fail(nullptr, FIB_EIO, "cannot open %s for writing", path);
  const bool ok = fwrite(text.data(), 1, text.size(), f) == text.size();
  if (fclose(f) != 0 || !ok) return fail(nullptr, FIB_EIO, "cannot write %s", path);
  return FIB_OK;
}

fib_status fibers_autotune_cache_load(const char* path) {
  if (!path) return fail(nullptr, FIB_EINVAL, "path is NULL");
  FILE* f = fopen(path, "r");
  if (!f) return fail(nullptr, FIB_EIO, "cannot open %s", path);
  std::string text;
  char buf[65536];
  size_t got;
  while ((got = fread(buf, 1, sizeof(buf), f)) > 0) text.append(buf, got);
  const bool read_ok = !ferror(f);
  fclose(f);
  if (!read_ok) return fail(nullptr, FIB_EIO, "cannot read %s", path);
  std::vector<std::pair<TuneKey, TuneChoice>> entries;
  size_t pos = 0, line_no = 0;
  while (pos < text.size()) {
    size_t end = text.find('\n', pos);
    if (end == std::string::npos) end = text.size();
    const std::string line = text.substr(pos, end - pos);
    pos = end + 1;
    ++line_no;
    if (line_no == 1) {
      if (line != "fibers-autotune-cache 1") return fail(nullptr, FIB_EINVAL, "%s: not an autotune cache file", path);
      continue;
    }
    if (line.empty()) continue;
    TuneKey k;
    TuneChoice v;
    if (!parse_tune_line(line, &k, &v)) return fail(nullptr, FIB_EINVAL, "%s:%zu: malformed entry", path, line_no);
    entries.emplace_back(std::move(k), v);
  }
  if (line_no == 0) return fail(nullptr, FIB_EINVAL, "%s: empty file", path);
  std::lock_guard<std::mutex> lock(g_tune_mu);
  for (auto& e : entries) g_tune_cache[std::move(e.first)] = e.second;
  return FIB_OK;
}

int64_t fibers_kernel_launches(const fib_ctx* c) { return c ? c->launches : 0; }

fib_status fibers_rest_state(const fib_params* p, float* out) {
  fib_status st = validate(p);
  if (st != FIB_OK) return st;
  if (!out) return fail(nullptr, FIB_EINVAL, "out is NULL");
  double m0, h0, n0;
  rest_gates(0.0, &m0, &h0, &n0, (p->flags & FIB_FLAG_EXP_APPROX) != 0);
  out[0] = (float)p->Vrest;
  out[1] = (float)m0;
  out[2] = (float)h0;
  out[3] = (float)n0;
  return FIB_OK;
}

fib_status fibers_solver_tables(int32_t K, double r, int32_t n_nodes, int32_t fp64_solve, int32_t* levels,
                                int32_t* threads, double* rows, double* recs) {
  if (K != 4 && K != 8 && K != 12 && K != 16) return fail(nullptr, FIB_EINVAL, "K must be 4, 8, 12 or 16");
  if (n_nodes < 1 || warps_for(n_nodes, K) > kMaxWarpsPerCta)
    return fail(nullptr, FIB_EINVAL, "n_nodes must be in [1, %d] at K = %d", 32 * kMaxWarpsPerCta * K, K);
  if (!(r >= 0.0) || !std::isfinite(r)) return fail(nullptr, FIB_EINVAL, "r must be finite and >= 0");
  const int32_t tw = 32 * warps_for(n_nodes, K);
  SolverTables tab;
  if (!build_solver_tables(K, r, {n_nodes}, {tw}, fp64_solve != 0, &tab))
    return fail(nullptr, FIB_EINVAL, "tridiagonal tables: zero pivot (r = %g)", r);
  if (levels) *levels = tab.levels;
  if (threads) *threads = tw;
  if (rows) std::copy(tab.rows.begin(), tab.rows.end(), rows);
  if (recs) std::copy(tab.recs.begin(), tab.recs.end(), recs);
  return FIB_OK;
}

const char* fibers_last_error(const fib_ctx* c) {
  if (!c) return g_create_error.c_str();
  return c->err.c_str();
}

fib_status fibers_load_surrogate(fib_ctx* c, const float* blob, size_t n_floats) {
  if (!c) return fail(nullptr, FIB_EINVAL, "ctx is NULL");
  if (c->p.mode != FIB_MODE_SURROGATE) return fail(c, FIB_ESTATE, "context was not created in surrogate mode");
  const size_t head = 3 + 2 * kIn + 2 * kOut + 4 * kIn;
  if (!blob || n_floats != head + (size_t)kNumParams)
    return fail(c, FIB_EINVAL, "surrogate blob must hold %zu floats", head + (size_t)kNumParams);
  if ((int)blob[0] != kIn || (int)blob[1] != kHid || (int)blob[2] != kOut)
    return fail(c, FIB_EINVAL, "surrogate blob shape is not 5 -> 128 -> 128 -> 4");
  for (size_t i = 0; i < n_floats; ++i)
    if (!std::isfinite(blob[i])) return fail(c, FIB_EINVAL, "surrogate blob has a non-finite value at %zu", i);
  const float* q = blob + 3;
  for (int k = 0; k < kIn; ++k) {
    c->in_mu[k] = q[k];
    if (!(q[kIn + k] > 0)) return fail(c, FIB_EINVAL, "input scale %d must be > 0", k);
    c->in_inv_sigma[k] = 1.0f / q[kIn + k];
  }
  q += 2 * kIn;
  for (int k = 0; k < kOut; ++k) {
    c->out_mu[k] = q[k];
    c->out_sigma[k] = q[kOut + k];
  }
  q += 2 * kOut;
  for (int k = 0; k < kIn; ++k) {
    c->env_lo[k] = q[k];
    c->env_hi[k] = q[kIn + k];
    c->quiet_lo[k] = q[2 * kIn + k];
    c->quiet_hi[k] = q[3 * kIn + k];
  }
  const float* th = q + 4 * kIn;
  auto bf = [](float v) {
    const __nv_bfloat16 b = __float2bfloat16_rn(v);
    return *reinterpret_cast<const uint16_t*>(&b);
  };
  const size_t n_w = (size_t)kHid * kW1Stride + (size_t)kHid * kW2Stride + 8 * (size_t)kW2Stride;
  std::vector<uint16_t> w(n_w, 0);
  uint16_t* W1 = w.data();
  uint16_t* W2 = W1 + kHid * kW1Stride;
  uint16_t* W3 = W2 + kHid * kW2Stride;
  for (int j = 0; j < kHid; ++j)
    for (int k = 0; k < kIn; ++k) {
      W1[j * kW1Stride + k] = bf(th[kOffW1 + j * kIn + k]);        // multiplies the bf16 high part
      W1[j * kW1Stride + kIn + k] = bf(th[kOffW1 + j * kIn + k]);  // and the low part of each input
    }
  for (int j = 0; j < kHid; ++j)
    for (int k = 0; k < kHid; ++k) W2[j * kW2Stride + k] = bf(th[kOffW2 + j * kHid + k]);
  for (int i = 0; i < kOut; ++i)
    for (int k = 0; k < kHid; ++k) W3[i * kW2Stride + k] = bf(th[kOffW3 + i * kHid + k]);
  std::vector<float> bias(2 * kHid + 8, 0.0f);
  for (int j = 0; j < kHid; ++j) {
    bias[j] = th[kOffB1 + j];
    bias[kHid + j] = th[kOffB2 + j];
  }
  for (int i = 0; i < kOut; ++i) bias[2 * kHid + i] = th[kOffB3 + i];
  if (set_device(c) != FIB_OK) return FIB_ECUDA;
  CU(c, cudaStreamSynchronize(c->stream));
  if (!c->d_sur_wts) CU(c, cudaMalloc(&c->d_sur_wts, sizeof(uint16_t) * n_w));
  if (!c->d_sur_bias) CU(c, cudaMalloc(&c->d_sur_bias, sizeof(float) * bias.size()));
  if (!c->d_fallback) {
    CU(c, cudaMalloc(&c->d_fallback, sizeof(unsigned long long)));
    CU(c, cudaMemset(c->d_fallback, 0, sizeof(unsigned long long)));
  }
  CU(c, cudaMemcpy(c->d_sur_wts, w.data(), sizeof(uint16_t) * n_w, cudaMemcpyHostToDevice));
  CU(c, cudaMemcpy(c->d_sur_bias, bias.data(), sizeof(float) * bias.size(), cudaMemcpyHostToDevice));
  CU(c, (cudaError_t)sur_set_smem_attributes());
  c->sur_loaded = true;
  if (c->graph) cudaGraphExecDestroy(c->graph);  // captured normalisation and envelope changed
  c->graph = nullptr;
  return FIB_OK;
}

fib_status fibers_hh_reaction(const fib_params* p, int64_t count, const float* in, const uint8_t* stim_mask,
                              float* out, void* cuda_stream) {
  fib_status st = validate(p);
  if (st != FIB_OK) return st;
  if (count < 0 || (count > 0 && (!in || !out))) return fail(nullptr, FIB_EINVAL, "bad count or NULL buffer");
  const double EL = std::isnan(p->EL) ? exact_leak_reversal(*p) : p->EL;
  const int n_sub = (int)std::nearbyint(p->dt_split / p->dt_0d);
  if (n_sub > 8) return fail(nullptr, FIB_EINVAL, "the reaction kernel handles at most 8 substeps per split step");
  const int e = launch_hh_reaction(hh_const(*p, EL), (float)p->Vrest, n_sub, count, in, stim_mask, out, cuda_stream);
  if (e) return fail(nullptr, FIB_ECUDA, "reaction kernel: %s", cudaGetErrorString((cudaError_t)e));
  return FIB_OK;
}

fib_status fibers_mlp_train_step(const float* theta, int32_t quantize, const float* x, const float* target,
                                 int64_t batch, float* workspace, float* grad, float* loss, void* cuda_stream) {
  if (batch < 1 || !theta || !x || !target || !workspace || !grad || !loss)
    return fail(nullptr, FIB_EINVAL, "bad batch or NULL buffer");
  int e = sur_set_smem_attributes();
  if (!e) e = launch_mlp_train_step(theta, quantize, x, target, batch, workspace, grad, loss, cuda_stream);
  if (e) return fail(nullptr, FIB_ECUDA, "training kernels: %s", cudaGetErrorString((cudaError_t)e));
  return FIB_OK;
}

fib_status fibers_mlp_forward(const float* theta, int32_t quantize, const float* x, int64_t batch, float* workspace,
                              float* out, void* cuda_stream) {
  if (batch < 1 || !theta || !x || !workspace || !out) return fail(nullptr, FIB_EINVAL, "bad batch or NULL buffer");
  int e = sur_set_smem_attributes();
  if (!e) e = launch_mlp_forward(theta, quantize, x, batch, workspace, out, cuda_stream);
  if (e) return fail(nullptr, FIB_ECUDA, "forward kernel: %s", cudaGetErrorString((cudaError_t)e));
  return FIB_OK;
}

fib_status fibers_adam_step(float* theta, float* m, float* v, const float* grad, int64_t n, float lr, float beta1,
                            float beta2, float eps, int64_t t, float* theta_avg, float avg_decay, void* cuda_stream) {
  if (n < 1 || t < 1 || !theta || !m || !v || !grad) return fail(nullptr, FIB_EINVAL, "bad size, step or buffer");
  if (theta_avg && !(avg_decay >= 0.0f && avg_decay <= 1.0f))
    return fail(nullptr, FIB_EINVAL, "avg_decay must be in [0, 1]");
  const int e = launch_adam(theta, m, v, grad, n, lr, beta1, beta2, eps, t, theta_avg, avg_decay, cuda_stream);
  if (e) return fail(nullptr, FIB_ECUDA, "adam kernel: %s", cudaGetErrorString((cudaError_t)e));
  return FIB_OK;
}

fib_status fibers_feature_stats(const float* X, int64_t n, int32_t cols, double* out, void* cuda_stream) {
  if (n < 1 || cols < 1 || cols > 64 || !X || !out) return fail(nullptr, FIB_EINVAL, "bad size or buffer");
  double* d = nullptr;
  cudaError_t e = cudaMalloc(&d, sizeof(double) * 4 * cols);
  if (e != cudaSuccess) return fail(nullptr, FIB_ENOMEM, "stats buffer: %s", cudaGetErrorString(e));
  int le = launch_stats(X, n, cols, d, cuda_stream);
  if (!le) e = cudaMemcpyAsync(out, d, sizeof(double) * 4 * cols, cudaMemcpyDeviceToHost, (cudaStream_t)cuda_stream);
  if (!le && e == cudaSuccess) e = cudaStreamSynchronize((cudaStream_t)cuda_stream);
  cudaFree(d);
  if (le) return fail(nullptr, FIB_ECUDA, "stats kernel: %s", cudaGetErrorString((cudaError_t)le));
  if (e != cudaSuccess) return fail(nullptr, FIB_ECUDA, "stats: %s", cudaGetErrorString(e));
  return FIB_OK;
}

void fibers_destroy(fib_ctx* c) {
  if (!c) return;
  cudaSetDevice(c->device);
  if (c->stream) cudaStreamSynchronize(c->stream);
  free_async(c);
  free_layout(c);
  dfree(c->d_mu_off);
  dfree(c->d_fire_k);
  dfree(c->d_step);
  dfree(c->d_flag);
  dfree(c->d_quiet);
  dfree(c->d_skipped);
  dfree(c->d_stage);
  dfree(c->d_sur_wts);
  dfree(c->d_sur_bias);
  dfree(c->d_fallback);
  if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
  delete c;
}

}  // extern "C"
