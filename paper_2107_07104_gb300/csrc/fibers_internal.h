// Internal types shared by the host library and the sm_103a kernels.
// Nothing here is part of the public ABI (include/fibers.h).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

#include "fibers.h"

namespace fib {

// Per-row coefficients of the partitioned tridiagonal solve (see
// solver_tables.cpp): F1 = 1/den, F2 = a/den (forward elimination),
// G = gamma (back substitution), Ap = alpha', Bt = beta (recovery).
constexpr int kCoefPerRow = 5;
// Per-thread record: 1/B, A/B, C/B, c0, kE, kD, kDn, then (ib, ka, kc) per
// cyclic-reduction level.
constexpr int kRecBase = 7;
constexpr int kRecPerLevel = 3;
constexpr int kMaxFibersPerCta = 15;  // named barriers 1..15 (0 is __syncthreads)
constexpr int kMaxWarpsPerCta = 8;    // 256 threads: the kernels' launch bound
constexpr int kMaxLevels = 12;
// Shape of the split-role kernel (split_step_ws.cu): a fiber's slot of
// kWsSlot nodes is covered by kWsReactWarps reaction warps of kWsKR nodes
// per lane, and by the diffusion warps at kWsKC nodes per lane; a CTA holds
// two fibers and kWsMinBlocks CTAs share an SM.
constexpr int kWsSlot = 1536;
constexpr int kWsReactWarps = 12;
constexpr int kWsKR = 4;
constexpr int kWsKC = 12;
constexpr int kWsMinBlocks = 2;
constexpr int kWsCnThreads = kWsSlot / kWsKC;
constexpr int kWsWarps = kWsReactWarps + kWsCnThreads / 32;
static_assert(32 * kWsReactWarps * kWsKR == kWsSlot, "reaction warps cover the slot");
static_assert(kWsCnThreads * kWsKC == kWsSlot && kWsCnThreads % 32 == 0, "diffusion warps cover the slot");
static_assert(kWsKR % 4 == 0 && kWsKC % 4 == 0, "slot rows move as float4");
static_assert(kWsReactWarps * 32 >= kWsCnThreads, "the CTA stages both fibers' tables");

struct FiberDesc {
  int64_t slot;      // index of node 0 in the padded state arrays
  int64_t coff;      // index of node 0 in ragged (compact) order
  int64_t rec;       // offset (elements) of the fiber's per-thread records
  int32_t n;         // nodes
  int32_t junction;  // junction node
  int32_t mu;        // motor unit, -1 = never stimulated
  int32_t last_set;  // offset (elements) of the last-chunk row set
  int32_t slot_len;  // padded nodes of the slot (32 * warps * K)
  int32_t pad;
};

struct WarpMap {       // one entry per warp of every CTA
  int32_t fiber;       // -1: idle warp
  int16_t first_warp;  // first warp of that fiber in the CTA
  int16_t n_warps;     // warps of that fiber
  int32_t slot;        // fiber index within the CTA (barrier id = slot + 1)
  int32_t pad;
};

struct HHConst {  // Hodgkin-Huxley constants in the depolarisation u = V - Vrest
  float gNa, gK, gL;  // conductances / Cm
  float uNa, uK, uL;  // reversal potentials - Vrest
  float stim;         // stimulus amplitude / Cm
  float dt0;          // Heun substep width
  float gNa_uNa, gK_uK, gL_uL;  // products of the above, rounded once from FP64
  // The state arrays hold each gate as its deviation from the resting value
  // (g - g0), as u holds V - Vrest: near rest FP32 then resolves the slow
  // gates' relaxation, which in absolute form stalls once an increment falls
  // below half an ulp of g.  Zero for callers whose gates are absolute.
  float m0, h0, n0;
};


struct StepArgs {
  float* u;  // SoA state in the padded layout; u = V - Vrest
  float* m;
  float* h;
  float* n;
  const FiberDesc* fibers;
  const WarpMap* warps;    // n_ctas * W entries
  const void* rows;        // row sets (float or double): interior set at 0
  const void* recs;        // per-thread records (float or double)
  const int64_t* mu_off;   // [n_mu + 1]
  const int64_t* fire_k;   // firing substep index, sorted within each MU
  const int64_t* step_base;  // device-resident index of the next split step
  int32_t* flag;           // bit 0: non-finite state seen; bit 1: surrogate node list overflowed;
                           // bit 2: a bounded wait between warp roles gave up
  HHConst hh;
  double r;                // tridiagonal-table parameter: c dt_1d / h^2 (CN), 2 c dt_1d / h^2 (IE)
  int64_t step_offset;     // this launch starts at *step_base + step_offset
  int32_t n_steps;         // split steps in this launch
  int32_t n_sub;           // Heun substeps per split step
  // One split step runs: reaction substeps [0, k_split), n_cn diffusion
  // steps, reaction substeps [k_split, n_sub), n_cn2 diffusion steps.
  int32_t k_split;
  int32_t n_cn;            // diffusion steps of the first diffusion phase
  int32_t n_cn2;           // diffusion steps of the second diffusion phase
  int32_t implicit_euler;  // 1: right-hand side u (eq:lumping_implicit_euler_2); 0: CN
  int32_t exp_approx;      // 1: rates with exp* (eq:apx-e-function), FP32 solve only
  int32_t pulse;           // stimulus length in substeps
  int32_t hw;              // stimulus half width (nodes)
  int32_t n_mu;
  int32_t n_levels;        // cyclic-reduction levels kept
  int32_t rec_stride;      // elements per thread record
  int32_t W;               // warps per CTA
  int32_t packed;          // 1: reaction step on node pairs with FP32x2 arithmetic
  int32_t occ;             // the kernel's register budget, as CTAs of 256 threads per SM (2, 3 or 4)
  int32_t phases;          // bit 0: first diffusion phase, bit 1: reaction, bit 2: second diffusion phase
  // adaptive computation: skip fibers in equilibrium with no pulse due
  uint8_t* quiet;          // per fiber: 1 = passed the equilibrium test at the end of its last launch
  unsigned long long* skipped;  // fiber-steps skipped
  int32_t adaptive;
  float eq_tol;            // relative change that still counts as equilibrium
  // surrogate mode (SUR instantiations, one split step per launch): nodes
  // outside the envelope or inside the quiet box take the plain step here;
  // the others are listed with their state before the reaction, for the
  // network pass, which overwrites them
  float* sur_list;         // per parity 6 arrays of sur_cap: slot (int bits), u, m, h, n, stimulus fraction
  unsigned int* sur_count; // [2] entries listed, by step parity
  int64_t sur_cap;
  float sur_env_lo[5], sur_env_hi[5], sur_quiet_lo[5], sur_quiet_hi[5];
  float inv_n_sub;
  float vrest;             // resting potential (the test uses V = u + Vrest)
  int32_t n_fib;           // fibers of the context (split-role kernel: two per CTA)
};

// Host-built solver tables for one (K, r, fiber-length set).
struct SolverTables {
  int K = 0;
  int levels = 0;
  int rec_stride = 0;
  std::vector<double> rows;         // [interior set][class 0 last set]...
  std::vector<double> recs;         // per class: threads x rec_stride
  std::vector<int64_t> class_last;  // offset of each class's last set in rows
  std::vector<int64_t> class_rec;   // offset of each class's records in recs
};

// Builds the tables for fiber lengths `lengths` (distinct values, one class
// each), K nodes per thread, threads_per_class[i] threads for class i, and
// CN coefficient r; fp64_solve selects the PCR cutoff of the FP64 solve.
// Returns false on a zero pivot.
bool build_solver_tables(int K, double r, const std::vector<int32_t>& lengths,
                         const std::vector<int32_t>& threads_per_class, bool fp64_solve, SolverTables* out);

// Device entry points (split_step.cu).
int launch_split_step(int K, bool fp64_solve, const StepArgs& a, int n_ctas, void* stream);
// The exp* instantiations (split_step_expapx.cu) and the adaptive ones
// (split_step_adaptive.cu).
int launch_split_step_expapx(int K, const StepArgs& a, int n_ctas, void* stream);
int launch_split_step_adaptive(int K, bool fp64_solve, const StepArgs& a, int n_ctas, void* stream);
// Split roles (split_step_ws.cu): reaction and diffusion warps, two fibers
// of at most kWsSlot nodes per CTA, tables for K = kWsKC.
int launch_split_step_ws(const StepArgs& a, int n_ctas, void* stream);
size_t split_step_ws_smem_bytes();
// Surrogate mode's split step (one per launch) with the network-node list
// (surrogate.cu).
int launch_split_step_sur(int K, const StepArgs& a, int n_ctas, void* stream);
int launch_advance(int64_t* step_base, int64_t n, void* stream);
// dst[coff + i] = src[slot + i] + add for the n real nodes of every fiber.
int launch_gather(const FiberDesc* fibers, int32_t n_fibers, const float* src, float* dst,
                  float add, void* stream);
// launch_gather that also ORs into *out_flag bit 0 for a non-finite value and
// the step kernels' error bits (*kflag).
int launch_gather_checked(const FiberDesc* fibers, int32_t n_fibers, const float* src, float* dst, float add,
                          const int32_t* kflag, int32_t* out_flag, void* stream);
// dst[slot + i] = src[coff + i] + add for real nodes; padding nodes keep dst.
int launch_scatter(const FiberDesc* fibers, int32_t n_fibers, const float* src, float* dst,
                   float add, void* stream);
// Fills every slot: u = vm0 - vrest on real nodes (0 without vm0 and on
// padding), gates = (m0, h0, n0) everywhere (the contexts pass zeros: their
// state holds gate deviations from rest).
int launch_fill_layout(const FiberDesc* fibers, int32_t n_fibers, float* u, float* m, float* h,
                       float* n, const float* vm0_compact, float vrest, float m0, float h0, float n0,
                       void* stream);
size_t split_step_smem_bytes(int K, bool fp64_solve, int W, bool adaptive);

}  // namespace fib

// Read-only view of a context for entry points outside fibers_api.cu.
struct fib_ctx;
namespace fib {
struct CtxView {
  int device;
  cudaStream_t stream;
  const FiberDesc* fibers;
  int32_t n_fibers;
  const float* u;       // depolarisation array of the padded layout
  int64_t total;        // real nodes
  float vrest;
  const int32_t* flag;  // device non-finite flag
  int64_t* launches;    // the context's kernel-launch counter
  const int32_t* n_nodes;  // host: nodes of every fiber (ragged order)
  double h;             // mesh width along the fibers (cm)
};
fib_status ctx_view(fib_ctx* c, CtxView* out);
fib_status ctx_fail(fib_ctx* c, fib_status s, const char* msg);
// Looks up read_vm_static's staging array on `device` (which must be
// current), loading its module and so reserving the array now rather than
// inside the first read_vm_static call.  Returns a cudaError_t.
int prepare_static_stage(int device);
}  // namespace fib
