// Learned surrogate of the 0D reaction step (the Heun substeps of the HH model
// inside one Strang split step, eq:monodomain_strang / eq:heun).  The thesis
// has no learned component on this path; these kernels implement the
// surrogate the build adds:
//   * hh_reaction_kernel: the plain reaction step on independent nodes, which
//     generates training targets and serves as the per-node fallback;
//   * training kernels (FP32 master weights, optional bfloat16 rounding of
//     weights and activations in the forward pass, straight-through
//     gradients) and an Adam update;
//   * the surrogate step: the split-step kernel (SUR instantiations, in this
//     file) integrates every node with the plain HH step and lists the nodes
//     inside the training data's range and away from rest; sur_net_kernel
//     evaluates the listed nodes on BF16 tensor cores (mma.sync m16n8k16,
//     FP32 accumulation) in full tiles of 16 and writes them over.
// Network: x (5) -> 128 -> SiLU -> 128 -> SiLU -> 4, predicting the change of
// (u, m, h, n) over one split step in normalised units.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "fibers_internal.h"
#include "hh_device.cuh"
#include "split_step_kernel.cuh"
#include "surrogate_internal.h"

namespace fib {
namespace {

constexpr int kFwdSmem = 4 * (kHid * kHid + kOut * kHid + 2 * kHid);
constexpr int kBwdSmem = 4 * (kHid * kHid + kOut * kHid + kOut + kHid);

__device__ __forceinline__ float silu(float z) { return z * rcp_approx(1.0f + ex2_approx(-kLog2e * z)); }
__device__ __forceinline__ float silu_grad(float z) {
  const float s = 1.0f / (1.0f + __expf(-z));
  return s * (1.0f + z * (1.0f - s));
}
__device__ __forceinline__ float q_bf16(float x, int quantize) {
  return quantize ? __bfloat162float(__float2bfloat16_rn(x)) : x;
}

// ---------------------------------------------------------------------------
// Plain reaction step on independent nodes (targets and fallback)
// ---------------------------------------------------------------------------

// Heun substeps of one node with the stimulus on for substeps whose bit is
// set in `mask`.  Same arithmetic as the split-step kernel's reaction phase.
__device__ __forceinline__ void reaction_node(float& u, float& m, float& h, float& n, uint32_t mask, int n_sub,
                                              const HHConst& c) {
  float uu[1] = {u}, mm[1] = {m}, hh[1] = {h}, nn[1] = {n};
  for (int k = 0; k < n_sub; ++k) {
    if ((mask >> k) & 1u) heun_nodes<1, true>(uu, mm, hh, nn, c, 1u);
    else heun_nodes<1, false>(uu, mm, hh, nn, c, 0u);
  }
  u = uu[0];
  m = mm[0];
  h = hh[0];
  n = nn[0];
}

__global__ void hh_reaction_kernel(HHConst c, float vrest, int n_sub, int64_t count, const float* in,
                                   const uint8_t* stim, float* out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x) {
    float u = in[i] - vrest, m = in[count + i], h = in[2 * count + i], n = in[3 * count + i];
    reaction_node(u, m, h, n, stim ? stim[i] : 0u, n_sub, c);
    out[i] = u + vrest;
    out[count + i] = m;
    out[2 * count + i] = h;
    out[3 * count + i] = n;
  }
}

// ---------------------------------------------------------------------------
// Training kernels (one CTA of 128 threads per sample for the per-sample
// passes; one thread per weight for the reductions over the batch)
// ---------------------------------------------------------------------------

// Forward pass of a chunk of samples per CTA.  W2 is staged transposed in
// shared memory (thread j reads column j: conflict-free), rounded to bf16
// when quantising.
__global__ void __launch_bounds__(kHid) mlp_fwd_kernel(const float* __restrict__ th, int quantize,
                                                       const float* __restrict__ x, int64_t B, float* z1, float* a1,
                                                       float* z2, float* a2, float* out) {
  extern __shared__ float sm[];
  float* sW2T = sm;                    // [k][j]
  float* sW3 = sW2T + kHid * kHid;     // [i][k]
  float* s_a1 = sW3 + kOut * kHid;
  float* s_a2 = s_a1 + kHid;
  const int j = threadIdx.x;
  const float* W1 = th + kOffW1;
  const float* b1 = th + kOffB1;
  const float* W2 = th + kOffW2;
  const float* b2 = th + kOffB2;
  const float* W3 = th + kOffW3;
  const float* b3 = th + kOffB3;
  for (int i = j; i < kHid * kHid; i += kHid) sW2T[(i % kHid) * kHid + i / kHid] = q_bf16(W2[i], quantize);
  for (int i = j; i < kOut * kHid; i += kHid) sW3[i] = q_bf16(W3[i], quantize);
  float w1[kIn];
  for (int k = 0; k < kIn; ++k) w1[k] = q_bf16(W1[j * kIn + k], quantize);
  __syncthreads();
  for (int64_t b = blockIdx.x; b < B; b += gridDim.x) {
    float acc = b1[j];
    for (int k = 0; k < kIn; ++k) acc += w1[k] * q_bf16(x[b * kIn + k], quantize);
    z1[b * kHid + j] = acc;
    const float v1 = q_bf16(acc / (1.0f + __expf(-acc)), quantize);
    a1[b * kHid + j] = v1;
    s_a1[j] = v1;
    __syncthreads();
    acc = b2[j];
    for (int k = 0; k < kHid; ++k) acc += sW2T[k * kHid + j] * s_a1[k];
    z2[b * kHid + j] = acc;
    const float v2 = q_bf16(acc / (1.0f + __expf(-acc)), quantize);
    a2[b * kHid + j] = v2;
    s_a2[j] = v2;
    __syncthreads();
    if (j < kOut) {
      float o = b3[j];
      for (int k = 0; k < kHid; ++k) o += sW3[j * kHid + k] * s_a2[k];
      out[b * kOut + j] = o;
    }
    __syncthreads();
  }
}

// Per-sample backward: d(out) of the mean-squared error, then dz2 and dz1.
// W2 is staged row-major (thread j reads column j of row i: conflict-free).
__global__ void __launch_bounds__(kHid) mlp_bwd_kernel(const float* __restrict__ th, int quantize, int64_t B,
                                                       const float* z1, const float* z2, const float* out,
                                                       const float* target, float* dout, float* dz1, float* dz2) {
  extern __shared__ float sm[];
  float* sW2 = sm;                     // [i][j]
  float* sW3 = sW2 + kHid * kHid;      // [i][k]
  float* s_do = sW3 + kOut * kHid;
  float* s_dz2 = s_do + kOut;
  const int j = threadIdx.x;
  const float* W2 = th + kOffW2;
  const float* W3 = th + kOffW3;
  for (int i = j; i < kHid * kHid; i += kHid) sW2[i] = q_bf16(W2[i], quantize);
  for (int i = j; i < kOut * kHid; i += kHid) sW3[i] = q_bf16(W3[i], quantize);
  __syncthreads();
  const float scale = 2.0f / (float)(B * kOut);
  for (int64_t b = blockIdx.x; b < B; b += gridDim.x) {
    if (j < kOut) {
      const float d = scale * (out[b * kOut + j] - target[b * kOut + j]);
      s_do[j] = d;
      dout[b * kOut + j] = d;
    }
    __syncthreads();
    float da2 = 0.0f;
    for (int i = 0; i < kOut; ++i) da2 += s_do[i] * sW3[i * kHid + j];
    const float g2 = da2 * silu_grad(z2[b * kHid + j]);
    dz2[b * kHid + j] = g2;
    s_dz2[j] = g2;
    __syncthreads();
    float da1 = 0.0f;
    for (int i = 0; i < kHid; ++i) da1 += s_dz2[i] * sW2[i * kHid + j];
    dz1[b * kHid + j] = da1 * silu_grad(z1[b * kHid + j]);
    __syncthreads();
  }
}

// grad(W)[r, k] = sum_b D[b, r] X[b, k] (rows x cols weights), grad(b)[r] = sum_b D[b, r].
__global__ void wgrad_kernel(const float* D, int rows, const float* X, int cols, int64_t B, int quantize_x,
                             float* gW, float* gb) {
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t nW = (int64_t)rows * cols;
  if (idx < nW) {
    const int r = (int)(idx / cols), k = (int)(idx % cols);
    float acc = 0.0f;
    for (int64_t b = 0; b < B; ++b) acc += D[b * rows + r] * q_bf16(X[b * cols + k], quantize_x);
    gW[idx] = acc;
  } else if (idx < nW + rows) {
    const int r = (int)(idx - nW);
    float acc = 0.0f;
    for (int64_t b = 0; b < B; ++b) acc += D[b * rows + r];
    gb[r] = acc;
  }
}

__global__ void mse_kernel(const float* out, const float* target, int64_t n, float* loss) {
  __shared__ float part[256];
  float acc = 0.0f;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
    const float d = out[i] - target[i];
    acc += d * d;
  }
  part[threadIdx.x] = acc;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) part[threadIdx.x] += part[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) *loss = part[0] / (float)n;
}

__global__ void adam_kernel(float* th, float* m, float* v, const float* g, int64_t n, float lr, float b1, float b2,
                            float eps, float c1, float c2, float* avg, float d) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float mi = b1 * m[i] + (1.0f - b1) * g[i];
    const float vi = b2 * v[i] + (1.0f - b2) * g[i] * g[i];
    m[i] = mi;
    v[i] = vi;
    const float ti = th[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    th[i] = ti;
    if (avg != nullptr) avg[i] = d * avg[i] + (1.0f - d) * ti;  // exponential weight average
  }
}

// Column statistics of an (n x 5) feature matrix: mean, std, min, max (FP64).
__global__ void stats_kernel(const float* X, int64_t n, int cols, double* out) {
  __shared__ double s1[256], s2[256], mn[256], mx[256];
  const int c = blockIdx.x;
  double a = 0, b = 0, lo = 1e300, hi = -1e300;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
    const double v = X[i * cols + c];
    a += v;
    b += v * v;
    lo = v < lo ? v : lo;
    hi = v > hi ? v : hi;
  }
  s1[threadIdx.x] = a;
  s2[threadIdx.x] = b;
  mn[threadIdx.x] = lo;
  mx[threadIdx.x] = hi;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      s1[threadIdx.x] += s1[threadIdx.x + s];
      s2[threadIdx.x] += s2[threadIdx.x + s];
      mn[threadIdx.x] = mn[threadIdx.x + s] < mn[threadIdx.x] ? mn[threadIdx.x + s] : mn[threadIdx.x];
      mx[threadIdx.x] = mx[threadIdx.x + s] > mx[threadIdx.x] ? mx[threadIdx.x + s] : mx[threadIdx.x];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double mean = s1[0] / (double)n;
    const double var = s2[0] / (double)n - mean * mean;
    out[4 * c + 0] = mean;
    out[4 * c + 1] = var > 0 ? sqrt(var) : 0.0;
    out[4 * c + 2] = mn[0];
    out[4 * c + 3] = mx[0];
  }
}

// ---------------------------------------------------------------------------
// Inference on BF16 tensor cores
// ---------------------------------------------------------------------------

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);  // .x = lo (low half), .y = hi
  return *reinterpret_cast<const uint32_t*>(&v);
}

// D = A (16x16 bf16, row) * B (16x8 bf16, col) + C, FP32 accumulate.
__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// Bias + SiLU on the accumulators of two adjacent n-tiles, packed into one
// bf16 A fragment of the next layer (a C fragment of m16n8 pairs maps onto
// the A fragment of m16k16).
__device__ __forceinline__ void to_a_frag(const float (&c0)[4], const float (&c1)[4], const float* bias0,
                                          const float* bias1, int t, uint32_t (&a)[4]) {
  const float b00 = bias0[2 * t], b01 = bias0[2 * t + 1], b10 = bias1[2 * t], b11 = bias1[2 * t + 1];
  a[0] = pack_bf16(silu(c0[0] + b00), silu(c0[1] + b01));
  a[1] = pack_bf16(silu(c0[2] + b00), silu(c0[3] + b01));
  a[2] = pack_bf16(silu(c1[0] + b10), silu(c1[1] + b11));
  a[3] = pack_bf16(silu(c1[2] + b10), silu(c1[3] + b11));
}

// Per-warp staging of one tile of network nodes: normalised features, the
// state before the step, and the slot.
constexpr int kTileRows = 16;
constexpr int kStageFloats = kTileRows * (kIn + 4 + 1);
constexpr int kSurThreads = 128;

// Inference tile: rows g and g + 8 of 16 staged nodes starting at `base`.
__device__ __forceinline__ void network_tile(const SurArgs& a, const uint16_t* sW1, const uint16_t* sW2,
                                             const uint16_t* sW3, const float* sB, const float* sx, const float* sy,
                                             const int* sq, int base, int count, int g, int t) {
  const int r0 = base + g, r1 = base + g + 8;
  const bool ok0 = r0 < count, ok1 = r1 < count;
  // features split into bf16 hi + lo parts (FP32-accurate inputs)
  auto feat = [&](int r, bool ok, int col) -> float {
    if (!ok || col >= 2 * kIn) return 0.0f;
    const float x = sx[r * kIn + (col < kIn ? col : col - kIn)];
    const float hi = __bfloat162float(__float2bfloat16_rn(x));
    return col < kIn ? hi : x - hi;
  };
  uint32_t A1[4];
  A1[0] = pack_bf16(feat(r0, ok0, 2 * t), feat(r0, ok0, 2 * t + 1));
  A1[1] = pack_bf16(feat(r1, ok1, 2 * t), feat(r1, ok1, 2 * t + 1));
  A1[2] = pack_bf16(feat(r0, ok0, 2 * t + 8), feat(r0, ok0, 2 * t + 9));
  A1[3] = pack_bf16(feat(r1, ok1, 2 * t + 8), feat(r1, ok1, 2 * t + 9));
  // layer 1: 16 n-tiles of 8 neurons, one k-tile
  uint32_t A2[8][4];
#pragma unroll
  for (int kk = 0; kk < 8; ++kk) {
    float c0[4] = {0, 0, 0, 0}, c1[4] = {0, 0, 0, 0};
    const uint32_t* w0 = reinterpret_cast<const uint32_t*>(sW1 + (16 * kk + g) * kW1Stride);
    const uint32_t* w1 = reinterpret_cast<const uint32_t*>(sW1 + (16 * kk + 8 + g) * kW1Stride);
    mma_bf16(c0, A1, w0[t], w0[t + 4]);
    mma_bf16(c1, A1, w1[t], w1[t + 4]);
    to_a_frag(c0, c1, sB + 16 * kk, sB + 16 * kk + 8, t, A2[kk]);
  }
  // layer 2: 16 n-tiles, 8 k-tiles
  uint32_t A3[8][4];
#pragma unroll
  for (int kk = 0; kk < 8; ++kk) {
    float c0[4] = {0, 0, 0, 0}, c1[4] = {0, 0, 0, 0};
    const uint32_t* w0 = reinterpret_cast<const uint32_t*>(sW2 + (16 * kk + g) * kW2Stride);
    const uint32_t* w1 = reinterpret_cast<const uint32_t*>(sW2 + (16 * kk + 8 + g) * kW2Stride);
#pragma unroll
    for (int k2 = 0; k2 < 8; ++k2) {
      mma_bf16(c0, A2[k2], w0[8 * k2 + t], w0[8 * k2 + t + 4]);
      mma_bf16(c1, A2[k2], w1[8 * k2 + t], w1[8 * k2 + t + 4]);
    }
    to_a_frag(c0, c1, sB + kHid + 16 * kk, sB + kHid + 16 * kk + 8, t, A3[kk]);
  }
  // layer 3: one n-tile (4 outputs padded to 8), 8 k-tiles
  float o[4] = {0, 0, 0, 0};
  {
    const uint32_t* w = reinterpret_cast<const uint32_t*>(sW3 + g * kW2Stride);
#pragma unroll
    for (int k2 = 0; k2 < 8; ++k2) mma_bf16(o, A3[k2], w[8 * k2 + t], w[8 * k2 + t + 4]);
  }
  // lane t = 0 holds outputs 0, 1 (du, dm) and t = 1 outputs 2, 3 (dh, dn)
  // of rows r0 (o[0], o[1]) and r1 (o[2], o[3])
  if (t < 2) {
    const int k0 = 2 * t, k1 = 2 * t + 1;
    const float b0 = sB[2 * kHid + k0], b1 = sB[2 * kHid + k1];
    float* dst0 = k0 == 0 ? a.u : a.h;
    float* dst1 = k1 == 1 ? a.m : a.n;
    // the listed state is absolute; the arrays hold gates as deviations from rest
    const float off0 = a.rest[k0], off1 = a.rest[k1];
    if (ok0) {
      const int64_t q = sq[r0];
      dst0[q] = (sy[r0 * 4 + k0] + fmaf(o[0] + b0, a.out_sigma[k0], a.out_mu[k0])) - off0;
      dst1[q] = (sy[r0 * 4 + k1] + fmaf(o[1] + b1, a.out_sigma[k1], a.out_mu[k1])) - off1;
    }
    if (ok1) {
      const int64_t q = sq[r1];
      dst0[q] = (sy[r1 * 4 + k0] + fmaf(o[2] + b0, a.out_sigma[k0], a.out_mu[k0])) - off0;
      dst1[q] = (sy[r1 * 4 + k1] + fmaf(o[3] + b1, a.out_sigma[k1], a.out_mu[k1])) - off1;
    }
  }
}

// Network pass of a surrogate split step: the nodes the step kernel listed
// (with their state before the reaction) in tiles of 16 on the tensor
// cores, written over the plain step's result.  Each warp stages one tile's
// inputs in shared memory, then evaluates it.  Node results do not depend
// on the list's order.  Block 0 also empties the other parity's list for
// the next step and counts the step's plain-path node updates.
__global__ void __launch_bounds__(kSurThreads) sur_net_kernel(const SurArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  uint16_t* sW1 = reinterpret_cast<uint16_t*>(smem_raw);  // [kHid][kW1Stride]
  uint16_t* sW2 = sW1 + kHid * kW1Stride;                  // [kHid][kW2Stride]
  uint16_t* sW3 = sW2 + kHid * kW2Stride;                  // [8][kW2Stride]
  float* sB = reinterpret_cast<float*>(sW3 + 8 * kW2Stride);  // b1[128], b2[128], b3[8]
  float* stage = sB + 2 * kHid + 8;
  const int64_t stp = *a.step_base + a.step_offset;
  const int par = (int)(stp & 1);
  const int64_t listed = a.list_count[par];
  const int64_t count = listed < a.list_cap ? listed : a.list_cap;  // overflow is flagged by the step kernel
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    a.list_count[par ^ 1] = 0;
    atomicAdd(a.fallback_count, (unsigned long long)(a.real_nodes - count));
  }
  if (count == 0) return;
  {
    const uint32_t* gw = reinterpret_cast<const uint32_t*>(a.wts);
    uint32_t* sw = reinterpret_cast<uint32_t*>(smem_raw);
    const int words = (kHid * kW1Stride + kHid * kW2Stride + 8 * kW2Stride) / 2;
    for (int i = threadIdx.x; i < words; i += blockDim.x) sw[i] = gw[i];
    for (int i = threadIdx.x; i < 2 * kHid + 8; i += blockDim.x) sB[i] = a.bias[i];
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  float* sx = stage + (threadIdx.x >> 5) * kStageFloats;  // [kTileRows][kIn]
  float* sy = sx + kTileRows * kIn;                       // [kTileRows][4]
  int* sq = reinterpret_cast<int*>(sy + kTileRows * 4);   // [kTileRows]
  const float* L = a.list + par * 6 * a.list_cap;
  const int64_t warps_total = (int64_t)gridDim.x * (blockDim.x >> 5);
  const int64_t n_tiles = (count + kTileRows - 1) / kTileRows;
  for (int64_t tile = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); tile < n_tiles;
       tile += warps_total) {
    const int64_t e0 = tile * kTileRows;
    const int rows = (int)(count - e0 < kTileRows ? count - e0 : kTileRows);
    if (lane < rows) {
      const int64_t e = e0 + lane;
      float raw[kIn];
#pragma unroll
      for (int k = 0; k < kIn; ++k) raw[k] = L[(1 + k) * a.list_cap + e];
#pragma unroll
      for (int k = 0; k < kIn; ++k) sx[lane * kIn + k] = (raw[k] - a.in_mu[k]) * a.in_inv_sigma[k];
#pragma unroll
      for (int k = 0; k < 4; ++k) sy[lane * 4 + k] = raw[k];
      sq[lane] = __float_as_int(L[e]);
    }
    __syncwarp();
    network_tile(a, sW1, sW2, sW3, sB, sx, sy, sq, 0, rows, g, t);
    __syncwarp();  // the staging area is rewritten by the next tile
  }
}

// ---------------------------------------------------------------------------
// Training on BF16 tensor cores (quantised mode)
// ---------------------------------------------------------------------------
//
// Every matrix product of a training step is C = A B with mma.sync
// m16n8k16 BF16 x BF16 -> FP32.  B operands are always exact in bf16 (the
// quantised weights, or activations and inputs already rounded to bf16 by
// the forward pass).  A operands that are FP32 (the backward pass's dz and
// dout) are split into bf16 high and low parts, A = A_hi + A_lo, and both
// are multiplied, so the product keeps about 16 bits of A's mantissa.  The
// weight gradients reduce over the batch in fixed chunks of kChunk samples
// whose partial products are summed in chunk order (deterministic).

constexpr int kGemmBM = 64, kGemmBN = 64, kGemmBK = 16, kGemmThreads = 128, kChunk = 256;

// A(m, k) = A[m * a_m + k * a_k], B(k, n) = B[k * b_k + n * b_n] (FP32 arrays).
struct GemmOp {
  const float* A;
  int64_t a_m, a_k;
  const float* B;
  int64_t b_k, b_n;
  int M, N;
  int64_t K;
  int split_a;   // A is FP32: multiply its bf16 high and low parts
};

enum EpiKind { kEpiSilu, kEpiOut, kEpiDz, kEpiPartial };

struct Epilogue {
  int kind;
  const float* bias;     // kEpiSilu, kEpiOut: per-column bias
  float* z;              // kEpiSilu: pre-activation out (M x N row-major)
  float* a;              // kEpiSilu: bf16-rounded SiLU out; kEpiDz: dz out
  const float* zin;      // kEpiDz: pre-activation whose SiLU derivative scales the product
  float* out;            // kEpiOut: network output; kEpiPartial: partial tiles [chunk][M][N]
  const float* target;   // kEpiOut
  float* dout;           // kEpiOut: 2 (out - target) / (B * 4)
  float scale;
  int quantize;
};

__device__ __forceinline__ uint16_t bf16_bits(float v) {
  const __nv_bfloat16 b = __float2bfloat16_rn(v);
  return *reinterpret_cast<const uint16_t*>(&b);
}

// One CTA: a kGemmBM x kGemmBN tile of C over k in [k0, k1); 4 warps, each
// a 32 x 32 quarter as 2 x 4 m16n8 tiles.
__global__ void __launch_bounds__(kGemmThreads) gemm_bf16_kernel(GemmOp g, Epilogue e, int64_t k_chunk) {
  __shared__ __align__(16) uint16_t sAh[kGemmBM][kGemmBK + 8];
  __shared__ __align__(16) uint16_t sAl[kGemmBM][kGemmBK + 8];
  __shared__ __align__(16) uint16_t sB[kGemmBN][kGemmBK + 8];  // [n][k]: col-major B
  const int m0 = blockIdx.x * kGemmBM, n0 = blockIdx.y * kGemmBN;
  const int64_t k0 = (int64_t)blockIdx.z * k_chunk;
  const int64_t k1 = min(g.K, k0 + k_chunk);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, gq = lane >> 2, tq = lane & 3;
  const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;
  float acc[2][4][4] = {};
  for (int64_t kb = k0; kb < k1; kb += kGemmBK) {
    for (int i = threadIdx.x; i < kGemmBM * kGemmBK; i += kGemmThreads) {
      const int mm = i / kGemmBK, kk = i % kGemmBK;
      const int64_t m = m0 + mm, k = kb + kk;
      float v = 0.0f;
      if (m < g.M && k < k1) v = g.A[m * g.a_m + k * g.a_k];
      const uint16_t hi = bf16_bits(v);
      sAh[mm][kk] = hi;
      if (g.split_a) {
        __nv_bfloat16 hb;
        *reinterpret_cast<uint16_t*>(&hb) = hi;
        sAl[mm][kk] = bf16_bits(v - __bfloat162float(hb));
      }
    }
    for (int i = threadIdx.x; i < kGemmBN * kGemmBK; i += kGemmThreads) {
      const int nn = i / kGemmBK, kk = i % kGemmBK;
      const int64_t n = n0 + nn, k = kb + kk;
      float v = 0.0f;
      if (n < g.N && k < k1) v = g.B[k * g.b_k + n * g.b_n];
      sB[nn][kk] = bf16_bits(v);  // bf16 values stay exact; FP32 weights round to nearest even
    }
    __syncthreads();
#pragma unroll
    for (int mt = 0; mt < 2; ++mt) {
      const int r = wm + 16 * mt + gq;
      uint32_t ah[4], al[4];
      ah[0] = *reinterpret_cast<const uint32_t*>(&sAh[r][2 * tq]);
      ah[1] = *reinterpret_cast<const uint32_t*>(&sAh[r + 8][2 * tq]);
      ah[2] = *reinterpret_cast<const uint32_t*>(&sAh[r][2 * tq + 8]);
      ah[3] = *reinterpret_cast<const uint32_t*>(&sAh[r + 8][2 * tq + 8]);
      if (g.split_a) {
        al[0] = *reinterpret_cast<const uint32_t*>(&sAl[r][2 * tq]);
        al[1] = *reinterpret_cast<const uint32_t*>(&sAl[r + 8][2 * tq]);
        al[2] = *reinterpret_cast<const uint32_t*>(&sAl[r][2 * tq + 8]);
        al[3] = *reinterpret_cast<const uint32_t*>(&sAl[r + 8][2 * tq + 8]);
      }
#pragma unroll
      for (int nt = 0; nt < 4; ++nt) {
        const int c = wn + 8 * nt + gq;
        const uint32_t b0 = *reinterpret_cast<const uint32_t*>(&sB[c][2 * tq]);
        const uint32_t b1 = *reinterpret_cast<const uint32_t*>(&sB[c][2 * tq + 8]);
        mma_bf16(acc[mt][nt], ah, b0, b1);
        if (g.split_a) mma_bf16(acc[mt][nt], al, b0, b1);
      }
    }
    __syncthreads();
  }
  // epilogue: element (m, n) of the tile
#pragma unroll
  for (int mt = 0; mt < 2; ++mt)
#pragma unroll
    for (int nt = 0; nt < 4; ++nt)
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int m = m0 + wm + 16 * mt + gq + (q >= 2 ? 8 : 0);
        const int n = n0 + wn + 8 * nt + 2 * tq + (q & 1);
        if (m >= g.M || n >= g.N) continue;
        const float v = acc[mt][nt][q];
        const int64_t o = (int64_t)m * g.N + n;
        if (e.kind == kEpiSilu) {
          const float zz = v + e.bias[n];
          e.z[o] = zz;
          e.a[o] = q_bf16(zz / (1.0f + __expf(-zz)), e.quantize);
        } else if (e.kind == kEpiOut) {
          const float oo = v + e.bias[n];
          e.out[o] = oo;
          if (e.target) e.dout[o] = e.scale * (oo - e.target[o]);
        } else if (e.kind == kEpiDz) {
          e.a[o] = v * silu_grad(e.zin[o]);
        } else {
          e.out[(int64_t)blockIdx.z * g.M * g.N + o] = v;
        }
      }
}

// W[o] = sum over chunks of partial[c][o] in chunk order; bias gradients as
// column sums of D (B x cols) over the batch, in fixed order.
__global__ void reduce_partials_kernel(const float* part, int chunks, int64_t n, float* out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    float acc = 0.0f;
    for (int c = 0; c < chunks; ++c) acc += part[(int64_t)c * n + i];
    out[i] = acc;
  }
}

__global__ void column_sum_kernel(const float* D, int64_t B, int cols, float* out) {
  __shared__ float part[256];
  const int c = blockIdx.x;
  float acc = 0.0f;
  for (int64_t b = threadIdx.x; b < B; b += blockDim.x) acc += D[b * cols + c];
  part[threadIdx.x] = acc;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) part[threadIdx.x] += part[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[c] = part[0];
}

void gemm(const GemmOp& g, const Epilogue& e, int64_t k_chunk, int chunks, cudaStream_t s) {
  dim3 grid((g.M + kGemmBM - 1) / kGemmBM, (g.N + kGemmBN - 1) / kGemmBN, chunks);
  gemm_bf16_kernel<<<grid, kGemmThreads, 0, s>>>(g, e, k_chunk);
}

// Forward pass of the quantised network on tensor cores: z1, a1, z2, a2,
// out, and with a target also dout = 2 (out - target) / (B * 4).
void mma_forward(const float* th, const float* xq, int64_t B, float* z1, float* a1, float* z2, float* a2, float* out,
                 const float* target, float* dout, cudaStream_t s) {
  const int Bi = (int)B;
  Epilogue e{};
  e.quantize = 1;
  e.kind = kEpiSilu;
  GemmOp g1{xq, kIn, 1, th + kOffW1, 1, kIn, Bi, kHid, kIn, 0};  // B(k, j) = W1[j][k]
  e.bias = th + kOffB1;
  e.z = z1;
  e.a = a1;
  gemm(g1, e, kIn, 1, s);
  GemmOp g2{a1, kHid, 1, th + kOffW2, 1, kHid, Bi, kHid, kHid, 0};
  e.bias = th + kOffB2;
  e.z = z2;
  e.a = a2;
  gemm(g2, e, kHid, 1, s);
  GemmOp g3{a2, kHid, 1, th + kOffW3, 1, kHid, Bi, kOut, kHid, 0};
  Epilogue eo{};
  eo.kind = kEpiOut;
  eo.bias = th + kOffB3;
  eo.out = out;
  eo.target = target;
  eo.dout = dout;
  eo.scale = 2.0f / (float)(B * kOut);
  gemm(g3, eo, kHid, 1, s);
}

// Weight gradient W(M x N) = sum_b A(m, b) B(b, n) over the batch in chunks
// of about kChunk samples (as many as `part_floats` of partials hold), then
// the chunk partials summed in order; a single chunk writes W directly.
void mma_wgrad(GemmOp g, float* part, int64_t part_floats, float* gW, cudaStream_t s) {
  const int64_t n = (int64_t)g.M * g.N;
  int64_t chunks = std::max<int64_t>(1, std::min<int64_t>((g.K + kChunk - 1) / kChunk, part_floats / n));
  int64_t k_chunk = (g.K + chunks - 1) / chunks;
  k_chunk = (k_chunk + kGemmBK - 1) / kGemmBK * kGemmBK;
  chunks = (g.K + k_chunk - 1) / k_chunk;
  Epilogue e{};
  e.kind = kEpiPartial;
  e.out = chunks == 1 ? gW : part;
  gemm(g, e, k_chunk, (int)chunks, s);
  if (chunks > 1) reduce_partials_kernel<<<(int)((n + 255) / 256), 256, 0, s>>>(part, (int)chunks, n, gW);
}

__global__ void quantize_kernel(const float* x, int64_t n, float* y) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = q_bf16(x[i], 1);
}

}  // namespace

size_t sur_smem_bytes() {
  return 2 * ((size_t)kHid * kW1Stride + (size_t)kHid * kW2Stride + 8 * (size_t)kW2Stride) +
         4 * (2 * (size_t)kHid + 8) + 4 * (size_t)kStageFloats * (kSurThreads / 32);
}

int launch_hh_reaction(const HHConst& c, float vrest, int n_sub, int64_t count, const float* in,
                       const uint8_t* stim, float* out, void* stream) {
  if (count <= 0) return 0;
  const int64_t blocks = (count + 255) / 256;
  hh_reaction_kernel<<<(int)(blocks < 65535 ? blocks : 65535), 256, 0, (cudaStream_t)stream>>>(c, vrest, n_sub, count,
                                                                                                in, stim, out);
  return (int)cudaGetLastError();
}

int launch_mlp_train_step(const float* th, int quantize, const float* x, const float* target, int64_t B, float* ws,
                          float* grad, float* loss, void* stream) {
  cudaStream_t s = (cudaStream_t)stream;
  float* z1 = ws;
  float* a1 = z1 + B * kHid;
  float* z2 = a1 + B * kHid;
  float* a2 = z2 + B * kHid;
  float* out = a2 + B * kHid;
  float* dout = out + B * kOut;
  float* dz1 = dout + B * kOut;
  float* dz2 = dz1 + B * kHid;
  if (quantize) {
    // BF16 tensor cores: forward, backward and the weight gradients
    float* xq = dz2 + B * kHid;                 // B x 5
    float* part = xq + B * kIn;                 // chunk partials of the weight gradients
    quantize_kernel<<<(int)((B * kIn + 255) / 256), 256, 0, s>>>(x, B * kIn, xq);
    mma_forward(th, xq, B, z1, a1, z2, a2, out, target, dout, s);
    mse_kernel<<<1, 256, 0, s>>>(out, target, B * kOut, loss);
    const int Bi = (int)B;
    Epilogue e{};
    e.kind = kEpiDz;
    GemmOp d2{dout, kOut, 1, th + kOffW3, kHid, 1, Bi, kHid, kOut, 1};  // da2 = dout W3
    e.a = dz2;
    e.zin = z2;
    gemm(d2, e, kOut, 1, s);
    GemmOp d1{dz2, kHid, 1, th + kOffW2, kHid, 1, Bi, kHid, kHid, 1};   // da1 = dz2 W2
    e.a = dz1;
    e.zin = z1;
    gemm(d1, e, kHid, 1, s);
    const int64_t part_floats = B * (kWorkPerSample - 6 * kHid - 2 * kOut - kIn);
    mma_wgrad(GemmOp{dout, 1, kOut, a2, kHid, 1, kOut, kHid, B, 1}, part, part_floats, grad + kOffW3, s);
    mma_wgrad(GemmOp{dz2, 1, kHid, a1, kHid, 1, kHid, kHid, B, 1}, part, part_floats, grad + kOffW2, s);
    mma_wgrad(GemmOp{dz1, 1, kHid, xq, kIn, 1, kHid, kIn, B, 1}, part, part_floats, grad + kOffW1, s);
    column_sum_kernel<<<kOut, 256, 0, s>>>(dout, B, kOut, grad + kOffB3);
    column_sum_kernel<<<kHid, 256, 0, s>>>(dz2, B, kHid, grad + kOffB2);
    column_sum_kernel<<<kHid, 256, 0, s>>>(dz1, B, kHid, grad + kOffB1);
    return (int)cudaGetLastError();
  }
  const int grid = (int)(B < 152 * 8 ? B : 152 * 8);
  mlp_fwd_kernel<<<grid, kHid, kFwdSmem, s>>>(th, quantize, x, B, z1, a1, z2, a2, out);
  mse_kernel<<<1, 256, 0, s>>>(out, target, B * kOut, loss);
  mlp_bwd_kernel<<<grid, kHid, kBwdSmem, s>>>(th, quantize, B, z1, z2, out, target, dout, dz1, dz2);
  auto wg = [&](const float* D, int rows, const float* X, int cols, int qx, int64_t offW, int64_t offB) {
    const int64_t n = (int64_t)rows * cols + rows;
    wgrad_kernel<<<(int)((n + 255) / 256), 256, 0, s>>>(D, rows, X, cols, B, qx, grad + offW, grad + offB);
  };
  wg(dout, kOut, a2, kHid, 0, kOffW3, kOffB3);
  wg(dz2, kHid, a1, kHid, 0, kOffW2, kOffB2);
  wg(dz1, kHid, x, kIn, quantize, kOffW1, kOffB1);
  return (int)cudaGetLastError();
}

int launch_mlp_forward(const float* th, int quantize, const float* x, int64_t B, float* ws, float* out, void* stream) {
  float* z1 = ws;
  float* a1 = z1 + B * kHid;
  float* z2 = a1 + B * kHid;
  float* a2 = z2 + B * kHid;
  if (quantize) {
    float* xq = a2 + B * kHid;
    quantize_kernel<<<(int)((B * kIn + 255) / 256), 256, 0, (cudaStream_t)stream>>>(x, B * kIn, xq);
    mma_forward(th, xq, B, z1, a1, z2, a2, out, nullptr, nullptr, (cudaStream_t)stream);
    return (int)cudaGetLastError();
  }
  const int grid = (int)(B < 152 * 8 ? B : 152 * 8);
  mlp_fwd_kernel<<<grid, kHid, kFwdSmem, (cudaStream_t)stream>>>(th, quantize, x, B, z1, a1, z2, a2, out);
  return (int)cudaGetLastError();
}

int launch_adam(float* th, float* m, float* v, const float* g, int64_t n, float lr, float b1, float b2, float eps,
                int64_t t, float* avg, float avg_decay, void* stream) {
  const float c1 = 1.0f - powf(b1, (float)t), c2 = 1.0f - powf(b2, (float)t);
  adam_kernel<<<(int)((n + 255) / 256), 256, 0, (cudaStream_t)stream>>>(th, m, v, g, n, lr, b1, b2, eps, c1, c2,
                                                                         avg, avg_decay);
  return (int)cudaGetLastError();
}

int launch_stats(const float* X, int64_t n, int cols, double* out, void* stream) {
  stats_kernel<<<cols, 256, 0, (cudaStream_t)stream>>>(X, n, cols, out);
  return (int)cudaGetLastError();
}

int launch_sur_net(const SurArgs& a, void* stream) {
  // the list's length exists on the device only: a fixed grid strides over it
  sur_net_kernel<<<152 * 4, kSurThreads, sur_smem_bytes(), (cudaStream_t)stream>>>(a);
  return (int)cudaGetLastError();
}

int launch_split_step_sur(int K, const StepArgs& a, int n_ctas, void* stream) {
  return launch_family<float, false, false, true>(K, a, n_ctas, stream);
}

int sur_set_smem_attributes() {
  cudaError_t e = cudaFuncSetAttribute(sur_net_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)sur_smem_bytes());
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(mlp_fwd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kFwdSmem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(mlp_bwd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kBwdSmem);
  return (int)e;
}

}  // namespace fib
