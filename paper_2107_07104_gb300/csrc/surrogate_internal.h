// Internal declarations of the reaction-step surrogate (surrogate.cu).
#pragma once

#include <cstdint>

#include "fibers_internal.h"

namespace fib {

constexpr int kIn = 5, kHid = 128, kOut = 4;
// FP32 parameter vector: W1 (128 x 5), b1, W2 (128 x 128), b2, W3 (4 x 128), b3.
constexpr int64_t kOffW1 = 0;
constexpr int64_t kOffB1 = kOffW1 + kHid * kIn;
constexpr int64_t kOffW2 = kOffB1 + kHid;
constexpr int64_t kOffB2 = kOffW2 + kHid * kHid;
constexpr int64_t kOffW3 = kOffB2 + kHid;
constexpr int64_t kOffB3 = kOffW3 + kOut * kHid;
constexpr int64_t kNumParams = kOffB3 + kOut;
// Floats of training workspace per sample: z1, a1, z2, a2, out, dout, dz1, dz2.
constexpr int64_t kWorkPerSample = 6 * kHid + 2 * kOut;
// bf16 row strides of the inference weight images (padded for conflict-free
// shared-memory fragment loads): W1 rows hold [x_hi (5) | x_lo (5) | 0].
constexpr int kW1Stride = 24;
constexpr int kW2Stride = 136;

struct SurArgs {
  float *u, *m, *h, *n;         // padded state arrays (u = V - Vrest)
  const int32_t* slot_code;     // per slot: -1 padding, else (fiber << 1) | (node in its junction's stimulus range)
  const uint8_t* fiber_stim;    // stimulus substep mask of each fiber for this step
  const uint16_t* wts;          // bf16 images W1 | W2 | W3
  const float* bias;            // b1 (128) | b2 (128) | b3 (8)
  unsigned long long* fallback_count;
  int32_t* net_list;            // slots of the step's network nodes (capacity n_slots)
  unsigned int* net_count;      // their number (reset by the step's stimulus kernel)
  int64_t n_slots;
  HHConst hh;
  float in_mu[kIn], in_inv_sigma[kIn];
  float out_mu[kOut], out_sigma[kOut];
  float env_lo[kIn], env_hi[kIn];      // training envelope: outside -> plain HH
  float quiet_lo[kIn], quiet_hi[kIn];  // neighbourhood of rest: inside -> plain HH
  int32_t n_sub, hw;
  float inv_n_sub;              // 1 / n_sub (stimulus fraction of a split step)
};

size_t sur_smem_bytes();
int sur_set_smem_attributes();
int launch_hh_reaction(const HHConst& c, float vrest, int n_sub, int64_t count, const float* in,
                       const uint8_t* stim, float* out, void* stream);
int launch_mlp_train_step(const float* th, int quantize, const float* x, const float* target, int64_t B, float* ws,
                          float* grad, float* loss, void* stream);
int launch_mlp_forward(const float* th, int quantize, const float* x, int64_t B, float* ws, float* out, void* stream);
int launch_adam(float* th, float* m, float* v, const float* g, int64_t n, float lr, float b1, float b2, float eps,
                int64_t t, void* stream);
int launch_stats(const float* X, int64_t n, int cols, double* out, void* stream);
int launch_sur_step(const SurArgs& a, void* stream);
int launch_fiber_stim(const FiberDesc* fibers, int32_t n_fibers, const int64_t* mu_off, const int64_t* fire_k,
                      int32_t n_mu, const int64_t* step_base, int64_t step_offset, int n_sub, int pulse, uint8_t* out,
                      unsigned int* net_count, void* stream);

}  // namespace fib
