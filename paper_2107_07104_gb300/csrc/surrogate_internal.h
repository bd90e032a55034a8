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
// Floats of training workspace per sample: z1, a1, z2, a2, out, dout, dz1,
// dz2, the bf16-rounded inputs (5) and the weight gradients' partial sums
// over chunks of 256 samples (128 x 128 / 256 = 64), rounded up to 848.
constexpr int64_t kWorkPerSample = 848;
// bf16 row strides of the inference weight images (padded for conflict-free
// shared-memory fragment loads): W1 rows hold [x_hi (5) | x_lo (5) | 0].
constexpr int kW1Stride = 24;
constexpr int kW2Stride = 136;

struct SurArgs {
  float *u, *m, *h, *n;         // padded state arrays (u = V - Vrest)
  const float* list;            // per parity 6 arrays of list_cap: slot (int bits), u, m, h, n, stimulus fraction
  unsigned int* list_count;     // [2] entries of each parity's list
  int64_t list_cap;
  const int64_t* step_base;     // device step counter; this step is *step_base + step_offset
  int64_t step_offset;
  int64_t real_nodes;           // nodes of the context (plain-path count)
  const uint16_t* wts;          // bf16 images W1 | W2 | W3
  const float* bias;            // b1 (128) | b2 (128) | b3 (8)
  unsigned long long* fallback_count;
  float in_mu[kIn], in_inv_sigma[kIn];
  float out_mu[kOut], out_sigma[kOut];
  float rest[kOut];             // 0, m0, h0, n0: the state arrays hold gates minus their rest values
};

size_t sur_smem_bytes();
int sur_set_smem_attributes();
int launch_hh_reaction(const HHConst& c, float vrest, int n_sub, int64_t count, const float* in,
                       const uint8_t* stim, float* out, void* stream);
int launch_mlp_train_step(const float* th, int quantize, const float* x, const float* target, int64_t B, float* ws,
                          float* grad, float* loss, void* stream);
int launch_mlp_forward(const float* th, int quantize, const float* x, int64_t B, float* ws, float* out, void* stream);
int launch_adam(float* th, float* m, float* v, const float* g, int64_t n, float lr, float b1, float b2, float eps,
                int64_t t, float* avg, float avg_decay, void* stream);
int launch_stats(const float* X, int64_t n, int cols, double* out, void* stream);
int launch_sur_net(const SurArgs& a, void* stream);

}  // namespace fib
