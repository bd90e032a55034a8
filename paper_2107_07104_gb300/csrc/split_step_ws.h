// Entry points of the split-role kernels (split_step_ws.cu) that the host
// runtime needs beyond fibers_internal.h.
#pragma once

#include <cstddef>

#include "fibers_internal.h"

namespace fib {

// The wide split-role shape: one 1024-thread CTA per SM holding 8 fibers of
// at most kWsSlot nodes (solver tables for K = kWsKC and kWsCnThreads
// threads per fiber, like the two-fiber shape).
int launch_split_step_ws8(const StepArgs& a, int n_ctas, void* stream);
size_t split_step_ws8_smem_bytes();
int split_step_ws8_fibers_per_cta();
int split_step_ws8_warps();

}  // namespace fib
