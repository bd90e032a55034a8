// Split-step kernel instantiations with adaptive computation
// (sec:adaptive_computation_for_fiber_based): fiber-level launch skipping.
// Kept in its own translation unit so
// that it compiles in parallel with the plain instantiations, and so that
// the plain kernels carry none of its code.
#include "split_step_kernel.cuh"

namespace fib {

int launch_split_step_adaptive(int K, bool fp64, const StepArgs& a, int n_ctas, void* stream) {
  return fp64 ? launch_family<double, false, true>(K, a, n_ctas, stream)
              : launch_family<float, false, true>(K, a, n_ctas, stream);
}

}  // namespace fib
