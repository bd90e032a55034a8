// Split-step kernel instantiations with the thesis's approximated
// exponential exp*(x) = (1 + x/1024)^1024 (eq:apx-e-function) in place of
// every exponential of the Hodgkin-Huxley rates; FP32 solve only.  Kept in
// its own translation unit so that it compiles in parallel with the exact
// instantiations.
#include "split_step_kernel.cuh"

namespace fib {

int launch_split_step_expapx(int K, const StepArgs& a, int n_ctas, void* stream) {
  return a.adaptive ? launch_family<float, true, true>(K, a, n_ctas, stream)
                    : launch_family<float, true, false>(K, a, n_ctas, stream);
}

}  // namespace fib
