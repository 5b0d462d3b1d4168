// Three-flavour step kernels of the exponential integrators (commutator-free Lie RK4, the
// exponential midpoint rule and the adaptive Lie RK4 with Richardson control): FP64 and mixed, one
// 256-thread block per SM.  The propagators are the eigen-decomposition form of Eq. U for 3 x 3
// generators (propagate3).  A translation unit of its own, so that it compiles in parallel with
// the others.
#include "step_kernel.cuh"
#include "kernels.h"

namespace xflat {

const void* step_kernel_ptr_3f_exp(int precision, int integrator) {
  if (precision == 0) {
    if (integrator == kLieRK4) return (const void*)&step_kernel<Phys3<double>, TabCF4, double, true, 1>;
    if (integrator == kExpMid) return (const void*)&step_kernel<Phys3<double>, TabEM2, double, true, 1>;
    if (integrator == kLieAdaptive) return (const void*)&step_kernel<Phys3<double>, TabCFR, double, true, 1>;
  } else {
    if (integrator == kLieRK4) return (const void*)&step_kernel<Phys3<float>, TabCF4, float, true, 1>;
    if (integrator == kExpMid) return (const void*)&step_kernel<Phys3<float>, TabEM2, float, true, 1>;
    if (integrator == kLieAdaptive) return (const void*)&step_kernel<Phys3<float>, TabCFR, float, true, 1>;
  }
  return nullptr;
}

}  // namespace xflat
