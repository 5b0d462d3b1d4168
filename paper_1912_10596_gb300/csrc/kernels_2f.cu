// Two-flavour step kernels: FP64 and mixed precision, RK4 / DP45 / commutator-free Lie RK4.
#include "step_kernel.cuh"
#include "kernels.h"

namespace xflat {

const void* step_kernel_ptr_2f(int precision, int integrator) {
  if (precision == 0) {
    if (integrator == kRK4) return (const void*)&step_kernel<Phys2<double>, TabRK4, double, false>;
    if (integrator == kDP45) return (const void*)&step_kernel<Phys2<double>, TabDP45, double, false>;
    if (integrator == kLieRK4) return (const void*)&step_kernel<Phys2<double>, TabCF4, double, true>;
  } else {
    if (integrator == kRK4) return (const void*)&step_kernel<Phys2<float>, TabRK4, float, false>;
    if (integrator == kDP45) return (const void*)&step_kernel<Phys2<float>, TabDP45, float, false>;
    if (integrator == kLieRK4) return (const void*)&step_kernel<Phys2<float>, TabCF4, float, true>;
  }
  return nullptr;
}

}  // namespace xflat
