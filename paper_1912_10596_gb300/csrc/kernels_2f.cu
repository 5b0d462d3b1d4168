// Two-flavour step kernels: FP64 and mixed precision, RK4 / DP45 / commutator-free Lie RK4.
// The mixed kernels exist at two register budgets (3 or 2 resident blocks per SM).
#include "step_kernel.cuh"
#include "kernels.h"

namespace xflat {

template <int B>
const void* mixed_2f(int integrator) {
  if (integrator == kRK4) return (const void*)&step_kernel<Phys2<float>, TabRK4, float, false, B>;
  if (integrator == kDP45) return (const void*)&step_kernel<Phys2<float>, TabDP45, float, false, B>;
  if (integrator == kLieRK4) return (const void*)&step_kernel<Phys2<float>, TabCF4, float, true, B>;
  return nullptr;
}

const void* step_kernel_ptr_2f(int precision, int integrator, int blocks_per_sm) {
  if (precision == 0) {
    if (integrator == kRK4) return (const void*)&step_kernel<Phys2<double>, TabRK4, double, false, 1>;
    if (integrator == kDP45) return (const void*)&step_kernel<Phys2<double>, TabDP45, double, false, 1>;
    if (integrator == kLieRK4) return (const void*)&step_kernel<Phys2<double>, TabCF4, double, true, 1>;
    return nullptr;
  }
  return blocks_per_sm >= 3 ? mixed_2f<3>(integrator) : mixed_2f<2>(integrator);
}

}  // namespace xflat
