// Two-flavour step kernels: FP64 and mixed precision, RK4 / DP45 / commutator-free Lie RK4 /
// exponential midpoint rule.
// The mixed kernels exist at two register budgets (768 or 512 resident threads per SM), the
// 512-thread one as 256 x 2 and as one 512-thread block.
#include "step_kernel.cuh"
#include "kernels.h"

namespace xflat {

template <int B, int T>
const void* mixed_2f(int integrator) {
  if (integrator == kRK4) return (const void*)&step_kernel<Phys2<float>, TabRK4, float, false, B, T>;
  if (integrator == kDP45) return (const void*)&step_kernel<Phys2<float>, TabDP45, float, false, B, T>;
  if (integrator == kLieRK4) return (const void*)&step_kernel<Phys2<float>, TabCF4, float, true, B, T>;
  if (integrator == kExpMid) return (const void*)&step_kernel<Phys2<float>, TabEM2, float, true, B, T>;
  return nullptr;
}

const void* step_kernel_ptr_2f(int precision, int integrator, int block, int blocks_per_sm) {
  if (integrator == kLieAdaptive) return step_kernel_ptr_lie(precision, block, blocks_per_sm);
  if (block > 256) return (precision == 1 && block == 512) ? mixed_2f<1, 512>(integrator) : nullptr;
  if (precision == 0) {
    if (integrator == kRK4) return (const void*)&step_kernel<Phys2<double>, TabRK4, double, false, 1>;
    if (integrator == kDP45) return (const void*)&step_kernel<Phys2<double>, TabDP45, double, false, 1>;
    if (integrator == kLieRK4) return (const void*)&step_kernel<Phys2<double>, TabCF4, double, true, 1>;
    if (integrator == kExpMid) return (const void*)&step_kernel<Phys2<double>, TabEM2, double, true, 1>;
    return nullptr;
  }
  return blocks_per_sm >= 3 ? mixed_2f<3, 256>(integrator) : mixed_2f<2, 256>(integrator);
}

}  // namespace xflat
