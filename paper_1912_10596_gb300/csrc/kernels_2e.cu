// Two-flavour step kernels of the extended bulb model (azimuthal bins, Sec. 2 Eq. int-v / Eq. F):
// FP64 and mixed precision, RK4 / DP45 / commutator-free Lie RK4 / exponential midpoint rule.
#include "step_kernel.cuh"
#include "kernels.h"

namespace xflat {

template <typename Real>
const void* ext_2f(int integrator) {
  using P = Phys2E<Real>;
  if (integrator == kRK4) return (const void*)&step_kernel<P, TabRK4, Real, false, 1>;
  if (integrator == kDP45) return (const void*)&step_kernel<P, TabDP45, Real, false, 1>;
  if (integrator == kLieRK4) return (const void*)&step_kernel<P, TabCF4, Real, true, 1>;
  if (integrator == kExpMid) return (const void*)&step_kernel<P, TabEM2, Real, true, 1>;
  return nullptr;
}

const void* step_kernel_ptr_2e(int precision, int integrator, int block) {
  if (block > 256) return nullptr;
  return precision == 0 ? ext_2f<double>(integrator) : ext_2f<float>(integrator);
}

}  // namespace xflat
