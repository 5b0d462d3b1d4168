// Two-flavour step kernels of the extended bulb model (azimuthal bins, Sec. 2 Eq. int-v / Eq. F):
// FP64 and mixed precision, RK4 / DP45 / commutator-free Lie RK4 / exponential midpoint rule.
#include "step_kernel.cuh"
#include "kernels.h"

namespace xflat {

// FP64 kernels: one 256-thread block per SM (the FP64 pipe is the bound).  FP32 kernels: two per
// SM (128 registers), so twice the warps hide the latency of the per-beam chains.
template <typename Real, int kMinB>
const void* ext_2f(int integrator) {
  using P = Phys2E<Real>;
  if (integrator == kRK4) return (const void*)&step_kernel<P, TabRK4, Real, false, kMinB>;
  if (integrator == kDP45) return (const void*)&step_kernel<P, TabDP45, Real, false, kMinB>;
  if (integrator == kLieRK4) return (const void*)&step_kernel<P, TabCF4, Real, true, kMinB>;
  if (integrator == kExpMid) return (const void*)&step_kernel<P, TabEM2, Real, true, kMinB>;
  return nullptr;
}

const void* step_kernel_ptr_2e(int precision, int integrator, int block) {
  if (block > 256) return nullptr;
  return precision == 0 ? ext_2f<double, 1>(integrator) : ext_2f<float, 2>(integrator);
}

}  // namespace xflat
