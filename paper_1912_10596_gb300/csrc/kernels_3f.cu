// Three-flavour step kernels (3x3 Hermitian density matrices): FP64 and mixed, RK4 / DP45 (the
// exponential integrators in kernels_3f_lie.cu), and the dispatch over flavours and models.
#include "step_kernel.cuh"
#include "kernels.h"

namespace xflat {

const void* step_kernel_ptr_2f(int precision, int integrator, int block, int blocks_per_sm);

const void* step_kernel_ptr(int n_flavor, int precision, int integrator, int block, int blocks_per_sm,
                            bool extended) {
  if (extended) return n_flavor == 2 ? step_kernel_ptr_2e(precision, integrator, block) : nullptr;
  if (n_flavor == 2) return step_kernel_ptr_2f(precision, integrator, block, blocks_per_sm);
  if (n_flavor != 3 || block > 256) return nullptr;
  if (integrator == kLieRK4 || integrator == kExpMid || integrator == kLieAdaptive)
    return step_kernel_ptr_3f_exp(precision, integrator);
  if (precision == 0) {
    if (integrator == kRK4) return (const void*)&step_kernel<Phys3<double>, TabRK4, double, false, 1>;
    if (integrator == kDP45) return (const void*)&step_kernel<Phys3<double>, TabDP45, double, false, 1>;
  } else {
    if (integrator == kRK4) return (const void*)&step_kernel<Phys3<float>, TabRK4, float, false, 1>;
    if (integrator == kDP45) return (const void*)&step_kernel<Phys3<float>, TabDP45, float, false, 1>;
  }
  return nullptr;
}

}  // namespace xflat
