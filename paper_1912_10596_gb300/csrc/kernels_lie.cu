// Two-flavour step kernels of the adaptive commutator-free Lie RK4 (Richardson step-size control,
// TabCFR): FP64, and mixed precision at the register budgets of the other mixed kernels (768 or
// 512 resident threads per SM).  A translation unit of its own, so that it compiles in parallel
// with the others.
#include "step_kernel.cuh"
#include "kernels.h"

namespace xflat {

const void* step_kernel_ptr_lie(int precision, int block, int blocks_per_sm) {
  if (precision == 0) return block <= 256 ? (const void*)&step_kernel<Phys2<double>, TabCFR, double, true, 1> : nullptr;
  if (block > 256) return block == 512 ? (const void*)&step_kernel<Phys2<float>, TabCFR, float, true, 1, 512> : nullptr;
  return blocks_per_sm >= 3 ? (const void*)&step_kernel<Phys2<float>, TabCFR, float, true, 3, 256>
                            : (const void*)&step_kernel<Phys2<float>, TabCFR, float, true, 2, 256>;
}

}  // namespace xflat
