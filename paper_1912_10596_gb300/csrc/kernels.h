// Registry of the persistent step kernels (instantiated in kernels_2f.cu / kernels_3f.cu).
#pragma once

namespace xflat {
struct KParams;
// Returns the __global__ step kernel for (n_flavor, precision, integrator), or nullptr.
const void* step_kernel_ptr(int n_flavor, int precision, int integrator);
}  // namespace xflat
