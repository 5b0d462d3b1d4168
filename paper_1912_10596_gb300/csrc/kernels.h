// Registry of the persistent step kernels (instantiated in kernels_2f.cu / kernels_3f.cu).
#pragma once

namespace xflat {
struct KParams;
// The __global__ step kernel for (n_flavor, precision, integrator) built for the requested number
// of resident blocks per SM (mixed two-flavour kernels: 2 or 3; all others: 1), or nullptr.
const void* step_kernel_ptr(int n_flavor, int precision, int integrator, int blocks_per_sm);
}  // namespace xflat
