// Registry of the persistent step kernels (instantiated in kernels_2f.cu / kernels_3f.cu).
#pragma once

namespace xflat {
struct KParams;
// The __global__ step kernel for (n_flavor, precision, integrator) built for the requested block
// size and resident blocks per SM (mixed two-flavour kernels: 256 x 2 or 3, or 512 x 1; all others:
// up to 256 threads, one block), or nullptr.
const void* step_kernel_ptr(int n_flavor, int precision, int integrator, int block, int blocks_per_sm,
                            bool extended = false);
// The adaptive Lie integrator's step kernels (two flavours, bulb model; kernels_lie.cu).
const void* step_kernel_ptr_lie(int precision, int block, int blocks_per_sm);
// The three-flavour exponential integrators' step kernels (kernels_3f_lie.cu).
const void* step_kernel_ptr_3f_exp(int precision, int integrator);
// The extended bulb model's step kernels (two flavours, up to 256 threads, one block per SM).
const void* step_kernel_ptr_2e(int precision, int integrator, int block);
}  // namespace xflat
