// Allocation-free moment reduction (two flavours): xflat_moments_2f_noalloc.
//
// Some callers cannot allocate device memory when they need the moments: a host framework that
// owns the whole device memory pool through its own allocator, or a time-critical loop that must
// not stall, because cudaMalloc/cudaFree can synchronise the device and can fail under memory
// pressure.  This entry point computes the same two moments as xflat_moments, but takes everything
// as caller-owned device pointers and keeps its only scratch -- one row of partial sums per
// (species, angle) bin plus a completion counter -- in a fixed-size array that lives in the
// library image on every device that loads the library, for the lifetime of the process.
//
// The reduction follows the paper's layering (energy integral inside each angle bin, then the
// angular integral): one block per (species, angle) row sums its energies, writes its row to the
// scratch array, and the last block to finish sums the rows in row order (deterministic).
#include <cstdint>
#include <mutex>

#include <cuda_runtime.h>

#include "../../include/xflat.h"

namespace {

constexpr uint32_t kRows = 2 * XFLAT_NOALLOC_MAX_ANGLES;   // (species, angle) rows
constexpr int kRowLen = 6;                                 // j0 (3), j1 (3)

// element 0: completion counter (bits of an unsigned 64-bit integer); then kRows x kRowLen doubles
static __device__ __align__(256) double g_noalloc_scratch[1 + kRows * kRowLen];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
double* g_scratch_ptr[kMaxDevices] = {};

__global__ void k_moments_rows(const double* __restrict__ s, uint32_t n_energy, uint32_t n_angle,
                               const double* __restrict__ g, const double* __restrict__ u,
                               const double* __restrict__ du, double x, double* scratch,
                               double* __restrict__ out) {
  const uint32_t jj = blockIdx.x;                     // species * n_angle + j
  const uint32_t sigma = jj >= n_angle ? 1u : 0u;
  const uint32_t j = jj - sigma * n_angle;
  const uint64_t nb = 2ull * n_angle * n_energy;
  const double* gk = g + (size_t)sigma * n_energy;
  double a[3] = {0, 0, 0};
  for (uint32_t k = threadIdx.x; k < n_energy; k += blockDim.x) {
    const uint64_t b = (uint64_t)jj * n_energy + k;
    const double w = gk[k];
    a[0] += w * s[b];
    a[1] += w * s[nb + b];
    a[2] += w * s[2 * nb + b];
  }
  // fixed shuffle tree, then fixed tree over warps
  __shared__ double red[32][3];
  __shared__ bool last;
  for (int i = 0; i < 3; ++i)
    for (int o = 16; o > 0; o >>= 1) a[i] += __shfl_down_sync(0xffffffffu, a[i], o);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  if (lane == 0)
    for (int i = 0; i < 3; ++i) red[warp][i] = a[i];
  __syncthreads();
  double* rows = scratch + 1;
  if (threadIdx.x == 0) {
    double t[3] = {0, 0, 0};
    for (int w = 0; w < nw; ++w)
      for (int i = 0; i < 3; ++i) t[i] += red[w][i];
    const double c = sqrt(1.0 - u[j] * x);            // cos(theta) of this angle bin at radius r
    for (int i = 0; i < 3; ++i) {
      rows[(size_t)jj * kRowLen + i] = du[j] * t[i] / c;     // contribution to J0
      rows[(size_t)jj * kRowLen + 3 + i] = du[j] * t[i];     // contribution to J1
    }
    __threadfence();
    unsigned long long* counter = reinterpret_cast<unsigned long long*>(scratch);
    const unsigned long long done = atomicAdd(counter, 1ull);
    last = (done == (unsigned long long)gridDim.x - 1);
  }
  __syncthreads();
  if (!last) return;
  // the last block: rows in fixed order, one component per thread, then reset the counter
  __threadfence();
  if (threadIdx.x < kRowLen) {
    double sum = 0;
    for (uint32_t r = 0; r < gridDim.x; ++r) sum += __ldcg(rows + (size_t)r * kRowLen + threadIdx.x);
    out[threadIdx.x] = sum;
  }
  __syncthreads();
  if (threadIdx.x == 0) *reinterpret_cast<unsigned long long*>(scratch) = 0ull;
}

}  // namespace

extern "C" int xflat_moments_2f_noalloc(const double* d_state, uint32_t n_energy, uint32_t n_angle,
                                        const double* d_g, const double* d_u, const double* d_du,
                                        double R_km, double r_km, double* d_J, void* cuda_stream) {
  if (!d_state || !d_g || !d_u || !d_du || !d_J) return XFLAT_ERR_INVAL;
  if (n_energy < 1 || n_angle < 1) return XFLAT_ERR_INVAL;
  if (n_angle > XFLAT_NOALLOC_MAX_ANGLES) return XFLAT_ERR_INVAL;   // scratch holds 2 rows per angle
  if (!(R_km > 0) || !(r_km >= R_km)) return XFLAT_ERR_INVAL;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return XFLAT_ERR_CUDA;
  double* scratch = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_ptr[dev]) {
      // once per device, with that device current: the device address of the scratch array (in
      // host code its name is only a stand-in, not a device address)
      void* p = nullptr;
      if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return XFLAT_ERR_CUDA;
      g_scratch_ptr[dev] = static_cast<double*>(p);
    }
    scratch = g_scratch_ptr[dev];
  }
  cudaStream_t stream = static_cast<cudaStream_t>(cuda_stream);
  // the completion counter must start at zero (the rows are fully overwritten by every call)
  if (cudaMemsetAsync(scratch, 0, sizeof(double), stream) != cudaSuccess) return XFLAT_ERR_CUDA;
  const double x = (R_km * R_km) / (r_km * r_km);
  // cudaLaunchKernel returns this launch's own error: an unrelated error left pending on the thread
  // by earlier work is neither reported as this call's failure nor cleared
  void* args[] = {(void*)&d_state, (void*)&n_energy, (void*)&n_angle, (void*)&d_g, (void*)&d_u,
                  (void*)&d_du, (void*)&x, (void*)&scratch, (void*)&d_J};
  const cudaError_t e = cudaLaunchKernel((const void*)k_moments_rows, dim3(2 * n_angle), dim3(256),
                                         args, 0, stream);
  return e == cudaSuccess ? XFLAT_OK : XFLAT_ERR_CUDA;
}
