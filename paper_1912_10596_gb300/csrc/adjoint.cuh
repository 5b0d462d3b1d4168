// Parameters of the discrete-adjoint kernel (two flavours, FP64, classical RK4); see adjoint_2f.cu.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "xflat_internal.cuh"

namespace xflat {

constexpr int kAdjStageVals = 10;   // per stage: mu D (3), mu J1 (3), lambda, R^2/r^2, mu, pad
constexpr int kAdjPartStride = 8;   // doubles per block partial

enum AdjMode : int { kAdjForward = 0, kAdjBackward = 1 };
// broadcast slots: [0, kAdjStageVals) stage constants, then the adjoint moments, then J
constexpr int kGlobAdj = 16, kGlobJ = 24, kGlobWords = 32;

struct AdjParams {
  // problem (instance 0 of a handle)
  uint32_t n_beams, n_energy, n_angle;  // n_beams = 2 n_angle n_energy, beam = (sigma, j, k)
  int32_t mode;                         // kAdjForward / kAdjBackward
  const double* omega;                  // [n_energy] omega_k = dm2 / (2 E_k), 1/km (nubar: -omega_k)
  const double* g;                      // [2][n_energy] signed normalised weights g_{sigma,k}
  const double* u;                      // [n_angle] u_j
  const double* du;                     // [n_angle] du_j
  const double* objw;                   // [n_energy] N_e,k / sum_{j,k} du_j N_e,k
  InstConst ic;                         // B, R^2, mu(r), lambda(r)
  double r0, h;                         // fixed step grid r_n = r0 + n h
  int32_t n_steps, ck_every;            // steps; checkpoint interval (segment length)
  int32_t seg_first, seg_count;         // backward: the segment's first step and length
  // state and scratch, SoA [3][n_beams] unless noted
  double* y;                            // forward working state
  double* ksum;                         // k1 + 2 k2 + 2 k3 (+ k4) of the current step
  double* klast;                        // last stage derivative
  double* ck;                           // [n_ck][3][n]: state at steps 0, K, 2K, ...
  double* seg;                          // [K][3][n]: states at the segment's step starts
  double* stage_sc;                     // [K][4][kAdjStageVals] stage constants of those steps
  double* ystage;                       // [3][3][n]: stage states Y2, Y3, Y4 of the current step
  double* a;                            // adjoint of the state
  double* ybar;                         // adjoint contributions of the stages so far this step
  double* v;                            // cotangent of the current stage derivative
  double* gw;                           // [n] dJ/dw_b (w_b = du_j g_{sigma,k})
  double* gth;                          // [n] dJ/dtheta_v per beam
  double* part;                         // [grid][kAdjPartStride] block partials
  double* glob;                         // [kGlobWords] broadcast values
  Barrier* bar;
  unsigned long long timeout_ns;
  int* status;
};

// Cooperative launch of the adjoint kernel on `stream` with `grid` x kAdjBlock threads.
cudaError_t adjoint_launch(const AdjParams& p, int grid, cudaStream_t stream);
// Resident blocks per SM of the adjoint kernel (0 on error).
int adjoint_blocks_per_sm();
constexpr int kAdjBlock = 256;

// Per-energy sums over angle bins of the final quantities (one thread per (sigma, k)):
//   pee_sum[k]    = sum_j du_j (P_ee(nu, j, k) - J)         (k < n_energy; J from the forward launch)
//   gw_sum[s][k]  = sum_j du_j gw[(s, j, k)]
//   gth_sum[s][k] = sum_j gth[(s, j, k)]
cudaError_t adjoint_energy_sums(const AdjParams& p, double* pee_sum, double* gw_sum, double* gth_sum,
                                cudaStream_t stream);

}  // namespace xflat
