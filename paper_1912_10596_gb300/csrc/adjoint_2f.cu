// Discrete adjoint of classical RK4 for the two-flavour bulb model, FP64.
//
// Forward map (Sec. 2, Eq. eom in the Bloch form of the step kernel): every beam b obeys
// ds_b/dr = K_b x s_b with K_b = q_b [eta omega_k B(theta_v) + lambda(r) z + mu(r) (D + t2_b J1)],
// q = 1/cos th_b, t2 = 1 - cos th_b, and the moments D = sum_b w_b t1_b s_b, J1 = sum_b w_b s_b,
// t1 = 1/cos - 1, w_b = du_j g_{sigma,k}.  Objective: J = sum over nu beams of
// du_j objw_k (1 + s_z)/2, the number-flux weighted mean survival probability.
//
// Adjoint of one evaluation k = f(s) with cotangent v (per beam):
//   p_b = s_b x v_b                        (adjoint of K_b)
//   Dbar = mu sum_b q_b p_b,  J1bar = mu sum_b t1_b p_b    (two grid reductions of 3-vectors)
//   sbar_b = v_b x K_b + w_b (t1_b Dbar + J1bar)
//   dJ/dw_b      += s_b . (t1_b Dbar + J1bar)
//   dJ/dtheta_v  += q_b eta omega_k p_b . dB/dtheta
// and RK4 is reversed stage by stage (a' the adjoint of the step's result):
//   v4 = h/6 a',  v3 = h/3 a' + h sbar4,  v2 = h/3 a' + h/2 sbar3,  v1 = h/6 a' + h/2 sbar2,
//   a = a' + sbar4 + sbar3 + sbar2 + sbar1.
//
// Memory: the forward launch stores the state every K steps (checkpoints); each backward launch
// re-runs one segment of K steps forward from its checkpoint, storing every step's start state and
// stage constants, then runs the segment's steps backwards.  Every pass over the beams ends in a
// device-wide barrier whose last block sums the block partials in block order (deterministic).
#include "adjoint.cuh"
#include "step_kernel.cuh"

namespace xflat {
namespace {

constexpr int kAdjGeoSets = 5;       // radii per pass whose geometry is tabulated
constexpr int kAdjGeoRows = 64;      // angle rows per block the table holds

struct AdjShared {
  Geo geo[kAdjGeoSets][kAdjGeoRows];    // per pass: geometry of this block's angle rows
  double scratch[32 * 6];
  double tot[8];
  double scf[kAdjStageVals];            // constants of the stage finished in this pass
  double scs[4][kAdjStageVals];         // constants of the formed stage's step (backward: all 4)
  double gl[8];                         // broadcast adjoint moments of the finished stage
  int flag;
  unsigned int gen;
};

struct BeamC {
  double eo, w, u, ow;                  // eta omega, moment weight, u_j, objective weight (nu)
  uint32_t jj;                          // combined row sigma n_angle + j
};

__device__ __forceinline__ BeamC beam_consts(const AdjParams& p, uint32_t b) {
  const uint32_t per = p.n_angle * p.n_energy;
  const uint32_t sig = b >= per ? 1u : 0u;
  const uint32_t rem = b - sig * per;
  const uint32_t j = rem / p.n_energy, k = rem - j * p.n_energy;
  BeamC c;
  c.eo = sig ? -p.omega[k] : p.omega[k];
  c.w = p.du[j] * p.g[sig * p.n_energy + k];
  c.u = p.u[j];
  c.ow = sig ? 0.0 : p.du[j] * p.objw[k];
  c.jj = sig * p.n_angle + j;
  return c;
}

// Geometry (1/cos, 1/cos - 1, 1 - cos) of every angle row of the beams [b0, b1) at up to
// kAdjGeoSets radii (R^2/r^2 = xof(set)): one FP64 square root and two divisions per (row,
// radius) instead of per beam, which GB300 would run on its two-lane FP64 pipe.  Returns whether
// the rows fit the table (same answer in every thread); if not, callers compute per beam.  The
// caller's __syncthreads publishes the table.
template <class XOf>
__device__ bool fill_geo(const AdjParams& p, AdjShared& S, uint32_t b0, uint32_t b1, XOf xof, uint32_t& row0) {
  row0 = b0 / p.n_energy;
  const uint32_t last = b1 > b0 ? (b1 - 1) / p.n_energy : row0;
  const int rows = (int)(last - row0 + 1);
  if (b1 <= b0 || rows > kAdjGeoRows) return false;
  for (int t = threadIdx.x; t < kAdjGeoSets * rows; t += blockDim.x) {
    const int set = t / rows, r = t - set * rows;
    const uint32_t jj = row0 + r;
    const uint32_t j = jj >= p.n_angle ? jj - p.n_angle : jj;
    S.geo[set][r] = geometry(p.u[j], xof(set));
  }
  return true;
}

__device__ __forceinline__ void ld3(const double* base, uint64_t n, uint32_t b, double (&x)[3]) {
  x[0] = base[b];
  x[1] = base[n + b];
  x[2] = base[2 * n + b];
}
__device__ __forceinline__ void st3(double* base, uint64_t n, uint32_t b, const double (&x)[3]) {
  base[b] = x[0];
  base[n + b] = x[1];
  base[2 * n + b] = x[2];
}
__device__ __forceinline__ void cross(const double (&a)[3], const double (&b)[3], double (&c)[3]) {
  c[0] = a[1] * b[2] - a[2] * b[1];
  c[1] = a[2] * b[0] - a[0] * b[2];
  c[2] = a[0] * b[1] - a[1] * b[0];
}
__device__ __forceinline__ double dot(const double (&a)[3], const double (&b)[3]) {
  return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}

// K_b at a stage with constants sc (mu D, mu J1, lambda, x) and geometry g.
__device__ __forceinline__ void kvec(const double* sc, const Geo& g, double eo, const double* B, double (&K)[3]) {
  K[0] = g.q * (eo * B[0] + sc[0] + g.t2 * sc[3]);
  K[1] = g.q * (sc[1] + g.t2 * sc[4]);
  K[2] = g.q * (eo * B[2] + sc[6] + sc[2] + g.t2 * sc[5]);
}

// RK4: stage s (1..4) forms Y_s = y + a_s h k_{s-1}; weights of k_s in the update.
__device__ __forceinline__ double rk_a(int s) { return s == 4 ? 1.0 : 0.5; }
__device__ __forceinline__ double rk_w(int s) { return (s == 1 || s == 4) ? 1.0 : 2.0; }
__device__ __forceinline__ double rk_c(int s) { return s == 1 ? 0.0 : (s == 4 ? 1.0 : 0.5); }

__device__ __forceinline__ double stage_radius(const AdjParams& p, int n, int s) {
  return (p.r0 + (double)n * p.h) + rk_c(s) * p.h;
}

// Block partials -> grid barrier -> the last block sums them in block order into S.tot.
template <int NV>
__device__ int grid_reduce(const AdjParams& p, AdjShared& S, double (&v)[NV]) {
  block_sum<NV>(v, S.scratch);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int c = 0; c < NV; ++c) p.part[(size_t)blockIdx.x * kAdjPartStride + c] = v[c];
  }
  const int res = barrier_arrive(p.bar, gridDim.x, p.timeout_ns, p.status, &S.flag, &S.gen) & 0xf;
  if (res == kBarLast) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (warp < NV) {
      double s = 0.0;
      for (unsigned b = lane; b < gridDim.x; b += 32) s += __ldcg(&p.part[(size_t)b * kAdjPartStride + warp]);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
      if (lane == 0) S.tot[warp] = s;
    }
    __syncthreads();
  }
  return res;
}

__device__ __forceinline__ void release(const AdjParams& p, AdjShared& S) {
  __threadfence();
  barrier_release(p.bar, 0, &S.gen);
}

// Forward RK4 over steps [n_first, n_first + count) from p.y.  store_seg: each step's start state
// to seg[m] and its stage constants to stage_sc[m]; store_ck: the start state of every step with
// n % K == 0 to ck[n / K]; finish: complete the last step (else stop after its last reduction).
__device__ bool forward_steps(const AdjParams& p, AdjShared& S, int n_first, int count, bool store_seg,
                              bool store_ck, bool finish) {
  const uint64_t n = p.n_beams;
  const uint32_t b0 = (uint32_t)(n * blockIdx.x / gridDim.x), b1 = (uint32_t)(n * (blockIdx.x + 1) / gridDim.x);
  const int P = 4 * count;
  for (int pp = 0; pp <= P; ++pp) {
    if (pp == P && !finish) break;
    const int sp = pp > 0 ? ((pp - 1) & 3) + 1 : 0;        // stage finished in this pass
    const int s = (pp & 3) + 1, m = pp >> 2;                // stage formed in this pass
    const int nstep = n_first + m;
    if (pp > 0 && threadIdx.x < kAdjStageVals) S.scf[threadIdx.x] = __ldcg(&p.glob[threadIdx.x]);
    const double x_s = pp < P ? p.ic.R2 / (stage_radius(p, nstep, s) * stage_radius(p, nstep, s)) : 0.0;
    // geometry sets: 0 the finished stage (its R^2/r^2 was published with its constants), 1 the
    // formed stage
    uint32_t row0;
    const bool tab = fill_geo(p, S, b0, b1, [&](int set) {
      return set == 0 ? (pp > 0 ? __ldcg(&p.glob[7]) : 0.0) : set == 1 ? x_s : 0.0;
    }, row0);
    __syncthreads();
    double acc[6] = {0, 0, 0, 0, 0, 0};
    for (uint32_t b = b0 + threadIdx.x; b < b1; b += blockDim.x) {
      const BeamC c = beam_consts(p, b);
      double y[3], kl[3];
      ld3(p.y, n, b, y);
      ld3(p.klast, n, b, kl);
      if (pp > 0) {
        double ys[3], K[3], k[3], ks[3];
        const double as = sp == 1 ? 0.0 : rk_a(sp) * p.h;
        for (int i = 0; i < 3; ++i) ys[i] = sp == 1 ? y[i] : y[i] + as * kl[i];
        const Geo g = tab ? S.geo[0][c.jj - row0] : geometry(c.u, S.scf[7]);
        kvec(S.scf, g, c.eo, p.ic.B, K);
        cross(K, ys, k);
        if (sp == 1) {
          for (int i = 0; i < 3; ++i) ks[i] = k[i];
        } else {
          ld3(p.ksum, n, b, ks);
          for (int i = 0; i < 3; ++i) ks[i] += rk_w(sp) * k[i];
        }
        if (sp == 4) {
          for (int i = 0; i < 3; ++i) y[i] = y[i] + (p.h / 6.0) * ks[i];
          st3(p.y, n, b, y);
        } else {
          st3(p.ksum, n, b, ks);
        }
        for (int i = 0; i < 3; ++i) kl[i] = k[i];
        st3(p.klast, n, b, kl);
      }
      if (pp < P) {
        if (s == 1) {
          if (store_seg) st3(p.seg + (size_t)m * 3 * n, n, b, y);
          if (store_ck && nstep % p.ck_every == 0) st3(p.ck + (size_t)(nstep / p.ck_every) * 3 * n, n, b, y);
        }
        double ys[3];
        const double as = s == 1 ? 0.0 : rk_a(s) * p.h;
        for (int i = 0; i < 3; ++i) ys[i] = s == 1 ? y[i] : y[i] + as * kl[i];
        const Geo g = tab ? S.geo[1][c.jj - row0] : geometry(c.u, x_s);
        const double wt = c.w * g.t1;
        for (int i = 0; i < 3; ++i) {
          acc[i] += wt * ys[i];
          acc[3 + i] += c.w * ys[i];
        }
      }
    }
    if (pp == P) break;
    const int res = grid_reduce<6>(p, S, acc);
    if (res == kBarAbort) return false;
    if (res == kBarLast) {
      if (threadIdx.x == 0) {
        const double r = stage_radius(p, nstep, s);
        double mu, lam;
        strengths(p.ic, r, mu, lam);
        double sc[kAdjStageVals];
        for (int i = 0; i < 6; ++i) sc[i] = mu * S.tot[i];
        sc[6] = lam;
        sc[7] = x_s;
        sc[8] = mu;
        sc[9] = 0.0;
        for (int i = 0; i < kAdjStageVals; ++i) p.glob[i] = sc[i];
        if (store_seg)
          for (int i = 0; i < kAdjStageVals; ++i) p.stage_sc[((size_t)m * 4 + (s - 1)) * kAdjStageVals + i] = sc[i];
      }
      release(p, S);
    }
  }
  return true;
}

// Objective J and the adjoint of the final state; zero the parameter accumulators.
__device__ bool objective(const AdjParams& p, AdjShared& S) {
  const uint64_t n = p.n_beams;
  const uint32_t b0 = (uint32_t)(n * blockIdx.x / gridDim.x), b1 = (uint32_t)(n * (blockIdx.x + 1) / gridDim.x);
  double acc[1] = {0.0};
  for (uint32_t b = b0 + threadIdx.x; b < b1; b += blockDim.x) {
    const BeamC c = beam_consts(p, b);
    const double sz = p.y[2 * n + b];
    acc[0] += c.ow * 0.5 * (1.0 + sz);
    const double a[3] = {0.0, 0.0, 0.5 * c.ow};
    st3(p.a, n, b, a);
    p.gw[b] = 0.0;
    p.gth[b] = 0.0;
  }
  const int res = grid_reduce<1>(p, S, acc);
  if (res == kBarAbort) return false;
  if (res == kBarLast) {
    if (threadIdx.x == 0) p.glob[kGlobJ] = S.tot[0];
    release(p, S);
  }
  return true;
}

// Backward over the segment's steps [seg_first, seg_first + seg_count), stage by stage.
__device__ bool backward_steps(const AdjParams& p, AdjShared& S) {
  const uint64_t n = p.n_beams;
  const uint32_t b0 = (uint32_t)(n * blockIdx.x / gridDim.x), b1 = (uint32_t)(n * (blockIdx.x + 1) / gridDim.x);
  const int count = p.seg_count;
  const int P = 4 * count;
  const double c2 = -p.ic.B[2], s2 = p.ic.B[0];              // B = (sin 2th, 0, -cos 2th)
  const double dB[3] = {2.0 * c2, 0.0, 2.0 * s2};             // dB / dtheta_v
  const double h = p.h;
  for (int pp = 0; pp <= P; ++pp) {
    const int sp = pp > 0 ? 4 - ((pp - 1) & 3) : 0;         // stage finished (its moments reduced)
    const int mp = pp > 0 ? count - 1 - ((pp - 1) >> 2) : 0;
    const int s = 4 - (pp & 3), m = count - 1 - (pp >> 2);  // stage formed
    if (threadIdx.x < 4 * kAdjStageVals && pp < P)
      S.scs[threadIdx.x / kAdjStageVals][threadIdx.x % kAdjStageVals] =
          __ldcg(&p.stage_sc[(size_t)m * 4 * kAdjStageVals + threadIdx.x]);
    if (pp > 0) {
      if (threadIdx.x < kAdjStageVals)
        S.scf[threadIdx.x] = __ldcg(&p.stage_sc[((size_t)mp * 4 + (sp - 1)) * kAdjStageVals + threadIdx.x]);
      if (threadIdx.x < 6) S.gl[threadIdx.x] = __ldcg(&p.glob[kGlobAdj + threadIdx.x]);
    }
    // geometry sets: 0 the finished stage, 1..4 the stages of the formed stage's step
    uint32_t row0;
    const bool tab = fill_geo(p, S, b0, b1, [&](int set) {
      if (set == 0) return pp > 0 ? __ldcg(&p.stage_sc[((size_t)mp * 4 + (sp - 1)) * kAdjStageVals + 7]) : 0.0;
      return pp < P ? __ldcg(&p.stage_sc[((size_t)m * 4 + (set - 1)) * kAdjStageVals + 7]) : 0.0;
    }, row0);
    __syncthreads();
    double acc[6] = {0, 0, 0, 0, 0, 0};
    for (uint32_t b = b0 + threadIdx.x; b < b1; b += blockDim.x) {
      const BeamC c = beam_consts(p, b);
      double a[3];
      ld3(p.a, n, b, a);
      double vnext[3] = {0, 0, 0};
      if (pp > 0) {
        double ys[3], v[3], K[3], pv[3], t[3];
        if (sp == 1) ld3(p.seg + (size_t)mp * 3 * n, n, b, ys);
        else ld3(p.ystage + (size_t)(sp - 2) * 3 * n, n, b, ys);
        ld3(p.v, n, b, v);
        const Geo g = tab ? S.geo[0][c.jj - row0] : geometry(c.u, S.scf[7]);
        kvec(S.scf, g, c.eo, p.ic.B, K);
        double br[3];
        for (int i = 0; i < 3; ++i) br[i] = g.t1 * S.gl[i] + S.gl[3 + i];
        cross(v, K, t);
        double sb[3];
        for (int i = 0; i < 3; ++i) sb[i] = t[i] + c.w * br[i];
        p.gw[b] += dot(ys, br);
        cross(ys, v, pv);
        p.gth[b] += g.q * c.eo * dot(pv, dB);
        double yb[3];
        if (sp == 4) {
          for (int i = 0; i < 3; ++i) { yb[i] = sb[i]; vnext[i] = (h / 3.0) * a[i] + h * sb[i]; }
        } else {
          ld3(p.ybar, n, b, yb);
          for (int i = 0; i < 3; ++i) yb[i] += sb[i];
          if (sp == 3) for (int i = 0; i < 3; ++i) vnext[i] = (h / 3.0) * a[i] + (0.5 * h) * sb[i];
          if (sp == 2) for (int i = 0; i < 3; ++i) vnext[i] = (h / 6.0) * a[i] + (0.5 * h) * sb[i];
        }
        if (sp == 1) {
          for (int i = 0; i < 3; ++i) a[i] += yb[i];
          st3(p.a, n, b, a);
        } else {
          st3(p.ybar, n, b, yb);
        }
      }
      if (pp < P) {
        double ys[3], v[3];
        if (s == 4) {
          // stage states of step m from its start state and stored stage constants
          double y[3], k[3], K[3], yy[3];
          ld3(p.seg + (size_t)m * 3 * n, n, b, y);
          for (int i = 0; i < 3; ++i) yy[i] = y[i];
          for (int st = 1; st <= 3; ++st) {
            const Geo g = tab ? S.geo[st][c.jj - row0] : geometry(c.u, S.scs[st - 1][7]);
            kvec(S.scs[st - 1], g, c.eo, p.ic.B, K);
            cross(K, yy, k);
            const double as = rk_a(st + 1) * h;
            for (int i = 0; i < 3; ++i) yy[i] = y[i] + as * k[i];
            st3(p.ystage + (size_t)(st - 1) * 3 * n, n, b, yy);
          }
          for (int i = 0; i < 3; ++i) { ys[i] = yy[i]; v[i] = (h / 6.0) * a[i]; }
        } else {
          if (s == 1) ld3(p.seg + (size_t)m * 3 * n, n, b, ys);
          else ld3(p.ystage + (size_t)(s - 2) * 3 * n, n, b, ys);
          for (int i = 0; i < 3; ++i) v[i] = vnext[i];
        }
        st3(p.v, n, b, v);
        double pv[3];
        cross(ys, v, pv);
        const Geo g = tab ? S.geo[s][c.jj - row0] : geometry(c.u, S.scs[s - 1][7]);
        for (int i = 0; i < 3; ++i) {
          acc[i] += g.q * pv[i];
          acc[3 + i] += g.t1 * pv[i];
        }
      }
    }
    if (pp == P) break;
    const int res = grid_reduce<6>(p, S, acc);
    if (res == kBarAbort) return false;
    if (res == kBarLast) {
      if (threadIdx.x == 0) {
        const double mu = S.scs[s - 1][8];
        for (int i = 0; i < 6; ++i) p.glob[kGlobAdj + i] = mu * S.tot[i];
      }
      release(p, S);
    }
  }
  return true;
}

__global__ void __launch_bounds__(kAdjBlock, 1) adjoint_kernel(AdjParams p) {
  __shared__ AdjShared S;
  if (threadIdx.x == 0) S.gen = ld_acquire(&p.bar->gen);
  __syncthreads();
  if (p.mode == kAdjForward) {
    if (!forward_steps(p, S, 0, p.n_steps, false, true, true)) return;
    objective(p, S);
    return;
  }
  // backward over one segment: re-run it forward from its checkpoint, then reverse it
  const uint64_t n = p.n_beams;
  const uint32_t b0 = (uint32_t)(n * blockIdx.x / gridDim.x), b1 = (uint32_t)(n * (blockIdx.x + 1) / gridDim.x);
  const double* ck = p.ck + (size_t)(p.seg_first / p.ck_every) * 3 * n;
  for (uint32_t b = b0 + threadIdx.x; b < b1; b += blockDim.x) {
    double y[3];
    ld3(ck, n, b, y);
    st3(p.y, n, b, y);
  }
  if (!forward_steps(p, S, p.seg_first, p.seg_count, true, false, false)) return;
  backward_steps(p, S);
}

__global__ void adjoint_sums_kernel(AdjParams p, double* pee_sum, double* gw_sum, double* gth_sum) {
  const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 2 * p.n_energy) return;
  const uint32_t sig = t / p.n_energy, k = t - sig * p.n_energy;
  const uint64_t n = p.n_beams;
  const double J = p.glob[kGlobJ];
  double ps = 0.0, gs = 0.0, ts = 0.0;
  for (uint32_t j = 0; j < p.n_angle; ++j) {
    const uint32_t b = (sig * p.n_angle + j) * p.n_energy + k;
    if (!sig) ps += p.du[j] * (0.5 * (1.0 + p.y[2 * n + b]) - J);
    gs += p.du[j] * p.gw[b];
    ts += p.gth[b];
  }
  if (!sig) pee_sum[k] = ps;
  gw_sum[t] = gs;
  gth_sum[t] = ts;
}

}  // namespace

cudaError_t adjoint_launch(const AdjParams& p, int grid, cudaStream_t stream) {
  AdjParams q = p;
  void* args[] = {&q};
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(kAdjBlock);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelExC(&cfg, (const void*)adjoint_kernel, args);
}

int adjoint_blocks_per_sm() {
  int occ = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, adjoint_kernel, kAdjBlock, 0) != cudaSuccess) return 0;
  return occ;
}

cudaError_t adjoint_energy_sums(const AdjParams& p, double* pee_sum, double* gw_sum, double* gth_sum,
                                cudaStream_t stream) {
  const unsigned nt = 2 * p.n_energy;
  adjoint_sums_kernel<<<(nt + 127) / 128, 128, 0, stream>>>(p, pee_sum, gw_sum, gth_sum);
  return cudaGetLastError();
}

}  // namespace xflat
