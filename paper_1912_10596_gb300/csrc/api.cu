// C ABI of the bulb-model solver: argument checks, tables, memory, launches (see include/xflat.h).
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/xflat.h"
#include "adjoint.cuh"
#include "kernels.h"
#include "xflat_internal.cuh"
#include "step_kernel.cuh"

#include <nvtx3/nvToolsExt.h>

using namespace xflat;

namespace {

// ---- tracing and allocation-failure injection ---------------------------------------------------
// Every exported call is one NVTX range named after the call (visible in any NVTX-aware profiler;
// a check of one pointer when none is attached).
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
};
#define XFLAT_TRACE() NvtxRange xflat_trace_range_(__func__)

// Allocation-failure injection for tests of the cleanup paths: after xflat_debug_fail_alloc(n),
// the n-th device or pinned-host allocation the library makes fails as if memory were exhausted
// (process-wide, once; 0 disarms).
std::atomic<long> g_fail_alloc{0};
bool injected_failure() {
  long v = g_fail_alloc.load();
  while (v > 0)
    if (g_fail_alloc.compare_exchange_weak(v, v - 1)) return v == 1;
  return false;
}
template <class T>
cudaError_t dev_alloc(T** p, size_t bytes) {
  if (injected_failure()) {
    *p = nullptr;
    return cudaErrorMemoryAllocation;
  }
  return cudaMalloc(reinterpret_cast<void**>(p), bytes);
}
template <class T>
cudaError_t host_alloc(T** p, size_t bytes) {
  if (injected_failure()) {
    *p = nullptr;
    return cudaErrorMemoryAllocation;
  }
  return cudaMallocHost(reinterpret_cast<void**>(p), bytes);
}

// ---- physical constants (CODATA 2018 / SI 2019) ------------------------------------------------
constexpr double kGF = 1.1663787e-5;                       // G_F / (hbar c)^3, GeV^-2
constexpr double kHbarcEvKm = 197.3269804e6 * 1e-18;       // hbar c in eV km
constexpr double kHbarcGevKm = 197.3269804e-3 * 1e-18;     // hbar c in GeV km
constexpr double kCkms = 299792.458;                       // km / s
constexpr double kMuG = 1.66053906660e-24;                 // atomic mass unit, g
constexpr double kPi = 3.14159265358979323846;
// sqrt(2) G_F (hbar c)^2: multiplies a number density in 1/km^3 to give 1/km
const double kSqrt2GFhc2 = std::sqrt(2.0) * kGF * kHbarcGevKm * kHbarcGevKm;

constexpr uint32_t kMaxJJ = 128;          // combined angle bins per piece (shared-memory table rows)
constexpr uint32_t kAlignBeams = 4;       // instance offsets and piece starts: 16-byte vectors
uint32_t max_jj_cap(int nf, size_t real_size, bool ext = false);

struct HostInst {
  xflat_config cfg;
  uint32_t n_beams = 0, n_pad = 0;
  uint64_t off = 0;
  std::vector<double> u, du;
  std::vector<double> N;                  // [2][nf][ne]
  bool spectra = false;
  std::vector<double> mtab;               // matter table [n][3]: r_i, lambda_i, exponent p_i
  uint32_t e_off = 0, a_off = 0;
};

}  // namespace

struct xflat_s {
  std::vector<HostInst> inst;
  int nf = 2, precision = 0, integrator = 0;
  bool extended = false;                   // extended bulb model (azimuthal bins)
  size_t real_size = 8;
  int nc = 3;
  cudaStream_t stream = nullptr;
  int device = 0, sm_count = 0;
  // device memory
  void* planes = nullptr;                  // [2][nc][stride] Real
  void* escr = nullptr;                    // DP45: error partial + scale planes [nc + 1][stride] Real
  void* kst = nullptr;                     // FP64 RK4 / DP45: stage derivatives + one stage state [n + 1][nc][stride] Real
  uint64_t stride = 0;
  InstConst* d_ic = nullptr;
  InstDyn* d_dyn = nullptr;
  Piece* d_pieces = nullptr;
  int* d_blk = nullptr;
  unsigned long long* d_acc = nullptr;
  unsigned long long* d_errmax = nullptr;
  int* d_nonfinite = nullptr;
  void* d_etab = nullptr;
  double* d_u = nullptr;
  double* d_du = nullptr;
  Barrier* d_bar = nullptr;
  int* d_words = nullptr;                  // [0] status, [1] all_done
  int* h_words = nullptr;                  // pinned mirror
  double* d_stage = nullptr;               // staging for conversions
  double* d_mtab = nullptr;                // every instance's matter table, concatenated
  size_t stage_bytes = 0;
  // allocation sizes in bytes (the checked build hands them to the kernel with the pointers)
  size_t planes_bytes = 0, escr_bytes = 0, kst_bytes = 0, etab_bytes = 0, angle_bytes = 0;
  // host mirrors
  std::vector<InstConst> ic;
  std::vector<InstDyn> dyn;
  std::vector<Piece> pieces;
  std::vector<int> blk;
  const void* kernel = nullptr;
  int block = 256, grid = 0;
  size_t smem = 0;
  int max_jj = 1;
  uint64_t launches = 0;
  uint32_t steps_per_launch = 64;
  uint64_t timeout_ns = 2000000000ull;
  uint32_t debug_extra = 0;
  unsigned long long* d_trace = nullptr;   // pass trace (xflat_debug_trace)
  uint32_t trace_passes = 0;
  cudaGraph_t graph = nullptr;             // captured launches of xflat_advance_graph
  cudaGraphExec_t graph_exec = nullptr;
  uint32_t graph_launches = 0, graph_steps = 0;
  bool moments_valid = false;
  bool advancing = false;                  // last call was an xflat_advance launch
  // beam shard of one instance (xflat_create_shard): the handle integrates beams [shard_lo,
  // shard_hi) only, one pass per launch, and the host exchanges the stage moments between passes
  bool shard = false;
  uint32_t shard_lo = 0, shard_hi = 0;
  // dynamic piece scheduling (several instances): blocks take pieces from a device-wide counter
  bool dyn_sched = false;
  int shard_last = -2;                     // the last pass launched (-1: moment pass), -2: none
  std::string err;
};

namespace {

int fail(xflat_t h, int code, const std::string& msg) {
  if (h) h->err = msg;
  return code;
}

#define CUDA_TRY(h, call)                                                                  \
  do {                                                                                     \
    cudaError_t e_ = (call);                                                               \
    if (e_ != cudaSuccess)                                                                 \
      return fail(h, XFLAT_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

bool is_fin(double x) { return std::isfinite(x); }
// combined angle bins (u x phi) of an instance: n_angle, times n_phi for the extended bulb model
uint32_t angle_bins(const xflat_config& c) { return c.n_angle * (c.n_phi >= 2 ? c.n_phi : 1u); }
// integrators with embedded error control (adaptive step size)
bool adaptive(uint32_t integrator) {
  return integrator == XFLAT_DP45 || integrator == XFLAT_EXP_MIDPOINT || integrator == XFLAT_LIE_ADAPTIVE;
}
// stage slots (0..S) of the integrator's tableau: the rows of the step kernel's shared-memory table
int table_stages(int integrator) {
  return integrator == XFLAT_DP45 ? 8 : integrator == XFLAT_EXP_MIDPOINT ? 4 : integrator == XFLAT_LIE_ADAPTIVE ? 12 : 5;
}

int check_config(const xflat_config& c, std::string& why) {
  if (c.abi_version != XFLAT_ABI_VERSION) { why = "abi_version mismatch"; return XFLAT_ERR_INVAL; }
  if (c.n_flavor != 2 && c.n_flavor != 3) { why = "n_flavor must be 2 or 3"; return XFLAT_ERR_INVAL; }
  if (c.n_energy < 1 || c.n_angle < 1) { why = "n_energy and n_angle must be >= 1"; return XFLAT_ERR_INVAL; }
  if (c.n_phi >= 2 && c.n_flavor != 2) { why = "the extended bulb model is two-flavour only"; return XFLAT_ERR_UNSUPPORTED; }
  if (c.n_phi > 4096) { why = "n_phi must be <= 4096"; return XFLAT_ERR_INVAL; }
  const uint64_t nb = 2ull * c.n_energy * c.n_angle * (c.n_phi >= 2 ? c.n_phi : 1u);
  if (nb >= (1ull << 31)) { why = "too many beams in one instance"; return XFLAT_ERR_INVAL; }
  if (nb * (uint64_t)c.n_energy >= (1ull << 40)) { why = "n_beams * n_energy must be < 2^40"; return XFLAT_ERR_INVAL; }
  if (c.precision > 1) { why = "precision must be FP64 or MIXED"; return XFLAT_ERR_INVAL; }
  if (c.integrator > 4) { why = "unknown integrator"; return XFLAT_ERR_INVAL; }
  if (c.integrator == XFLAT_LIE_ADAPTIVE && c.n_phi >= 2) {
    why = "the adaptive Lie integrator is built for the bulb model only"; return XFLAT_ERR_UNSUPPORTED;
  }
  if (c.matter_kind > 3) { why = "unknown matter_kind"; return XFLAT_ERR_INVAL; }
  if (c.geometry > 2) { why = "unknown geometry"; return XFLAT_ERR_INVAL; }
  if (c.geometry != XFLAT_GEOMETRY_BULB && c.n_phi >= 2) {
    why = "the extended bulb model has the bulb geometry only"; return XFLAT_ERR_UNSUPPORTED;
  }
  if (c.geometry == XFLAT_GEOMETRY_HOMOGENEOUS && !is_fin(c.mu_const_kmi)) {
    why = "mu_const_kmi must be finite"; return XFLAT_ERR_INVAL;
  }
  if (!(c.R_km > 0) || !is_fin(c.R_km)) { why = "R_km must be > 0"; return XFLAT_ERR_INVAL; }
  if (!(c.E_min_MeV > 0) || !(c.E_max_MeV > c.E_min_MeV) || !is_fin(c.E_max_MeV)) { why = "need 0 < E_min < E_max"; return XFLAT_ERR_INVAL; }
  for (int i = 0; i < 2; ++i) if (!is_fin(c.dm2_eV2[i])) { why = "dm2 not finite"; return XFLAT_ERR_INVAL; }
  for (int i = 0; i < 3; ++i) if (!is_fin(c.theta[i])) { why = "theta not finite"; return XFLAT_ERR_INVAL; }
  if (adaptive(c.integrator)) {
    if (!(c.rtol >= 0) || !(c.atol >= 0) || !(c.rtol + c.atol > 0)) { why = "need rtol, atol >= 0, not both 0"; return XFLAT_ERR_INVAL; }
    if (!(c.h0_km > 0) || !(c.h_min_km >= 0)) { why = "need h0 > 0 and h_min >= 0"; return XFLAT_ERR_INVAL; }
  } else if (!(c.fixed_dr_km > 0)) { why = "fixed-step integrators need fixed_dr_km > 0"; return XFLAT_ERR_INVAL; }
  if (c.matter_kind == XFLAT_MATTER_POWER_LAW &&
      (!(c.rho0_gcc >= 0) || !(c.r_ref_km > 0) || !is_fin(c.power) || !(c.Ye >= 0))) {
    why = "bad power-law matter parameters"; return XFLAT_ERR_INVAL;
  }
  if (c.matter_kind == XFLAT_MATTER_CONSTANT && !is_fin(c.lambda_const_kmi)) { why = "bad lambda_const"; return XFLAT_ERR_INVAL; }
  if (c.block_size != 0 && c.block_size != 128 && c.block_size != 256 && c.block_size != 512) {
    why = "block_size must be 0, 128, 256 or 512"; return XFLAT_ERR_INVAL;
  }
  return XFLAT_OK;
}

// Real three-flavour mixing U = R23 R13 R12 and the unit vacuum matrices U diag(0,1,0) U^T,
// U diag(0,0,1) U^T (entries 00, 11, 22, 01, 02, 12).
void vacuum_matrices_3f(const double th[3], double M21[6], double M31[6]) {
  const double c12 = std::cos(th[0]), s12 = std::sin(th[0]);
  const double c13 = std::cos(th[1]), s13 = std::sin(th[1]);
  const double c23 = std::cos(th[2]), s23 = std::sin(th[2]);
  const double R12[3][3] = {{c12, s12, 0}, {-s12, c12, 0}, {0, 0, 1}};
  const double R13[3][3] = {{c13, 0, s13}, {0, 1, 0}, {-s13, 0, c13}};
  const double R23[3][3] = {{1, 0, 0}, {0, c23, s23}, {0, -s23, c23}};
  double T[3][3] = {}, U[3][3] = {};
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b)
      for (int k = 0; k < 3; ++k) T[a][b] += R13[a][k] * R12[k][b];
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b)
      for (int k = 0; k < 3; ++k) U[a][b] += R23[a][k] * T[k][b];
  const int ia[6] = {0, 1, 2, 0, 0, 1}, ib[6] = {0, 1, 2, 1, 2, 2};
  for (int e = 0; e < 6; ++e) {
    M21[e] = U[ia[e]][1] * U[ib[e]][1];
    M31[e] = U[ia[e]][2] * U[ib[e]][2];
  }
}

// ---- small device kernels (state set-up, conversions, observables) ---------------------------
template <typename Real>
__global__ void k_initial_state(Real* planes, uint64_t stride, uint64_t n_total, int nf) {
  const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_total) return;
  const int nc = nf == 2 ? 3 : 9;
  for (int b = 0; b < 2; ++b)
    for (int c = 0; c < nc; ++c) {
      Real v = 0;
      if (nf == 2 && c == 2) v = 1;      // s = z: P = diag(1, 0)
      if (nf == 3 && c == 0) v = 1;      // P = diag(1, 0, 0)
      planes[((uint64_t)b * nc + c) * stride + i] = v;
    }
}

// native (Real, internal convention) -> double dst in the requested layout
template <typename Real>
__global__ void k_export(const Real* src, uint64_t stride, uint32_t n, uint32_t n_nu, int nf, int layout,
                         double* dst) {
  const uint32_t b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= n) return;
  const bool bar = b >= n_nu;
  if (layout == XFLAT_LAYOUT_NATIVE) {
    const int nc = nf == 2 ? 3 : 9;
    for (int c = 0; c < nc; ++c) dst[(uint64_t)c * n + b] = (double)src[(uint64_t)c * stride + b];
    return;
  }
  double* m = dst + (uint64_t)b * 2 * nf * nf;
  const double sg = bar ? -1.0 : 1.0;       // antineutrinos: the paper's Pbar = conj(internal)
  if (nf == 2) {
    const double sx = src[b], sy = src[stride + b], sz = src[2 * stride + b];
    m[0] = 0.5 * (1 + sz); m[1] = 0;
    m[2] = 0.5 * sx;       m[3] = -0.5 * sy * sg;
    m[4] = 0.5 * sx;       m[5] = 0.5 * sy * sg;
    m[6] = 0.5 * (1 - sz); m[7] = 0;
  } else {
    double v[9];
    for (int c = 0; c < 9; ++c) v[c] = (double)src[(uint64_t)c * stride + b];
    const double re[3][3] = {{v[0], v[3], v[5]}, {v[3], v[1], v[7]}, {v[5], v[7], v[2]}};
    const double im[3][3] = {{0, v[4], v[6]}, {-v[4], 0, v[8]}, {-v[6], -v[8], 0}};
    for (int a = 0; a < 3; ++a)
      for (int c = 0; c < 3; ++c) {
        m[(a * 3 + c) * 2] = re[a][c];
        m[(a * 3 + c) * 2 + 1] = sg * im[a][c];
      }
  }
}

template <typename Real>
__global__ void k_import(const double* srcd, uint64_t stride, uint32_t n, uint32_t n_nu, int nf, int layout,
                         Real* dst) {
  const uint32_t b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= n) return;
  const bool bar = b >= n_nu;
  if (layout == XFLAT_LAYOUT_NATIVE) {
    const int nc = nf == 2 ? 3 : 9;
    for (int c = 0; c < nc; ++c) dst[(uint64_t)c * stride + b] = (Real)srcd[(uint64_t)c * n + b];
    return;
  }
  const double* m = srcd + (uint64_t)b * 2 * nf * nf;
  const double sg = bar ? -1.0 : 1.0;
  if (nf == 2) {
    // P = (1 + s.sigma)/2: sx = 2 Re P01, sy = -2 Im P01, sz = P00 - P11 (nubar: conjugate first)
    dst[b] = (Real)(2 * m[2]);
    dst[stride + b] = (Real)(-2 * sg * m[3]);
    dst[2 * stride + b] = (Real)(m[0] - m[6]);
  } else {
    const int d[3] = {0, 4, 8};
    for (int a = 0; a < 3; ++a) dst[(uint64_t)a * stride + b] = (Real)m[d[a] * 2];
    const int off[3] = {1, 2, 5};   // (0,1), (0,2), (1,2)
    for (int e = 0; e < 3; ++e) {
      dst[(uint64_t)(3 + 2 * e) * stride + b] = (Real)m[off[e] * 2];
      dst[(uint64_t)(4 + 2 * e) * stride + b] = (Real)(sg * m[off[e] * 2 + 1]);
    }
  }
}

// P_ee per beam and the deterministic weighted mean over nu beams (one block, fixed tree).
template <typename Real>
__global__ void k_pee(const Real* src, uint64_t stride, uint32_t n, int nf, double* pee) {
  const uint32_t b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= n) return;
  pee[b] = nf == 2 ? 0.5 * (1.0 + (double)src[2 * stride + b]) : (double)src[b];
}

// Number-flux weighted mean of P_ee over nu beams, deterministic and spread over the GPU (the
// sums are FP64, whose pipe is narrow: one block would take milliseconds at 2M beams).  One warp
// per angle bin sums N_e,k P_ee over energies (lanes in a fixed order, then a fixed shuffle tree);
// one block then sums du_j times the rows in a fixed tree.
__global__ void k_pee_rows(const double* pee, const double* N_e, uint32_t ne, uint32_t na, double* rows) {
  const uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (warp >= na) return;
  double s = 0.0;
  for (uint32_t k = lane; k < ne; k += 32) s += N_e[k] * pee[(uint64_t)warp * ne + k];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if (lane == 0) rows[warp] = s;
}

__global__ void k_pee_final(const double* rows, const double* du, uint32_t na, double den, double* out) {
  __shared__ double sn[1024];
  double num = 0.0;
  for (uint32_t j = threadIdx.x; j < na; j += blockDim.x) num += du[j] * rows[j];
  sn[threadIdx.x] = num;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) sn[threadIdx.x] += sn[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[0] = den > 0 ? sn[0] / den : 0.0;
}

// Number-flux energy spectra: one thread per (species, flavour a, energy k), angle bins summed in
// order: Phi = sum_j du_j [N_e P_ea + N_x (1 - P_ea)], P_ea the a-a entry of the electron-flavour
// state (unitarity: the x states carry 1 - P_ea into flavour a).
template <typename Real>
__global__ void k_flux_spectra(const Real* src, uint64_t stride, uint32_t ne, uint32_t na, int nf,
                               const double* N, const double* du, double* flux) {
  const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 2u * nf * ne) return;
  const uint32_t sig = t / (nf * ne), a = (t / ne) % nf, k = t % ne;
  const double Ne = N[(sig * nf + 0) * ne + k], Nx = N[(sig * nf + 1) * ne + k];
  double f = 0.0;
  for (uint32_t j = 0; j < na; ++j) {
    const uint64_t b = ((uint64_t)sig * na + j) * ne + k;
    double P;
    if (nf == 2) {
      const double sz = (double)src[2 * stride + b];
      P = a == 0 ? 0.5 * (1.0 + sz) : 0.5 * (1.0 - sz);
    } else {
      P = (double)src[(uint64_t)a * stride + b];
    }
    f += du[j] * (Ne * P + Nx * (1.0 - P));
  }
  flux[t] = f;
}

// ---- host helpers ------------------------------------------------------------------------------
void build_tables(xflat_t h, HostInst& I, std::vector<double>& et, InstConst& ic) {
  const xflat_config& c = I.cfg;
  const uint32_t ne = c.n_energy, nf = c.n_flavor;
  const double dE = (c.E_max_MeV - c.E_min_MeV) / ne;
  const int ntab = nf == 2 ? 3 : 4;
  et.assign((size_t)ntab * ne, 0.0);
  // weight scale: total number luminosity of every listed species, flavour and bin
  double S = 0;
  for (double v : I.N) S += std::fabs(v);
  const double wscale = S > 0 ? S : 1.0;
  for (uint32_t k = 0; k < ne; ++k) {
    const double E = c.E_min_MeV + (k + 0.5) * dE;
    const double inv2E = 1.0 / (2.0 * E * 1e6 * kHbarcEvKm);     // 1/(2E) per eV^2, in 1/km
    const double Ne = I.N[(0 * nf + 0) * ne + k], Nx = I.N[(0 * nf + 1) * ne + k];
    const double Nbe = I.N[(1 * nf + 0) * ne + k], Nbx = I.N[(1 * nf + 1) * ne + k];
    if (nf == 2) {
      et[k] = c.dm2_eV2[0] * inv2E;
      et[ne + k] = (Ne - Nx) / wscale;
      et[2 * ne + k] = -(Nbe - Nbx) / wscale;
    } else {
      et[k] = c.dm2_eV2[0] * inv2E;
      et[ne + k] = c.dm2_eV2[1] * inv2E;
      et[2 * ne + k] = (Ne - Nx) / wscale;
      et[3 * ne + k] = -(Nbe - Nbx) / wscale;
    }
  }
  ic.wscale = wscale;
  ic.mu_coef = kSqrt2GFhc2 * wscale / (4.0 * kPi * kCkms);
  (void)h;
}

void fill_inst_const(HostInst& I, InstConst& ic) {
  const xflat_config& c = I.cfg;
  ic.beam_off = I.off;
  ic.n_beams = I.n_beams;
  ic.n_energy = c.n_energy;
  ic.n_angle = angle_bins(c);
  ic.n_phi = c.n_phi >= 2 ? c.n_phi : 1u;
  ic.e_off = I.e_off;
  ic.a_off = I.a_off;
  ic.div_magic = (1ull << 40) / c.n_energy + 1;
  ic.R2 = c.R_km * c.R_km;
  ic.matter = (int)c.matter_kind;
  ic.adaptive = adaptive(c.integrator);
  ic.r_ref = c.r_ref_km > 0 ? c.r_ref_km : 1.0;
  ic.power = c.power;
  ic.lam_coef = c.matter_kind == XFLAT_MATTER_POWER_LAW ? kSqrt2GFhc2 * c.Ye * c.rho0_gcc / kMuG * 1e15 : 0.0;
  ic.lam_const = c.lambda_const_kmi;
  ic.geom = (int)c.geometry;
  ic.mu_const = c.mu_const_kmi;
  ic.B[0] = std::sin(2 * c.theta[0]);
  ic.B[1] = 0.0;
  ic.B[2] = -std::cos(2 * c.theta[0]);
  if (c.n_flavor == 3) vacuum_matrices_3f(c.theta, ic.M21, ic.M31);
  ic.rtol = c.rtol;
  ic.atol = c.atol;
  ic.h_min = c.h_min_km;
  ic.h_max = c.h_max_km > 0 ? c.h_max_km : INFINITY;
}

int upload_inst(xflat_t h) {
  CUDA_TRY(h, cudaMemcpyAsync(h->d_ic, h->ic.data(), sizeof(InstConst) * h->ic.size(), cudaMemcpyHostToDevice, h->stream));
  return XFLAT_OK;
}
int upload_dyn(xflat_t h) {
  CUDA_TRY(h, cudaMemcpyAsync(h->d_dyn, h->dyn.data(), sizeof(InstDyn) * h->dyn.size(), cudaMemcpyHostToDevice, h->stream));
  return XFLAT_OK;
}
int download_dyn(xflat_t h) {
  CUDA_TRY(h, cudaMemcpyAsync(h->dyn.data(), h->d_dyn, sizeof(InstDyn) * h->dyn.size(), cudaMemcpyDeviceToHost, h->stream));
  CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  return XFLAT_OK;
}

int upload_tables(xflat_t h, uint32_t i) {
  HostInst& I = h->inst[i];
  std::vector<double> et;
  build_tables(h, I, et, h->ic[i]);
  const size_t n = et.size();
  if (h->real_size == 8) {
    CUDA_TRY(h, cudaMemcpy((double*)h->d_etab + I.e_off, et.data(), n * 8, cudaMemcpyHostToDevice));
  } else {
    // Mixed kernels hand each thread's FP32 moment partial sums to integers in units of 2^-S (see
    // the step kernel): the weights are uploaded times 2^S, with S the largest integer for which
    // 2 B 2^S <= 2^52, B = sum_b |w_b| / cos(theta_b)(R) bounding every partial sum of states with
    // |Y| <= 2 (|t1|, |q| and the extended model's |tan theta| are at most 1/cos theta, largest at
    // r = R).  The kernel accepts thread and block partials below 2^52 units, so no integer sum
    // can overflow; the resolution 2^-S of the normalised moments is 2^-50 or finer for B <= 2.
    const uint32_t ne = I.cfg.n_energy, na = (uint32_t)I.u.size();
    const int wrow = I.cfg.n_flavor == 2 ? 1 : 2;     // first of the two weight rows (nu, nubar)
    double B = 0.0;
    for (uint32_t a = 0; a < na; ++a) {
      double gs = 0.0;
      for (int sp = 0; sp < 2; ++sp)
        for (uint32_t k = 0; k < ne; ++k) gs += std::fabs(et[(size_t)(wrow + sp) * ne + k]);
      B += std::fabs(I.du[a]) * gs / std::sqrt(1.0 - I.u[a]);
    }
    const int S = B > 0 ? std::min(100, 51 - (int)std::ceil(std::log2(B))) : 50;
    h->ic[i].acc_unit = std::ldexp(1.0, -S);
    std::vector<float> ef(n);
    for (size_t t = 0; t < n; ++t) {
      const bool weight = t >= (size_t)wrow * ne && t < (size_t)(wrow + 2) * ne;
      ef[t] = (float)(weight ? std::ldexp(et[t], S) : et[t]);
    }
    CUDA_TRY(h, cudaMemcpy((float*)h->d_etab + I.e_off, ef.data(), n * 4, cudaMemcpyHostToDevice));
  }
  CUDA_TRY(h, cudaMemcpy(h->d_u + I.a_off, I.u.data(), I.u.size() * 8, cudaMemcpyHostToDevice));
  CUDA_TRY(h, cudaMemcpy(h->d_du + I.a_off, I.du.data(), I.du.size() * 8, cudaMemcpyHostToDevice));
  return XFLAT_OK;
}

void reset_dyn(xflat_t h, uint32_t i, double r0) {
  InstDyn& d = h->dyn[i];
  const xflat_config& c = h->inst[i].cfg;
  std::memset(&d, 0, sizeof(InstDyn));
  d.r = r0;
  d.r_end = r0;
  d.h = adaptive(c.integrator) ? c.h0_km : c.fixed_dr_km;
  d.done = 1;
}

// Cut all instances into G slices and slices into pieces; blk[b]..blk[b+1] are block b's pieces.
// Dynamic scheduling: blocks take pieces in list order from a counter.  The list holds first every
// instance's leading beams in pieces of about kDynBig vector iterations per thread, then the last
// kDynTailPct percent of every instance in pieces of kDynSmall iterations (each at most the table's
// rows): the large pieces keep the per-piece set-up rare, the small ones at the end of the list let
// the blocks finish a pass within a small piece of one another.
constexpr uint32_t kDynBig = 64, kDynSmall = 8, kDynTailPct = 15;
void build_dynamic_pieces(xflat_t h) {
  h->pieces.clear();
  h->blk.assign(h->grid + 1, 0);
  h->max_jj = 1;
  auto cut = [&](uint32_t i, uint64_t a0, uint64_t a1, uint32_t iters) {
    const HostInst& I = h->inst[i];
    const uint32_t ne = I.cfg.n_energy;
    const uint64_t rows_cap = std::max<uint64_t>(kAlignBeams, ((uint64_t)(max_jj_cap(h->nf, h->real_size, h->extended) - 1) * ne) / kAlignBeams * kAlignBeams);
    const uint64_t len = std::min<uint64_t>((uint64_t)iters * 2 * h->block, rows_cap);
    for (uint64_t a = a0; a < a1; a += len) {
      Piece p{};
      p.inst = (int)i;
      p.start = (uint32_t)a;
      p.len = (uint32_t)std::min<uint64_t>(len, a1 - a);
      p.jj_lo = p.start / ne;
      p.n_jj = (p.start + p.len - 1) / ne - p.jj_lo + 1;
      h->max_jj = std::max<int>(h->max_jj, (int)p.n_jj);
      h->pieces.push_back(p);
    }
  };
  std::vector<uint64_t> split(h->inst.size());
  for (uint32_t i = 0; i < h->inst.size(); ++i) {
    split[i] = ((uint64_t)h->inst[i].n_beams * (100 - kDynTailPct) / 100) / kAlignBeams * kAlignBeams;
    cut(i, 0, split[i], kDynBig);
  }
  for (uint32_t i = 0; i < h->inst.size(); ++i) cut(i, split[i], h->inst[i].n_beams, kDynSmall);
}

void build_pieces(xflat_t h, int G) {
  if (h->dyn_sched) {
    build_dynamic_pieces(h);
    return;
  }
  uint64_t T = 0, A = 0;                   // the beams [A, A + T) of the planes the grid covers
  for (auto& I : h->inst) T = std::max<uint64_t>(T, I.off + I.n_pad);
  if (h->shard) {
    A = h->inst[0].off + h->shard_lo;
    T = h->shard_hi - h->shard_lo;
  }
  h->pieces.clear();
  h->blk.assign(G + 1, 0);
  h->max_jj = 1;
  for (int b = 0; b < G; ++b) {
    h->blk[b] = (int)h->pieces.size();
    uint64_t s0 = A + (T * (uint64_t)b / G) / kAlignBeams * kAlignBeams;
    uint64_t s1 = A + ((b == G - 1) ? T : (T * (uint64_t)(b + 1) / G) / kAlignBeams * kAlignBeams);
    for (uint32_t i = 0; i < h->inst.size(); ++i) {
      const HostInst& I = h->inst[i];
      const uint64_t lo = std::max<uint64_t>(s0, I.off), hi = std::min<uint64_t>(s1, I.off + I.n_beams);
      if (lo >= hi) continue;
      const uint32_t ne = I.cfg.n_energy;
      const uint64_t maxlen = std::max<uint64_t>(kAlignBeams, ((uint64_t)(max_jj_cap(h->nf, h->real_size, h->extended) - 1) * ne) / kAlignBeams * kAlignBeams);
      for (uint64_t a = lo; a < hi; a += maxlen) {
        const uint64_t e = std::min<uint64_t>(hi, a + maxlen);
        Piece p{};
        p.inst = (int)i;
        p.start = (uint32_t)(a - I.off);
        p.len = (uint32_t)(e - a);
        p.jj_lo = p.start / ne;
        p.n_jj = (p.start + p.len - 1) / ne - p.jj_lo + 1;
        h->max_jj = std::max<int>(h->max_jj, (int)p.n_jj);
        h->pieces.push_back(p);
      }
    }
  }
  h->blk[G] = (int)h->pieces.size();
}

// Values per (stage, angle bin) table row of the step kernel (Phys2<float>::KT, Phys2<double>::KT,
// Phys3::KT), and the cap on angle bins per piece that bounds the table's shared memory.
int table_row_values(int nf, size_t real_size, bool ext = false) {
  if (ext) return real_size == 4 ? 18 : 10;
  return nf == 2 ? (real_size == 4 ? 24 : 8) : 4;
}
// combined angle rows per piece: bounded by the shared-memory table ([stage slots][rows][row values]);
// the extended model has ten times the rows per beam, so its rows are kept narrow and a block's
// share of a 4M-beam problem (about 130 rows at two blocks per SM) fits one piece
uint32_t max_jj_cap(int nf, size_t real_size, bool ext) {
  if (nf == 2 && real_size == 4) return ext ? 160u : 48u;
  return kMaxJJ;
}

// Dynamic shared memory of a step-kernel block: reduction scratch, the table rows, the angle
// weights and positions, and (FP32 two-flavour bulb kernels) the threads' state rings,
// kStateRingDepth + 1 slots of 3 components x 2 beams per thread.
size_t smem_bytes(int nf, size_t real_size, int max_jj, int stages, int block, bool ext = false) {
  size_t s = 32 * kNMMax * sizeof(double);
  s += (size_t)stages * max_jj * table_row_values(nf, real_size, ext) * real_size;
  s += (size_t)max_jj * real_size;                 // angle weights
  s = (s + 7) / 8 * 8 + (size_t)max_jj * sizeof(double);   // angle positions
  s = (s + 15) / 16 * 16;
  if (nf == 2 && real_size == 4 && !ext) s += (size_t)block * (kStateRingDepth + 1) * 3 * 2 * sizeof(float);
  return s;
}

KParams make_params(xflat_t h, int n_steps, int init_only) {
  KParams p{};
  p.n_inst = (int)h->inst.size();
  p.n_pieces = (int)h->pieces.size();
  p.ic = h->d_ic;
  p.dyn = h->d_dyn;
  p.pieces = h->d_pieces;
  p.blk_piece = h->d_blk;
  p.acc = h->d_acc;
  p.errmax = h->d_errmax;
  p.nonfinite = h->d_nonfinite;
  p.planeA = h->planes;
  p.planeB = (char*)h->planes + (size_t)h->nc * h->stride * h->real_size;
  p.escr = h->escr;
  p.kst = h->kst;
  p.plane_stride = h->stride;
  p.etab = h->d_etab;
  p.u_tab = h->d_u;
  p.du_tab = h->d_du;
  p.bar = h->d_bar;
  p.timeout_ns = h->timeout_ns;
  p.status = h->d_words;
  p.all_done = h->d_words + 1;
  p.n_steps = n_steps;
  p.init_only = init_only;
  p.max_jj = h->max_jj;
  p.integrator = h->integrator;
  p.trace = init_only ? nullptr : h->d_trace;
  p.dyn_sched = h->dyn_sched ? 1 : 0;
  p.trace_passes = (int)h->trace_passes;
#ifdef XFLAT_BOUNDS
  p.span[kSpanPlanes] = Span{(const char*)h->planes, h->planes_bytes};
  p.span[kSpanEscr] = Span{(const char*)h->escr, h->escr_bytes};
  p.span[kSpanKst] = Span{(const char*)h->kst, h->kst_bytes};
  p.span[kSpanEtab] = Span{(const char*)h->d_etab, h->etab_bytes};
  p.span[kSpanU] = Span{(const char*)h->d_u, h->angle_bytes};
  p.span[kSpanDu] = Span{(const char*)h->d_du, h->angle_bytes};
#endif
  return p;
}

int launch(xflat_t h, int n_steps, int init_only, cudaStream_t stream, int shard_mode = kShardOff,
           int shard_pass = 0) {
  KParams p = make_params(h, n_steps, init_only);
  p.shard_mode = shard_mode;
  p.shard_pass = shard_pass;
  void* args[] = {&p};
  cudaLaunchConfig_t cfg{};
  const bool serial_only = shard_mode == kShardSerialInit || shard_mode == kShardSerialFinal;
  cfg.gridDim = dim3(serial_only ? 1 : h->grid);
  cfg.blockDim = dim3(h->block);
  cfg.dynamicSmemBytes = h->smem;
  cfg.stream = stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  CUDA_TRY(h, cudaLaunchKernelExC(&cfg, h->kernel, args));
  h->launches++;
  return XFLAT_OK;
}
int launch(xflat_t h, int n_steps, int init_only) { return launch(h, n_steps, init_only, h->stream); }

void drop_graph(xflat_t h) {
  if (h->graph_exec) cudaGraphExecDestroy(h->graph_exec);
  if (h->graph) cudaGraphDestroy(h->graph);
  h->graph_exec = nullptr;
  h->graph = nullptr;
  h->graph_launches = h->graph_steps = 0;
}

// Capture n_launches persistent launches of max_steps steps each, followed by the read-back of the
// status words, into one executable graph.  Capture runs on a private stream (the legacy default
// stream cannot be captured); the graph is launched on the handle's stream.
int capture_graph(xflat_t h, uint32_t n_launches, uint32_t max_steps) {
  drop_graph(h);
  cudaStream_t cs = nullptr;
  CUDA_TRY(h, cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  const uint64_t launches0 = h->launches;
  int rc = XFLAT_OK;
  if (e == cudaSuccess) {
    for (uint32_t i = 0; i < n_launches && rc == XFLAT_OK; ++i) rc = launch(h, (int)max_steps, 0, cs);
    if (rc == XFLAT_OK)
      e = cudaMemcpyAsync(h->h_words, h->d_words, 2 * sizeof(int), cudaMemcpyDeviceToHost, cs);
    cudaGraph_t g = nullptr;
    const cudaError_t e2 = cudaStreamEndCapture(cs, &g);
    if (e == cudaSuccess) e = e2;
    if (rc == XFLAT_OK && e == cudaSuccess) {
      h->graph = g;
      e = cudaGraphInstantiate(&h->graph_exec, g, 0);
    } else if (g) {
      cudaGraphDestroy(g);
    }
  }
  cudaStreamDestroy(cs);
  h->launches = launches0;               // captured, not yet launched
  if (rc == XFLAT_OK && e != cudaSuccess) rc = fail(h, XFLAT_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
  if (rc != XFLAT_OK) {
    cudaGetLastError();
    drop_graph(h);
    return rc;
  }
  h->graph_launches = n_launches;
  h->graph_steps = max_steps;
  return XFLAT_OK;
}

int clear_sync_words(xflat_t h) {
  Barrier b{};
  b.extra = h->debug_extra;
  CUDA_TRY(h, cudaMemcpyAsync(h->d_bar, &b, sizeof(Barrier), cudaMemcpyHostToDevice, h->stream));
  CUDA_TRY(h, cudaMemsetAsync(h->d_words, 0, 2 * sizeof(int), h->stream));
  CUDA_TRY(h, cudaMemsetAsync(h->d_nonfinite, 0, h->inst.size() * sizeof(int), h->stream));
  CUDA_TRY(h, cudaMemsetAsync(h->d_errmax, 0, h->inst.size() * sizeof(unsigned long long), h->stream));
  CUDA_TRY(h, cudaMemsetAsync(h->d_acc, 0, h->inst.size() * kAccWordsPerInst * sizeof(unsigned long long), h->stream));
  return XFLAT_OK;
}

int read_words(xflat_t h, int& status, int& all_done) {
  CUDA_TRY(h, cudaMemcpyAsync(h->h_words, h->d_words, 2 * sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  status = h->h_words[0];
  all_done = h->h_words[1];
#ifdef XFLAT_BOUNDS
  // checked build: name the first access the kernel found outside its allocation
  Barrier b{};
  CUDA_TRY(h, cudaMemcpy(&b, h->d_bar, sizeof(Barrier), cudaMemcpyDeviceToHost));
  if (b.bounds_site) {
    status = XFLAT_ERR_CUDA;
    return fail(h, XFLAT_ERR_CUDA, "bounds check failed at site " + std::to_string(b.bounds_site) +
                                       ", byte offset " + std::to_string(b.bounds_off));
  }
#endif
  return XFLAT_OK;
}

// Compute the moments of the current state of every instance (stage 1 constants).
int refresh_moments(xflat_t h) {
  std::vector<unsigned long long> evals(h->dyn.size());
  for (size_t i = 0; i < h->dyn.size(); ++i) {
    InstDyn& d = h->dyn[i];
    evals[i] = d.stage_evals;
    d.rs[1] = d.r;
    d.xs[1] = h->ic[i].R2 / (d.r * d.r);
    d.status = 0;
    d.done = 0;            // the init pass skips finished instances
  }
  int rc = upload_dyn(h);
  if (rc) return rc;
  if ((rc = clear_sync_words(h))) return rc;
  if ((rc = launch(h, 0, 1))) return rc;
  if ((rc = download_dyn(h))) return rc;
  int st, ad;
  if ((rc = read_words(h, st, ad))) return rc;
  for (size_t i = 0; i < h->dyn.size(); ++i) {
    h->dyn[i].done = 1;
    h->dyn[i].stage_evals = evals[i];   // an export is not an integration stage
  }
  if ((rc = upload_dyn(h))) return rc;
  if (st) return fail(h, st, "device status after the moment reduction");
  for (auto& d : h->dyn)
    if (d.status) return fail(h, d.status, "non-finite moments");
  h->moments_valid = true;
  return XFLAT_OK;
}

int setup_launch_shape(xflat_t h, const xflat_config& c) {
  // mixed two-flavour kernels exist at two register budgets: 768 resident threads per SM (80
  // registers) and 512 (128 registers); the request picks the one that fits.  Every other kernel
  // is built for one 256-thread block per SM.  Default for the mixed two-flavour bulb kernels: one
  // 512-thread block per SM while both state buffers fit the L2 (the passes are then bound by
  // issue: the 80-register budget spills, and two co-resident blocks finish their passes at
  // different times), three 256-thread blocks once the state streams from HBM (more loads in
  // flight); 256 threads otherwise.  (GB300, DP45, 28M beams in 64 instances with dynamic piece
  // scheduling: 1.86 ms per step at 256 x 3 against 1.96 ms at 256 x 2 and about 2.2 ms at
  // 512 x 1; 4M beams in one instance: 0.186 ms per one-step launch at 512 x 1 against 0.224 ms
  // at 256 x 3.)
  const bool mixed_2f = h->nf == 2 && !h->extended && h->real_size == 4;
  int l2_bytes = 0;
  cudaDeviceGetAttribute(&l2_bytes, cudaDevAttrL2CacheSize, h->device);
  const uint64_t state_bytes = 2ull * h->nc * h->stride * h->real_size;
  const bool resident = state_bytes <= (uint64_t)l2_bytes;
  h->block = c.block_size ? (int)c.block_size : (mixed_2f && !c.blocks_per_sm && resident ? 512 : 256);
  const int want_bps = c.blocks_per_sm ? (int)c.blocks_per_sm : ((mixed_2f ? 512 : 768) / h->block);
  h->kernel = step_kernel_ptr(h->nf, h->precision, h->integrator, h->block, want_bps * h->block >= 768 ? 3 : 2,
                              h->extended);
  if (!h->kernel) return fail(h, XFLAT_ERR_UNSUPPORTED, "no kernel for this flavour/precision/integrator");
  const size_t smax = smem_bytes(h->nf, h->real_size, max_jj_cap(h->nf, h->real_size, h->extended),
                                 table_stages(h->integrator), h->block, h->extended);
  CUDA_TRY(h, cudaFuncSetAttribute(h->kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smax));
  int occ = 0;
  CUDA_TRY(h, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, h->kernel, h->block, smax));
  if (occ < 1) return fail(h, XFLAT_ERR_CUDA, "kernel does not fit on an SM");
  if (c.blocks_per_sm) occ = std::min<int>(occ, (int)c.blocks_per_sm);
  uint64_t T = 0;
  for (auto& I : h->inst) T += I.n_pad;
  if (h->shard) T = h->shard_hi - h->shard_lo;
  int G = occ * h->sm_count;
  // at least one vector of work per thread
  const uint64_t per_block = (uint64_t)h->block * kAlignBeams;
  G = (int)std::max<uint64_t>(1, std::min<uint64_t>((uint64_t)G, (T + per_block - 1) / per_block));
  h->grid = G;
  h->dyn_sched = h->inst.size() > 1 && !h->shard;
  build_pieces(h, G);
  h->smem = smem_bytes(h->nf, h->real_size, h->max_jj, table_stages(h->integrator), h->block, h->extended);
  if (h->d_pieces) cudaFree(h->d_pieces);
  if (h->d_blk) cudaFree(h->d_blk);
  h->d_pieces = nullptr;
  h->d_blk = nullptr;
  CUDA_TRY(h, dev_alloc(&h->d_pieces, sizeof(Piece) * std::max<size_t>(1, h->pieces.size())));
  CUDA_TRY(h, dev_alloc(&h->d_blk, sizeof(int) * h->blk.size()));
  CUDA_TRY(h, cudaMemcpy(h->d_pieces, h->pieces.data(), sizeof(Piece) * h->pieces.size(), cudaMemcpyHostToDevice));
  CUDA_TRY(h, cudaMemcpy(h->d_blk, h->blk.data(), sizeof(int) * h->blk.size(), cudaMemcpyHostToDevice));
  return XFLAT_OK;
}

int ensure_stage(xflat_t h, size_t bytes) {
  if (h->stage_bytes >= bytes) return XFLAT_OK;
  if (h->d_stage) cudaFree(h->d_stage);
  h->d_stage = nullptr;
  h->stage_bytes = 0;
  CUDA_TRY(h, dev_alloc(&h->d_stage, bytes));
  h->stage_bytes = bytes;
  return XFLAT_OK;
}

void* cur_plane(xflat_t h, uint32_t i) {
  const int par = h->dyn[i].parity;
  return (char*)h->planes + ((size_t)par * h->nc * h->stride + h->inst[i].off) * h->real_size;
}

// Targets of an evolve or advance: per instance the radius r1 (null: the previous target), the
// fixed-step grid or the adaptive state, and the current radius as stage 1; *any = some instance
// still has work, *changed = the moments of the current state must be recomputed.
int prepare_targets(xflat_t h, const double* r1, bool& any, bool& changed) {
  int rc;
  if ((rc = download_dyn(h))) return rc;
  any = false;
  changed = !h->moments_valid;
  for (size_t i = 0; i < h->inst.size(); ++i) {
    if (!h->inst[i].spectra) return fail(h, XFLAT_ERR_STATE, "set_spectra before evolve");
    if (h->inst[i].cfg.matter_kind == XFLAT_MATTER_TABLE && h->inst[i].mtab.empty())
      return fail(h, XFLAT_ERR_STATE, "xflat_set_matter_table before evolve");
    InstDyn& d = h->dyn[i];
    const xflat_config& c = h->inst[i].cfg;
    const double target = r1 ? r1[i] : d.r_end;
    if (!is_fin(target)) return fail(h, XFLAT_ERR_INVAL, "non-finite target radius");
    if (target < c.R_km) return fail(h, XFLAT_ERR_INVAL, "target radius below R");
    d.status = 0;
    if (r1 || d.r_end != target) {
      changed = true;
      d.r_end = target;
      d.done = d.r >= target ? 1 : 0;
      if (!adaptive(c.integrator)) {
        const double span = target - d.r;
        long long n = (long long)std::ceil(span / c.fixed_dr_km - 1e-9);
        if (n < 1) n = 1;
        d.r0_fixed = d.r;
        d.n_fixed = 0;
        d.n_fixed_total = n;
        d.h_fixed = span / (double)n;
      } else {
        d.last = 0;
        if (!(d.h > 0)) d.h = c.h0_km;
      }
    }
    d.rs[1] = d.r;
    d.xs[1] = h->ic[i].R2 / (d.r * d.r);
    any = any || !d.done;
  }
  return XFLAT_OK;
}

int do_evolve(xflat_t h, const double* r1, bool sync_loop, uint32_t max_steps, int* done_out) {
  int rc;
  if (h->shard) return fail(h, XFLAT_ERR_STATE, "a beam-shard handle advances with the xflat_shard_* calls");
  if (!sync_loop && r1 == nullptr && h->moments_valid && h->advancing) {
    // continuing an advance: device state, moments and step geometry are already in place
    if (done_out) *done_out = h->h_words[1];
    if ((rc = launch(h, (int)max_steps, 0))) return rc;
    CUDA_TRY(h, cudaMemcpyAsync(h->h_words, h->d_words, 2 * sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    return XFLAT_OK;
  }
  h->advancing = false;
  bool any = false, changed = false;
  if ((rc = prepare_targets(h, r1, any, changed))) return rc;
  if (done_out) *done_out = any ? 0 : 1;
  if (!any) return XFLAT_OK;
  if ((rc = upload_dyn(h))) return rc;
  if ((rc = clear_sync_words(h))) return rc;
  // moments of the current state and the first step's geometry, unless the previous launch left
  // both in place (same targets, state untouched since)
  if (changed && (rc = launch(h, 0, 1))) return rc;
  if (!sync_loop) {
    if ((rc = launch(h, (int)max_steps, 0))) return rc;
    CUDA_TRY(h, cudaMemcpyAsync(h->h_words, h->d_words, 2 * sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    // the step kernel keeps the moments of the current state (stage 1) up to date
    h->moments_valid = true;
    h->advancing = true;
    return XFLAT_OK;
  }
  for (;;) {
    if ((rc = launch(h, (int)h->steps_per_launch, 0))) return rc;
    int st, ad;
    if ((rc = read_words(h, st, ad))) return rc;
    if (st || ad) break;
  }
  if ((rc = download_dyn(h))) return rc;
  h->moments_valid = true;
  int st, ad;
  if ((rc = read_words(h, st, ad))) return rc;
  for (auto& d : h->dyn)
    if (d.status) return fail(h, d.status, std::string("device status: ") + xflat_status_string(d.status));
  if (st) return fail(h, st, std::string("device status: ") + xflat_status_string(st));
  return XFLAT_OK;
}

int create_impl(const xflat_config* cfgs, uint32_t n, xflat_t* out) {
  if (!cfgs || !out || n == 0) return XFLAT_ERR_INVAL;
  std::string why;
  for (uint32_t i = 0; i < n; ++i) {
    int rc = check_config(cfgs[i], why);
    if (rc) { (void)why; return rc; }
    if (cfgs[i].n_flavor != cfgs[0].n_flavor || cfgs[i].precision != cfgs[0].precision ||
        cfgs[i].integrator != cfgs[0].integrator || (cfgs[i].n_phi >= 2) != (cfgs[0].n_phi >= 2))
      return XFLAT_ERR_INVAL;
  }
  xflat_t h = new (std::nothrow) xflat_s();
  if (!h) return XFLAT_ERR_NOMEM;
  auto bail = [&](int rc) { xflat_destroy(h); return rc; };
  h->nf = (int)cfgs[0].n_flavor;
  h->extended = cfgs[0].n_phi >= 2;
  h->precision = (int)cfgs[0].precision;
  h->integrator = (int)cfgs[0].integrator;
  h->real_size = h->precision == XFLAT_FP64 ? 8 : 4;
  h->nc = h->nf == 2 ? 3 : 9;
  h->stream = (cudaStream_t)cfgs[0].cuda_stream;
  h->timeout_ns = cfgs[0].barrier_timeout_ns ? cfgs[0].barrier_timeout_ns : 2000000000ull;
  h->steps_per_launch = cfgs[0].steps_per_launch ? cfgs[0].steps_per_launch : 64;
  if (cudaGetDevice(&h->device) != cudaSuccess) return bail(XFLAT_ERR_CUDA);
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, h->device) != cudaSuccess) return bail(XFLAT_ERR_CUDA);
  if (prop.major * 10 + prop.minor != 103) return bail(XFLAT_ERR_CUDA);
  h->sm_count = prop.multiProcessorCount;
  // layout
  h->inst.resize(n);
  uint64_t off = 0;
  uint32_t eoff = 0, aoff = 0;
  for (uint32_t i = 0; i < n; ++i) {
    HostInst& I = h->inst[i];
    I.cfg = cfgs[i];
    const uint32_t na_tot = angle_bins(I.cfg), nphi = I.cfg.n_phi >= 2 ? I.cfg.n_phi : 1u;
    I.n_beams = 2u * I.cfg.n_energy * na_tot;
    I.n_pad = (I.n_beams + kAlignBeams - 1) / kAlignBeams * kAlignBeams;
    I.off = off;
    off += I.n_pad;
    I.e_off = eoff;
    eoff += (h->nf == 2 ? 3 : 4) * I.cfg.n_energy;
    I.a_off = aoff;
    aoff += na_tot;
    // combined angle bins a = j n_phi + p: u_j and du_j / n_phi (the azimuthal measure dphi / 2 pi)
    I.u.resize(na_tot);
    I.du.resize(na_tot);
    for (uint32_t a = 0; a < na_tot; ++a) {
      const uint32_t j = a / nphi;
      I.u[a] = (j + 0.5) / I.cfg.n_angle;
      I.du[a] = 1.0 / I.cfg.n_angle / nphi;
    }
    I.N.assign(2ull * h->nf * I.cfg.n_energy, 0.0);
  }
  h->stride = (off + 63) / 64 * 64;
  const size_t plane_bytes = 2ull * h->nc * h->stride * h->real_size;
  h->planes_bytes = plane_bytes;
  h->etab_bytes = (size_t)eoff * h->real_size;
  h->angle_bytes = sizeof(double) * aoff;
  if (dev_alloc(&h->planes, plane_bytes) != cudaSuccess) return bail(XFLAT_ERR_NOMEM);
  // FP64 DP45: error partial (nc planes) and error scale (one plane) of the step in flight
  if (h->integrator == XFLAT_DP45 && h->real_size == 8) {
    h->escr_bytes = (size_t)(h->nc + 1) * h->stride * h->real_size;
    if (dev_alloc(&h->escr, h->escr_bytes) != cudaSuccess) return bail(XFLAT_ERR_NOMEM);
  }
  // FP64 RK4 / DP45: the stage derivatives a step stores (k_1..k_3 of RK4, k_1..k_5 of DP45, whose
  // pass forming y5 keeps the error partial instead of k_6), then one stage state
  const int n_kst = h->real_size != 8 ? 0 : h->integrator == XFLAT_RK4 ? 3 : h->integrator == XFLAT_DP45 ? 5 : 0;
  if (n_kst) {
    h->kst_bytes = (size_t)(n_kst + 1) * h->nc * h->stride * h->real_size;
    if (dev_alloc(&h->kst, h->kst_bytes) != cudaSuccess) return bail(XFLAT_ERR_NOMEM);
  }
  if (dev_alloc(&h->d_ic, sizeof(InstConst) * n) != cudaSuccess ||
      dev_alloc(&h->d_dyn, sizeof(InstDyn) * n) != cudaSuccess ||
      dev_alloc(&h->d_acc, sizeof(unsigned long long) * n * kAccWordsPerInst) != cudaSuccess ||
      dev_alloc(&h->d_errmax, sizeof(unsigned long long) * n) != cudaSuccess ||
      dev_alloc(&h->d_nonfinite, sizeof(int) * n) != cudaSuccess ||
      dev_alloc(&h->d_etab, (size_t)eoff * h->real_size) != cudaSuccess ||
      dev_alloc(&h->d_u, sizeof(double) * aoff) != cudaSuccess ||
      dev_alloc(&h->d_du, sizeof(double) * aoff) != cudaSuccess ||
      dev_alloc(&h->d_bar, sizeof(Barrier)) != cudaSuccess ||
      dev_alloc(&h->d_words, 2 * sizeof(int)) != cudaSuccess ||
      host_alloc(&h->h_words, 2 * sizeof(int)) != cudaSuccess)
    return bail(XFLAT_ERR_NOMEM);
  cudaMemset(h->d_etab, 0, (size_t)eoff * h->real_size);
  h->ic.assign(n, InstConst{});
  h->dyn.assign(n, InstDyn{});
  for (uint32_t i = 0; i < n; ++i) {
    fill_inst_const(h->inst[i], h->ic[i]);
    h->ic[i].wscale = 1.0;
    h->ic[i].mu_coef = 0.0;
    h->ic[i].acc_unit = std::ldexp(1.0, -50);
    reset_dyn(h, i, h->inst[i].cfg.R_km);
  }
  int rc = setup_launch_shape(h, cfgs[0]);
  if (rc) return bail(rc);
  if ((rc = upload_inst(h)) || (rc = upload_dyn(h))) return bail(rc);
  const uint64_t tot = h->stride;
  if (h->real_size == 8) k_initial_state<double><<<(unsigned)((tot + 255) / 256), 256, 0, h->stream>>>((double*)h->planes, h->stride, tot, h->nf);
  else k_initial_state<float><<<(unsigned)((tot + 255) / 256), 256, 0, h->stream>>>((float*)h->planes, h->stride, tot, h->nf);
  if (cudaStreamSynchronize(h->stream) != cudaSuccess) return bail(XFLAT_ERR_CUDA);
  *out = h;
  return XFLAT_OK;
}

}  // namespace

// ==== exported C ABI ============================================================================
extern "C" {

int xflat_default_config(xflat_config* c) {
  XFLAT_TRACE();
  if (!c) return XFLAT_ERR_INVAL;
  std::memset(c, 0, sizeof(*c));
  c->abi_version = XFLAT_ABI_VERSION;
  c->n_flavor = 2;
  c->n_energy = 64;
  c->n_angle = 32;
  c->precision = XFLAT_FP64;
  c->integrator = XFLAT_RK4;
  c->matter_kind = XFLAT_MATTER_NONE;
  c->R_km = 11.0;
  c->E_min_MeV = 1.0;
  c->E_max_MeV = 60.0;
  c->dm2_eV2[0] = -2.4e-3;
  c->theta[0] = 0.1;
  c->rtol = 1e-9;
  c->atol = 1e-9;
  c->h0_km = 1e-4;
  c->h_min_km = 1e-14;
  c->h_max_km = 0.0;
  c->fixed_dr_km = 0.0945;
  c->rho0_gcc = 1e7;
  c->r_ref_km = 100.0;
  c->power = 3.0;
  c->Ye = 0.5;
  return XFLAT_OK;
}

int xflat_create(const xflat_config* cfg, xflat_t* out) {
  XFLAT_TRACE(); return create_impl(cfg, 1, out); }

int xflat_create_batch(const xflat_config* cfgs, uint32_t n_inst, xflat_t* out) {
  XFLAT_TRACE();
  return create_impl(cfgs, n_inst, out);
}

int xflat_destroy(xflat_t h) {
  XFLAT_TRACE();
  if (!h) return XFLAT_OK;
  if (h->stream || true) cudaStreamSynchronize(h->stream);
  drop_graph(h);
  void* ptrs[] = {h->planes, h->escr, h->kst, h->d_ic, h->d_dyn, h->d_pieces, h->d_blk, h->d_acc, h->d_errmax,
                  h->d_nonfinite, h->d_etab, h->d_u, h->d_du, h->d_bar, h->d_words, h->d_stage,
                  h->d_trace, h->d_mtab};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  if (h->h_words) cudaFreeHost(h->h_words);
  delete h;
  return XFLAT_OK;
}

// Upload every instance's matter table into one device array and point the instance constants
// at their rows (the array is replaced whenever a table changes).
int upload_matter_tables(xflat_t h) {
  std::vector<double> all;
  std::vector<size_t> off(h->inst.size());
  for (size_t i = 0; i < h->inst.size(); ++i) {
    off[i] = all.size();
    all.insert(all.end(), h->inst[i].mtab.begin(), h->inst[i].mtab.end());
  }
  // the new array is filled before the old one is released: a failure leaves the device copy and
  // the instance constants as they were
  double* fresh = nullptr;
  if (!all.empty()) {
    if (dev_alloc(&fresh, all.size() * sizeof(double)) != cudaSuccess)
      return fail(h, XFLAT_ERR_NOMEM, "matter table");
    if (cudaMemcpy(fresh, all.data(), all.size() * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess) {
      cudaFree(fresh);
      return fail(h, XFLAT_ERR_CUDA, "matter table upload");
    }
  }
  if (h->d_mtab) cudaFree(h->d_mtab);
  h->d_mtab = fresh;
  for (size_t i = 0; i < h->inst.size(); ++i) {
    h->ic[i].mt_n = (int32_t)(h->inst[i].mtab.size() / 3);
    h->ic[i].mtab = h->ic[i].mt_n ? h->d_mtab + off[i] : nullptr;
  }
  return upload_inst(h);
}

int xflat_set_matter_table(xflat_t h, uint32_t inst, const double* r_km, const double* lambda_kmi,
                           uint32_t n) {
  XFLAT_TRACE();
  if (!h) return XFLAT_ERR_INVAL;
  if (inst >= h->inst.size()) return fail(h, XFLAT_ERR_INVAL, "instance index out of range");
  HostInst& I = h->inst[inst];
  if (I.cfg.matter_kind != XFLAT_MATTER_TABLE) return fail(h, XFLAT_ERR_STATE, "matter_kind is not XFLAT_MATTER_TABLE");
  if (!r_km || !lambda_kmi || n < 1) return fail(h, XFLAT_ERR_INVAL, "need n >= 1 points");
  for (uint32_t i = 0; i < n; ++i) {
    if (!is_fin(r_km[i]) || !(r_km[i] > 0) || !is_fin(lambda_kmi[i]) || !(lambda_kmi[i] > 0))
      return fail(h, XFLAT_ERR_INVAL, "table radii and strengths must be finite and > 0");
    if (i && !(r_km[i] > r_km[i - 1])) return fail(h, XFLAT_ERR_INVAL, "table radii must increase");
  }
  std::vector<double> t(3ull * n);
  for (uint32_t i = 0; i < n; ++i) {
    t[3 * i] = r_km[i];
    t[3 * i + 1] = lambda_kmi[i];
    t[3 * i + 2] = i + 1 < n ? std::log(lambda_kmi[i + 1] / lambda_kmi[i]) / std::log(r_km[i + 1] / r_km[i]) : 0.0;
  }
  int rc;
  if ((rc = download_dyn(h))) return rc;
  std::vector<double> previous = std::move(I.mtab);
  I.mtab = std::move(t);
  if ((rc = upload_matter_tables(h))) {
    I.mtab = std::move(previous);           // the device still holds the previous tables
    return rc;
  }
  // the stage strengths of the current step were computed with the previous profile
  h->moments_valid = false;
  return XFLAT_OK;
}

int xflat_set_spectra_inst(xflat_t h, uint32_t inst, const double* nnu, const double* u_bins,
                           const double* u_weights) {
  XFLAT_TRACE();
  if (!h) return XFLAT_ERR_INVAL;
  if (inst >= h->inst.size()) return fail(h, XFLAT_ERR_INVAL, "instance index out of range");
  if (!nnu) return fail(h, XFLAT_ERR_INVAL, "nnu is NULL");
  if ((u_bins == nullptr) != (u_weights == nullptr)) return fail(h, XFLAT_ERR_INVAL, "u_bins and u_weights go together");
  HostInst& I = h->inst[inst];
  const uint32_t ne = I.cfg.n_energy, na = I.cfg.n_angle, nf = I.cfg.n_flavor;
  std::vector<double> N(nnu, nnu + 2ull * nf * ne);
  for (double v : N)
    if (!is_fin(v)) return fail(h, XFLAT_ERR_INVAL, "non-finite luminosity");
  if (nf == 3)
    for (int s = 0; s < 2; ++s)
      for (uint32_t k = 0; k < ne; ++k)
        if (N[(s * 3 + 1) * ne + k] != N[(s * 3 + 2) * ne + k])
          return fail(h, XFLAT_ERR_INVAL, "mu and tau spectra must be equal");
  if (u_bins) {
    for (uint32_t j = 0; j < na; ++j) {
      if (!(u_bins[j] >= 0.0 && u_bins[j] < 1.0)) return fail(h, XFLAT_ERR_INVAL, "u outside [0, 1)");
      if (!is_fin(u_weights[j]) || u_weights[j] < 0) return fail(h, XFLAT_ERR_INVAL, "bad u weight");
    }
    const uint32_t nphi = I.cfg.n_phi >= 2 ? I.cfg.n_phi : 1u;
    for (uint32_t a = 0; a < na * nphi; ++a) {
      I.u[a] = u_bins[a / nphi];
      I.du[a] = u_weights[a / nphi] / nphi;
    }
  }
  I.N = N;
  I.spectra = true;
  int rc;
  if ((rc = download_dyn(h))) return rc;
  fill_inst_const(I, h->ic[inst]);
  if ((rc = upload_tables(h, inst))) return rc;
  if ((rc = upload_inst(h))) return rc;
  reset_dyn(h, inst, I.cfg.R_km);
  if ((rc = upload_dyn(h))) return rc;
  // initial condition of this instance in both buffers (the kernel writes both)
  const size_t nb = I.n_pad;
  if (h->real_size == 8)
    k_initial_state<double><<<(unsigned)((nb + 255) / 256), 256, 0, h->stream>>>((double*)h->planes + I.off, h->stride, nb, h->nf);
  else
    k_initial_state<float><<<(unsigned)((nb + 255) / 256), 256, 0, h->stream>>>((float*)h->planes + I.off, h->stride, nb, h->nf);
  CUDA_TRY(h, cudaGetLastError());
  h->moments_valid = false;
  return XFLAT_OK;
}

int xflat_set_spectra(xflat_t h, const double* nnu, const double* u_bins, const double* u_weights) {
  XFLAT_TRACE();
  return xflat_set_spectra_inst(h, 0, nnu, u_bins, u_weights);
}

int xflat_reset(xflat_t h, double r0_km) {
  XFLAT_TRACE();
  if (!h) return XFLAT_ERR_INVAL;
  if (!is_fin(r0_km)) return fail(h, XFLAT_ERR_INVAL, "r0 not finite");
  int rc;
  for (size_t i = 0; i < h->inst.size(); ++i) {
    if (r0_km < h->inst[i].cfg.R_km) return fail(h, XFLAT_ERR_INVAL, "r0 below R");
    reset_dyn(h, (uint32_t)i, r0_km);
  }
  const uint64_t tot = h->stride;
  if (h->real_size == 8) k_initial_state<double><<<(unsigned)((tot + 255) / 256), 256, 0, h->stream>>>((double*)h->planes, h->stride, tot, h->nf);
  else k_initial_state<float><<<(unsigned)((tot + 255) / 256), 256, 0, h->stream>>>((float*)h->planes, h->stride, tot, h->nf);
  CUDA_TRY(h, cudaGetLastError());
  if ((rc = upload_dyn(h))) return rc;
  h->moments_valid = false;
  return XFLAT_OK;
}

int xflat_evolve_batch(xflat_t h, const double* r1) {
  XFLAT_TRACE();
  if (!h || !r1) return fail(h, XFLAT_ERR_INVAL, "NULL argument");
  return do_evolve(h, r1, true, 0, nullptr);
}

int xflat_evolve(xflat_t h, double r0_km, double r1_km) {
  XFLAT_TRACE();
  if (!h) return XFLAT_ERR_INVAL;
  int rc;
  if ((rc = download_dyn(h))) return rc;
  const double r = h->dyn[0].r;
  if (!is_fin(r0_km) || std::fabs(r0_km - r) > 1e-12 * std::max(1.0, std::fabs(r)))
    return fail(h, XFLAT_ERR_STATE, "r0 does not match the current radius");
  if (!(r1_km >= r0_km)) return fail(h, XFLAT_ERR_INVAL, "need r1 >= r0");
  std::vector<double> t(h->inst.size(), r1_km);
  return do_evolve(h, t.data(), true, 0, nullptr);
}

int xflat_advance(xflat_t h, const double* r1, uint32_t max_steps, int* done_out) {
  XFLAT_TRACE();
  if (!h) return XFLAT_ERR_INVAL;
  if (max_steps == 0) return fail(h, XFLAT_ERR_INVAL, "max_steps must be >= 1");
  return do_evolve(h, r1, false, max_steps, done_out);
}

int xflat_advance_graph(xflat_t h, uint32_t n_launches, uint32_t max_steps, int* done_out) {
  XFLAT_TRACE();
  if (!h) return XFLAT_ERR_INVAL;
  if (n_launches == 0 || max_steps == 0) return fail(h, XFLAT_ERR_INVAL, "n_launches and max_steps must be >= 1");
  if (!(h->advancing && h->moments_valid))
    return fail(h, XFLAT_ERR_STATE, "xflat_advance must precede xflat_advance_graph");
  int rc;
  if (!h->graph_exec || h->graph_launches != n_launches || h->graph_steps != max_steps)
    if ((rc = capture_graph(h, n_launches, max_steps))) return rc;
  if (done_out) *done_out = h->h_words[1];
  CUDA_TRY(h, cudaGraphLaunch(h->graph_exec, h->stream));
  h->launches += n_launches;
  return XFLAT_OK;
}

int xflat_moments_inst(xflat_t h, uint32_t inst, double* J0, double* J1) {
  XFLAT_TRACE();
  if (!h || !J0 || !J1) return fail(h, XFLAT_ERR_INVAL, "NULL argument");
  if (inst >= h->inst.size()) return fail(h, XFLAT_ERR_INVAL, "instance index out of range");
  if (!h->inst[inst].spectra) return fail(h, XFLAT_ERR_STATE, "set_spectra first");
  int rc;
  if ((rc = download_dyn(h))) return rc;
  if (!h->moments_valid && (rc = refresh_moments(h))) return rc;
  const InstDyn& d = h->dyn[inst];
  const double ws = h->ic[inst].wscale;
  const int nf = h->nf;
  const int ncomp = nf == 2 ? 3 : 9;
  for (int t = 0; t < 2; ++t) {
    // the device reduces D = J0 - J1 (slots 0..ncomp-1) and J1 (slots ncomp..2 ncomp-1)
    double m[9];
    for (int c = 0; c < ncomp; ++c) m[c] = d.mom[1][ncomp + c] + (t == 0 ? d.mom[1][c] : 0.0);
    double* J = t == 0 ? J0 : J1;
    std::memset(J, 0, sizeof(double) * 2 * nf * nf);
    if (nf == 2) {
      J[0] = 0.5 * ws * m[2];
      J[2] = 0.5 * ws * m[0];
      J[3] = -0.5 * ws * m[1];
      J[4] = 0.5 * ws * m[0];
      J[5] = 0.5 * ws * m[1];
      J[6] = -0.5 * ws * m[2];
    } else {
      const double tr = (m[0] + m[1] + m[2]) / 3.0;
      const double re[3][3] = {{m[0] - tr, m[3], m[5]}, {m[3], m[1] - tr, m[7]}, {m[5], m[7], m[2] - tr}};
      const double im[3][3] = {{0, m[4], m[6]}, {-m[4], 0, m[8]}, {-m[6], -m[8], 0}};
      for (int a = 0; a < 3; ++a)
        for (int c = 0; c < 3; ++c) {
          J[(a * 3 + c) * 2] = ws * re[a][c];
          J[(a * 3 + c) * 2 + 1] = ws * im[a][c];
        }
    }
  }
  return XFLAT_OK;
}

int xflat_moments(xflat_t h, double* J0, double* J1) {
  XFLAT_TRACE(); return xflat_moments_inst(h, 0, J0, J1); }

int xflat_moments_phi(xflat_t h, uint32_t inst, double* Jc, double* Js) {
  XFLAT_TRACE();
  if (!h || !Jc || !Js) return fail(h, XFLAT_ERR_INVAL, "NULL argument");
  if (!h->extended) return fail(h, XFLAT_ERR_UNSUPPORTED, "azimuthal moments need the extended bulb model");
  if (inst >= h->inst.size()) return fail(h, XFLAT_ERR_INVAL, "instance index out of range");
  if (!h->inst[inst].spectra) return fail(h, XFLAT_ERR_STATE, "set_spectra first");
  int rc;
  if ((rc = download_dyn(h))) return rc;
  if (!h->moments_valid && (rc = refresh_moments(h))) return rc;
  const InstDyn& d = h->dyn[inst];
  const double ws = h->ic[inst].wscale;
  for (int t = 0; t < 2; ++t) {
    const double* m = &d.mom[1][6 + 3 * t];
    double* J = t == 0 ? Jc : Js;
    J[0] = 0.5 * ws * m[2];  J[1] = 0;
    J[2] = 0.5 * ws * m[0];  J[3] = -0.5 * ws * m[1];
    J[4] = 0.5 * ws * m[0];  J[5] = 0.5 * ws * m[1];
    J[6] = -0.5 * ws * m[2]; J[7] = 0;
  }
  return XFLAT_OK;
}

int xflat_get_rho_inst(xflat_t h, uint32_t inst, void* dst, int dst_is_device, int layout) {
  XFLAT_TRACE();
  if (!h || !dst) return fail(h, XFLAT_ERR_INVAL, "NULL argument");
  if (inst >= h->inst.size()) return fail(h, XFLAT_ERR_INVAL, "instance index out of range");
  if (layout != XFLAT_LAYOUT_MATRIX && layout != XFLAT_LAYOUT_NATIVE) return fail(h, XFLAT_ERR_INVAL, "bad layout");
  int rc;
  if ((rc = download_dyn(h))) return rc;
  const HostInst& I = h->inst[inst];
  const uint32_t n = I.n_beams, n_nu = n / 2;
  const size_t bytes = layout == XFLAT_LAYOUT_MATRIX ? (size_t)n * 2 * h->nf * h->nf * 8 : (size_t)n * h->nc * 8;
  double* target = (double*)dst;
  if (!dst_is_device) {
    if ((rc = ensure_stage(h, bytes))) return rc;
    target = h->d_stage;
  }
  const void* src = cur_plane(h, inst);
  const unsigned nb = (n + 255) / 256;
  if (h->real_size == 8) k_export<double><<<nb, 256, 0, h->stream>>>((const double*)src, h->stride, n, n_nu, h->nf, layout, target);
  else k_export<float><<<nb, 256, 0, h->stream>>>((const float*)src, h->stride, n, n_nu, h->nf, layout, target);
  CUDA_TRY(h, cudaGetLastError());
  if (!dst_is_device) CUDA_TRY(h, cudaMemcpyAsync(dst, target, bytes, cudaMemcpyDeviceToHost, h->stream));
  CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  return XFLAT_OK;
}

int xflat_get_rho(xflat_t h, void* dst, int dst_is_device, int layout) {
  XFLAT_TRACE();
  return xflat_get_rho_inst(h, 0, dst, dst_is_device, layout);
}

int xflat_set_rho_inst(xflat_t h, uint32_t inst, const void* src, int src_is_device, int layout, double r_km) {
  XFLAT_TRACE();
  if (!h || !src) return fail(h, XFLAT_ERR_INVAL, "NULL argument");
  if (inst >= h->inst.size()) return fail(h, XFLAT_ERR_INVAL, "instance index out of range");
  if (layout != XFLAT_LAYOUT_MATRIX && layout != XFLAT_LAYOUT_NATIVE) return fail(h, XFLAT_ERR_INVAL, "bad layout");
  if (!is_fin(r_km) || r_km < h->inst[inst].cfg.R_km) return fail(h, XFLAT_ERR_INVAL, "radius below R or not finite");
  int rc;
  if ((rc = download_dyn(h))) return rc;
  const HostInst& I = h->inst[inst];
  const uint32_t n = I.n_beams, n_nu = n / 2;
  const size_t bytes = layout == XFLAT_LAYOUT_MATRIX ? (size_t)n * 2 * h->nf * h->nf * 8 : (size_t)n * h->nc * 8;
  const double* from = (const double*)src;
  if (!src_is_device) {
    if ((rc = ensure_stage(h, bytes))) return rc;
    CUDA_TRY(h, cudaMemcpyAsync(h->d_stage, src, bytes, cudaMemcpyHostToDevice, h->stream));
    from = h->d_stage;
  }
  void* dstp = cur_plane(h, inst);
  const unsigned nb = (n + 255) / 256;
  if (h->real_size == 8) k_import<double><<<nb, 256, 0, h->stream>>>(from, h->stride, n, n_nu, h->nf, layout, (double*)dstp);
  else k_import<float><<<nb, 256, 0, h->stream>>>(from, h->stride, n, n_nu, h->nf, layout, (float*)dstp);
  CUDA_TRY(h, cudaGetLastError());
  InstDyn& d = h->dyn[inst];
  d.r = r_km;
  d.r_end = r_km;
  d.done = 1;
  d.status = 0;
  if ((rc = upload_dyn(h))) return rc;
  CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  h->moments_valid = false;
  return XFLAT_OK;
}

int xflat_set_rho(xflat_t h, const void* src, int src_is_device, int layout, double r_km) {
  XFLAT_TRACE();
  return xflat_set_rho_inst(h, 0, src, src_is_device, layout, r_km);
}

int xflat_pee_inst(xflat_t h, uint32_t inst, double* pee_per_beam, double* pee_mean) {
  XFLAT_TRACE();
  if (!h) return XFLAT_ERR_INVAL;
  if (inst >= h->inst.size()) return fail(h, XFLAT_ERR_INVAL, "instance index out of range");
  int rc;
  if ((rc = download_dyn(h))) return rc;
  const HostInst& I = h->inst[inst];
  const uint32_t n = I.n_beams, ne = I.cfg.n_energy, na = angle_bins(I.cfg);
  const size_t need = ((size_t)n + ne + na + 2) * 8;
  if ((rc = ensure_stage(h, need))) return rc;
  double* pee = h->d_stage;
  double* Ne = pee + n;
  double* rows = Ne + ne;
  double* mean = rows + na;
  const void* src = cur_plane(h, inst);
  const unsigned nb = (n + 255) / 256;
  if (h->real_size == 8) k_pee<double><<<nb, 256, 0, h->stream>>>((const double*)src, h->stride, n, h->nf, pee);
  else k_pee<float><<<nb, 256, 0, h->stream>>>((const float*)src, h->stride, n, h->nf, pee);
  CUDA_TRY(h, cudaMemcpyAsync(Ne, I.N.data(), sizeof(double) * ne, cudaMemcpyHostToDevice, h->stream));
  // denominator sum_j du_j sum_k N_e,k (host, fixed order)
  double sN = 0.0, sdu = 0.0;
  for (uint32_t k = 0; k < ne; ++k) sN += I.N[k];
  for (uint32_t j = 0; j < na; ++j) sdu += I.du[j];
  k_pee_rows<<<(unsigned)((32ull * na + 255) / 256), 256, 0, h->stream>>>(pee, Ne, ne, na, rows);
  k_pee_final<<<1, 1024, 0, h->stream>>>(rows, h->d_du + I.a_off, na, sN * sdu, mean);
  CUDA_TRY(h, cudaGetLastError());
  if (pee_per_beam) CUDA_TRY(h, cudaMemcpyAsync(pee_per_beam, pee, sizeof(double) * n, cudaMemcpyDeviceToHost, h->stream));
  if (pee_mean) CUDA_TRY(h, cudaMemcpyAsync(pee_mean, mean, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  return XFLAT_OK;
}

int xflat_pee(xflat_t h, double* pee_per_beam, double* pee_mean) {
  XFLAT_TRACE();
  return xflat_pee_inst(h, 0, pee_per_beam, pee_mean);
}

int xflat_flux_spectra(xflat_t h, uint32_t inst, double* flux) {
  XFLAT_TRACE();
  if (!h || !flux) return fail(h, XFLAT_ERR_INVAL, "NULL argument");
  if (inst >= h->inst.size()) return fail(h, XFLAT_ERR_INVAL, "instance index out of range");
  if (!h->inst[inst].spectra) return fail(h, XFLAT_ERR_STATE, "set_spectra first");
  int rc;
  if ((rc = download_dyn(h))) return rc;
  const HostInst& I = h->inst[inst];
  const uint32_t ne = I.cfg.n_energy, na = angle_bins(I.cfg);
  const int nf = h->nf;
  const size_t nval = 2ull * nf * ne;
  if ((rc = ensure_stage(h, 2 * nval * sizeof(double)))) return rc;
  double* dN = h->d_stage;
  double* dflux = dN + nval;
  CUDA_TRY(h, cudaMemcpyAsync(dN, I.N.data(), nval * sizeof(double), cudaMemcpyHostToDevice, h->stream));
  const void* src = cur_plane(h, inst);
  const unsigned nb = (unsigned)((nval + 127) / 128);
  if (h->real_size == 8) k_flux_spectra<double><<<nb, 128, 0, h->stream>>>((const double*)src, h->stride, ne, na, nf, dN, h->d_du + I.a_off, dflux);
  else k_flux_spectra<float><<<nb, 128, 0, h->stream>>>((const float*)src, h->stride, ne, na, nf, dN, h->d_du + I.a_off, dflux);
  CUDA_TRY(h, cudaGetLastError());
  CUDA_TRY(h, cudaMemcpyAsync(flux, dflux, nval * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  return XFLAT_OK;
}

int xflat_get_stats_inst(xflat_t h, uint32_t inst, xflat_stats* out) {
  XFLAT_TRACE();
  if (!h || !out) return fail(h, XFLAT_ERR_INVAL, "NULL argument");
  if (inst >= h->inst.size()) return fail(h, XFLAT_ERR_INVAL, "instance index out of range");
  int rc;
  if ((rc = download_dyn(h))) return rc;
  std::memset(out, 0, sizeof(*out));
  const InstDyn& d = h->dyn[inst];
  out->r_km = d.r;
  out->h_km = adaptive(h->inst[inst].cfg.integrator) ? d.h : d.h_fixed;
  out->last_err = d.err;
  out->accepted = d.accepted;
  out->rejected = d.rejected;
  out->stage_evals = d.stage_evals;
  uint64_t bsu = 0;
  for (size_t i = 0; i < h->inst.size(); ++i) bsu += (uint64_t)h->inst[i].n_beams * h->dyn[i].stage_evals;
  out->beam_stage_updates = bsu;
  out->launches = h->launches;
  out->n_beams = h->inst[inst].n_beams;
  out->n_instances = (uint32_t)h->inst.size();
  out->status = d.status;
  out->grid_blocks = (uint32_t)h->grid;
  out->block_size = (uint32_t)h->block;
  return XFLAT_OK;
}

int xflat_get_stats(xflat_t h, xflat_stats* out) {
  XFLAT_TRACE(); return xflat_get_stats_inst(h, 0, out); }

int xflat_adjoint(xflat_t h, double r0_km, double r1_km, uint32_t n_steps, uint32_t checkpoint_every,
                  double* dJ_dN, double* dJ_dtheta, double* J_out) {
  XFLAT_TRACE();
  if (!h) return XFLAT_ERR_INVAL;
  if (h->nf != 2 || h->inst.size() != 1 || h->extended || h->inst[0].cfg.geometry != XFLAT_GEOMETRY_BULB ||
      h->inst[0].cfg.matter_kind == XFLAT_MATTER_TABLE)
    return fail(h, XFLAT_ERR_UNSUPPORTED,
                "the adjoint is built for one two-flavour bulb-model instance (bulb geometry, no matter table)");
  HostInst& I = h->inst[0];
  if (!I.spectra) return fail(h, XFLAT_ERR_STATE, "set_spectra before the adjoint");
  if (!is_fin(r0_km) || !is_fin(r1_km) || r0_km < I.cfg.R_km || !(r1_km > r0_km))
    return fail(h, XFLAT_ERR_INVAL, "need R <= r0 < r1, finite");
  if (n_steps == 0 || checkpoint_every == 0) return fail(h, XFLAT_ERR_INVAL, "n_steps and checkpoint_every must be >= 1");
  const uint32_t ne = I.cfg.n_energy, na = I.cfg.n_angle, n = I.n_beams;
  const uint32_t K = std::min(checkpoint_every, n_steps);
  const uint32_t n_ck = (n_steps + K - 1) / K;
  // host tables (the forward step kernel's tables, in double)
  InstConst ic = h->ic[0];
  std::vector<double> et;
  build_tables(h, I, et, ic);
  double SW = 0.0;
  for (uint32_t j = 0; j < na; ++j)
    for (uint32_t k = 0; k < ne; ++k) SW += I.du[j] * I.N[k];
  if (!(SW > 0)) return fail(h, XFLAT_ERR_INVAL, "the objective needs a positive nu_e luminosity");
  std::vector<double> objw(ne);
  for (uint32_t k = 0; k < ne; ++k) objw[k] = I.N[k] / SW;
  int G = adjoint_blocks_per_sm() * h->sm_count;
  if (G < 1) return fail(h, XFLAT_ERR_CUDA, "adjoint kernel does not fit on an SM");
  G = (int)std::max<uint64_t>(1, std::min<uint64_t>((uint64_t)G, ((uint64_t)n + kAdjBlock - 1) / kAdjBlock));
  // device buffers
  const size_t n3 = 3ull * n;
  const size_t words = ne + 2ull * ne + 2 * na + ne                // omega, g, u, du, objw
                     + 3 * n3 + (size_t)n_ck * n3 + (size_t)K * n3 // y, ksum, klast, ck, seg
                     + (size_t)K * 4 * kAdjStageVals + 3 * n3      // stage_sc, ystage
                     + 3 * n3 + 2ull * n                           // a, ybar, v, gw, gth
                     + (size_t)G * kAdjPartStride + kGlobWords     // part, glob
                     + 5ull * ne;                                  // pee_sum, gw_sum, gth_sum
  double* base = nullptr;
  Barrier* bar = nullptr;
  int* status = nullptr;
  if (dev_alloc(&base, words * sizeof(double)) != cudaSuccess) return fail(h, XFLAT_ERR_NOMEM, "adjoint buffers");
  if (dev_alloc(&bar, sizeof(Barrier)) != cudaSuccess || dev_alloc(&status, sizeof(int)) != cudaSuccess) {
    cudaFree(base);
    if (bar) cudaFree(bar);
    return fail(h, XFLAT_ERR_NOMEM, "adjoint barrier");
  }
  auto release_all = [&]() { cudaFree(base); cudaFree(bar); cudaFree(status); };
  double* q = base;
  auto take = [&](size_t cnt) { double* r = q; q += cnt; return r; };
  AdjParams p{};
  p.n_beams = n;
  p.n_energy = ne;
  p.n_angle = na;
  double* d_omega = take(ne);
  double* d_g = take(2ull * ne);
  double* d_u = take(na);
  double* d_du = take(na);
  double* d_objw = take(ne);
  p.omega = d_omega; p.g = d_g; p.u = d_u; p.du = d_du; p.objw = d_objw;
  p.ic = ic;
  p.r0 = r0_km;
  p.h = (r1_km - r0_km) / (double)n_steps;
  p.n_steps = (int)n_steps;
  p.ck_every = (int)K;
  p.y = take(n3); p.ksum = take(n3); p.klast = take(n3);
  p.ck = take((size_t)n_ck * n3);
  p.seg = take((size_t)K * n3);
  p.stage_sc = take((size_t)K * 4 * kAdjStageVals);
  p.ystage = take(3 * n3);
  p.a = take(n3); p.ybar = take(n3); p.v = take(n3);
  p.gw = take(n); p.gth = take(n);
  p.part = take((size_t)G * kAdjPartStride);
  p.glob = take(kGlobWords);
  double* d_pee = take(ne);
  double* d_gws = take(2ull * ne);
  double* d_gths = take(2ull * ne);
  p.bar = bar;
  p.timeout_ns = h->timeout_ns;
  p.status = status;
  cudaStream_t st = h->stream;
  int rc = XFLAT_OK;
  auto check = [&](cudaError_t e, const char* what) {
    if (e != cudaSuccess && rc == XFLAT_OK) rc = fail(h, XFLAT_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
    return rc == XFLAT_OK;
  };
  auto device_status = [&]() {
    int s = 0;
    if (!check(cudaMemcpyAsync(&s, status, sizeof(int), cudaMemcpyDeviceToHost, st), "status read")) return false;
    if (!check(cudaStreamSynchronize(st), "adjoint launch")) return false;
    if (s) rc = fail(h, s, std::string("adjoint device status: ") + xflat_status_string(s));
    return rc == XFLAT_OK;
  };
  // the initial condition of Sec. 3.4: s = z (P = diag(1, 0)) for every beam
  std::vector<double> y0(n3, 0.0);
  for (uint32_t b = 0; b < n; ++b) y0[2ull * n + b] = 1.0;
  std::vector<double> pee(ne), gws(2ull * ne), gths(2ull * ne);
  double J = 0.0;
  check(cudaMemcpyAsync(d_omega, et.data(), ne * 8, cudaMemcpyHostToDevice, st), "upload") &&
  check(cudaMemcpyAsync(d_g, et.data() + ne, 2ull * ne * 8, cudaMemcpyHostToDevice, st), "upload") &&
  check(cudaMemcpyAsync(d_u, I.u.data(), na * 8, cudaMemcpyHostToDevice, st), "upload") &&
  check(cudaMemcpyAsync(d_du, I.du.data(), na * 8, cudaMemcpyHostToDevice, st), "upload") &&
  check(cudaMemcpyAsync(d_objw, objw.data(), ne * 8, cudaMemcpyHostToDevice, st), "upload") &&
  check(cudaMemcpyAsync(p.y, y0.data(), n3 * 8, cudaMemcpyHostToDevice, st), "upload") &&
  check(cudaMemsetAsync(bar, 0, sizeof(Barrier), st), "memset") &&
  check(cudaMemsetAsync(status, 0, sizeof(int), st), "memset") &&
  check(cudaMemsetAsync(p.klast, 0, n3 * 8, st), "memset");
  if (rc == XFLAT_OK) {
    p.mode = kAdjForward;
    if (check(adjoint_launch(p, G, st), "adjoint forward launch") && device_status()) {
      check(adjoint_energy_sums(p, d_pee, d_gws, d_gths, st), "energy sums");
      check(cudaMemcpyAsync(pee.data(), d_pee, ne * 8, cudaMemcpyDeviceToHost, st), "download");
      check(cudaMemcpyAsync(&J, p.glob + kGlobJ, 8, cudaMemcpyDeviceToHost, st), "download");
    }
  }
  for (int c = (int)n_ck - 1; c >= 0 && rc == XFLAT_OK; --c) {
    p.mode = kAdjBackward;
    p.seg_first = c * (int)K;
    p.seg_count = std::min<int>((int)K, (int)n_steps - c * (int)K);
    if (!check(adjoint_launch(p, G, st), "adjoint backward launch")) break;
    if (c == 0 || (c % 16) == 0) device_status();
  }
  if (rc == XFLAT_OK) {
    check(adjoint_energy_sums(p, d_pee, d_gws, d_gths, st), "energy sums");
    check(cudaMemcpyAsync(gws.data(), d_gws, 2ull * ne * 8, cudaMemcpyDeviceToHost, st), "download");
    check(cudaMemcpyAsync(gths.data(), d_gths, 2ull * ne * 8, cudaMemcpyDeviceToHost, st), "download");
    check(cudaStreamSynchronize(st), "adjoint");
  }
  release_all();
  if (rc != XFLAT_OK) return rc;
  // chain rule to the per-bin luminosities: g_nu,k = (N_e - N_x)/ws, g_nubar,k = -(Nbar_e - Nbar_x)/ws
  // (mu carries ws, so J depends on N only through the products mu g), plus the objective's own
  // weights du_j N_e,k
  const double ws = ic.wscale;
  if (dJ_dN) {
    for (uint32_t k = 0; k < ne; ++k) {
      const double gn = gws[k] / ws, gb = gws[ne + k] / ws;
      dJ_dN[0 * ne + k] = gn + pee[k] / SW;                // N[nu][e][k]
      dJ_dN[1 * ne + k] = -gn;                             // N[nu][x][k]
      dJ_dN[2 * ne + k] = -gb;                             // N[nubar][e][k]
      dJ_dN[3 * ne + k] = gb;                              // N[nubar][x][k]
    }
  }
  if (dJ_dtheta) {
    double t = 0.0;
    for (size_t i = 0; i < gths.size(); ++i) t += gths[i];
    *dJ_dtheta = t;
  }
  if (J_out) *J_out = J;
  return XFLAT_OK;
}

// ---- beam shards: one problem over several GPUs (Sec. 3.3's decomposition of the angle bins and
// the sum of the Eq. F integrals over ranks at every evaluation) ---------------------------------
int xflat_create_shard(const xflat_config* cfg, uint32_t beam_lo, uint32_t beam_hi, xflat_t* out) {
  XFLAT_TRACE();
  if (!cfg || !out) return XFLAT_ERR_INVAL;
  xflat_t h = nullptr;
  int rc = create_impl(cfg, 1, &h);
  if (rc) return rc;
  const uint32_t nb = h->inst[0].n_beams;
  if (!(beam_lo < beam_hi && beam_hi <= nb) || beam_lo % kAlignBeams != 0 ||
      (beam_hi % kAlignBeams != 0 && beam_hi != nb)) {
    xflat_destroy(h);
    return XFLAT_ERR_INVAL;
  }
  h->shard = true;
  h->shard_lo = beam_lo;
  h->shard_hi = beam_hi;
  h->ic[0].rec_start = beam_lo;
  if ((rc = setup_launch_shape(h, *cfg)) || (rc = upload_inst(h))) {
    xflat_destroy(h);
    return rc;
  }
  *out = h;
  return XFLAT_OK;
}

int xflat_shard_info(xflat_t h, uint32_t* passes_per_step, uint32_t* n_words) {
  XFLAT_TRACE();
  if (!h || !h->shard) return h ? fail(h, XFLAT_ERR_STATE, "not a beam-shard handle") : XFLAT_ERR_INVAL;
  const int it = h->integrator;
  const uint32_t passes = it == XFLAT_DP45 ? 7 : it == XFLAT_EXP_MIDPOINT ? 2 : it == XFLAT_LIE_ADAPTIVE ? 11 : 4;
  const uint32_t nm = h->extended ? 12 : (h->nf == 2 ? kNM2 : kNM3);
  if (passes_per_step) *passes_per_step = passes;
  if (n_words) *n_words = 2 * nm + 2;
  return XFLAT_OK;
}

int xflat_shard_begin(xflat_t h, double r1_km) {
  XFLAT_TRACE();
  if (!h || !h->shard) return h ? fail(h, XFLAT_ERR_STATE, "not a beam-shard handle") : XFLAT_ERR_INVAL;
  bool any = false, changed = false;
  int rc;
  if ((rc = prepare_targets(h, &r1_km, any, changed))) return rc;
  if ((rc = upload_dyn(h))) return rc;
  if ((rc = clear_sync_words(h))) return rc;
  h->shard_last = -2;
  h->moments_valid = false;
  return XFLAT_OK;
}

int xflat_shard_pass(xflat_t h, int32_t pass) {
  XFLAT_TRACE();
  if (!h || !h->shard) return h ? fail(h, XFLAT_ERR_STATE, "not a beam-shard handle") : XFLAT_ERR_INVAL;
  uint32_t passes = 0;
  xflat_shard_info(h, &passes, nullptr);
  if (pass < -1 || pass >= (int32_t)passes) return fail(h, XFLAT_ERR_INVAL, "pass out of range");
  int rc;
  if ((rc = launch(h, 0, 0, h->stream, kShardPass, pass))) return rc;
  h->shard_last = pass;
  return XFLAT_OK;
}

// The accumulator slot the last pass reduced into: the moment pass slot 1, stage pass p slot p + 2,
// the final pass slot 0 (the new state's moments, where the integrator forms them).
int shard_slot(xflat_t h) {
  uint32_t passes = 0;
  xflat_shard_info(h, &passes, nullptr);
  if (h->shard_last == -1) return 1;
  return h->shard_last == (int)passes - 1 ? 0 : h->shard_last + 2;
}

int xflat_shard_partials(xflat_t h, int64_t* words) {
  XFLAT_TRACE();
  if (!h || !h->shard) return h ? fail(h, XFLAT_ERR_STATE, "not a beam-shard handle") : XFLAT_ERR_INVAL;
  if (!words) return fail(h, XFLAT_ERR_INVAL, "words is NULL");
  if (h->shard_last < -1) return fail(h, XFLAT_ERR_STATE, "no pass launched");
  uint32_t nw = 0;
  xflat_shard_info(h, nullptr, &nw);
  const int nm = (int)(nw - 2) / 2, slot = shard_slot(h);
  constexpr int kWords = kAccCopies * kNMMax * 2;
  std::vector<unsigned long long> acc(kWords);
  unsigned long long em = 0;
  int nonfin = 0;
  CUDA_TRY(h, cudaMemcpyAsync(acc.data(), h->d_acc + (size_t)slot * kWords, kWords * 8, cudaMemcpyDeviceToHost, h->stream));
  CUDA_TRY(h, cudaMemcpyAsync(&em, h->d_errmax, 8, cudaMemcpyDeviceToHost, h->stream));
  CUDA_TRY(h, cudaMemcpyAsync(&nonfin, h->d_nonfinite, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  for (int c = 0; c < nm; ++c) {
    unsigned __int128 t = 0;
    for (int cp = 0; cp < kAccCopies; ++cp) {
      const unsigned long long* w = acc.data() + ((size_t)cp * kNMMax + c) * 2;
      if (h->real_size == 4) t += (unsigned __int128)(__int128)(long long)w[0];   // one signed word
      else t += ((unsigned __int128)w[1] << 64) | (unsigned __int128)w[0];
    }
    words[2 * c] = (int64_t)(unsigned long long)t;
    words[2 * c + 1] = (int64_t)(unsigned long long)(t >> 64);
  }
  words[2 * nm] = (int64_t)em;
  words[2 * nm + 1] = nonfin;
  return XFLAT_OK;
}

int xflat_shard_set_totals(xflat_t h, const int64_t* words) {
  XFLAT_TRACE();
  if (!h || !h->shard) return h ? fail(h, XFLAT_ERR_STATE, "not a beam-shard handle") : XFLAT_ERR_INVAL;
  if (!words) return fail(h, XFLAT_ERR_INVAL, "words is NULL");
  if (h->shard_last < -1) return fail(h, XFLAT_ERR_STATE, "no pass launched");
  uint32_t nw = 0;
  xflat_shard_info(h, nullptr, &nw);
  const int nm = (int)(nw - 2) / 2, slot = shard_slot(h);
  constexpr int kWords = kAccCopies * kNMMax * 2;
  std::vector<unsigned long long> acc(kWords, 0ull);    // the total in copy 0, the other copies 0
  for (int c = 0; c < nm; ++c) {
    acc[(size_t)c * 2] = (unsigned long long)words[2 * c];
    acc[(size_t)c * 2 + 1] = h->real_size == 4 ? 0ull : (unsigned long long)words[2 * c + 1];
    if (h->real_size == 4) {
      // a mixed accumulator is one signed 64-bit word: the total must fit it
      const long long lo = words[2 * c], hi = words[2 * c + 1];
      if (hi != (lo < 0 ? -1 : 0)) return fail(h, XFLAT_ERR_INVAL, "moment total out of range");
    }
  }
  const unsigned long long em = (unsigned long long)words[2 * nm];
  const int nonfin = words[2 * nm + 1] ? 1 : 0;
  CUDA_TRY(h, cudaMemcpy(h->d_acc + (size_t)slot * kWords, acc.data(), kWords * 8, cudaMemcpyHostToDevice));
  CUDA_TRY(h, cudaMemcpy(h->d_errmax, &em, 8, cudaMemcpyHostToDevice));
  CUDA_TRY(h, cudaMemcpy(h->d_nonfinite, &nonfin, sizeof(int), cudaMemcpyHostToDevice));
  return XFLAT_OK;
}

int xflat_shard_serial(xflat_t h, int32_t after_moment_pass, int* done_out) {
  XFLAT_TRACE();
  if (!h || !h->shard) return h ? fail(h, XFLAT_ERR_STATE, "not a beam-shard handle") : XFLAT_ERR_INVAL;
  uint32_t passes = 0;
  xflat_shard_info(h, &passes, nullptr);
  const bool init = after_moment_pass != 0;
  if (init ? h->shard_last != -1 : h->shard_last != (int)passes - 1)
    return fail(h, XFLAT_ERR_STATE, "the serial section follows the moment pass or a step's final pass");
  int rc;
  if ((rc = launch(h, 0, 0, h->stream, init ? kShardSerialInit : kShardSerialFinal, 0))) return rc;
  int st, ad;
  if ((rc = read_words(h, st, ad))) return rc;
  h->moments_valid = true;
  if (done_out) *done_out = ad;
  if (st) {
    if ((rc = download_dyn(h))) return rc;
    return fail(h, st, std::string("device status: ") + xflat_status_string(st));
  }
  return XFLAT_OK;
}

const char* xflat_status_string(int s) {
  switch (s) {
    case XFLAT_OK: return "ok";
    case XFLAT_ERR_INVAL: return "invalid argument";
    case XFLAT_ERR_NOMEM: return "out of memory";
    case XFLAT_ERR_CUDA: return "CUDA error";
    case XFLAT_ERR_TIMEOUT: return "device barrier timeout";
    case XFLAT_ERR_NONFINITE: return "non-finite value";
    case XFLAT_ERR_STEP: return "step size underflow";
    case XFLAT_ERR_STATE: return "call order violated";
    case XFLAT_ERR_UNSUPPORTED: return "unsupported";
    default: return "unknown status";
  }
}

const char* xflat_last_error(xflat_t h) { return h ? h->err.c_str() : "NULL handle"; }

int xflat_debug_fail_alloc(uint32_t nth) {
  XFLAT_TRACE();
  g_fail_alloc.store((long)nth);
  return XFLAT_OK;
}

int xflat_debug_barrier_extra(xflat_t h, uint32_t extra) {
  XFLAT_TRACE();
  if (!h) return XFLAT_ERR_INVAL;
  h->debug_extra = extra;
  return XFLAT_OK;
}

int xflat_debug_trace(xflat_t h, uint32_t n_passes, uint64_t* host_out, uint32_t* grid_out) {
  XFLAT_TRACE();
  if (!h) return XFLAT_ERR_INVAL;
  if (grid_out) *grid_out = (uint32_t)h->grid;
  if (host_out) {
    if (!h->d_trace) return fail(h, XFLAT_ERR_STATE, "trace not armed");
    CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    CUDA_TRY(h, cudaMemcpy(host_out, h->d_trace, (size_t)h->trace_passes * h->grid * 4 * 8, cudaMemcpyDeviceToHost));
    return XFLAT_OK;
  }
  if (h->d_trace) {
    cudaStreamSynchronize(h->stream);
    cudaFree(h->d_trace);
    h->d_trace = nullptr;
    h->trace_passes = 0;
  }
  if (n_passes == 0) return XFLAT_OK;
  const size_t bytes = (size_t)n_passes * h->grid * 4 * 8;
  CUDA_TRY(h, dev_alloc(&h->d_trace, bytes));
  CUDA_TRY(h, cudaMemset(h->d_trace, 0, bytes));
  h->trace_passes = n_passes;
  return XFLAT_OK;
}

}  // extern "C"
