// Internal device-side data structures of the bulb-model solver (not part of the C ABI).
//
// Work decomposition.  All instances' beams live in one set of SoA planes.  The beams of the whole
// problem are cut into G equal contiguous slices, one per persistent block; the intersection of a
// slice with an instance is a "piece".  A block processes its pieces one after the other and adds
// each piece's moments to its instance's fixed-point accumulators; the last block to arrive at the
// device-wide barrier converts them and derives the next stage's constants before it releases the
// other blocks.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace xflat {

constexpr int kMaxStages = 12;      // stage slots 0..11 (Richardson-controlled CF4: 11 stages)
constexpr int kStateRingDepth = 3;  // FP32 two-flavour bulb passes: state vectors in flight per thread
constexpr int kNM2 = 6;             // 2 flavours: j0 (3) and j1 (3) Bloch components
constexpr int kNM3 = 18;            // 3 flavours: j0 and j1, 9 reals each
constexpr int kNSC2 = 8;            // stage constants: mu*j0 (3), mu*j1 (3), lambda, R^2/r^2
constexpr int kNSC3 = 20;           // mu*j0 (9), mu*j1 (9), lambda, R^2/r^2
constexpr int kNMMax = 18;
constexpr int kNSCMax = 20;
// Blocks add their moment partials to one of kAccCopies copies of an instance's accumulators
// (block index mod kAccCopies), so the integer atomics of hundreds of blocks spread over several
// L2 lines instead of queueing on one; the last block sums the copies (exact integer sums).
constexpr int kAccCopies = 8;
// accumulator words per instance: [stage slot][copy][component][2]
constexpr int kAccWordsPerInst = kMaxStages * kAccCopies * kNMMax * 2;

enum Integrator : int { kRK4 = 0, kDP45 = 1, kLieRK4 = 2, kExpMid = 3, kLieAdaptive = 4 };
enum Matter : int { kMatterNone = 0, kMatterPower = 1, kMatterConst = 2, kMatterTable = 3 };
enum Geometry : int { kGeomBulb = 0, kGeomSingleAngle = 1, kGeomHomogeneous = 2 };
enum ShardMode : int { kShardOff = 0, kShardPass = 1, kShardSerialInit = 2, kShardSerialFinal = 3 };

// Instance constants, written by the host before a launch.
struct InstConst {
  uint64_t beam_off;        // first beam of the instance in the planes
  uint32_t n_beams;         // 2 * n_angle * n_energy
  uint32_t n_energy, n_angle;
  uint32_t e_off, a_off;    // offsets into the energy and angle tables
  uint32_t n_phi;           // azimuthal bins of the extended bulb model (n_angle counts u x phi)
  uint64_t div_magic;       // floor(2^40 / n_energy) + 1: q = (l * magic) >> 40 is l / n_energy
  double R2;                // R^2 (km^2)
  double mu_coef;           // mu(r) = mu_coef / r^2, includes the weight scale wscale
  double wscale;            // physical per-bin number luminosity of a unit table weight (1/s)
  double acc_unit;          // mixed kernels: value of one unit of the fixed-point moment sums (2^-S)
  double lam_coef, power, lam_const, r_ref;   // lambda(r) = lam_coef (r_ref / r)^power
  const double* mtab;       // matter table: [mt_n][3] (r_i, lambda_i, exponent p_i of the interval
  int32_t mt_n;             // after r_i: lambda = lambda_i (r/r_i)^p_i), device memory, or null
  int32_t geom;             // Geometry
  uint32_t rec_start;       // first beam of the instance this handle integrates (beam shards; else 0):
                            // the block holding it records the stage moments and constants
  double mu_const;          // homogeneous geometry: the constant nu-nu strength mu0 (1/km)
  int32_t matter;
  int32_t adaptive;
  double B[3];              // 2 flavours: unit vacuum vector (sin 2th, 0, -cos 2th)
  double M21[6], M31[6];    // 3 flavours: U diag(0,1,0) U^T, U diag(0,0,1) U^T (00,11,22,01,02,12)
  double rtol, atol, h_min, h_max;
};

// Instance dynamics, owned by the device during a launch.
struct InstDyn {
  double r, h, r_end;       // current radius, next step size, target
  double r0_fixed, h_fixed; // fixed-step grid: r_n = r0_fixed + n h_fixed
  long long n_fixed, n_fixed_total;
  double err;               // last error norm
  double rs[kMaxStages];    // stage radii of the current step
  double xs[kMaxStages];    // R^2 / rs^2
  double mus[kMaxStages];   // mu(rs): nu-nu strength at the stage radii
  double lams[kMaxStages];  // lambda(rs): matter strength at the stage radii
  int32_t status, done, last, parity;
  int32_t geo_pending, pad_geo;   // stage geometry of the next step still to be computed
  unsigned long long accepted, rejected, stage_evals;
  double mom[kMaxStages][kNMMax];   // raw moments (weights normalised by wscale) per stage
  double sc[kMaxStages][kNSCMax];   // stage constants per stage
};

struct Piece {
  int32_t inst;
  uint32_t start;           // first local beam of the piece within the instance
  uint32_t len;             // beams in the piece
  uint32_t jj_lo;           // first combined angle index (species * n_angle + j) touched
  uint32_t n_jj;            // combined angle indices touched
  uint32_t pad;
};

struct Barrier {
  unsigned int count;
  unsigned int pad0[31];
  unsigned int gen;
  unsigned int pad1[31];
  int abort;
  int timeout_hits;
  unsigned int extra;       // test hook: additional arrivals expected
  // dynamic piece scheduling: the pass after barrier generation g (which steps by 2, bit 0 being a
  // flag) takes pieces from chunk[(g >> 1) & 1]; the last block at a barrier zeroes the counter
  // of the pass that follows it before the release
  unsigned int chunk[2];
  // checked build (-DXFLAT_BOUNDS): the first access found outside its allocation (site number,
  // byte offset from the allocation's start)
  int bounds_site;
  long long bounds_off;
  int pad2[24];
};

// Checked build: the allocations the step kernel's pass body reads and writes, by role.
struct Span {
  const char* lo;
  unsigned long long bytes;
};
enum SpanId : int { kSpanPlanes = 0, kSpanEscr, kSpanKst, kSpanEtab, kSpanU, kSpanDu, kSpanCount };

// ---------------------------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long globaltimer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ unsigned int ld_acquire(const unsigned int* p) {
  unsigned int v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ int ld_acquire_int(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ uint32_t fast_div(uint32_t l, uint64_t magic) {
  return (uint32_t)(((uint64_t)l * magic) >> 40);
}

// Deterministic block sum of NV doubles per thread (fixed shuffle tree, then fixed smem tree).
// Result valid in thread 0.  scratch: >= 32 * NV doubles.
template <int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV], double* scratch) {
#pragma unroll
  for (int i = 0; i < NV; ++i) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[i] += __shfl_down_sync(0xffffffffu, v[i], o);
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  __syncthreads();
  if (lane == 0) {
#pragma unroll
    for (int i = 0; i < NV; ++i) scratch[warp * NV + i] = v[i];
  }
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int i = 0; i < NV; ++i) {
      double s = lane < nw ? scratch[lane * NV + i] : 0.0;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
      v[i] = s;
    }
  }
}

__device__ __forceinline__ double block_max(double v, double* scratch) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  __syncthreads();
  if (lane == 0) scratch[warp] = v;
  __syncthreads();
  if (warp == 0) {
    double s = lane < nw ? scratch[lane] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s = fmax(s, __shfl_down_sync(0xffffffffu, s, o));
    v = s;
  }
  return v;
}

// Device-wide barrier.  Returns kBarLast in every thread of the one block that arrived last (that
// block must call barrier_release after its serial work), kBarReleased elsewhere after the
// release, or kBarAbort.  Every wait is bounded by timeout_ns: on expiry the block records
// XFLAT_ERR_TIMEOUT in *status_word, raises the abort flag and returns kBarAbort; a block that sees
// the abort flag while waiting also returns kBarAbort, so every block leaves the kernel.
enum BarrierResult : int { kBarReleased = 0, kBarLast = 1, kBarAbort = 2 };

__device__ __forceinline__ int barrier_arrive(Barrier* bar, unsigned int n_blocks,
                                             unsigned long long timeout_ns, int* status_word,
                                             int* s_flag, unsigned int* s_gen) {
  // *s_gen: in, the generation this block last saw; out (released blocks), the new one
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned int g = *s_gen;                 // generation of the last barrier this block passed
    __threadfence();                               // this block's writes before its arrival
    const unsigned int ticket = atomicAdd(&bar->count, 1u);
    const unsigned int expected = n_blocks + bar->extra;
    int res = (ticket == expected - 1) ? kBarLast : kBarReleased;
    unsigned int gnow = g;
    if (res == kBarLast) {
      __threadfence();                             // acquire: every other block's writes
    } else {
      const unsigned long long t0 = globaltimer_ns();
      while ((gnow = ld_acquire(&bar->gen)) == g) {   // acquire load: no further fence needed
        if (ld_acquire_int(&bar->abort)) { res = kBarAbort; break; }
        if (globaltimer_ns() - t0 > timeout_ns) {
          atomicAdd(&bar->timeout_hits, 1);
          atomicCAS(status_word, 0, 4 /* XFLAT_ERR_TIMEOUT */);
          atomicExch(&bar->abort, 1);
          res = kBarAbort;
          break;
        }
        __nanosleep(20);
      }
    }
    if (res == kBarReleased) *s_gen = gnow;
    *s_flag = res | (int)((gnow & 1u) << 4);       // bit 4: the flag carried by the release
  }
  __syncthreads();
  return *s_flag;
}

// Release the barrier (last block only, after its serial work; every thread that wrote shared
// results must have executed __threadfence() before the __syncthreads here).  The generation word
// advances by 2 and its low bit carries one flag to every waiting block (the kernels use it for
// "every instance finished"), so a released block learns it from the load that saw the release.
// The count is reset before the new generation is published with release ordering.
__device__ __forceinline__ void barrier_release(Barrier* bar, int flag, unsigned int* s_gen) {
  __syncthreads();
  if (threadIdx.x == 0) {
    bar->count = 0;
    const unsigned int ng = ((*s_gen & ~1u) + 2u) | (flag ? 1u : 0u);
    *s_gen = ng;
    unsigned int old;
    asm volatile("atom.release.gpu.global.exch.b32 %0, [%1], %2;" : "=r"(old) : "l"(&bar->gen), "r"(ng) : "memory");
  }
}

__device__ __forceinline__ bool barrier_aborted(Barrier* bar, int* s_flag) {
  __syncthreads();
  if (threadIdx.x == 0) *s_flag = ld_acquire_int(&bar->abort);
  __syncthreads();
  return *s_flag != 0;
}

}  // namespace xflat
