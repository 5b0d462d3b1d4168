// Persistent radial-step kernel of the bulb model (arXiv:1912.10596, Sec. 2 and Sec. 3.4).
//
// One cooperative launch advances every active instance by up to n_steps radial steps.  A step is a
// sequence of passes over all beams separated by device-wide barriers, because every stage of the
// integrator needs the angular moments of *all* beams (Eq. Hnu / Eq. F):
//
//   pass p (p = 0 .. S-2): form the stage state Y_{p+2} of every beam from the step's initial
//       state y and the stage derivatives k_1..k_{p+1}, and reduce the moments of Y_{p+2}.  FP32
//       kernels recompute k_1..k_{p+1} in registers from y and the earlier stages' constants (the
//       stage vectors are not stored); FP64 RK4 / DP45 kernels read k_1..k_p and Y_{p+1} back from
//       HBM planes and evaluate only k_{p+1} (stored_stages);
//   final pass: form the new state (and, for DP45, the embedded error), write it to the second
//       state buffer and reduce either the moments of the new state (fixed step) or the error norm
//       (DP45).
//
// So every pass reads each beam's state once (vector loads of the SoA planes, or the per-thread
// cp.async ring of the FP32 two-flavour bulb kernels) and a step writes it once; the FP64 kernels
// also move their stage planes.  The exponential integrators (commutator-free Lie RK4, the
// exponential midpoint rule, the adaptive Lie RK4 with Richardson control) build every stage state
// from y by exact propagators exp(-i Om) y exp(i Om) of Eq. U instead: a rotation of the Bloch
// vector for two flavours, an eigen-decomposition of the 3 x 3 generator for three (propagate3).
//
// Moments without cancellation.  With the measure of Eq. Hnu in u-bins, the nu-nu term of beam b is
// mu(r) (J0 - cos(th_b) J1), J0 = sum w s / cos(th), J1 = sum w s.  Far from the neutrino sphere
// J0 and J1 agree to O(R^2/r^2) and the difference cancels catastrophically in FP32.  The kernel
// therefore reduces J1 and D = J0 - J1 = sum w s (1/cos(th) - 1), and assembles
// J0 - cos(th_b) J1 = D + (1 - cos(th_b)) J1, with 1 - cos = u x / (1 + cos), x = R^2/r^2, and
// 1/cos - 1 = (1 - cos)/cos: every term is computed without cancellation.
//
// Reduction.  FP64 path: each thread accumulates its beams' contributions in double, each block
// reduces them with a fixed shuffle/shared-memory tree in double and adds its partial to the
// instance accumulator as a 128-bit fixed-point integer (exact to 2^-64).  Mixed path: each beam's
// contribution is formed in FP32 (per-beam algebra) and summed per thread without rounding loss as
// an unevaluated (hi, lo) pair (TwoSum); at the end of the pass the pair goes to integers in units
// of the instance's 2^-S (the FP32 weights carry that power-of-two scale), and the warp shuffle
// trees, the sum over warps and the grid sum are integer additions.  So the moments are the
// FP64-accurate sums of the FP32 contributions, with no FP64 instruction per beam (GB300's FP64
// pipe is ~1/68 of its FP32 rate).  Integer addition is associative, so either grid-level sum is
// identical whatever order the blocks arrive in.  Every block derives a stage's constants
// mu(r_s) D, mu(r_s) J1, lambda(r_s) from the integer sums; the last block to arrive at a step's
// final barrier runs the step-size controller in double.
#pragma once

#include "xflat_internal.cuh"

namespace xflat {

// --------------------------------------------------------------------------------------------
// Butcher tableaus (1-based stage indices).
// Traits of every tableau: S stages (stage radii r + c_s h), kPasses passes per step,
// kAdaptive (embedded error control), kErrPow (the controller's exponent is -1/kErrPow),
// kFinalMoments (the final pass reduces the moments of the new state: stage 1 of the next step),
// kEvalsPerStep (new stage evaluations per step), kEM2 (exponential midpoint rule).
struct TabRK4 {
  static constexpr bool kRichardson = false;
  static constexpr int S = 4;
  static constexpr int kPasses = 4;
  static constexpr bool kAdaptive = false;
  static constexpr int kErrPow = 5;
  static constexpr bool kFinalMoments = true;
  static constexpr int kEvalsPerStep = 4;
  static constexpr bool kEM2 = false;
  __host__ __device__ static constexpr double a(int i, int j) {
    return (i == 2 && j == 1) ? 0.5 : (i == 3 && j == 2) ? 0.5 : (i == 4 && j == 3) ? 1.0 : 0.0;
  }
  __host__ __device__ static constexpr double c(int i) {
    return i == 1 ? 0.0 : (i == 4 ? 1.0 : 0.5);
  }
  __host__ __device__ static constexpr double b(int i) {
    return (i == 1 || i == 4) ? 1.0 / 6.0 : 1.0 / 3.0;
  }
  __host__ __device__ static constexpr double e(int) { return 0.0; }
};

// Dormand & Prince (1980) 5(4) pair; b = row 7 of A (first same as last), e = b - bhat.
struct TabDP45 {
  static constexpr bool kRichardson = false;
  static constexpr int S = 7;
  static constexpr int kPasses = 7;
  static constexpr bool kAdaptive = true;
  static constexpr int kErrPow = 5;
  static constexpr bool kFinalMoments = false;   // first same as last: stage 7 is the new state
  static constexpr int kEvalsPerStep = 6;
  static constexpr bool kEM2 = false;
  __host__ __device__ static constexpr double a(int i, int j) {
    return i == 2 ? (j == 1 ? 1.0 / 5 : 0.0)
         : i == 3 ? (j == 1 ? 3.0 / 40 : j == 2 ? 9.0 / 40 : 0.0)
         : i == 4 ? (j == 1 ? 44.0 / 45 : j == 2 ? -56.0 / 15 : j == 3 ? 32.0 / 9 : 0.0)
         : i == 5 ? (j == 1 ? 19372.0 / 6561 : j == 2 ? -25360.0 / 2187 : j == 3 ? 64448.0 / 6561
                                             : j == 4 ? -212.0 / 729 : 0.0)
         : i == 6 ? (j == 1 ? 9017.0 / 3168 : j == 2 ? -355.0 / 33 : j == 3 ? 46732.0 / 5247
                     : j == 4 ? 49.0 / 176 : j == 5 ? -5103.0 / 18656 : 0.0)
         : i == 7 ? b(j) : 0.0;
  }
  __host__ __device__ static constexpr double c(int i) {
    return i == 1 ? 0.0 : i == 2 ? 0.2 : i == 3 ? 0.3 : i == 4 ? 0.8 : i == 5 ? 8.0 / 9 : 1.0;
  }
  __host__ __device__ static constexpr double b(int j) {
    return j == 1 ? 35.0 / 384 : j == 3 ? 500.0 / 1113 : j == 4 ? 125.0 / 192
         : j == 5 ? -2187.0 / 6784 : j == 6 ? 11.0 / 84 : 0.0;
  }
  // b - bhat, bhat = (5179/57600, 0, 7571/16695, 393/640, -92097/339200, 187/2100, 1/40)
  __host__ __device__ static constexpr double e(int j) {
    return j == 1 ? 71.0 / 57600 : j == 3 ? -71.0 / 16695 : j == 4 ? 71.0 / 1920
         : j == 5 ? -17253.0 / 339200 : j == 6 ? 22.0 / 525 : j == 7 ? -1.0 / 40 : 0.0;
  }
};

// Commutator-free Lie RK4 (Celledoni, Marthinsen & Owren 2003): stage radii as classical RK4.
struct TabCF4 {
  static constexpr bool kRichardson = false;
  static constexpr int S = 4;
  static constexpr int kPasses = 4;
  static constexpr bool kAdaptive = false;
  static constexpr int kErrPow = 5;
  static constexpr bool kFinalMoments = true;
  static constexpr int kEvalsPerStep = 4;
  static constexpr bool kEM2 = false;
  __host__ __device__ static constexpr double a(int, int) { return 0.0; }
  __host__ __device__ static constexpr double b(int) { return 0.0; }
  __host__ __device__ static constexpr double e(int) { return 0.0; }
  __host__ __device__ static constexpr double c(int i) { return TabRK4::c(i); }
};

// Exponential midpoint rule (Lie-group Runge-Kutta-Munthe-Kaas method with Runge's midpoint
// tableau) with its exponential-Euler partner as the embedded first-order estimate: stage 1 at r
// (generator K1), stage 2 at r + h/2 from the half step Y_half = exp(h/2 K1) y, the new state
// exp(h K2) y, the estimate exp(h K1) y; stage 3 is the new state at r + h (the next step's stage 1).
struct TabEM2 {
  static constexpr bool kRichardson = false;
  static constexpr int S = 3;
  static constexpr int kPasses = 2;
  static constexpr bool kAdaptive = true;
  static constexpr int kErrPow = 2;
  static constexpr bool kFinalMoments = true;
  static constexpr int kEvalsPerStep = 2;
  static constexpr bool kEM2 = true;
  __host__ __device__ static constexpr double a(int, int) { return 0.0; }
  __host__ __device__ static constexpr double b(int) { return 0.0; }
  __host__ __device__ static constexpr double e(int) { return 0.0; }
  __host__ __device__ static constexpr double c(int i) { return i == 1 ? 0.0 : (i == 2 ? 0.5 : 1.0); }
};

// Commutator-free Lie RK4 (as TabCF4) with Richardson step-size control: every attempt takes the
// full step of size h and two half steps from the same state, keeps the two half steps and
// estimates their local error as (y_two - y_full) / (2^4 - 1) (error norm, acceptance and
// controller as DP45, exponent 1/5).  Stage slots and radii r + c h:
//   1 (c = 0): y;  full step: 2 (1/2), 3 (1/2), 4 (1);  first half step: 5 (1/4), 6 (1/4), 7 (1/2);
//   8 (1/2): the first half step's result y_a;  second half step from y_a: 9 (3/4), 10 (3/4), 11 (1).
// Pass p reduces slot p + 2; the final pass forms y_b (two half steps) and y_full, the error, and
// the moments of y_b at r + h (the next step's slot 1).
struct TabCFR {
  static constexpr bool kRichardson = true;
  static constexpr int S = 11;
  static constexpr int kPasses = 11;
  static constexpr bool kAdaptive = true;
  static constexpr int kErrPow = 5;
  static constexpr bool kFinalMoments = true;
  static constexpr int kEvalsPerStep = 11;
  static constexpr bool kEM2 = false;
  __host__ __device__ static constexpr double a(int, int) { return 0.0; }
  __host__ __device__ static constexpr double b(int) { return 0.0; }
  __host__ __device__ static constexpr double e(int) { return 0.0; }
  __host__ __device__ static constexpr double c(int i) {
    return i == 1 ? 0.0 : (i == 2 || i == 3 || i == 7 || i == 8) ? 0.5 : (i == 5 || i == 6) ? 0.25
         : (i == 9 || i == 10) ? 0.75 : 1.0;
  }
};

// Largest finite value of the working precision.
template <typename Real>
__host__ __device__ constexpr Real rbig() { return sizeof(Real) == 4 ? Real(3.0e38) : Real(1.7e308); }

// Geometry of one (stage radius, angle bin): cos, 1/cos, 1 - cos, 1/cos - 1 without cancellation.
// The kernels use q (path-length factor 1/cos of Eq. eom), t1 (the weight of the moment D) and t2
// (the factor of mu J1 in the nu-nu term): K = q [eta omega B + lambda z + mu (D + t2 J1)].
//   bulb: q = 1/cos th, t1 = 1/cos th - 1, t2 = 1 - cos th (Eq. Hnu with the measure in u-bins);
//   single angle: every beam radial (q = 1, D = 0) and t2 = (1 - sqrt(1 - x))^2 / x, the
//     geometric factor of Eq. Hnu integrated over emission uniform in u (x = R^2 / r^2);
//   homogeneous test geometry: q = 1, D = 0, t2 = 1 (H_nunu = mu0 J1, mu0 constant).
struct Geo { double q, t1, t2; };
__device__ __forceinline__ Geo geometry(double u, double x, int geom = kGeomBulb) {
  if (geom == kGeomSingleAngle) {
    const double s = 1.0 + sqrt(1.0 - x);       // (1 - sqrt(1 - x))^2 / x = x / (1 + sqrt(1 - x))^2
    return {1.0, 0.0, x / (s * s)};
  }
  if (geom == kGeomHomogeneous) return {1.0, 0.0, 1.0};
  const double c = sqrt(fma(-u, x, 1.0));
  const double t2 = u * x / (1.0 + c);          // 1 - cos
  const double q = 1.0 / c;                     // 1 / cos
  return {q, t2 * q, t2};                       // t1 = 1/cos - 1 = (1 - cos)/cos
}
__device__ __forceinline__ void geometry_f(double u, double x, float& q, float& t1, float& t2,
                                           int geom = kGeomBulb) {
  if (geom != kGeomBulb) {
    const Geo g = geometry(u, x, geom);
    q = (float)g.q;
    t1 = (float)g.t1;
    t2 = (float)g.t2;
    return;
  }
  const float om = (float)fma(-u, x, 1.0);      // 1 - u x in double (no cancellation), then FP32
  const float ux = (float)(u * x);
  const float c = sqrtf(om);
  q = 1.0f / c;
  t2 = ux / (1.0f + c);
  t1 = t2 * q;
}

// --------------------------------------------------------------------------------------------
// Per-thread moment accumulators.  FP64 kernels add each beam's contribution w s by FMA into a
// double.  Mixed kernels form each contribution w s in FP32 (per-beam algebra) and sum the
// contributions without rounding loss: a component's running sum is the unevaluated pair hi + lo,
// and TwoSum (Knuth, TAOCP vol. 2, 4.2.2) splits hi + c into the rounded sum and its exact
// rounding error, which lo collects (lo's own roundings stay near 2^-48 of the sum, as in a
// double accumulator).  At the end of a pass each thread's pair goes exactly to integers
// (f32_to_fix) and every further sum is an integer addition.  The FP32 weights carry a
// per-instance power-of-two scale (InstConst::acc_unit = 2^-S) so that the integers are in units
// of 2^-S; no FP64 instruction is issued per beam (GB300's FP64 pipe is ~1/68 of its FP32 rate).
__device__ __forceinline__ void two_sum_acc(float& hi, float& lo, float c) {
  const float s = __fadd_rn(hi, c);
  const float bv = __fsub_rn(s, hi);
  const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bv)), __fsub_rn(c, bv));
  hi = s;
  lo = __fadd_rn(lo, err);
}

template <typename Real, int NM> struct MomAcc;
template <int NM> struct MomAcc<double, NM> {
  double v[NM];
  __device__ __forceinline__ void zero() {
#pragma unroll
    for (int i = 0; i < NM; ++i) v[i] = 0.0;
  }
  __device__ __forceinline__ void add(int i, double w, double y) { v[i] = fma(w, y, v[i]); }
};
template <int NM> struct MomAcc<float, NM> {
  float hi[NM], lo[NM];
  __device__ __forceinline__ void zero() {
#pragma unroll
    for (int i = 0; i < NM; ++i) { hi[i] = 0.0f; lo[i] = 0.0f; }
  }
  __device__ __forceinline__ void add(int i, float w, float y) { two_sum_acc(hi[i], lo[i], __fmul_rn(w, y)); }
};

// A float that holds a count of 2^-S units (possibly with a fraction) as the nearest int64 (halves
// away from zero), from its bits on the integer pipe, branch-free (no FP64 instruction).  Sets ovf
// when |v| >= 2^52 or v is not finite: a partial that large voids the scale's guarantee.
__device__ __forceinline__ long long f32_to_fix(float v, int& ovf) {
  const unsigned int b = __float_as_uint(v);
  const unsigned int ef = (b >> 23) & 0xffu;
  ovf |= ef >= 127u + 52u ? 1 : 0;
  const unsigned int m = ef ? ((b & 0x7fffffu) | 0x800000u) : 0u;   // below 2^-126: zero
  const int e = (int)ef - 150;                                       // |v| = m 2^e
  const int rs = min(max(-e, 0), 31);
  const unsigned int mr = rs ? ((m + (1u << (rs - 1))) >> rs) : m;
  const unsigned long long r = (unsigned long long)mr << min(max(e, 0), 63);
  return (b >> 31) ? -(long long)r : (long long)r;
}
constexpr long long kFixLimit = 1ll << 52;               // largest block partial accepted

// --------------------------------------------------------------------------------------------
// Physics policies.  "Real" is the working precision of the per-beam algebra.
//
// Two flavours: the state of a beam is the Bloch vector s of P = (1 + s.sigma)/2 (antineutrinos:
// of conj(Pbar)), and every beam obeys ds/dr = K x s with
//   K = [eta omega_k B + lambda(r) z + mu(r) (D + (1 - cos th) J1)] / cos th,
// eta = +1 / -1 for nu / nubar, B = (sin 2 theta_v, 0, -cos 2 theta_v): this is
// d(rho)/dr = -i [H, rho] / cos(th) of Eq. eom with H = (1/2) h.sigma.
//
// Per (stage, angle bin) table row: t1 = 1/cos - 1, q = 1/cos, q Bx, q Bz, G0x, G0y, G0z with
// G0 = q (lambda z + mu D + (1 - cos) mu J1), so that K = eta omega (q Bx, 0, q Bz) + G0, followed
// (FP32 only) by the negated q Bx, q Bz, G0.  FP64 rows hold the 7 values (KT = 8).  FP32 rows hold
// 12 values each stored twice (KT = 24): a 64-bit load then yields a packed f32x2 operand for the
// two beams a thread processes together (both share the angle bin), see PairRK.
template <typename Real>
struct Phys2 {
  static constexpr bool kF32 = sizeof(Real) == 4;
  static constexpr bool kPairable = kF32;       // FP32 passes run beam pairs (PairRK)
  static constexpr bool kNegated = kF32;        // FP32 rows carry -G0_y (saves a multiply per stage)
  static constexpr int NC = 3, NM = kNM2, NSC = kNSC2, KT = kF32 ? 24 : 8;
  enum : int { vT1 = 0, vQ = 1, vQBX = 2, vQBZ = 3, vG0X = 4, vG0Y = 5, vG0Z = 6,
               vNQBX = 7, vNQBZ = 8, vNG0X = 9, vNG0Y = 10, vNG0Z = 11 };
  struct Consts { double B[3]; int geom; };
  struct Beam { Real eo; Real w; };   // eta * omega_k, signed weight du_j * g_{sigma,k}

  __device__ static inline Real val(const Real* t, int v) { return kF32 ? t[2 * v] : t[v]; }
  __device__ static inline void put(Real* t, int v, Real x) {
    if (kF32) { t[2 * v] = x; t[2 * v + 1] = x; } else { t[v] = x; }
  }
  __device__ static inline Real t1(const Real* t) { return val(t, vT1); }

  // sc: mu D (3), mu J1 (3), lambda
  __device__ static inline void fill(Real* t, const Geo& g, const double* sc, const Consts& C) {
    put(t, vT1, (Real)g.t1);
    put(t, vQ, (Real)g.q);
    put(t, vQBX, (Real)(g.q * C.B[0]));
    put(t, vQBZ, (Real)(g.q * C.B[2]));
    put(t, vG0X, (Real)(g.q * (sc[0] + g.t2 * sc[3])));
    put(t, vG0Y, (Real)(g.q * (sc[1] + g.t2 * sc[4])));
    put(t, vG0Z, (Real)(g.q * (sc[6] + sc[2] + g.t2 * sc[5])));
    if (!kF32) t[7] = 0;
  }
  __device__ static inline void fill_f(Real* t, float q, float t1v, float t2, const float* scf,
                                       const Consts& C) {
    const float qbx = q * (float)C.B[0], qbz = q * (float)C.B[2];
    const float gx = q * (scf[0] + t2 * scf[3]);
    const float gy = q * (scf[1] + t2 * scf[4]);
    const float gz = q * (scf[6] + scf[2] + t2 * scf[5]);
    put(t, vT1, t1v);
    put(t, vQ, q);
    put(t, vQBX, qbx);
    put(t, vQBZ, qbz);
    put(t, vG0X, gx);
    put(t, vG0Y, gy);
    put(t, vG0Z, gz);
    if (kF32) {
      put(t, vNQBX, -qbx);
      put(t, vNQBZ, -qbz);
      put(t, vNG0X, -gx);
      put(t, vNG0Y, -gy);
      put(t, vNG0Z, -gz);
    }
  }
  __device__ static inline void K(const Real* t, const Beam& bm, const Real*, const Real*,
                                  Real (&Kv)[3]) {
    Kv[0] = bm.eo * val(t, vQBX) + val(t, vG0X);
    Kv[1] = val(t, vG0Y);
    Kv[2] = bm.eo * val(t, vQBZ) + val(t, vG0Z);
  }
  __device__ static inline void f(const Real (&Kv)[3], const Real (&y)[3], Real (&k)[3]) {
    k[0] = Kv[1] * y[2] - Kv[2] * y[1];
    k[1] = Kv[2] * y[0] - Kv[0] * y[2];
    k[2] = Kv[0] * y[1] - Kv[1] * y[0];
  }
  // moments D (weight w t1) and J1 (weight w)
  template <class Acc>
  __device__ static inline void accum(Acc& acc, Real w, Real t1, const Real (&y)[3]) {
    const Real wt = w * t1;
#pragma unroll
    for (int i = 0; i < 3; ++i) { acc.add(i, wt, y[i]); acc.add(3 + i, w, y[i]); }
  }
  template <class Acc>
  __device__ static inline void accum_row(Acc& acc, Real w, const Real* row, const Real (&y)[3]) {
    accum(acc, w, t1(row), y);
  }
  // table row of (stage with constants sc / scf and R^2/r^2 = x, angle bin at u)
  __device__ static inline void fill_row(Real* row, double u, double x, const double* sc, const Real* scr,
                                         const Consts& C, int, int) {
    if constexpr (kF32) {
      float q, t1v, t2;
      geometry_f(u, x, q, t1v, t2, C.geom);
      fill_f(row, q, t1v, t2, reinterpret_cast<const float*>(scr), C);
    } else {
      fill(row, geometry(u, x, C.geom), sc, C);
    }
  }
  // Frobenius norm^2 of the traceless part of P = (1 + s.sigma)/2: |s|^2 / 2
  __device__ static inline Real tnorm2(const Real (&y)[3]) {
    return Real(0.5) * (y[0] * y[0] + y[1] * y[1] + y[2] * y[2]);
  }
  // Frobenius norm of the traceless matrix (e.sigma)/2, scaled so it cannot overflow; +inf if not finite
  __device__ static inline Real enorm(const Real (&e)[3]) {
    const Real m = fmax(fabs(e[0]), fmax(fabs(e[1]), fabs(e[2])));
    if (!(m <= rbig<Real>())) return Real(INFINITY);
    if (m == Real(0)) return Real(0);
    const Real inv = Real(1) / m;
    const Real a = e[0] * inv, b = e[1] * inv, c = e[2] * inv;
    return m * sqrt(Real(0.5) * (a * a + b * b + c * c));
  }
  __device__ static inline void normalise(Real (&y)[3]) {
    const Real n2 = y[0] * y[0] + y[1] * y[1] + y[2] * y[2];
    const Real inv = Real(1) / sqrt(n2);
#pragma unroll
    for (int i = 0; i < 3; ++i) y[i] *= inv;
  }
  // the pure-state projection of the exponential steps: for a Bloch vector, its unit length
  __device__ static inline void purify(Real (&y)[3]) { normalise(y); }
};

// Three flavours: the state is the full 3x3 Hermitian density matrix (9 reals: P00, P11, P22,
// Re P01, Im P01, Re P02, Im P02, Re P12, Im P12) of P (nu) or conj(Pbar) (nubar); the derivative
// is -i [K, P] with the Hermitian
//   K = [eta (omega21 M21 + omega31 M31) + lambda E_ee + mu (D + (1 - cos) J1)] / cos,
// M21/M31 the real unit vacuum matrices U diag(0,1,0) U^T and U diag(0,0,1) U^T.
// Table row (KT = 4): q, t1, t2, pad; the stage constants mu D, mu J1, lambda stay per stage.
template <typename Real>
struct Phys3 {
  static constexpr bool kPairable = false;
  static constexpr int NC = 9, NM = kNM3, NSC = kNSC3, KT = 4;
  struct Consts { double M21[6], M31[6]; int geom; };
  struct Beam { Real o21, o31; Real w; };

  __device__ static inline Real t1(const Real* t) { return t[1]; }
  __device__ static inline void fill(Real* t, const Geo& g, const double*, const Consts&) {
    t[0] = (Real)g.q;
    t[1] = (Real)g.t1;
    t[2] = (Real)g.t2;
    t[3] = 0;
  }
  __device__ static inline void fill_f(Real* t, float q, float t1, float t2, const float*, const Consts&) {
    t[0] = q;
    t[1] = t1;
    t[2] = t2;
    t[3] = 0;
  }
  // vac: the six real entries (00,11,22,01,02,12) of M21, M31 in working precision;
  // sc (working precision): mu D (9), mu J1 (9), lambda
  __device__ static inline void K(const Real* t, const Beam& bm, const Real* vac, const Real* sc,
                                  Real (&Kv)[9]) {
    const Real q = t[0], t2 = t[2];
    Real v[6];
#pragma unroll
    for (int i = 0; i < 6; ++i) v[i] = bm.o21 * vac[i] + bm.o31 * vac[6 + i];
    Kv[0] = q * (v[0] + sc[18] + sc[0] + t2 * sc[9]);
    Kv[1] = q * (v[1] + sc[1] + t2 * sc[10]);
    Kv[2] = q * (v[2] + sc[2] + t2 * sc[11]);
    Kv[3] = q * (v[3] + sc[3] + t2 * sc[12]);
    Kv[4] = q * (sc[4] + t2 * sc[13]);
    Kv[5] = q * (v[4] + sc[5] + t2 * sc[14]);
    Kv[6] = q * (sc[6] + t2 * sc[15]);
    Kv[7] = q * (v[5] + sc[7] + t2 * sc[16]);
    Kv[8] = q * (sc[8] + t2 * sc[17]);
  }
  // Z = -i [K, Y] for Hermitian K, Y; A = K Y, Z_aa = 2 Im A_aa, Z_ab = -i (A_ab - conj(A_ba)).
  __device__ static inline void f(const Real (&Kv)[9], const Real (&y)[9], Real (&z)[9]) {
    const Real kr[3][3] = {{Kv[0], Kv[3], Kv[5]}, {Kv[3], Kv[1], Kv[7]}, {Kv[5], Kv[7], Kv[2]}};
    const Real ki[3][3] = {{0, Kv[4], Kv[6]}, {-Kv[4], 0, Kv[8]}, {-Kv[6], -Kv[8], 0}};
    const Real yr[3][3] = {{y[0], y[3], y[5]}, {y[3], y[1], y[7]}, {y[5], y[7], y[2]}};
    const Real yi[3][3] = {{0, y[4], y[6]}, {-y[4], 0, y[8]}, {-y[6], -y[8], 0}};
    Real ar[3][3], ai[3][3];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        Real sr = 0, si = 0;
#pragma unroll
        for (int cc = 0; cc < 3; ++cc) {
          sr += kr[a][cc] * yr[cc][b] - ki[a][cc] * yi[cc][b];
          si += kr[a][cc] * yi[cc][b] + ki[a][cc] * yr[cc][b];
        }
        ar[a][b] = sr;
        ai[a][b] = si;
      }
    z[0] = 2 * ai[0][0];
    z[1] = 2 * ai[1][1];
    z[2] = 2 * ai[2][2];
    z[3] = ai[0][1] + ai[1][0];
    z[4] = ar[1][0] - ar[0][1];
    z[5] = ai[0][2] + ai[2][0];
    z[6] = ar[2][0] - ar[0][2];
    z[7] = ai[1][2] + ai[2][1];
    z[8] = ar[2][1] - ar[1][2];
  }
  template <class Acc>
  __device__ static inline void accum(Acc& acc, Real w, Real t1, const Real (&y)[9]) {
    const Real wt = w * t1;
#pragma unroll
    for (int i = 0; i < 9; ++i) { acc.add(i, wt, y[i]); acc.add(9 + i, w, y[i]); }
  }
  // ||P - tr(P)/3||_F^2 with off-diagonal entries counted twice
  __device__ static inline Real tnorm2(const Real (&y)[9]) {
    const Real t = (y[0] + y[1] + y[2]) * Real(1.0 / 3.0);
    const Real d0 = y[0] - t, d1 = y[1] - t, d2 = y[2] - t;
    return d0 * d0 + d1 * d1 + d2 * d2 +
           2 * (y[3] * y[3] + y[4] * y[4] + y[5] * y[5] + y[6] * y[6] + y[7] * y[7] + y[8] * y[8]);
  }
  // full Frobenius norm of the Hermitian matrix, scaled against overflow; +inf if not finite
  __device__ static inline Real enorm(const Real (&e)[9]) {
    Real m = 0;
#pragma unroll
    for (int i = 0; i < 9; ++i) m = fmax(m, fabs(e[i]));
    if (!(m <= rbig<Real>())) return Real(INFINITY);
    if (m == Real(0)) return Real(0);
    const Real inv = Real(1) / m;
    Real d = 0, o = 0;
#pragma unroll
    for (int i = 0; i < 3; ++i) d += (e[i] * inv) * (e[i] * inv);
#pragma unroll
    for (int i = 3; i < 9; ++i) o += (e[i] * inv) * (e[i] * inv);
    return m * sqrt(d + 2 * o);
  }
  __device__ static inline void normalise(Real (&)[9]) {}
  // Mixed-precision exponential steps: restore the idempotency of the (pure) density matrix that
  // the FP32 rounding of the propagators erodes step by step, P <- 3 P^2 - 2 P^3 (McWeeny
  // purification: an eigenvalue 1 - e goes to 1 - 3 e^2 + 2 e^3, a small one d to 3 d^2 - 2 d^3),
  // as the two-flavour path renormalises its Bloch vector.
  __device__ static inline void purify(Real (&y)[9]) {
    const Real pr[3][3] = {{y[0], y[3], y[5]}, {y[3], y[1], y[7]}, {y[5], y[7], y[2]}};
    const Real pi[3][3] = {{0, y[4], y[6]}, {-y[4], 0, y[8]}, {-y[6], -y[8], 0}};
    Real qr[3][3], qi[3][3];                          // P^2
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        Real sr = 0, si = 0;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          sr += pr[a][c] * pr[c][b] - pi[a][c] * pi[c][b];
          si += pr[a][c] * pi[c][b] + pi[a][c] * pr[c][b];
        }
        qr[a][b] = sr;
        qi[a][b] = si;
      }
    Real outr[3][3], outi[3][3];                      // 3 P^2 - 2 P^3, upper triangle
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = a; b < 3; ++b) {
        Real sr = 0, si = 0;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          sr += qr[a][c] * pr[c][b] - qi[a][c] * pi[c][b];
          si += qr[a][c] * pi[c][b] + qi[a][c] * pr[c][b];
        }
        outr[a][b] = Real(3) * qr[a][b] - Real(2) * sr;
        outi[a][b] = Real(3) * qi[a][b] - Real(2) * si;
      }
    y[0] = outr[0][0];
    y[1] = outr[1][1];
    y[2] = outr[2][2];
    y[3] = outr[0][1];
    y[4] = outi[0][1];
    y[5] = outr[0][2];
    y[6] = outi[0][2];
    y[7] = outr[1][2];
    y[8] = outi[1][2];
  }
  template <class Acc>
  __device__ static inline void accum_row(Acc& acc, Real w, const Real* row, const Real (&y)[NC]) {
    accum(acc, w, t1(row), y);
  }
  __device__ static inline void fill_row(Real* row, double u, double x, const double* sc, const Real* scr,
                                         const Consts& C, int, int) {
    if constexpr (sizeof(Real) == 4) {
      float q, t1v, t2;
      geometry_f(u, x, q, t1v, t2, C.geom);
      fill_f(row, q, t1v, t2, reinterpret_cast<const float*>(scr), C);
    } else {
      fill(row, geometry(u, x, C.geom), sc, C);
    }
  }
};
// Two flavours, extended bulb model (Sec. 2, Eq. int-v and Eq. F): beams also carry an azimuthal
// angle phi around the radial direction, the combined angle bin a = j n_phi + p holding u_j,
// du_j / n_phi and phi_p = 2 pi (p + 1/2) / n_phi.  Besides D and J1 the potential needs
//   Jc = sum_b w_b (sin th_b / cos th_b) cos phi_b s_b,   Js = the same with sin phi_b,
// and K = [eta omega B + lambda z + mu (D + (1 - cos th) J1 - sin th (cos phi Jc + sin phi Js))] / cos th.
// Table row: t1, q, q Bx, q Bz, G0 (3), (sin th / cos th) cos phi, (sin th / cos th) sin phi (FP64:
// KT = 10; FP32: each value twice, KT = 18, so FP32 passes run beam pairs as for the bulb model).
template <typename Real>
struct Phys2E {
  static constexpr bool kF32 = sizeof(Real) == 4;
  static constexpr bool kPairable = kF32;       // FP32 passes run beam pairs (PairRK)
  static constexpr bool kNegated = false;       // no negated copies: rows stay small (many rows)
  static constexpr int NC = 3, NM = 12, NSC = 14, KT = kF32 ? 18 : 10;
  // t1, q, q Bx, q Bz, G0 (3), then the azimuthal moment weights (sin th / cos th) cos phi and
  // (sin th / cos th) sin phi; FP32 rows store each value twice (one 64-bit load per packed operand)
  enum : int { vT1 = 0, vQ = 1, vQBX = 2, vQBZ = 3, vG0X = 4, vG0Y = 5, vG0Z = 6, vSCC = 7, vSCS = 8 };
  struct Consts { double B[3]; int n_phi; };
  using Beam = typename Phys2<Real>::Beam;

  __device__ static inline Real val(const Real* t, int v) { return kF32 ? t[2 * v] : t[v]; }
  __device__ static inline void put(Real* t, int v, Real x) {
    if (kF32) { t[2 * v] = x; t[2 * v + 1] = x; } else { t[v] = x; }
  }
  __device__ static inline Real t1(const Real* t) { return val(t, vT1); }
  // sc: mu D (3), mu J1 (3), mu Jc (3), mu Js (3), lambda
  __device__ static inline void fill_row(Real* t, double u, double x, const double* sc, const Real* scr,
                                         const Consts& C, int a, int) {
    const int pidx = a % C.n_phi;
    Real q, t1v, t2, so, sp, cp;
    if constexpr (kF32) {
      // FP32 rows in FP32 arithmetic (as Phys2's): the table holds floats anyway, and FP64 square
      // roots, divisions and sincospi per row would cost more than the row's beams on GB300
      geometry_f(u, x, q, t1v, t2);
      so = sqrtf((float)(u * x)) * q;                         // sin th / cos th, sin^2 th = u R^2 / r^2
      sincospif((2.0f * pidx + 1.0f) / C.n_phi, &sp, &cp);   // phi_p = 2 pi (p + 1/2) / n_phi
    } else {
      const Geo g = geometry(u, x);
      q = g.q;
      t1v = g.t1;
      t2 = g.t2;
      so = sqrt(u * x) * g.q;
      sincospi((2.0 * pidx + 1.0) / C.n_phi, &sp, &cp);
    }
    Real G0[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      if constexpr (kF32) {
        const float ext = cp * scr[6 + i] + sp * scr[9 + i];
        G0[i] = q * ((i == 2 ? scr[12] : 0.0f) + scr[i] + t2 * scr[3 + i]) - so * ext;
      } else {
        const double ext = cp * sc[6 + i] + sp * sc[9 + i];
        G0[i] = q * ((i == 2 ? sc[12] : 0.0) + sc[i] + t2 * sc[3 + i]) - so * ext;
      }
    }
    const Real qbx = q * (Real)C.B[0], qbz = q * (Real)C.B[2];
    put(t, vT1, t1v);
    put(t, vQ, q);
    put(t, vQBX, qbx);
    put(t, vQBZ, qbz);
    put(t, vG0X, G0[0]);
    put(t, vG0Y, G0[1]);
    put(t, vG0Z, G0[2]);
    put(t, vSCC, so * cp);
    put(t, vSCS, so * sp);
    if constexpr (!kF32) t[9] = 0;
  }
  __device__ static inline void K(const Real* t, const Beam& bm, const Real*, const Real*, Real (&Kv)[3]) {
    Kv[0] = bm.eo * val(t, vQBX) + val(t, vG0X);
    Kv[1] = val(t, vG0Y);
    Kv[2] = bm.eo * val(t, vQBZ) + val(t, vG0Z);
  }
  __device__ static inline void f(const Real (&Kv)[3], const Real (&y)[3], Real (&k)[3]) {
    Phys2<Real>::f(Kv, y, k);
  }
  template <class Acc>
  __device__ static inline void accum_row(Acc& acc, Real w, const Real* t, const Real (&y)[3]) {
    const Real wt = w * val(t, vT1), wc = w * val(t, vSCC), ws = w * val(t, vSCS);
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      acc.add(i, wt, y[i]);
      acc.add(3 + i, w, y[i]);
      acc.add(6 + i, wc, y[i]);
      acc.add(9 + i, ws, y[i]);
    }
  }
  __device__ static inline Real tnorm2(const Real (&y)[3]) { return Phys2<Real>::tnorm2(y); }
  __device__ static inline Real enorm(const Real (&e)[3]) { return Phys2<Real>::enorm(e); }
  __device__ static inline void normalise(Real (&y)[3]) { Phys2<Real>::normalise(y); }
  __device__ static inline void purify(Real (&y)[3]) { Phys2<Real>::normalise(y); }
};


// --------------------------------------------------------------------------------------------
struct KParams {
  int n_inst;
  int n_pieces;
  const InstConst* ic;
  InstDyn* dyn;
  const Piece* pieces;
  const int* blk_piece;          // [gridDim.x + 1]
  unsigned long long* acc;       // [n_inst][kMaxStages][kNMMax][2] fixed-point accumulators
  unsigned long long* errmax;    // [n_inst] error norm maxima (bit patterns of non-negative doubles)
  int* nonfinite;                // [n_inst]
  void* planeA;
  void* planeB;
  void* escr;                    // adaptive tableaus: error partial and scale planes [NC + 1][plane_stride]
  void* kst;                     // FP64 RK4 / DP45: stage derivatives k_1..k_n, then one stage state [n + 1][NC][plane_stride]
  uint64_t plane_stride;         // elements between component planes
  const void* etab;              // energy tables, Real, per instance at e_off: [n_tab][n_energy]
  const double* u_tab;           // angle positions u_j, at a_off
  const double* du_tab;          // angle weights du_j, at a_off
  Barrier* bar;
  unsigned long long timeout_ns;
  int* status;                   // global sticky status
  int* all_done;
  int n_steps;
  int init_only;
  // beam-shard mode (one problem split over several GPUs, the host exchanging the stage moments):
  // 0 off; kShardPass: only pass `shard_pass` of the current step (-1: the moment pass of the
  // current state), no device-wide barrier, no serial section; kShardSerialInit / Final: only the
  // serial section that follows the moment pass or a step's final pass (one block)
  int shard_mode;
  int shard_pass;
  // dynamic scheduling (handles with several instances): instead of a fixed list of pieces per
  // block, every block takes the next piece of the pass from a device-wide counter until none is
  // left, so blocks whose pieces run slower (small angle rows, more set-ups, memory placement) do
  // not hold the whole grid at the pass's barrier
  int dyn_sched;
  int max_jj;
  int integrator;
  // optional pass trace (NULL: off): per pass and block, %globaltimer at pass start, after the
  // block's beams and reduction, after the barrier released it, and 1 if it was the last block
  unsigned long long* trace;
  int trace_passes;
#ifdef XFLAT_BOUNDS
  Span span[kSpanCount];         // checked build: the allocations behind the pointers above
#endif
};

// Checked build (-DXFLAT_BOUNDS): every state-plane, stage-plane, energy-table and angle-table
// access of the pass body, the shared-memory row index of every beam and the piece list are tested
// before use.  An access outside its allocation (or off the alignment of its vector type) is
// skipped, a load yielding zeros; the first one is recorded in the barrier's bounds words and the
// launch status becomes XFLAT_ERR_CUDA.  Without the macro every check is the constant true.
#ifdef XFLAT_BOUNDS
static __device__ __noinline__ void bounds_fault(const KParams& p, int site, long long off) {
  if (atomicCAS(&p.bar->bounds_site, 0, site) == 0)
    atomicExch(reinterpret_cast<unsigned long long*>(&p.bar->bounds_off), (unsigned long long)off);
  atomicCAS(p.status, 0, 3 /* XFLAT_ERR_CUDA */);
}
__device__ __forceinline__ bool span_ok(const KParams& p, int id, const void* ptr, unsigned bytes, int site,
                                        unsigned align = 0) {
  const Span sp = p.span[id];
  const char* c = static_cast<const char*>(ptr);
  const bool ok = sp.lo != nullptr && c >= sp.lo && c + bytes <= sp.lo + sp.bytes &&
                  (reinterpret_cast<uintptr_t>(c) % (align ? align : bytes)) == 0;
  if (!ok) bounds_fault(p, site, sp.lo ? (long long)(c - sp.lo) : -1ll);
  return ok;
}
__device__ __forceinline__ bool index_ok(const KParams& p, bool ok, int site, long long v) {
  if (!ok) bounds_fault(p, site, v);
  return ok;
}
#define XFLAT_SPAN_OK(p, id, ptr, bytes, site) ::xflat::span_ok((p), (id), (ptr), (bytes), (site))
#define XFLAT_SPAN_OK_AL(p, id, ptr, bytes, align, site) ::xflat::span_ok((p), (id), (ptr), (bytes), (site), (align))
#define XFLAT_INDEX_OK(p, cond, site, v) ::xflat::index_ok((p), (cond), (site), (long long)(v))
#else
#define XFLAT_SPAN_OK(p, id, ptr, bytes, site) true
#define XFLAT_SPAN_OK_AL(p, id, ptr, bytes, align, site) true
#define XFLAT_INDEX_OK(p, cond, site, v) true
#endif

// Add x (|x| < 2^63) to a 128-bit fixed-point accumulator (acc2[0]: fraction in units of 2^-64,
// acc2[1]: signed integer part), truncating |x| below 2^-64.  The split is done on |x|, where
// |x| - floor(|x|) is exact, and the pair is negated as a 128-bit integer for x < 0 (x - floor(x)
// itself would round for small negative x).
__device__ __forceinline__ void fx_add(unsigned long long* acc2, double x) {
  const double ax = fabs(x);
  const double hi_d = floor(ax);
  const unsigned long long lo_a = (unsigned long long)((ax - hi_d) * 18446744073709551616.0);
  const long long hi_a = (long long)hi_d;
  const bool neg = x < 0.0;
  const unsigned long long lo = neg ? 0ull - lo_a : lo_a;
  const long long hi = neg ? -hi_a - (lo_a != 0ull ? 1ll : 0ll) : hi_a;
  const unsigned long long old = atomicAdd(&acc2[0], lo);
  const unsigned long long carry = (old + lo < old) ? 1ull : 0ull;
  atomicAdd(&acc2[1], (unsigned long long)hi + carry);
}

__device__ __forceinline__ double fx_read(const unsigned long long* acc2) {
  const long long hi = (long long)acc2[1];
  return (double)hi + (double)acc2[0] * 5.421010862427522e-20;   // 2^-64 (words already loaded)
}

template <class Tab>
__device__ __forceinline__ double stage_c(int i) { return Tab::c(i); }

// ------------------------------------------------------------------------------------------
// The last block to arrive: reduce accumulators, derive stage constants, run the controller.
// Every value another block may have written since this SM last looked is read through L2
// (__ldcg), never from a possibly stale L1 line; the loads are issued before any branch on them.
// 0.9 Err^(-1/P), the unclamped step-size factor, in double (P = 5 for the 5(4) pair, 2 for the
// 2(1) pair).  The caller clamps it to [0.2, 5], which decides alone below Err = (0.9/5)^P and
// above (0.9/0.2)^P, so only (a slightly wider) range is computed: a float seed refined by two
// Newton steps for y^-P = Err, y <- y ((P + 1) - Err y^P) / P, which need no division (one FP64
// pow costs ~5800 cycles of latency on this part, the two steps ~800) and converge to double
// accuracy.
template <int P>
__device__ __forceinline__ double controller_factor(double err) {
  constexpr double lo = P == 5 ? 1.5e-4 : 0.025, hi = P == 5 ? 2000.0 : 25.0;
  if (!(err > lo)) return 5.0;
  if (!(err < hi)) return 0.0;
  double y = (double)powf((float)err, -1.0f / (float)P);
  for (int it = 0; it < 2; ++it) {
    double yp = y;
#pragma unroll
    for (int q = 1; q < P; ++q) yp *= y;
    y = y * fma(err * (-1.0 / P), yp, (P + 1.0) / P);
  }
  return 0.9 * y;
}

// mu(r) and lambda(r) at one radius (double).
// mu(r) and lambda(r) from 1/r
// lambda(r) from a matter table: the interval [r_i, r_{i+1}) holding r by binary search, then
// lambda_i (r / r_i)^p_i (the end values outside the table)
__device__ inline double table_strength(const double* t, int n, double r) {
  if (r <= t[0]) return t[1];
  if (r >= t[3 * (n - 1)]) return t[3 * (n - 1) + 1];
  int lo = 0, hi = n - 1;                       // t[3 lo] <= r < t[3 hi]
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (t[3 * mid] <= r) lo = mid; else hi = mid;
  }
  return t[3 * lo + 1] * pow(r / t[3 * lo], t[3 * lo + 2]);
}
__device__ __forceinline__ void strengths_inv(const InstConst& ic, double inv, double& mu, double& lam) {
  mu = ic.geom == kGeomHomogeneous ? ic.mu_const : ic.mu_coef * inv * inv;
  lam = 0.0;
  if (ic.matter == kMatterPower) {
    const double x = ic.r_ref * inv;
    lam = ic.lam_coef * (ic.power == 3.0 ? x * x * x : pow(x, ic.power));
  } else if (ic.matter == kMatterConst) {
    lam = ic.lam_const;
  } else if (ic.matter == kMatterTable) {
    lam = table_strength(ic.mtab, ic.mt_n, 1.0 / inv);
  }
}
__device__ __forceinline__ void strengths(const InstConst& ic, double r, double& mu, double& lam) {
  strengths_inv(ic, 1.0 / r, mu, lam);
}

// Loads that must not hit a stale L1 line: instance dynamics change across barriers.
__device__ __forceinline__ double ldcg(const double* p) { return __ldcg(p); }
__device__ __forceinline__ int ldcg(const int* p) { return __ldcg(p); }

// Component c of a stage's moments: the kAccCopies fixed-point copies summed as integers (exact,
// so every block that reads them gets the same bits), then converted to double.
template <typename Real>
__device__ __forceinline__ double acc_component(const unsigned long long* acc_slot, int c, double unit) {
  if constexpr (sizeof(Real) == 4) {
    long long sum = 0;
#pragma unroll
    for (int cp = 0; cp < kAccCopies; ++cp) sum += (long long)__ldcg(acc_slot + ((size_t)cp * kNMMax + c) * 2);
    return (double)sum * unit;                                   // 2^-S of the instance
  } else {
    unsigned __int128 sum = 0;
#pragma unroll
    for (int cp = 0; cp < kAccCopies; ++cp) {
      const unsigned long long* w = acc_slot + ((size_t)cp * kNMMax + c) * 2;
      sum += ((unsigned __int128)__ldcg(w + 1) << 64) | (unsigned __int128)__ldcg(w);
    }
    return (double)(long long)(unsigned long long)(sum >> 64) +
           (double)(unsigned long long)sum * 5.421010862427522e-20;    // 2^-64
  }
}

// Hand-off of each instance's new r and h (and whether its next step needs stage geometry) from
// serial_update to serial_geometry inside the last block, through shared memory (instances past
// kGeoShared are read back from global memory).
constexpr int kGeoShared = 64;
struct GeoHandoff {
  double r[kGeoShared], h[kGeoShared];
  int pending[kGeoShared];
};
__device__ __forceinline__ GeoHandoff& geo_handoff() {
  __shared__ GeoHandoff g;
  return g;
}

template <class Phys, class Tab, typename Real>
__device__ int serial_update(const KParams& p, int slot, bool final_pass, bool init) {
  constexpr int NM = Phys::NM;
  constexpr int NCOMP = NM / 2;
  int all_finished = 1;                            // over this thread's instances
  for (int i = threadIdx.x; i < p.n_inst; i += blockDim.x) {
    const InstConst& ic = p.ic[i];
    InstDyn& d = p.dyn[i];
    const unsigned long long* acc = p.acc + (size_t)i * kAccWordsPerInst + (size_t)slot * kAccCopies * kNMMax * 2;
    const bool have_moments = !(final_pass && !Tab::kFinalMoments);
    const bool adaptive_final = final_pass && Tab::kAdaptive && !Tab::kFinalMoments;   // FSAL
    // ---- every load first (no store may sit between them) -------------------------------
    const int done = __ldcg(&d.done), status = __ldcg(&d.status), nonfin = __ldcg(&p.nonfinite[i]);
    const unsigned long long eb = __ldcg(&p.errmax[i]);
    double m[NM];
    if (have_moments) {
#pragma unroll
      for (int c = 0; c < NM; ++c) m[c] = acc_component<Real>(acc, c, ic.acc_unit);
    }
    double m7[NM], sc7[Phys::NSC];
    if (adaptive_final) {
#pragma unroll
      for (int c = 0; c < NM; ++c) m7[c] = __ldcg(&d.mom[Tab::S][c]);
#pragma unroll
      for (int c = 0; c < Phys::NSC; ++c) sc7[c] = __ldcg(&d.sc[Tab::S][c]);
    }
    const int gslot = slot == 0 ? Tab::S : slot;   // slot 0: new state's moments at r + h
    double mu = __ldcg(&d.mus[gslot]), lam = __ldcg(&d.lams[gslot]);
    double r = __ldcg(&d.r), hh = __ldcg(&d.h);
    const double r_end = __ldcg(&d.r_end), r0f = __ldcg(&d.r0_fixed), hf = __ldcg(&d.h_fixed);
    long long nfix = __ldcg(&d.n_fixed);
    const long long nfix_tot = __ldcg(&d.n_fixed_total);
    int last = __ldcg(&d.last), parity = __ldcg(&d.parity);
    unsigned long long accepted = __ldcg(&d.accepted), rejected = __ldcg(&d.rejected);
    unsigned long long evals = __ldcg(&d.stage_evals);
    const double h_min = ic.h_min, h_max = ic.h_max;
    if (done || status) continue;
    if (nonfin) {
      d.status = 5;  // XFLAT_ERR_NONFINITE
      atomicCAS(p.status, 0, 5);
      continue;
    }
    // ---- stage constants of the stage just reduced (the accumulators are cleared elsewhere) --
    if (have_moments) {
      if (init) strengths(ic, __ldcg(&d.rs[slot]), mu, lam);   // the host set only rs[1], xs[1]
      for (int c = 0; c < NM; ++c) d.mom[slot][c] = m[c];
      for (int c = 0; c < NCOMP; ++c) {
        d.sc[slot][c] = mu * m[c];
        d.sc[slot][NCOMP + c] = mu * m[NCOMP + c];
      }
      d.sc[slot][NM] = lam;
    }
    if (!final_pass && !init) {
      all_finished = 0;
      continue;
    }
    // ---- step bookkeeping ---------------------------------------------------------------
    bool fin = false, step_err = false;
    if (init) {
      evals += Tab::kAdaptive ? 1ull : 0ull;
    } else if (!Tab::kAdaptive) {
      parity ^= 1;
      accepted += 1;
      evals += Tab::kEvalsPerStep;
      nfix += 1;
      fin = nfix >= nfix_tot;
      r = fin ? r_end : r0f + (double)nfix * hf;
      // the final pass reduced the new state's moments at r + h (= stage S radius): stage 1 of
      // the next step
      for (int c = 0; c < NM; ++c) d.mom[1][c] = m[c];
      for (int c = 0; c < NCOMP; ++c) {
        d.sc[1][c] = mu * m[c];
        d.sc[1][NCOMP + c] = mu * m[NCOMP + c];
      }
      d.sc[1][NM] = lam;
    } else {
      const double err = __longlong_as_double((long long)eb);
      p.errmax[i] = 0ull;
      d.err = err;
      evals += Tab::kEvalsPerStep;
      const bool ok = err <= 1.0;
      const double q = controller_factor<Tab::kErrPow>(err);
      if (ok) {
        r = last ? r_end : r + hh;
        parity ^= 1;
        accepted += 1;
        if (Tab::kFinalMoments) {
          // the final pass reduced the new state's moments at r + h: stage 1 of the next step
          for (int c = 0; c < NM; ++c) d.mom[1][c] = m[c];
          for (int c = 0; c < NCOMP; ++c) {
            d.sc[1][c] = mu * m[c];
            d.sc[1][NCOMP + c] = mu * m[NCOMP + c];
          }
          d.sc[1][NM] = lam;
        } else {
          for (int c = 0; c < NM; ++c) d.mom[1][c] = m7[c];
          for (int c = 0; c < Phys::NSC; ++c) d.sc[1][c] = sc7[c];
        }
        fin = last != 0;
      } else {
        rejected += 1;
      }
      const double fac = ok ? fmin(5.0, fmax(0.2, q)) : fmax(0.2, q);
      hh = fmin(hh * fac, h_max);
      if (!fin && hh < h_min) {
        d.status = 6;  // XFLAT_ERR_STEP
        atomicCAS(p.status, 0, 6);
        step_err = true;
      }
    }
    // ---- the next step's clipped step size; its stage geometry follows in serial_geometry ----
    if (!fin && Tab::kAdaptive) {
      last = (r + hh >= r_end) ? 1 : 0;
      if (last) hh = r_end - r;
    }
    d.geo_pending = (!fin && !step_err) ? 1 : 0;
    if (i < kGeoShared) {
      GeoHandoff& g = geo_handoff();
      g.r[i] = r;
      g.h[i] = Tab::kAdaptive ? hh : hf;
      g.pending[i] = d.geo_pending;
    }
    d.r = r;
    d.h = hh;
    d.last = last;
    d.parity = parity;
    d.n_fixed = nfix;
    d.accepted = accepted;
    d.rejected = rejected;
    d.stage_evals = evals;
    if (fin) d.done = 1;
    if (!fin && !step_err) all_finished = 0;
  }
  return all_finished;
}

// Accumulator slots of the stages kPasses..S (no pass of their own index clears them), zeroed by
// the last block of the final barrier: nobody accumulates into or reads them until the next step
// (the fence in serial_geometry publishes the stores before the release).
template <class Tab>
__device__ void clear_late_slots(const KParams& p) {
  constexpr int kWords = kAccCopies * kNMMax * 2;
  constexpr int kLate = Tab::S - Tab::kPasses + 1;
  for (int t = threadIdx.x; t < p.n_inst * kLate * kWords; t += blockDim.x) {
    const int inst = t / (kLate * kWords), rem = t % (kLate * kWords);
    const int slot = Tab::kPasses + rem / kWords;
    p.acc[(size_t)inst * kAccWordsPerInst + (size_t)slot * kWords + rem % kWords] = 0ull;
  }
}

// The next step's stage radii, R^2/r^2, mu and lambda, one (instance, stage) per thread of the last
// block: FP64 divisions have a long latency on this part, so they run side by side, not in a chain.
// Takes r, h and the pending flag from serial_update (after a __syncthreads), then fences every
// thread's writes (those of serial_update included) before the barrier is released.
template <class Tab>
__device__ void serial_geometry(const KParams& p) {
  const GeoHandoff& g = geo_handoff();
  for (int t = threadIdx.x; t < p.n_inst * Tab::S; t += blockDim.x) {
    const int i = t / Tab::S, s = t % Tab::S + 1;
    InstDyn& d = p.dyn[i];
    const bool shared = i < kGeoShared;
    if (!(shared ? g.pending[i] : ldcg(&d.geo_pending))) continue;
    const InstConst& ic = p.ic[i];
    const double r = shared ? g.r[i] : ldcg(&d.r);
    const double h = shared ? g.h[i] : (Tab::kAdaptive ? ldcg(&d.h) : ldcg(&d.h_fixed));
    const double rs = (s == 1) ? r : __dadd_rn(r, __dmul_rn(stage_c<Tab>(s), h));
    const double inv = 1.0 / rs;
    double mus, lams;
    strengths_inv(ic, inv, mus, lams);
    d.rs[s] = rs;
    d.xs[s] = ic.R2 * inv * inv;
    d.mus[s] = mus;
    d.lams[s] = lams;
  }
  __threadfence();
}


// ---------------------------------------------------------------------------------------------
// State ring of the FP32 two-flavour bulb passes.  Each thread streams its beams' state through a
// private ring of kStateRingDepth + 1 slots in shared memory, filled by cp.async (LDGSTS)
// kStateRingDepth vectors ahead of the one being processed: several vectors' bytes in flight per
// thread without holding registers for them.  (Measured on GB300 against one register-held
// prefetch vector, against 2 and 5 vectors ahead, and against a per-warp ring of 256-byte bulk
// copies completing on mbarriers, which was slower on every launch shape.)  The slots are
// thread-private, so the only ordering needed is the thread's own cp.async.wait_group.
template <class Phys, typename Real>
__host__ __device__ constexpr bool state_ring() {
  return Phys::NC == 3 && Phys::NM == 6 && sizeof(Real) == 4;
}
__device__ __forceinline__ uint32_t smem_addr(const void* ptr) {
  return (uint32_t)__cvta_generic_to_shared(ptr);
}
__device__ __forceinline__ void cp_async8(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_addr(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
// wait until at most N of this thread's committed groups are pending
template <int N>
__device__ __forceinline__ void cp_async_wait_pending() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Per-thread state vectors: two consecutive beams per load (float2 / double2), so the loaded and
// the prefetched vectors fit the register budget; a warp still reads 256 or 512 contiguous bytes
// per plane.
template <typename Real> struct Vec16;
template <> struct Vec16<float> { using T = float2; static constexpr int N = 2; };
template <> struct Vec16<double> { using T = double2; static constexpr int N = 2; };

template <typename Real>
__device__ __forceinline__ void vload(const Real* p, Real (&v)[Vec16<Real>::N]) {
  const typename Vec16<Real>::T t = __ldcg(reinterpret_cast<const typename Vec16<Real>::T*>(p));
  const Real* a = reinterpret_cast<const Real*>(&t);
#pragma unroll
  for (int i = 0; i < Vec16<Real>::N; ++i) v[i] = a[i];
}
template <typename Real>
__device__ __forceinline__ void vstore(Real* p, const Real (&v)[Vec16<Real>::N]) {
  typename Vec16<Real>::T t;
  Real* a = reinterpret_cast<Real*>(&t);
#pragma unroll
  for (int i = 0; i < Vec16<Real>::N; ++i) a[i] = v[i];
  __stcg(reinterpret_cast<typename Vec16<Real>::T*>(p), t);
}

// Plane accesses of the pass body, checked in the checked build (site: where, for the record).
template <typename Real>
__device__ __forceinline__ void vload_at(const KParams& p, int span, const Real* ptr,
                                         Real (&v)[Vec16<Real>::N], int site) {
  if (XFLAT_SPAN_OK(p, span, ptr, sizeof(typename Vec16<Real>::T), site)) {
    vload(ptr, v);
  } else {
#pragma unroll
    for (int i = 0; i < Vec16<Real>::N; ++i) v[i] = Real(0);
  }
}
template <typename Real>
__device__ __forceinline__ void vstore_at(const KParams& p, int span, Real* ptr,
                                          const Real (&v)[Vec16<Real>::N], int site) {
  if (XFLAT_SPAN_OK(p, span, ptr, sizeof(typename Vec16<Real>::T), site)) vstore(ptr, v);
}

// Rotation of y about Om by |Om| (right-handed): y + a Om x y + b Om x (Om x y), the Bloch form of
// y -> U y U^dagger with U = exp(-i Om.sigma/2), i.e. the propagator of Eq. U.
template <typename Real>
__device__ __forceinline__ void rotate(const Real (&Om)[3], Real (&y)[3]) {
  const Real t2 = Om[0] * Om[0] + Om[1] * Om[1] + Om[2] * Om[2];
  Real a, b;
  const Real eps = sizeof(Real) == 4 ? Real(1e-3) : Real(1e-5);
  if (t2 > eps * eps) {
    const Real t = sqrt(t2);
    Real sh, ch;
    if (sizeof(Real) == 4) sincosf((float)(Real(0.5) * t), (float*)&sh, (float*)&ch);
    else sincos((double)(Real(0.5) * t), (double*)&sh, (double*)&ch);
    a = Real(2) * sh * ch / t;
    b = Real(2) * sh * sh / t2;
  } else {
    a = Real(1) - t2 * Real(1.0 / 6.0);
    b = Real(0.5) - t2 * Real(1.0 / 24.0);
  }
  const Real c0 = Om[1] * y[2] - Om[2] * y[1];
  const Real c1 = Om[2] * y[0] - Om[0] * y[2];
  const Real c2 = Om[0] * y[1] - Om[1] * y[0];
  const Real d0 = Om[1] * c2 - Om[2] * c1;
  const Real d1 = Om[2] * c0 - Om[0] * c2;
  const Real d2 = Om[0] * c1 - Om[1] * c0;
  y[0] += a * c0 + b * d0;
  y[1] += a * c1 + b * d1;
  y[2] += a * c2 + b * d2;
}

// Three flavours: one cyclic-Jacobi rotation of the Hermitian matrix A (real and imaginary parts)
// in the plane (p, q), accumulated into V: a phase makes A_pq real, then the real symmetric 2 x 2
// Schur rotation (Golub and Van Loan, Matrix Computations, Sec. 8.5.2) zeroes it.
template <typename Real>
__device__ __forceinline__ void jacobi3_rotate(Real (&ar)[3][3], Real (&ai)[3][3], Real (&vr)[3][3],
                                               Real (&vi)[3][3], int p, int q) {
  const Real br = ar[p][q], bi = ai[p][q];
  const Real mag = hypot(br, bi);                      // no underflow of the squares: |exp(i phi)| = 1
  // an entry below the rounding of the diagonal is dropped (also keeps converged entries, which
  // fall towards the underflow range sweep after sweep, from ever entering the phase)
  const Real tiny = sizeof(Real) == 8 ? Real(8.673617379884035e-19) : Real(9.313225746154785e-10);   // 2^-60, 2^-30
  if (!(mag > tiny * (fabs(ar[p][p]) + fabs(ar[q][q])))) {
    ar[p][q] = ar[q][p] = ai[p][q] = ai[q][p] = Real(0);
    return;
  }
  const Real er = br / mag, ei = bi / mag;             // exp(i phi) of A_pq
  // A <- D^dagger A D, V <- V D with D = diag(1, exp(-i phi)) in the plane: A_pq becomes |A_pq|
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const Real xr = ar[k][q], xi = ai[k][q];
    ar[k][q] = xr * er + xi * ei;
    ai[k][q] = xi * er - xr * ei;
    const Real wr = vr[k][q], wi = vi[k][q];
    vr[k][q] = wr * er + wi * ei;
    vi[k][q] = wi * er - wr * ei;
  }
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const Real xr = ar[q][k], xi = ai[q][k];
    ar[q][k] = xr * er - xi * ei;
    ai[q][k] = xi * er + xr * ei;
  }
  // real rotation J = [[c, s], [-s, c]] in the plane: A <- J^T A J, V <- V J
  const Real tau = (ar[q][q] - ar[p][p]) / (Real(2) * mag);
  const Real at = fabs(tau);
  const Real big = sizeof(Real) == 8 ? Real(1e150) : Real(1e18);
  const Real t = at > big ? Real(0.5) / tau : copysign(Real(1), tau) / (at + sqrt(Real(1) + tau * tau));
  const Real c = Real(1) / sqrt(Real(1) + t * t), sn = t * c;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    Real x = ar[k][p], y = ar[k][q];
    ar[k][p] = c * x - sn * y;
    ar[k][q] = sn * x + c * y;
    x = ai[k][p];
    y = ai[k][q];
    ai[k][p] = c * x - sn * y;
    ai[k][q] = sn * x + c * y;
    x = vr[k][p];
    y = vr[k][q];
    vr[k][p] = c * x - sn * y;
    vr[k][q] = sn * x + c * y;
    x = vi[k][p];
    y = vi[k][q];
    vi[k][p] = c * x - sn * y;
    vi[k][q] = sn * x + c * y;
  }
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    Real x = ar[p][k], y = ar[q][k];
    ar[p][k] = c * x - sn * y;
    ar[q][k] = sn * x + c * y;
    x = ai[p][k];
    y = ai[q][k];
    ai[p][k] = c * x - sn * y;
    ai[q][k] = sn * x + c * y;
  }
  ar[p][q] = ar[q][p] = ai[p][q] = ai[q][p] = Real(0);
}

// Three flavours: y <- U y U^dagger with U = exp(-i Om) for Hermitian Om (9 reals: the diagonal,
// then real and imaginary parts of the 01, 02 and 12 entries), the propagator of Eq. U for a
// 3 x 3 generator.  Om = V diag(l) V^dagger by cyclic Jacobi sweeps (a 3 x 3 Hermitian matrix
// converges quadratically: to the working precision in four sweeps, five in FP64); in the
// eigenbasis the entry (a, b) of V^dagger y V turns by exp(-i (l_a - l_b)), so U is never formed.
template <typename Real>
__device__ __noinline__ void propagate3(const Real (&Om)[9], Real (&y)[9]) {
  constexpr int kSweeps = sizeof(Real) == 8 ? 5 : 4;
  Real ar[3][3] = {{Om[0], Om[3], Om[5]}, {Om[3], Om[1], Om[7]}, {Om[5], Om[7], Om[2]}};
  Real ai[3][3] = {{0, Om[4], Om[6]}, {-Om[4], 0, Om[8]}, {-Om[6], -Om[8], 0}};
  Real vr[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
  Real vi[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
#pragma unroll 1
  for (int sw = 0; sw < kSweeps; ++sw) {
    jacobi3_rotate(ar, ai, vr, vi, 0, 1);
    jacobi3_rotate(ar, ai, vr, vi, 0, 2);
    jacobi3_rotate(ar, ai, vr, vi, 1, 2);
  }
  const Real yr[3][3] = {{y[0], y[3], y[5]}, {y[3], y[1], y[7]}, {y[5], y[7], y[2]}};
  const Real yi[3][3] = {{0, y[4], y[6]}, {-y[4], 0, y[8]}, {-y[6], -y[8], 0}};
  // T = Y V, W = V^dagger T
  Real tr[3][3], ti[3][3], wr[3][3], wi[3][3];
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      Real sr = 0, si = 0;
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        sr += yr[a][c] * vr[c][b] - yi[a][c] * vi[c][b];
        si += yr[a][c] * vi[c][b] + yi[a][c] * vr[c][b];
      }
      tr[a][b] = sr;
      ti[a][b] = si;
    }
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      Real sr = 0, si = 0;
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        sr += vr[c][a] * tr[c][b] + vi[c][a] * ti[c][b];
        si += vr[c][a] * ti[c][b] - vi[c][a] * tr[c][b];
      }
      wr[a][b] = sr;
      wi[a][b] = si;
    }
  // the phases of the off-diagonal entries in the eigenbasis (W stays Hermitian)
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = a + 1; b < 3; ++b) {
      Real sd, cd;
      if (sizeof(Real) == 4) sincosf((float)(ar[a][a] - ar[b][b]), (float*)&sd, (float*)&cd);
      else sincos((double)(ar[a][a] - ar[b][b]), (double*)&sd, (double*)&cd);
      const Real xr = wr[a][b], xi = wi[a][b];
      wr[a][b] = xr * cd + xi * sd;
      wi[a][b] = xi * cd - xr * sd;
      wr[b][a] = wr[a][b];
      wi[b][a] = -wi[a][b];
    }
  // T = V W, Y = T V^dagger (upper triangle)
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      Real sr = 0, si = 0;
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        sr += vr[a][c] * wr[c][b] - vi[a][c] * wi[c][b];
        si += vr[a][c] * wi[c][b] + vi[a][c] * wr[c][b];
      }
      tr[a][b] = sr;
      ti[a][b] = si;
    }
  Real outr[3][3], outi[3][3];
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = a; b < 3; ++b) {
      Real sr = 0, si = 0;
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        sr += tr[a][c] * vr[b][c] + ti[a][c] * vi[b][c];
        si += ti[a][c] * vr[b][c] - tr[a][c] * vi[b][c];
      }
      outr[a][b] = sr;
      outi[a][b] = si;
    }
  y[0] = outr[0][0];
  y[1] = outr[1][1];
  y[2] = outr[2][2];
  y[3] = outr[0][1];
  y[4] = outi[0][1];
  y[5] = outr[0][2];
  y[6] = outi[0][2];
  y[7] = outr[1][2];
  y[8] = outi[1][2];
}

// The propagator of Eq. U over one step for the generator Om (step length and coefficients folded
// in): y <- exp(-i Om) y exp(i Om).  Two flavours: the rotation of the Bloch vector; three
// flavours: by the eigen-decomposition of Om.
template <typename Real>
__device__ __forceinline__ void propagate(const Real (&Om)[3], Real (&y)[3]) { rotate(Om, y); }
template <typename Real>
__device__ __forceinline__ void propagate(const Real (&Om)[9], Real (&y)[9]) { propagate3(Om, y); }

// Per-block shared state of the piece being processed.
template <typename Real, class Phys>
struct BlockShared {
  double scd[kMaxStages][Phys::NSC];   // stage constants (double)
  double xs[kMaxStages];               // R^2 / r_s^2
  unsigned long long hA2[kMaxStages][kMaxStages];   // packed (h a_ij, h a_ij) for the FP32 pair path
  unsigned long long hB2[kMaxStages];
  unsigned long long hE2[kMaxStages];
  Real scr[kMaxStages][Phys::NSC];     // stage constants in working precision
  Real hA[kMaxStages][kMaxStages];
  Real hB[kMaxStages];
  Real hE[kMaxStages];
  Real vac[12];                        // three flavours: M21, M31 in working precision
  Real rtol, atol;
  double fx[kNMMax];
  int active;
  int parity;
  int flag;
  int pass_idx;                        // passes run by this block in this launch (pass trace)
  int next_piece;                      // dynamic scheduling: the piece this block processes next
  int keep;                            // single-piece block: launch-invariant set-up already loaded
  unsigned int gen_seen;               // barrier generation this block arrived in
};

// Table view: row (stage s, combined angle index tj) holds Phys::KT values.
template <typename Real, class Phys>
struct TabView {
  const Real* t;
  int n_jj;
  __device__ __forceinline__ const Real* row(int s, int tj) const {
    return t + ((size_t)s * n_jj + tj) * Phys::KT;
  }
};

// What a pass does (compile time).
enum PassKind : int { kStagePass = 0, kFinalPass = 1, kInitPass = 2 };

// Adaptive FP64 kernels split the last two passes of a step: the pass forming Y_S (= y5, first
// same as last) also stores y5, the error partial sum over stages 1..S-1 and the error scale, and
// the final pass only adds k_S -- the stage chain costs FP64 instructions on GB300's narrow FP64
// pipe.  FP32 kernels rebuild the chain in the final pass instead: their state, y5 and those
// partials together exceed the L2, and the extra DRAM traffic costs more than the FP32 chain.
template <class Tab, typename Real>
__host__ __device__ constexpr bool split_final() {
  return Tab::kAdaptive && !Tab::kFinalMoments && !Tab::kEM2 && sizeof(Real) == 8;   // DP45 in FP64
}

// FP64 commutator tableaus (RK4, DP45) keep their stage derivatives in HBM: the pass that
// evaluates k_s writes it, later passes of the step read it back instead of rebuilding the chain.
// On GB300 an FP64 stage evaluation costs far more time than moving its 8 bytes per component
// (the FP64 pipe runs at ~1/68 of the FP32 rate), so a DP45 step evaluates 7 stages instead of
// the 28 of the rebuilt chain.  FP32 kernels rebuild: their stage vectors would push the state out
// of the L2.  The stored values are bit-identical to rebuilt ones (same inputs, same arithmetic).
template <class Tab, typename Real>
__host__ __device__ constexpr bool stored_stages() {
  return !Tab::kEM2 && sizeof(Real) == 8;
}
// Stage derivatives a step stores (k_1 .. k_n): every stage whose derivative a later pass needs.
template <class Tab, typename Real>
__host__ __device__ constexpr int stored_stage_count() {
  return split_final<Tab, Real>() ? Tab::S - 2 : Tab::S - 1;
}

template <class Phys, class Tab, typename Real, bool kCF, int kPass, int kKind>
struct PassBody;

// Commutator-form Runge-Kutta (RK4 / DP45) ------------------------------------------------------
template <class Phys, class Tab, typename Real, int kPass, int kKind>
struct PassBody<Phys, Tab, Real, false, kPass, kKind> {
  static constexpr int NC = Phys::NC;
  static constexpr bool kSplit = split_final<Tab, Real>();
  // number of stage derivatives the pass needs before its stage state, rebuilt or (stored stages)
  // read back (split final pass: none, the pass forming Y_S left y5 and the error partial behind;
  // unsplit adaptive: S - 1, k_S follows from the new state)
  static constexpr int kChain =
      kKind == kInitPass ? 0
      : (kKind == kFinalPass ? (kSplit ? 0 : Tab::S - (Tab::kAdaptive ? 1 : 0)) : kPass + 1);
  // stored stage derivatives (stored_stages): all of the chain but its last stage are read back,
  // and a stage pass writes the one it evaluates when a later pass of the step reads it
  static constexpr bool kStore = stored_stages<Tab, Real>();
  static constexpr int kLoadK = (kStore && kChain > 0) ? kChain - 1 : 0;
  static constexpr bool kStoreK = kStore && kKind == kStagePass && kChain <= stored_stage_count<Tab, Real>();
  // the stage state the chain evaluates last, Y_kChain, is the one the previous pass formed for its
  // moments: stored there (plane set after the stage derivatives) and read back here
  static constexpr bool kLoadY = kStore && kChain >= 2;
  static constexpr bool kStoreY = kStore && kKind == kStagePass && !(kSplit && kPass + 2 == Tab::S);
  static constexpr int kYPlanes = stored_stage_count<Tab, Real>();
  // y: the step's state.  Split final pass: the pass forming Y_S replaces y by the new state
  // y5 = Y_S and sets ep = (error partial sum over stages 1..S-1, atol + rtol max(|y|, |y5|)); the
  // final pass gets y5 in y and that ep back.  kst: this beam's element of the stage-derivative
  // planes (component i of k_l at kst[((l - 1) NC + i) kstride]), read and written by this thread
  // only.
  template <class BS, class Acc>
  __device__ static inline void beam(const BS& bs, const typename Phys::Beam& bm,
                                     const TabView<Real, Phys>& tv, int tj, Real (&y)[NC],
                                     Real (&ep)[NC + 1],
                                     Acc& acc, Real& emax, int& bad, bool mixed,
                                     Real* kst, size_t kstride) {
    Real k[Tab::S + 1][NC];
#pragma unroll
    for (int l = 1; l <= kLoadK; ++l)
#pragma unroll
      for (int i = 0; i < NC; ++i) k[l][i] = kst[((size_t)(l - 1) * NC + i) * kstride];
#pragma unroll
    for (int l = kLoadK + 1; l <= kChain; ++l) {
      Real Y[NC];
      if constexpr (kLoadY) {
#pragma unroll
        for (int i = 0; i < NC; ++i) Y[i] = kst[((size_t)kYPlanes * NC + i) * kstride];
      } else {
#pragma unroll
        for (int i = 0; i < NC; ++i) {
          Real v = y[i];
#pragma unroll
          for (int m = 1; m < l; ++m)
            if (Tab::a(l, m) != 0.0) v += bs.hA[l][m] * k[m][i];
          Y[i] = v;
        }
      }
      Real Kv[NC];
      Phys::K(tv.row(l, tj), bm, bs.vac, bs.scr[l], Kv);
      Phys::f(Kv, Y, k[l]);
    }
    if constexpr (kStoreK) {
#pragma unroll
      for (int i = 0; i < NC; ++i) kst[((size_t)(kChain - 1) * NC + i) * kstride] = k[kChain][i];
    }
    if (kKind == kInitPass) {
      Phys::accum_row(acc, bm.w, tv.row(1, tj), y);
      return;
    }
    if (kKind == kStagePass) {
      constexpr int I = kPass + 2;
      Real Y[NC];
#pragma unroll
      for (int i = 0; i < NC; ++i) {
        Real v = y[i];
#pragma unroll
        for (int m = 1; m < I; ++m)
          if (Tab::a(I, m) != 0.0) v += bs.hA[I][m] * k[m][i];
        Y[i] = v;
      }
      if (kSplit && I == Tab::S) {
        // first same as last: Y_S is the new state y5 (row S of A is b).  Its error partial sum
        // over stages 1..S-1 and the error scale go with it, so the final pass needs only k_S.
        if (!(Phys::tnorm2(y) <= rbig<Real>())) bad = 1;   // non-finite input state: fatal
        if (mixed) Phys::normalise(Y);
#pragma unroll
        for (int i = 0; i < NC; ++i) {
          Real v = 0;
#pragma unroll
          for (int m = 1; m < Tab::S; ++m)
            if (Tab::e(m) != 0.0) v += bs.hE[m] * k[m][i];
          ep[i] = v;
        }
        ep[NC] = bs.atol + bs.rtol * sqrt(fmax(Phys::tnorm2(y), Phys::tnorm2(Y)));
        Phys::accum_row(acc, bm.w, tv.row(I, tj), Y);
#pragma unroll
        for (int i = 0; i < NC; ++i) y[i] = Y[i];
        return;
      }
      if (Tab::kAdaptive && I == Tab::S && mixed) Phys::normalise(Y);
      if constexpr (kStoreY) {
#pragma unroll
        for (int i = 0; i < NC; ++i) kst[((size_t)kYPlanes * NC + i) * kstride] = Y[i];
      }
      Phys::accum_row(acc, bm.w, tv.row(I, tj), Y);
      return;
    }
    if (Tab::kAdaptive && !kSplit) {
      // final pass: y5 from the rebuilt chain, k_S = f(y5), the embedded error and the squared
      // error ratio (its square root is taken once per block)
      Real yn[NC];
#pragma unroll
      for (int i = 0; i < NC; ++i) {
        Real v = y[i];
#pragma unroll
        for (int m = 1; m <= kChain; ++m)
          if (Tab::b(m) != 0.0) v += bs.hB[m] * k[m][i];
        yn[i] = v;
      }
      const bool ynok = Phys::tnorm2(yn) <= rbig<Real>();
      if (mixed && ynok) Phys::normalise(yn);
      if (!(Phys::tnorm2(y) <= rbig<Real>())) bad = 1;     // non-finite input state: fatal
      Real Kv[NC];
      Phys::K(tv.row(Tab::S, tj), bm, bs.vac, bs.scr[Tab::S], Kv);
      Phys::f(Kv, yn, k[Tab::S]);
      Real e[NC];
#pragma unroll
      for (int i = 0; i < NC; ++i) {
        Real v = 0;
#pragma unroll
        for (int m = 1; m <= Tab::S; ++m)
          if (Tab::e(m) != 0.0) v += bs.hE[m] * k[m][i];
        e[i] = v;
      }
      const Real den = bs.atol + bs.rtol * sqrt(fmax(Phys::tnorm2(y), Phys::tnorm2(yn)));
      Real r2 = Phys::tnorm2(e) / (den * den);
      if (!(r2 <= rbig<Real>()) || !ynok) r2 = Real(INFINITY);
      emax = fmax(emax, r2);
#pragma unroll
      for (int i = 0; i < NC; ++i) y[i] = yn[i];
      return;
    }
    if (Tab::kAdaptive) {
      // split final pass (y holds y5): k_S = f(y5) with the moments of y5, the embedded error,
      // and the squared error ratio (its square root is taken once per block)
      const bool ynok = Phys::tnorm2(y) <= rbig<Real>();
      Real Kv[NC], kS[NC], e[NC];
      Phys::K(tv.row(Tab::S, tj), bm, bs.vac, bs.scr[Tab::S], Kv);
      Phys::f(Kv, y, kS);
#pragma unroll
      for (int i = 0; i < NC; ++i) {
        Real v = ep[i];
        v += bs.hE[Tab::S] * kS[i];
        e[i] = v;
      }
      const Real den = ep[NC];
      Real r2 = Phys::tnorm2(e) / (den * den);
      // a trial step whose stages overflowed the working precision is rejected, not fatal
      if (!(r2 <= rbig<Real>()) || !ynok) r2 = Real(INFINITY);
      emax = fmax(emax, r2);
      return;
    }
    // final pass of a fixed-step tableau
    Real yn[NC];
#pragma unroll
    for (int i = 0; i < NC; ++i) {
      Real v = y[i];
#pragma unroll
      for (int m = 1; m <= kChain; ++m)
        if (Tab::b(m) != 0.0) v += bs.hB[m] * k[m][i];
      yn[i] = v;
    }
    const bool ynok = Phys::tnorm2(yn) <= rbig<Real>();
    if (mixed && ynok) Phys::normalise(yn);
    Phys::accum_row(acc, bm.w, tv.row(Tab::S, tj), yn);
#pragma unroll
    for (int i = 0; i < NC; ++i) y[i] = yn[i];
  }
};

// Commutator-free Lie RK4 on Bloch vectors (two flavours) ---------------------------------------
template <class Phys, class Tab, typename Real, int kPass, int kKind>
struct PassBody<Phys, Tab, Real, true, kPass, kKind> {
  static constexpr int NC = Phys::NC;          // 3: Bloch vectors; 9: Hermitian 3 x 3 matrices
  static constexpr bool kStore = false;
  // rotation of y by d K (the propagator of Eq. U over the path length d for generator K)
  __device__ static inline void rot(Real (&y)[NC], const Real (&K)[NC], Real d) {
    Real Om[NC];
#pragma unroll
    for (int i = 0; i < NC; ++i) Om[i] = d * K[i];
    propagate(Om, y);
  }
  // the fourth stage state of a CF4 step of size hh from y with generators Ka (its first stage)
  // and Kc (its third): exp(hh (Kc - Ka/2)) exp(hh/2 Ka) y
  __device__ static inline void cf4_stage4(Real (&y)[NC], const Real (&Ka)[NC], const Real (&Kc)[NC], Real hh) {
    rot(y, Ka, Real(0.5) * hh);
    Real D[NC];
#pragma unroll
    for (int i = 0; i < NC; ++i) D[i] = Kc[i] - Real(0.5) * Ka[i];
    rot(y, D, hh);
  }
  // the CF4 update of size hh from y with the step's four generators
  __device__ static inline void cf4_final(Real (&y)[NC], const Real (&K1)[NC], const Real (&K2)[NC],
                                          const Real (&K3)[NC], const Real (&K4)[NC], Real hh) {
    Real Om[NC];
#pragma unroll
    for (int i = 0; i < NC; ++i)
      Om[i] = hh * (Real(0.25) * K1[i] + Real(1.0 / 6.0) * (K2[i] + K3[i]) - Real(1.0 / 12.0) * K4[i]);
    propagate(Om, y);
#pragma unroll
    for (int i = 0; i < NC; ++i)
      Om[i] = hh * (Real(-1.0 / 12.0) * K1[i] + Real(1.0 / 6.0) * (K2[i] + K3[i]) + Real(0.25) * K4[i]);
    propagate(Om, y);
  }
  template <class BS>
  __device__ static inline void gen(const BS& bs, const typename Phys::Beam& bm, const TabView<Real, Phys>& tv,
                                    int tj, int s, Real (&K)[NC]) {
    Phys::K(tv.row(s, tj), bm, bs.vac, bs.scr[s], K);
  }
  // Richardson-controlled CF4 (TabCFR): pass p forms the stage state of slot p + 2 from y; the
  // final pass forms both results, the error ratio and the moments of the kept result.
  template <class BS, class Acc>
  __device__ static inline void richardson(const BS& bs, const typename Phys::Beam& bm,
                                           const TabView<Real, Phys>& tv, int tj, Real (&y)[NC], Acc& acc,
                                           Real& emax, int& bad, bool mixed) {
    const Real h = bs.hB[0], hh = Real(0.5) * h;
    constexpr int I = kKind == kFinalPass ? 0 : kPass + 2;   // slot formed by this pass
    Real K1[NC];
    gen(bs, bm, tv, tj, 1, K1);
    if constexpr (I >= 2 && I <= 4) {
      // full step: Y2 = exp(h/2 K1) y, Y3 = exp(h/2 K2) y, Y4 = exp(h (K3 - K1/2)) exp(h/2 K1) y
      if constexpr (I == 2) {
        rot(y, K1, hh);
      } else if constexpr (I == 3) {
        Real K2[NC];
        gen(bs, bm, tv, tj, 2, K2);
        rot(y, K2, hh);
      } else {
        Real K3[NC];
        gen(bs, bm, tv, tj, 3, K3);
        cf4_stage4(y, K1, K3, h);
      }
      Phys::accum_row(acc, bm.w, tv.row(I, tj), y);
      return;
    }
    if constexpr (I >= 5 && I <= 7) {
      // first half step: slots 5, 6, 7 as 2, 3, 4 with hh and generators K1, K5, K6
      if constexpr (I == 5) {
        rot(y, K1, Real(0.5) * hh);
      } else if constexpr (I == 6) {
        Real K5[NC];
        gen(bs, bm, tv, tj, 5, K5);
        rot(y, K5, Real(0.5) * hh);
      } else {
        Real K6[NC];
        gen(bs, bm, tv, tj, 6, K6);
        cf4_stage4(y, K1, K6, hh);
      }
      Phys::accum_row(acc, bm.w, tv.row(I, tj), y);
      return;
    }
    // everything later starts from the first half step's result y_a (slot 8)
    Real y0[NC];
#pragma unroll
    for (int i = 0; i < NC; ++i) y0[i] = y[i];
    {
      Real K5[NC], K6[NC], K7[NC];
      gen(bs, bm, tv, tj, 5, K5);
      gen(bs, bm, tv, tj, 6, K6);
      gen(bs, bm, tv, tj, 7, K7);
      cf4_final(y, K1, K5, K6, K7, hh);
    }
    if constexpr (I == 8) {
      Phys::accum_row(acc, bm.w, tv.row(8, tj), y);
      return;
    }
    Real K8[NC];
    gen(bs, bm, tv, tj, 8, K8);
    if constexpr (I >= 9 && I <= 11) {
      if constexpr (I == 9) {
        rot(y, K8, Real(0.5) * hh);
      } else if constexpr (I == 10) {
        Real K9[NC];
        gen(bs, bm, tv, tj, 9, K9);
        rot(y, K9, Real(0.5) * hh);
      } else {
        Real K10[NC];
        gen(bs, bm, tv, tj, 10, K10);
        cf4_stage4(y, K8, K10, hh);
      }
      Phys::accum_row(acc, bm.w, tv.row(I, tj), y);
      return;
    } else {
      // final pass: y_b = the second half step from y_a, y_full = the full step from y0
      {
        Real K9[NC], K10[NC], K11[NC];
        gen(bs, bm, tv, tj, 9, K9);
        gen(bs, bm, tv, tj, 10, K10);
        gen(bs, bm, tv, tj, 11, K11);
        cf4_final(y, K8, K9, K10, K11, hh);
      }
      Real yf[NC];
#pragma unroll
      for (int i = 0; i < NC; ++i) yf[i] = y0[i];
      {
        Real K2[NC], K3[NC], K4[NC];
        gen(bs, bm, tv, tj, 2, K2);
        gen(bs, bm, tv, tj, 3, K3);
        gen(bs, bm, tv, tj, 4, K4);
        cf4_final(yf, K1, K2, K3, K4, h);
      }
      Real e[NC];
#pragma unroll
      for (int i = 0; i < NC; ++i) e[i] = (y[i] - yf[i]) * Real(1.0 / 15.0);
      if (!(Phys::tnorm2(y0) <= rbig<Real>())) bad = 1;       // non-finite input state: fatal
      const bool ynok = Phys::tnorm2(y) <= rbig<Real>();
      const Real den = bs.atol + bs.rtol * sqrt(fmax(Phys::tnorm2(y0), Phys::tnorm2(y)));
      Real r2 = Phys::tnorm2(e) / (den * den);
      if (!(r2 <= rbig<Real>()) || !ynok) r2 = Real(INFINITY);
      emax = fmax(emax, r2);
      if (mixed && ynok) Phys::purify(y);
      Phys::accum_row(acc, bm.w, tv.row(11, tj), y);
    }
  }
  template <class BS, class Acc>
  __device__ static inline void beam(const BS& bs, const typename Phys::Beam& bm,
                                     const TabView<Real, Phys>& tv, int tj, Real (&y)[NC],
                                     Real (&)[NC + 1],
                                     Acc& acc, Real& emax, int& bad, bool mixed,
                                     Real*, size_t) {
    if (kKind == kInitPass) {
      Phys::accum_row(acc, bm.w, tv.row(1, tj), y);
      return;
    }
    const Real h = bs.hB[0];
    if constexpr (Tab::kRichardson) {
      richardson(bs, bm, tv, tj, y, acc, emax, bad, mixed);
      return;
    }
    if constexpr (Tab::kEM2) {
      // exponential midpoint rule: half step with K1 -> Y_half (moments at r + h/2); final pass:
      // y' = exp(h K2) y, the estimate exp(h K1) y, the error ratio, moments of y' at r + h
      Real K1[NC], Om[NC];
      Phys::K(tv.row(1, tj), bm, bs.vac, bs.scr[1], K1);
      if (kKind == kStagePass) {
#pragma unroll
        for (int i = 0; i < NC; ++i) Om[i] = Real(0.5) * h * K1[i];
        propagate(Om, y);
        Phys::accum_row(acc, bm.w, tv.row(2, tj), y);
        return;
      }
      Real K2[NC], yn[NC], ye[NC], e[NC];
      Phys::K(tv.row(2, tj), bm, bs.vac, bs.scr[2], K2);
#pragma unroll
      for (int i = 0; i < NC; ++i) { yn[i] = y[i]; ye[i] = y[i]; Om[i] = h * K2[i]; }
      propagate(Om, yn);
#pragma unroll
      for (int i = 0; i < NC; ++i) Om[i] = h * K1[i];
      propagate(Om, ye);
#pragma unroll
      for (int i = 0; i < NC; ++i) e[i] = yn[i] - ye[i];
      if (!(Phys::tnorm2(y) <= rbig<Real>())) bad = 1;       // non-finite input state: fatal
      const bool ynok = Phys::tnorm2(yn) <= rbig<Real>();
      const Real den = bs.atol + bs.rtol * sqrt(fmax(Phys::tnorm2(y), Phys::tnorm2(yn)));
      Real r2 = Phys::tnorm2(e) / (den * den);
      if (!(r2 <= rbig<Real>()) || !ynok) r2 = Real(INFINITY);
      emax = fmax(emax, r2);
      if (mixed && ynok) Phys::purify(yn);
      Phys::accum_row(acc, bm.w, tv.row(3, tj), yn);
#pragma unroll
      for (int i = 0; i < NC; ++i) y[i] = yn[i];
      return;
    }
    Real K1[NC], K2[NC], K3[NC], K4[NC], Om[NC];
    Phys::K(tv.row(1, tj), bm, bs.vac, bs.scr[1], K1);
    if (kKind == kStagePass && kPass == 0) {
#pragma unroll
      for (int i = 0; i < NC; ++i) Om[i] = Real(0.5) * h * K1[i];
      propagate(Om, y);
      Phys::accum_row(acc, bm.w, tv.row(2, tj), y);
      return;
    }
    Phys::K(tv.row(2, tj), bm, bs.vac, bs.scr[2], K2);
    if (kKind == kStagePass && kPass == 1) {
#pragma unroll
      for (int i = 0; i < NC; ++i) Om[i] = Real(0.5) * h * K2[i];
      propagate(Om, y);
      Phys::accum_row(acc, bm.w, tv.row(3, tj), y);
      return;
    }
    Phys::K(tv.row(3, tj), bm, bs.vac, bs.scr[3], K3);
    if (kKind == kStagePass && kPass == 2) {
#pragma unroll
      for (int i = 0; i < NC; ++i) Om[i] = Real(0.5) * h * K1[i];
      propagate(Om, y);
#pragma unroll
      for (int i = 0; i < NC; ++i) Om[i] = h * K3[i] - Real(0.5) * h * K1[i];
      propagate(Om, y);
      Phys::accum_row(acc, bm.w, tv.row(4, tj), y);
      return;
    }
    Phys::K(tv.row(4, tj), bm, bs.vac, bs.scr[4], K4);
#pragma unroll
    for (int i = 0; i < NC; ++i)
      Om[i] = h * (Real(0.25) * K1[i] + Real(1.0 / 6.0) * (K2[i] + K3[i]) - Real(1.0 / 12.0) * K4[i]);
    propagate(Om, y);
#pragma unroll
    for (int i = 0; i < NC; ++i)
      Om[i] = h * (Real(-1.0 / 12.0) * K1[i] + Real(1.0 / 6.0) * (K2[i] + K3[i]) + Real(0.25) * K4[i]);
    propagate(Om, y);
    if (mixed) Phys::purify(y);
    Phys::accum_row(acc, bm.w, tv.row(4, tj), y);
  }
};

// ----------------------------------------------------------------------------------------------
// FP32 two-flavour beams in pairs with packed f32x2 arithmetic (Blackwell fma/mul.rn.f32x2).
// A thread's two beams are consecutive energy bins of one angle bin, so every table value and step
// coefficient is shared: it is stored duplicated and loaded as one 64-bit operand, while the
// per-beam values (state, eta omega, weight) are packed once per pair.  Each packed instruction
// does the work of two scalar ones, in the same order, so a pair gives the same bits as two
// scalar beams would with contraction to FMA.
using F2 = unsigned long long;
__device__ __forceinline__ F2 pk(float a, float b) {
  F2 r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
  return r;
}
__device__ __forceinline__ void upk(F2 r, float& a, float& b) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(r));
}
__device__ __forceinline__ F2 fma2(F2 a, F2 b, F2 c) {
  F2 d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}
__device__ __forceinline__ F2 mul2(F2 a, F2 b) {
  F2 d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ F2 add2(F2 a, F2 b) {
  F2 d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ F2 sub2(F2 a, F2 b) {
  F2 d;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
// two_sum_acc on a pair (each half one beam): hi + c split into the rounded sum and its exact
// rounding error, collected in lo.
__device__ __forceinline__ void two_sum_acc2(F2& hi, F2& lo, F2 c) {
  const F2 s = add2(hi, c);
  const F2 bv = sub2(s, hi);
  const F2 err = add2(sub2(hi, sub2(s, bv)), sub2(c, bv));
  hi = s;
  lo = add2(lo, err);
}
// Moment accumulators of a thread's beam pairs: component i is the unevaluated sum hi[i] + lo[i].
template <int NM>
struct PairAcc {
  F2 hi[NM], lo[NM];
};
// A single (unpaired) beam of a pair kernel accumulates into the first half of the pair
// accumulators, so those kernels keep one set of accumulator registers.
template <int NM>
struct PairHalfAcc {
  PairAcc<NM>& a;
  __device__ __forceinline__ void add(int i, float w, float y) { two_sum_acc2(a.hi[i], a.lo[i], pk(__fmul_rn(w, y), 0.0f)); }
};

template <class P, class Tab, int kPass, int kKind>
struct PairRK {
  static constexpr int NM = P::NM;                 // 6 (bulb) or 12 (extended: + Jc, Js)
  static_assert(!split_final<Tab, float>(), "FP32 passes rebuild the chain in the final pass");
  static constexpr int kChain =
      kKind == kInitPass ? 0 : (kKind == kFinalPass ? Tab::S - (Tab::kAdaptive ? 1 : 0) : kPass + 1);

  // K and -K of stage row R (packed values) for the pair's eta omega; -K_x and -K_z by one packed
  // multiply by (-1, -1) each, -K_y = -G0_y from the row
  __device__ static inline void Kpair(const F2* R, F2 eo, F2 (&K)[3], F2 (&nK)[3]) {
    const F2 m1 = 0xbf800000bf800000ull;            // (-1.0f, -1.0f)
    K[0] = fma2(eo, R[P::vQBX], R[P::vG0X]);
    K[1] = R[P::vG0Y];
    K[2] = fma2(eo, R[P::vQBZ], R[P::vG0Z]);
    nK[0] = mul2(K[0], m1);
    if constexpr (P::kNegated) nK[1] = R[P::vNG0Y];
    else nK[1] = mul2(K[1], m1);
    nK[2] = mul2(K[2], m1);
  }
  // k = K x Y as K1 Y2 - K2 Y1, ... with the products of -K added by FMA
  __device__ static inline void cross(const F2 (&K)[3], const F2 (&nK)[3], const F2 (&Y)[3], F2 (&k)[3]) {
    k[0] = fma2(K[1], Y[2], mul2(nK[2], Y[1]));
    k[1] = fma2(K[2], Y[0], mul2(nK[0], Y[2]));
    k[2] = fma2(K[0], Y[1], mul2(nK[1], Y[0]));
  }
  // moments of the pair's states with the weights of row R: D (w t1), J1 (w) and, extended model,
  // Jc (w (sin th / cos th) cos phi), Js (w (sin th / cos th) sin phi)
  // (contributions formed in FP32, summed without loss: see MomAcc<float>)
  __device__ static inline void accum(PairAcc<NM>& acc, F2 w, const F2* R, const F2 (&y)[3]) {
    const F2 wt = mul2(w, R[P::vT1]);
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      two_sum_acc2(acc.hi[i], acc.lo[i], mul2(wt, y[i]));
      two_sum_acc2(acc.hi[3 + i], acc.lo[3 + i], mul2(w, y[i]));
    }
    if constexpr (NM == 12) {
      const F2 wc = mul2(w, R[P::vSCC]), ws = mul2(w, R[P::vSCS]);
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        two_sum_acc2(acc.hi[6 + i], acc.lo[6 + i], mul2(wc, y[i]));
        two_sum_acc2(acc.hi[9 + i], acc.lo[9 + i], mul2(ws, y[i]));
      }
    }
  }
  // 1/sqrt(n2) of a pair: hardware reciprocal square root refined by one Newton step
  // r <- r (3 - n2 r^2) / 2 (relative error ~1e-7, as a correctly rounded quotient would give)
  __device__ static inline F2 rnorm(F2 n2) {
    float a, b;
    upk(n2, a, b);
    const F2 r = pk(rsqrtf(a), rsqrtf(b));
    const F2 t = mul2(mul2(n2, r), r);                         // n2 r^2
    return mul2(mul2(r, 0xbf000000bf000000ull), fma2(t, 0x3f8000003f800000ull, 0xc0400000c0400000ull));
  }
  __device__ static inline void normalise(F2 (&y)[3]) {
    F2 n2 = mul2(y[0], y[0]);
    n2 = fma2(y[1], y[1], n2);
    n2 = fma2(y[2], y[2], n2);
    const F2 inv = rnorm(n2);
#pragma unroll
    for (int i = 0; i < 3; ++i) y[i] = mul2(y[i], inv);
  }

  // rows: table rows of this pair's angle bin, stage s at rows + s * rstride (in F2 units);
  // y, ep as in PassBody::beam
  template <class BS>
  __device__ static inline void run(const BS& bs, F2 eo, F2 w, const F2* rows, int rstride, F2 (&y)[3],
                                    F2 (&ep)[4], PairAcc<NM>& acc, float& emax, int& bad) {
    F2 k[Tab::S + 1][3];
    // adaptive final pass: y5 and the error accumulate as soon as each stage derivative exists
    // (same order of operations as summing after the chain), so the derivatives die early
    constexpr bool kFinalAdaptive = kKind == kFinalPass && Tab::kAdaptive;
    F2 yn[3] = {y[0], y[1], y[2]};
    F2 e[3] = {0ull, 0ull, 0ull};
#pragma unroll
    for (int l = 1; l <= kChain; ++l) {
      F2 Y[3] = {y[0], y[1], y[2]};
#pragma unroll
      for (int m = 1; m < l; ++m)
        if (Tab::a(l, m) != 0.0) {
          const F2 ha = bs.hA2[l][m];
#pragma unroll
          for (int i = 0; i < 3; ++i) Y[i] = fma2(ha, k[m][i], Y[i]);
        }
      F2 K[3], nK[3];
      Kpair(rows + l * rstride, eo, K, nK);
      cross(K, nK, Y, k[l]);
      if (kFinalAdaptive) {
        if (Tab::b(l) != 0.0) {
          const F2 hb = bs.hB2[l];
#pragma unroll
          for (int i = 0; i < 3; ++i) yn[i] = fma2(hb, k[l][i], yn[i]);
        }
        if (Tab::e(l) != 0.0) {
          const F2 he = bs.hE2[l];
#pragma unroll
          for (int i = 0; i < 3; ++i) e[i] = fma2(he, k[l][i], e[i]);
        }
      }
    }
    if (kKind == kInitPass) {
      accum(acc, w, rows + rstride * 1, y);
      return;
    }
    if (kKind == kStagePass) {
      constexpr int I = kPass + 2;
      F2 Y[3] = {y[0], y[1], y[2]};
#pragma unroll
      for (int m = 1; m < I; ++m)
        if (Tab::a(I, m) != 0.0) {
          const F2 ha = bs.hA2[I][m];
#pragma unroll
          for (int i = 0; i < 3; ++i) Y[i] = fma2(ha, k[m][i], Y[i]);
        }
      if (Tab::kAdaptive && I == Tab::S) normalise(Y);
      accum(acc, w, rows + rstride * I, Y);
      return;
    }
    if (Tab::kAdaptive) {
      // final pass: y5 from the rebuilt chain, k_S = f(y5), the embedded error and the squared
      // error ratio |e|_F^2 / scale^2 (its square root is taken once per block)
      F2 n2y = mul2(y[0], y[0]);
      n2y = fma2(y[1], y[1], n2y);
      n2y = fma2(y[2], y[2], n2y);
      F2 n2n = mul2(yn[0], yn[0]);
      n2n = fma2(yn[1], yn[1], n2n);
      n2n = fma2(yn[2], yn[2], n2n);
      float a0, a1, c0, c1;
      upk(n2y, a0, a1);
      upk(n2n, c0, c1);
      if (!(a0 <= 3.0e38f) || !(a1 <= 3.0e38f)) bad = 1;    // non-finite input state: fatal
      const bool ok0 = c0 <= 3.0e38f, ok1 = c1 <= 3.0e38f;
      if (ok0 && ok1) {
        const F2 inv = rnorm(n2n);
#pragma unroll
        for (int i = 0; i < 3; ++i) yn[i] = mul2(yn[i], inv);
      }
      F2 K[3], nK[3];
      Kpair(rows + Tab::S * rstride, eo, K, nK);
      cross(K, nK, yn, k[Tab::S]);
      if (Tab::e(Tab::S) != 0.0) {
        const F2 he = bs.hE2[Tab::S];
#pragma unroll
        for (int i = 0; i < 3; ++i) e[i] = fma2(he, k[Tab::S][i], e[i]);
      }
      F2 e2 = mul2(e[0], e[0]);
      e2 = fma2(e[1], e[1], e2);
      e2 = fma2(e[2], e[2], e2);
      F2 m2 = mul2(yn[0], yn[0]);
      m2 = fma2(yn[1], yn[1], m2);
      m2 = fma2(yn[2], yn[2], m2);
      float e20, e21, m20, m21;
      upk(e2, e20, e21);
      upk(m2, m20, m21);
      // |P~|_F = |s| / sqrt(2), |e|_F^2 = |e|^2 / 2
      const float atol = bs.atol, rtol = bs.rtol;
      const float s0 = atol + rtol * sqrtf(0.5f * fmaxf(a0, m20));
      const float s1 = atol + rtol * sqrtf(0.5f * fmaxf(a1, m21));
      float r0 = __fdiv_rn(0.5f * e20, s0 * s0);
      float r1 = __fdiv_rn(0.5f * e21, s1 * s1);
      if (!(r0 <= 3.0e38f) || !ok0) r0 = INFINITY;
      if (!(r1 <= 3.0e38f) || !ok1) r1 = INFINITY;
      emax = fmaxf(emax, fmaxf(r0, r1));
#pragma unroll
      for (int i = 0; i < 3; ++i) y[i] = yn[i];
      return;
    }
    // final pass of a fixed-step tableau
#pragma unroll
    for (int m = 1; m <= kChain; ++m)
      if (Tab::b(m) != 0.0) {
        const F2 hb = bs.hB2[m];
#pragma unroll
        for (int i = 0; i < 3; ++i) yn[i] = fma2(hb, k[m][i], yn[i]);
      }
    float a0[3], a1[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) upk(yn[i], a0[i], a1[i]);
    const bool ok0 = 0.5f * (a0[0] * a0[0] + a0[1] * a0[1] + a0[2] * a0[2]) <= 3.0e38f;
    const bool ok1 = 0.5f * (a1[0] * a1[0] + a1[1] * a1[1] + a1[2] * a1[2]) <= 3.0e38f;
    if (ok0 && ok1) normalise(yn);
    accum(acc, w, rows + rstride * Tab::S, yn);
#pragma unroll
    for (int i = 0; i < 3; ++i) y[i] = yn[i];
  }
};

// Load the beam constants of (species, energy k) and the angle weight du.
template <typename Real>
__device__ __forceinline__ void load_beam(const Real* et, int ne, int sigma, int k, Real du,
                                          typename Phys2<Real>::Beam& bm) {
  const Real om = et[k];
  bm.eo = sigma ? -om : om;
  bm.w = du * et[(1 + sigma) * ne + k];
}
template <typename Real>
__device__ __forceinline__ void load_beam(const Real* et, int ne, int sigma, int k, Real du,
                                          typename Phys3<Real>::Beam& bm) {
  const Real o21 = et[k], o31 = et[ne + k];
  bm.o21 = sigma ? -o21 : o21;
  bm.o31 = sigma ? -o31 : o31;
  bm.w = du * et[(2 + sigma) * ne + k];
}

// Checked build: a beam's energy-table entries (rows 0 .. 2 of the two-flavour tables, 0 .. 3 of
// the three-flavour ones), its row of the shared angle tables and (stored-stage bodies) its
// elements of the stage planes.  Always true without XFLAT_BOUNDS.
template <class Body, int NC, typename Real>
__device__ __forceinline__ bool beam_in_bounds(const KParams& p, const Real* et, int ne, int k, int tj,
                                               int n_jj, const Real* kst_beam) {
#ifdef XFLAT_BOUNDS
  constexpr int kERowMax = NC == 3 ? 2 : 3;
  bool ok = index_ok(p, tj >= 0 && tj < n_jj, 12, tj) && index_ok(p, k >= 0 && k < ne, 10, k) &&
            span_ok(p, kSpanEtab, et + k, sizeof(Real), 10) &&
            span_ok(p, kSpanEtab, et + (size_t)kERowMax * ne + k, sizeof(Real), 11);
  if constexpr (Body::kStore)
    ok = ok && span_ok(p, kSpanKst, kst_beam, sizeof(Real), 8) &&
         span_ok(p, kSpanKst, kst_beam + ((size_t)(Body::kYPlanes + 1) * NC - 1) * p.plane_stride,
                 sizeof(Real), 9);
  return ok;
#else
  return true;
#endif
}

// Stages whose table rows a pass reads (bit s set: row s needed).
template <class Tab, int kPass, int kKind>
__device__ __forceinline__ unsigned stages_needed() {
  if (kKind == kInitPass) return 1u << 1;
  if (kKind == kFinalPass) return ((1u << (Tab::S + 1)) - 1u) & ~1u;          // 1..S
  return ((1u << (kPass + 3)) - 1u) & ~1u;                                      // 1..kPass+2
}

// One pass over all pieces of this block.
template <class Phys, class Tab, typename Real, bool kCF, int kPass, int kKind>
__device__ void run_pass(const KParams& p, BlockShared<Real, Phys>& bs, unsigned char* dyn_smem) {
  constexpr int NC = Phys::NC, NM = Phys::NM, VN = Vec16<Real>::N;
  using Body = PassBody<Phys, Tab, Real, kCF, kPass, kKind>;
  double* red = reinterpret_cast<double*>(dyn_smem);                 // 32 * NM doubles
  constexpr int kTS = Tab::S + 1;                                    // table stage slots 0..S
  Real* tab = reinterpret_cast<Real*>(red + 32 * kNMMax);            // [kTS][max_jj][KT]
  Real* dut = tab + (size_t)kTS * p.max_jj * Phys::KT;               // [max_jj]
  double* ut = reinterpret_cast<double*>(                            // [max_jj], 8-byte aligned
      (reinterpret_cast<uintptr_t>(dut + p.max_jj) + 7) & ~uintptr_t(7));
  float* ring = reinterpret_cast<float*>(                            // [slots][NC][threads][2], 16-byte aligned
      (reinterpret_cast<uintptr_t>(ut + p.max_jj) + 15) & ~uintptr_t(15));
  const bool mixed = sizeof(Real) == 4;
  const int slot = kKind == kInitPass ? 1 : (kKind == kStagePass ? kPass + 2 : 0);
  // Clear accumulator slots nobody reads any more (block 0, while the other blocks already work).
  // Stage s (2 <= s < kPasses) is reduced in pass s - 2 and read by every block in the set-up of
  // pass s - 1, so it is cleared at the start of pass s; pass 0 clears the final pass's slot 0 and
  // the moment launch's slot 1, both read by serial updates that finish before their barrier
  // opens.  Stages with no pass of their own index (kPasses <= s <= S: stage S of RK4 / DP45,
  // stages 2 and 3 of the exponential midpoint rule) are cleared by the final pass's serial section
  // (clear_late_slots) while every other block waits at the final barrier.  Nothing accumulates
  // into a cleared slot until at least one barrier later, and block 0's stores are fenced at its
  // next arrival.
  if (kKind != kInitPass && blockIdx.x == 0) {
    constexpr int kWords = kAccCopies * kNMMax * 2;
    constexpr int kSlots = kPass == 0 ? 2 : (kPass >= 2 ? 1 : 0);
    for (int t = threadIdx.x; t < p.n_inst * kSlots * kWords; t += blockDim.x) {
      const int inst = t / (kSlots * kWords), rem = t % (kSlots * kWords), q = rem / kWords;
      const int zslot = kPass == 0 ? q : kPass;
      p.acc[(size_t)inst * kAccWordsPerInst + (size_t)zslot * kWords + rem % kWords] = 0ull;
    }
  }
  const unsigned need = stages_needed<Tab, kPass, kKind>();
  // the stage whose moments the previous pass reduced (0: none of this step, its constants come
  // from the serial update of the previous step or of the moment launch)
  constexpr int kNewest = (kKind != kInitPass && kPass >= 1) ? kPass + 1 : 0;
  const bool dyn = p.dyn_sched != 0;
  const int b0 = dyn ? 0 : p.blk_piece[blockIdx.x], b1 = dyn ? 0 : p.blk_piece[blockIdx.x + 1];
  // A block with a single piece keeps its set-up in shared memory for the whole step: after pass
  // 0 only the newest stage's constants and the table rows of the newest and the formed stage
  // change (flags, step size, coefficients, radii, angle tables and older rows stay valid).
  const bool single = !dyn && b1 - b0 == 1;
  const bool incremental = single && kNewest >= 1 && !p.shard_mode;
  for (int it = 0;; ++it) {
    int pi = b0 + it;
    if (dyn) {
      __syncthreads();                           // next_piece of the previous piece has been read
      if (threadIdx.x == 0) bs.next_piece = (int)atomicAdd(&p.bar->chunk[(bs.gen_seen >> 1) & 1u], 1u);
      __syncthreads();
      pi = bs.next_piece;
      if (pi >= p.n_pieces) break;
    } else if (pi >= b1) {
      break;
    }
    if (!XFLAT_INDEX_OK(p, pi >= 0 && pi < p.n_pieces, 13, pi)) break;
    const Piece pc = p.pieces[pi];
    if (!XFLAT_INDEX_OK(p, pc.inst >= 0 && pc.inst < p.n_inst && (int)pc.n_jj <= p.max_jj &&
                               (uint64_t)pc.start + pc.len <= p.ic[pc.inst].n_beams, 14, pi))
      continue;
    const InstConst& ic = p.ic[pc.inst];
    const InstDyn* d = p.dyn + pc.inst;
    __syncthreads();
    if (incremental) {
      if (threadIdx.x < Phys::NSC) {
        const int c = threadIdx.x;
        double v = 0.0;
        const unsigned long long* accs = p.acc + (size_t)pc.inst * kAccWordsPerInst +
                                         (size_t)kNewest * kAccCopies * kNMMax * 2;
        InstDyn* dw = p.dyn + pc.inst;
        if (c < Phys::NM) {
          const double m = acc_component<Real>(accs, c, ic.acc_unit);
          v = ldcg(&d->mus[kNewest]) * m;
          if (pc.start == ic.rec_start) dw->mom[kNewest][c] = m;
        } else if (c == Phys::NM) {
          v = ldcg(&d->lams[kNewest]);
        }
        if (pc.start == ic.rec_start && c <= Phys::NM) dw->sc[kNewest][c] = v;
        bs.scd[kNewest][c] = v;
        bs.scr[kNewest][c] = (Real)v;
      }
      __syncthreads();
    }
    if (!incremental) {
    // one parallel load phase: flags, step size, stage constants, radii, angle weights (every
    // load issued before any of them is used, so the phase costs one L2 round trip)
    if (threadIdx.x == 0) {
      const int dn = ldcg(&d->done), st = ldcg(&d->status), par = ldcg(&d->parity);
      bs.active = (dn == 0 && st == 0) ? 1 : 0;
      bs.parity = par;
    }
    const double h = Tab::kAdaptive ? ldcg(&d->h) : ldcg(&d->h_fixed);
    for (int t = threadIdx.x; t < kTS * Phys::NSC; t += blockDim.x) {
      const int s = t / Phys::NSC, c = t % Phys::NSC;
      double v = 0.0;
      if (s == kNewest) {
        // the stage reduced by the previous pass: every block derives its constants mu m (and
        // lambda) from the accumulators itself (integer sums: the same bits everywhere), so that
        // barrier needs no serial section; the block holding the instance's first beams records
        // the moments and constants for later passes and the host
        const unsigned long long* accs = p.acc + (size_t)pc.inst * kAccWordsPerInst +
                                         (size_t)s * kAccCopies * kNMMax * 2;
        InstDyn* dw = p.dyn + pc.inst;
        if (c < Phys::NM) {
          const double m = acc_component<Real>(accs, c, ic.acc_unit);
          v = ldcg(&d->mus[s]) * m;
          if (pc.start == ic.rec_start) dw->mom[s][c] = m;
        } else if (c == Phys::NM) {
          v = ldcg(&d->lams[s]);
        }
        if (pc.start == ic.rec_start && c <= Phys::NM) dw->sc[s][c] = v;
      } else if ((need >> s) & 1u) {
        v = ldcg(&d->sc[s][c]);
      }
      bs.scd[s][c] = v;
      bs.scr[s][c] = (Real)v;
    }
    if (threadIdx.x < kMaxStages) bs.xs[threadIdx.x] = ldcg(&d->xs[threadIdx.x]);
    if (threadIdx.x < kMaxStages * kMaxStages) {
      const int i = threadIdx.x / kMaxStages, j = threadIdx.x % kMaxStages;
      bs.hA[i][j] = (Real)(h * ((i >= 1 && j >= 1) ? Tab::a(i, j) : 0.0));
      const float fa = (float)bs.hA[i][j];
      bs.hA2[i][j] = pk(fa, fa);
    }
    if (threadIdx.x < kMaxStages) {
      const int i = threadIdx.x;
      if (kCF) {
        bs.hB[i] = (Real)h;
        bs.hE[i] = 0;
      } else {
        bs.hB[i] = (Real)(h * (i >= 1 ? Tab::b(i) : 0.0));
        bs.hE[i] = (Real)(h * (i >= 1 ? Tab::e(i) : 0.0));
      }
      const float fb = (float)bs.hB[i], fe = (float)bs.hE[i];
      bs.hB2[i] = pk(fb, fb);
      bs.hE2[i] = pk(fe, fe);
    }
    // launch-invariant part (vacuum matrices, tolerances, angle tables): a single-piece block
    // loads it once per launch
    if (!(single && bs.keep)) {
      if (threadIdx.x < 6) {
        bs.vac[threadIdx.x] = (Real)ic.M21[threadIdx.x];
        bs.vac[6 + threadIdx.x] = (Real)ic.M31[threadIdx.x];
      }
      if (threadIdx.x == 0) {
        bs.rtol = (Real)ic.rtol;
        bs.atol = (Real)ic.atol;
      }
      for (int t = threadIdx.x; t < (int)pc.n_jj; t += blockDim.x) {
        const int jj = pc.jj_lo + t;
        const int j = jj >= (int)ic.n_angle ? jj - (int)ic.n_angle : jj;
        if (!(XFLAT_INDEX_OK(p, j >= 0 && j < (int)ic.n_angle, 15, jj) &&
              XFLAT_SPAN_OK(p, kSpanDu, p.du_tab + ic.a_off + j, sizeof(double), 16) &&
              XFLAT_SPAN_OK(p, kSpanU, p.u_tab + ic.a_off + j, sizeof(double), 16))) {
          dut[t] = Real(0);
          ut[t] = 0.0;
          continue;
        }
        dut[t] = (Real)p.du_tab[ic.a_off + j];
        ut[t] = p.u_tab[ic.a_off + j];
      }
    }
    __syncthreads();
    if (single && threadIdx.x == 0) bs.keep = 1;     // read after later barriers only
    }
    const int n_jj = pc.n_jj;
    if (!bs.active) continue;
    typename Phys::Consts C;
    if constexpr (Phys::NC == 3) {
      C.B[0] = ic.B[0]; C.B[1] = ic.B[1]; C.B[2] = ic.B[2];
      if constexpr (Phys::NM == 12) C.n_phi = (int)ic.n_phi;
      else C.geom = ic.geom;
    } else {
#pragma unroll
      for (int i = 0; i < 6; ++i) { C.M21[i] = ic.M21[i]; C.M31[i] = ic.M31[i]; }
      C.geom = ic.geom;
    }
    // table rows: every needed stage, or (incremental) only the newest and the formed stage
    const unsigned fill = incremental ? (need & (3u << kNewest)) : need;
    for (int t = threadIdx.x; t < kTS * n_jj; t += blockDim.x) {
      const int s = t / n_jj, tj = t % n_jj;
      if (!((fill >> s) & 1u)) continue;
      Real* row = tab + ((size_t)s * n_jj + tj) * Phys::KT;
      const int jj = (int)pc.jj_lo + tj;
      const int a = jj >= (int)ic.n_angle ? jj - (int)ic.n_angle : jj;     // angle bin of its species
      Phys::fill_row(row, ut[tj], bs.xs[s], bs.scd[s], bs.scr[s], C, a, 0);
    }
    __syncthreads();
    const TabView<Real, Phys> tv{tab, n_jj};
    const Real* et = reinterpret_cast<const Real*>(p.etab) + ic.e_off;
    const Real* yin = reinterpret_cast<const Real*>(bs.parity ? p.planeB : p.planeA) + ic.beam_off;
    Real* yout = reinterpret_cast<Real*>(bs.parity ? p.planeA : p.planeB) + ic.beam_off;
    // split final pass (see split_final): the pass forming Y_S stores y5 (into the output planes),
    // the error partial and the error scale; the final pass reads those instead of the chain
    constexpr bool kSplitStore = split_final<Tab, Real>() && kKind == kStagePass && kPass + 2 == Tab::S;
    constexpr bool kSplitLoad = split_final<Tab, Real>() && kKind == kFinalPass;
    Real* escr = reinterpret_cast<Real*>(p.escr) + ic.beam_off;
    Real* kst = Body::kStore ? reinterpret_cast<Real*>(p.kst) + ic.beam_off : nullptr;
    const Real* ysrc = kSplitLoad ? yout : yin;
    const int ne = (int)ic.n_energy, na = (int)ic.n_angle;
    MomAcc<Real, NM> acc;
    acc.zero();
    Real emax = 0;
    int bad = 0;
    // FP32 two-flavour RK passes run beam pairs on packed f32x2 arithmetic (PairRK)
    constexpr bool kPair = Phys::kPairable && !kCF;
    PairAcc<NM> acc2;
#pragma unroll
    for (int i = 0; i < NM; ++i) { acc2.hi[i] = 0ull; acc2.lo[i] = 0ull; }
    float emax2 = 0.0f;
    const uint32_t end = pc.start + pc.len;
    const uint32_t vstep = VN * blockDim.x;
    // FP32 two-flavour bulb passes: the state comes through the thread's ring, kStateRingDepth vectors
    // ahead (see state_ring).  Other two-flavour passes: the next vector's state is loaded into
    // registers while this one is processed.  Either way the L2/HBM latency of the stream overlaps
    // the arithmetic.
    constexpr bool kRingLoad = state_ring<Phys, Real>();
    constexpr bool kPrefetch = NC == 3 && !kRingLoad;
    Real nxt[NC][VN];
    if (kPrefetch && pc.start + VN * threadIdx.x < end) {
#pragma unroll
      for (int c = 0; c < NC; ++c) vload_at(p, kSpanPlanes, ysrc + (size_t)c * p.plane_stride + pc.start + VN * threadIdx.x, nxt[c], 1);
    }
    constexpr int ring_d = kStateRingDepth;
    constexpr uint32_t ring_slots = (uint32_t)ring_d + 1u;
    uint32_t q_fill = 0, q_read = 0;
    // start the copies of the vector at beam l (if it is in the piece) into the next slot; one
    // commit group per vector, empty past the end, so the group count stays in step
    auto ring_fill = [&](uint32_t l) {
      if (l < end) {
#pragma unroll
        for (int c = 0; c < NC; ++c) {
          const Real* src = ysrc + (size_t)c * p.plane_stride + l;
          if (XFLAT_SPAN_OK(p, kSpanPlanes, src, 2 * sizeof(Real), 1))
            cp_async8(ring + (((size_t)q_fill * NC + c) * blockDim.x + threadIdx.x) * 2, src);
        }
      }
      cp_async_commit();
      q_fill = q_fill + 1u == ring_slots ? 0u : q_fill + 1u;
    };
    if constexpr (kRingLoad) {
      for (int j = 0; j < ring_d; ++j) ring_fill(pc.start + VN * threadIdx.x + (uint32_t)j * vstep);
    }
    for (uint32_t l0 = pc.start + VN * threadIdx.x; l0 < end; l0 += vstep) {
      Real ys[NC][VN];
      if constexpr (kRingLoad) {
        // the slot filled now is the one read in the previous iteration (kStateRingDepth + 1 slots)
        ring_fill(l0 + (uint32_t)ring_d * vstep);
        cp_async_wait_pending<ring_d>();
#pragma unroll
        for (int c = 0; c < NC; ++c) {
          const float2 t = *reinterpret_cast<const float2*>(ring + (((size_t)q_read * NC + c) * blockDim.x + threadIdx.x) * 2);
          ys[c][0] = t.x;
          ys[c][1] = t.y;
        }
        q_read = q_read + 1u == ring_slots ? 0u : q_read + 1u;
      } else if constexpr (kPrefetch) {
#pragma unroll
        for (int c = 0; c < NC; ++c)
#pragma unroll
          for (int v = 0; v < VN; ++v) ys[c][v] = nxt[c][v];
        if (l0 + vstep < end) {
#pragma unroll
          for (int c = 0; c < NC; ++c) vload_at(p, kSpanPlanes, ysrc + (size_t)c * p.plane_stride + l0 + vstep, nxt[c], 2);
        }
      } else {
#pragma unroll
        for (int c = 0; c < NC; ++c) vload_at(p, kSpanPlanes, ysrc + (size_t)c * p.plane_stride + l0, ys[c], 3);
      }
      Real ep[NC + 1][VN];
      if constexpr (kSplitLoad) {
#pragma unroll
        for (int c = 0; c <= NC; ++c) vload_at(p, kSpanEscr, escr + (size_t)c * p.plane_stride + l0, ep[c], 4);
      }
      int jj = (int)fast_div(l0, ic.div_magic);
      int k = (int)l0 - jj * ne;
      bool paired = false;
      if constexpr (kPair) {
        // both beams in the same angle bin (all but the rare pair that straddles two bins)
        if (l0 + 1 < end && k + 1 < ne &&
            beam_in_bounds<Body, NC, Real>(p, et, ne, k, jj - (int)pc.jj_lo, n_jj, nullptr) &&
            beam_in_bounds<Body, NC, Real>(p, et, ne, k + 1, jj - (int)pc.jj_lo, n_jj, nullptr)) {
          paired = true;
          const int sigma = jj >= na ? 1 : 0;
          const int tj = jj - (int)pc.jj_lo;
          typename Phys2<float>::Beam b0, b1;
          load_beam<float>(et, ne, sigma, k, dut[tj], b0);
          load_beam<float>(et, ne, sigma, k + 1, dut[tj], b1);
          F2 y2[3], ep2[4];
#pragma unroll
          for (int c = 0; c < 3; ++c) y2[c] = pk(ys[c][0], ys[c][1]);
          if constexpr (kSplitLoad) {
#pragma unroll
            for (int c = 0; c < 4; ++c) ep2[c] = pk(ep[c][0], ep[c][1]);
          }
          const F2* rows = reinterpret_cast<const F2*>(tab) + (size_t)tj * (Phys::KT / 2);
          PairRK<Phys, Tab, kPass, kKind>::run(bs, pk(b0.eo, b1.eo), pk(b0.w, b1.w), rows,
                                         n_jj * (Phys::KT / 2), y2, ep2, acc2, emax2, bad);
#pragma unroll
          for (int c = 0; c < 3; ++c) upk(y2[c], ys[c][0], ys[c][1]);
          if constexpr (kSplitStore) {
#pragma unroll
            for (int c = 0; c < 4; ++c) upk(ep2[c], ep[c][0], ep[c][1]);
          }
        }
      }
      if (!paired) {
#pragma unroll
        for (int v = 0; v < VN; ++v) {
          if (l0 + v < end &&
              beam_in_bounds<Body, NC, Real>(p, et, ne, k, jj - (int)pc.jj_lo, n_jj,
                                             Body::kStore ? kst + l0 + v : nullptr)) {
            const int sigma = jj >= na ? 1 : 0;
            const int tj = jj - (int)pc.jj_lo;
            typename Phys::Beam bm;
            load_beam<Real>(et, ne, sigma, k, dut[tj], bm);
            Real y[NC], ev[NC + 1];
#pragma unroll
            for (int c = 0; c < NC; ++c) y[c] = ys[c][v];
            if constexpr (kSplitLoad) {
#pragma unroll
              for (int c = 0; c <= NC; ++c) ev[c] = ep[c][v];
            }
            if constexpr (kPair) {
              PairHalfAcc<NM> hacc{acc2};
              Body::beam(bs, bm, tv, tj, y, ev, hacc, emax, bad, mixed, nullptr, p.plane_stride);
            } else {
              Body::beam(bs, bm, tv, tj, y, ev, acc, emax, bad, mixed, Body::kStore ? kst + l0 + v : nullptr,
                         p.plane_stride);
            }
#pragma unroll
            for (int c = 0; c < NC; ++c) ys[c][v] = y[c];
            if constexpr (kSplitStore) {
#pragma unroll
              for (int c = 0; c <= NC; ++c) ep[c][v] = ev[c];
            }
          }
          if (++k == ne) { k = 0; ++jj; }
        }
      }
      if constexpr (kKind == kFinalPass && !kSplitLoad) {
#pragma unroll
        for (int c = 0; c < NC; ++c) vstore_at(p, kSpanPlanes, yout + (size_t)c * p.plane_stride + l0, ys[c], 5);
      }
      if constexpr (kSplitStore) {
#pragma unroll
        for (int c = 0; c < NC; ++c) vstore_at(p, kSpanPlanes, yout + (size_t)c * p.plane_stride + l0, ys[c], 6);
#pragma unroll
        for (int c = 0; c <= NC; ++c) vstore_at(p, kSpanEscr, escr + (size_t)c * p.plane_stride + l0, ep[c], 7);
      }
    }
    if constexpr (kRingLoad) cp_async_wait_pending<0>();  // nothing in flight into the ring after the piece
    if constexpr (kPair) emax = fmax(emax, (Real)emax2);
    // the pass forming Y_S also checked the step's input state (non-finite: fatal)
    if constexpr (kSplitStore) {
      const int any_bad = __syncthreads_or(bad);
      if (any_bad && threadIdx.x == 0) atomicExch(&p.nonfinite[pc.inst], 1);
    }
    // reduce this piece into the instance accumulators: the error maximum (final pass of an
    // adaptive tableau) and the moments (every pass but a final one without moments); a
    // non-finite moment rejects an adaptive trial step and is fatal for a fixed step
    constexpr bool kErrMax = kKind == kFinalPass && Tab::kAdaptive;
    constexpr bool kMoments = kKind != kFinalPass || Tab::kFinalMoments;
    constexpr bool kRejectOverflow = Tab::kAdaptive;
    if constexpr (sizeof(Real) == 4) {
      // mixed precision: each thread's (hi, lo) partial sums go to integers of the instance's
      // acc_unit; the warp shuffle trees, the sum over warps and the accumulator atomics are
      // integer additions (exact, order-free).  A thread or block partial of 2^52 units or more
      // (only a runaway or non-finite state reaches it) rejects an adaptive trial step and is
      // fatal for a fixed step.  The error maximum is a max (exact); the square root of the
      // block's maximum is taken in double.
      const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
      float* redf = reinterpret_cast<float*>(red);
      if constexpr (kErrMax) {
        float em = (emax <= 3.0e38f) ? (float)emax : INFINITY;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) em = fmaxf(em, __shfl_down_sync(0xffffffffu, em, o));
        if (lane == 0) redf[warp] = em;
        const int any_bad = __syncthreads_or(bad);
        if (threadIdx.x == 0) {
          float m = 0.0f;
          for (int w = 0; w < nw; ++w) m = fmaxf(m, redf[w]);
          if (any_bad) atomicExch(&p.nonfinite[pc.inst], 1);
          // the beams gave squared error ratios
          atomicMax(&p.errmax[pc.inst], (unsigned long long)__double_as_longlong(sqrt((double)m)));
        }
      }
      if constexpr (kMoments) {
        if constexpr (kErrMax) __syncthreads();              // the scratch is reused
        long long* redl = reinterpret_cast<long long*>(red);  // [warp][NM]
        int ovf = 0;
#pragma unroll
        for (int i = 0; i < NM; ++i) {
          // the thread's partial (pair halves and scalar accumulator joined by TwoSum), then a warp
          // shuffle tree on the (hi, lo) pairs, each step a TwoSum with the error added to lo
          // (lo's FP32 additions round near 2^-48 of the partial), and lane 0 turns the warp's
          // pair into integers of 2^-S units
          float hi, lo;
          if constexpr (kPair) {
            float b, lb;
            upk(acc2.hi[i], hi, b);
            upk(acc2.lo[i], lo, lb);
            two_sum_acc(hi, lo, b);
            lo = __fadd_rn(lo, lb);
          } else {
            hi = acc.hi[i];
            lo = acc.lo[i];
          }
          long long v = f32_to_fix(hi, ovf) + f32_to_fix(lo, ovf);
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
          if (lane == 0) redl[warp * NM + i] = v;
        }
        const int any_ovf = __syncthreads_or(ovf);
        if (threadIdx.x < NM) {
          long long v = 0;
          for (int w = 0; w < nw; ++w) v += redl[w * NM + threadIdx.x];
          unsigned long long* a = p.acc + (size_t)pc.inst * kAccWordsPerInst +
                                  (((size_t)slot * kAccCopies + blockIdx.x % kAccCopies) * kNMMax + threadIdx.x) * 2;
          if (!any_ovf && v < kFixLimit && v > -kFixLimit) {
            atomicAdd(a, (unsigned long long)v);
          } else if (kRejectOverflow) {
            atomicMax(&p.errmax[pc.inst], 0x7ff0000000000000ull);   // overflowing trial step
          } else {
            atomicExch(&p.nonfinite[pc.inst], 1);
          }
        }
      }
    } else {
      if constexpr (kErrMax) {
        const double em = (emax <= rbig<Real>()) ? (double)emax : __longlong_as_double(0x7ff0000000000000ll);
        const int any_bad = __syncthreads_or(bad);
        const double bmax = block_max(em, red);
        if (threadIdx.x == 0) {
          if (any_bad) atomicExch(&p.nonfinite[pc.inst], 1);
          // the beams gave squared error ratios
          atomicMax(&p.errmax[pc.inst], (unsigned long long)__double_as_longlong(sqrt(bmax)));
        }
      }
      if constexpr (kMoments) {
        double v[NM];
#pragma unroll
        for (int i = 0; i < NM; ++i) v[i] = acc.v[i];
        block_sum<NM>(v, red);
        if (threadIdx.x == 0) {
          bool fin = true;
#pragma unroll
          for (int i = 0; i < NM; ++i) { bs.fx[i] = v[i]; fin = fin && (fabs(v[i]) <= 1.7e308); }
          bs.flag = fin ? 1 : 0;
          if (!fin) {
            if (kRejectOverflow)
              atomicMax(&p.errmax[pc.inst], 0x7ff0000000000000ull);
            else
              atomicExch(&p.nonfinite[pc.inst], 1);
          }
        }
        __syncthreads();
        if (bs.flag && threadIdx.x < NM) {
          unsigned long long* a = p.acc + (size_t)pc.inst * kAccWordsPerInst +
                                  (((size_t)slot * kAccCopies + blockIdx.x % kAccCopies) * kNMMax + threadIdx.x) * 2;
          fx_add(a, bs.fx[threadIdx.x]);
        }
      }
    }
  }
}

template <class Phys, class Tab, typename Real, bool kCF, int kPass>
__device__ __forceinline__ bool pass_and_sync(const KParams& p, BlockShared<Real, Phys>& bs,
                                              unsigned char* dyn_smem) {
  constexpr bool kFinal = kPass == Tab::kPasses - 1;
  constexpr int kKind = kFinal ? kFinalPass : kStagePass;
  unsigned long long t0 = 0, t1 = 0;
  if (p.trace && threadIdx.x == 0) t0 = globaltimer_ns();
  run_pass<Phys, Tab, Real, kCF, kPass, kKind>(p, bs, dyn_smem);
  if (p.trace && threadIdx.x == 0) t1 = globaltimer_ns();
  const int res = barrier_arrive(p.bar, gridDim.x, p.timeout_ns, p.status, &bs.flag, &bs.gen_seen);
  if ((res & 0xf) == kBarAbort) return false;
  if (p.trace && threadIdx.x == 0) {
    const int idx = bs.pass_idx++;
    if (idx < p.trace_passes) {
      unsigned long long* t = p.trace + ((size_t)idx * gridDim.x + blockIdx.x) * 4;
      t[0] = t0;
      t[1] = t1;
      t[2] = globaltimer_ns();
      t[3] = (res & 0xf) == kBarLast ? 1ull : 0ull;
    }
  }
  if ((res & 0xf) == kBarLast && p.dyn_sched && threadIdx.x == 0)
    p.bar->chunk[((bs.gen_seen >> 1) + 1u) & 1u] = 0u;   // the next pass's piece counter (released below)
  if ((res & 0xf) == kBarLast && !kFinal) {
    // stage pass: every block derives the new stage's constants from the accumulators in its next
    // set-up (run_pass), so the barrier opens at once (a non-finite partial is reported by the
    // final pass's serial update)
    if (threadIdx.x == 0) bs.flag = 0;
    barrier_release(p.bar, 0, &bs.gen_seen);
    if (p.trace && threadIdx.x == 0 && bs.pass_idx - 1 < p.trace_passes)
      p.trace[((size_t)(bs.pass_idx - 1) * gridDim.x + blockIdx.x) * 4 + 3] = globaltimer_ns() | (1ull << 63);
  } else if ((res & 0xf) == kBarLast) {
    const int mine = serial_update<Phys, Tab, Real>(p, 0, true, false);
    const int all = __syncthreads_and(mine);
    clear_late_slots<Tab>(p);
    serial_geometry<Tab>(p);
    if (threadIdx.x == 0) {
      *p.all_done = all;
      bs.flag = all ? 0x10 : 0;
    }
    unsigned long long ts = 0;
    if (p.trace && threadIdx.x == 0) ts = globaltimer_ns();
    barrier_release(p.bar, all, &bs.gen_seen);
    if (p.trace && threadIdx.x == 0 && bs.pass_idx - 1 < p.trace_passes) {
      // last block: stamp 3 = serial work done (bits 0..62), stamp 2 stays its arrival
      p.trace[((size_t)(bs.pass_idx - 1) * gridDim.x + blockIdx.x) * 4 + 3] = ts | (1ull << 63);
    }
  }
  return true;
}

template <class Phys, class Tab, typename Real, bool kCF, int kPass>
__device__ __forceinline__ bool all_passes(const KParams& p, BlockShared<Real, Phys>& bs,
                                           unsigned char* dyn_smem) {
  if constexpr (kPass < Tab::kPasses) {
    if (!pass_and_sync<Phys, Tab, Real, kCF, kPass>(p, bs, dyn_smem)) return false;
    return all_passes<Phys, Tab, Real, kCF, kPass + 1>(p, bs, dyn_smem);
  } else {
    return true;
  }
}

// Beam-shard mode: the beam work of one pass chosen at run time (no barrier, no serial section).
template <class Phys, class Tab, typename Real, bool kCF, int kPass>
__device__ __forceinline__ void one_pass(const KParams& p, BlockShared<Real, Phys>& bs, unsigned char* dyn_smem,
                                         int which) {
  if constexpr (kPass < Tab::kPasses) {
    if (which == kPass) {
      constexpr int kKind = kPass == Tab::kPasses - 1 ? kFinalPass : kStagePass;
      run_pass<Phys, Tab, Real, kCF, kPass, kKind>(p, bs, dyn_smem);
      return;
    }
    one_pass<Phys, Tab, Real, kCF, kPass + 1>(p, bs, dyn_smem, which);
  }
}

// kThreads x kMinB: the block size and resident blocks per SM the register budget is sized for.
// FP64 work runs on GB300's narrow FP64 pipe (about 1/68 of the FP32 rate), which one 256-thread
// block per SM already keeps busy, so FP64 kernels are built for that (whole register file, no
// spills).  The FP32 two-flavour kernels are latency-bound; they are built for 768 resident threads
// per SM (256 x 3) and for 512 (256 x 2, or one 512-thread block: the SM's two halves of the work
// then finish together instead of the older block's warps finishing first), and the launch shape
// is chosen by measurement (the autotuner in paper_1912_10596_gb300/autotune.py).
template <class Phys, class Tab, typename Real, bool kCF, int kMinB, int kThreads = 256>
__global__ void __launch_bounds__(kThreads, kMinB) step_kernel(KParams p) {
  extern __shared__ __align__(16) unsigned char dyn_smem[];
  __shared__ BlockShared<Real, Phys> bs;
  if (threadIdx.x == 0) {
    bs.pass_idx = 0;
    bs.keep = 0;
    bs.gen_seen = ld_acquire(&p.bar->gen);        // later barriers track the generation locally
  }
  if (p.shard_mode == kShardPass) {
    if (p.shard_pass < 0) run_pass<Phys, Tab, Real, kCF, 0, kInitPass>(p, bs, dyn_smem);
    else one_pass<Phys, Tab, Real, kCF, 0>(p, bs, dyn_smem, p.shard_pass);
    return;
  }
  if (p.shard_mode == kShardSerialInit || p.shard_mode == kShardSerialFinal) {
    // one block; the host has replaced the pass's partial sums by the totals over all shards
    if (blockIdx.x != 0) return;
    const bool init = p.shard_mode == kShardSerialInit;
    const int mine = serial_update<Phys, Tab, Real>(p, init ? 1 : 0, !init, init);
    const int all = __syncthreads_and(mine);
    if (!init) clear_late_slots<Tab>(p);
    serial_geometry<Tab>(p);
    if (threadIdx.x == 0) *p.all_done = all;
    return;
  }
  if (p.init_only) {
    run_pass<Phys, Tab, Real, kCF, 0, kInitPass>(p, bs, dyn_smem);
    const int res = barrier_arrive(p.bar, gridDim.x, p.timeout_ns, p.status, &bs.flag, &bs.gen_seen);
    if ((res & 0xf) == kBarLast) {
      if (p.dyn_sched && threadIdx.x == 0) p.bar->chunk[((bs.gen_seen >> 1) + 1u) & 1u] = 0u;
      const int mine = serial_update<Phys, Tab, Real>(p, 1, false, true);
      const int all = __syncthreads_and(mine);
      serial_geometry<Tab>(p);
      if (threadIdx.x == 0) *p.all_done = all;
      barrier_release(p.bar, 0, &bs.gen_seen);
    }
    return;
  }
  for (int step = 0; step < p.n_steps; ++step) {
    if (!all_passes<Phys, Tab, Real, kCF, 0>(p, bs, dyn_smem)) return;
    // the release of the final pass carried "every instance finished" in bit 4 of bs.flag
    if (bs.flag & 0x10) return;
  }
}

}  // namespace xflat
