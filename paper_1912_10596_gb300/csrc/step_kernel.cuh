// Persistent radial-step kernel of the bulb model (arXiv:1912.10596, Sec. 2 and Sec. 3.4).
//
// One cooperative launch advances every active instance by up to n_steps radial steps.  A step is a
// sequence of passes over all beams separated by device-wide barriers, because every stage of the
// integrator needs the two angular moments of *all* beams (Eq. Hnu / Eq. F):
//
//   pass p (p = 0 .. S-2): rebuild the stage state Y_{p+2} of every beam from the step's initial
//       state y and the stage constants of the earlier stages (the stage derivatives k_1..k_{p+1}
//       are recomputed in registers instead of being stored), and reduce the moments of Y_{p+2};
//   final pass: rebuild the chain once more, form the new state (and, for DP45, the embedded error),
//       write it to the second state buffer and reduce either the moments of the new state (fixed
//       step) or the error norm (DP45).
//
// So every pass reads each beam's state once (128-bit vector loads of the SoA planes) and a step
// writes it once: the algorithmic traffic of a streaming stage update.
//
// Moments.  Each thread accumulates its beams' contributions (working precision), each block
// reduces them with a fixed shuffle/shared-memory tree in double, and each block adds its double
// partial to the instance accumulator as a 128-bit fixed-point integer.  Integer addition is
// associative, so the grid-level sum is exact to 2^-64 and identical whatever order the blocks
// arrive in.  The last block to arrive at the barrier converts the accumulators, derives the stage
// constants mu(r_s) j0, mu(r_s) j1, lambda(r_s) and runs the step-size controller in double.
#pragma once

#include "xflat_internal.cuh"

namespace xflat {

// --------------------------------------------------------------------------------------------
// Butcher tableaus (1-based stage indices).
struct TabRK4 {
  static constexpr int S = 4;
  static constexpr int kPasses = 4;
  static constexpr bool kAdaptive = false;
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
  static constexpr int S = 7;
  static constexpr int kPasses = 7;
  static constexpr bool kAdaptive = true;
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
  static constexpr int S = 4;
  static constexpr int kPasses = 4;
  static constexpr bool kAdaptive = false;
  __host__ __device__ static constexpr double c(int i) { return TabRK4::c(i); }
};

// Largest finite value of the working precision.
template <typename Real>
__host__ __device__ constexpr Real rbig() { return sizeof(Real) == 4 ? Real(3.0e38) : Real(1.7e308); }

// --------------------------------------------------------------------------------------------
// Physics policies.  "Real" is the working precision of the per-beam algebra.
//
// Two flavours: the state of a beam is the Bloch vector s of P = (1 + s.sigma)/2 (antineutrinos:
// of conj(Pbar), so that every beam obeys ds/dr = K x s with
//   K = [eta omega_k B + lambda(r) z + mu(r) (j0 - cos(th) j1)] / cos(th),
// eta = +1 / -1 for nu / nubar, B = (sin 2 theta_v, 0, -cos 2 theta_v)), which is
// d(rho)/dr = -i [H, rho] / cos(th) of Eq. eom with H = (1/2) h.sigma.
template <typename Real>
struct Phys2 {
  static constexpr int NC = 3, NM = kNM2, NSC = kNSC2;
  struct Consts { Real B[3]; };
  struct Beam { Real eo; Real w; };   // eta*omega_k, signed weight du_j * g_{sigma,k}

  // stage constant block (Real): m0[3], m1[3], lam
  __device__ static inline void K(const Consts& C, const Beam& bm, const Real* sc, Real q, Real c,
                                  Real (&Kv)[3]) {
    Kv[0] = (bm.eo * C.B[0] + sc[0]) * q - sc[3];
    Kv[1] = sc[1] * q - sc[4];
    Kv[2] = (bm.eo * C.B[2] + sc[6] + sc[2]) * q - sc[5];
  }
  __device__ static inline void f(const Real (&Kv)[3], const Real (&y)[3], Real (&k)[3]) {
    k[0] = Kv[1] * y[2] - Kv[2] * y[1];
    k[1] = Kv[2] * y[0] - Kv[0] * y[2];
    k[2] = Kv[0] * y[1] - Kv[1] * y[0];
  }
  __device__ static inline void accum(Real (&acc)[NM], Real w, Real q, const Real (&y)[3]) {
    const Real wq = w * q;
#pragma unroll
    for (int i = 0; i < 3; ++i) { acc[i] += wq * y[i]; acc[3 + i] += w * y[i]; }
  }
  // Frobenius norm^2 of the traceless part of P = (1 + s.sigma)/2: |s|^2 / 2
  __device__ static inline Real tnorm2(const Real (&y)[3]) {
    return Real(0.5) * (y[0] * y[0] + y[1] * y[1] + y[2] * y[2]);
  }
  // Frobenius norm of a traceless matrix e = (e.sigma)/2 given by its Bloch vector, computed with a
  // scale so that it cannot overflow; +inf if a component is not finite
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
};

// Three flavours: the state is the full 3x3 Hermitian density matrix (9 reals: P00, P11, P22,
// Re P01, Im P01, Re P02, Im P02, Re P12, Im P12) of P (nu) or conj(Pbar) (nubar); the derivative
// is -i [K, P] with the Hermitian K = [eta (omega21 M21 + omega31 M31) + lambda E_ee + mu (J0 - cos J1)]
// / cos(th), M21/M31 the real unit vacuum matrices U diag(0,1,0) U^T and U diag(0,0,1) U^T.
template <typename Real>
struct Phys3 {
  static constexpr int NC = 9, NM = kNM3, NSC = kNSC3;
  struct Consts { Real M21[6], M31[6]; };
  struct Beam { Real o21, o31; Real w; };

  // stage constants: m0[9], m1[9], lam
  __device__ static inline void K(const Consts& C, const Beam& bm, const Real* sc, Real q, Real c,
                                  Real (&Kv)[9]) {
    // vacuum part (real symmetric): order 00,11,22,01,02,12
    const Real v00 = bm.o21 * C.M21[0] + bm.o31 * C.M31[0];
    const Real v11 = bm.o21 * C.M21[1] + bm.o31 * C.M31[1];
    const Real v22 = bm.o21 * C.M21[2] + bm.o31 * C.M31[2];
    const Real v01 = bm.o21 * C.M21[3] + bm.o31 * C.M31[3];
    const Real v02 = bm.o21 * C.M21[4] + bm.o31 * C.M31[4];
    const Real v12 = bm.o21 * C.M21[5] + bm.o31 * C.M31[5];
    Kv[0] = (v00 + sc[18] + sc[0]) * q - sc[9];
    Kv[1] = (v11 + sc[1]) * q - sc[10];
    Kv[2] = (v22 + sc[2]) * q - sc[11];
    Kv[3] = (v01 + sc[3]) * q - sc[12];
    Kv[4] = sc[4] * q - sc[13];
    Kv[5] = (v02 + sc[5]) * q - sc[14];
    Kv[6] = sc[6] * q - sc[15];
    Kv[7] = (v12 + sc[7]) * q - sc[16];
    Kv[8] = sc[8] * q - sc[17];
  }
  // Z = -i [K, Y] for Hermitian K, Y; A = K Y, Z_aa = 2 Im A_aa, Z_ab = -i (A_ab - conj(A_ba)).
  __device__ static inline void f(const Real (&Kv)[9], const Real (&y)[9], Real (&z)[9]) {
    // complex entries: K_ab = kr[a][b] + i ki[a][b]
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
    // Z_ab = -i (A_ab - conj(A_ba)) = (ai_ab + ai_ba) + i (-(ar_ab - ar_ba))
    z[3] = ai[0][1] + ai[1][0];
    z[4] = ar[1][0] - ar[0][1];
    z[5] = ai[0][2] + ai[2][0];
    z[6] = ar[2][0] - ar[0][2];
    z[7] = ai[1][2] + ai[2][1];
    z[8] = ar[2][1] - ar[1][2];
  }
  __device__ static inline void accum(Real (&acc)[NM], Real w, Real q, const Real (&y)[9]) {
    const Real wq = w * q;
#pragma unroll
    for (int i = 0; i < 9; ++i) { acc[i] += wq * y[i]; acc[9 + i] += w * y[i]; }
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
  int max_jj;
  int integrator;
};

__device__ __forceinline__ void fx_add(unsigned long long* acc2, double x) {
  const double hi_d = floor(x);
  const double frac = x - hi_d;                                   // exact, in [0, 1)
  const unsigned long long lo = (unsigned long long)(frac * 18446744073709551616.0);
  const long long hi = (long long)hi_d;
  const unsigned long long old = atomicAdd(&acc2[0], lo);
  const unsigned long long carry = (old + lo < old) ? 1ull : 0ull;
  atomicAdd(&acc2[1], (unsigned long long)hi + carry);
}

__device__ __forceinline__ double fx_read(const unsigned long long* acc2) {
  const long long hi = (long long)acc2[1];
  return (double)hi + (double)acc2[0] * 5.421010862427522e-20;   // 2^-64
}

template <class Tab>
__device__ __forceinline__ double stage_c(int i) { return Tab::c(i); }

// Per-block shared state for the piece being processed.
template <typename Real, int NSC>
struct PieceShared {
  Real sc[kMaxStages][NSC];      // stage constants in working precision
  Real hA[kMaxStages][kMaxStages];
  Real hB[kMaxStages];
  Real hE[kMaxStages];
  Real cB[3];                    // unused for 3 flavours
  int inst;
  int active;
};

// ------------------------------------------------------------------------------------------
// The last block to arrive: reduce accumulators, derive stage constants, run the controller.
template <class Phys, class Tab>
__device__ void serial_update(const KParams& p, int slot, bool final_pass, bool init) {
  constexpr int NM = Phys::NM;
  constexpr int NCOMP = NM / 2;
  for (int i = threadIdx.x; i < p.n_inst; i += blockDim.x) {
    const InstConst& ic = p.ic[i];
    InstDyn& d = p.dyn[i];
    if (d.done || d.status) continue;
    unsigned long long* acc = p.acc + ((size_t)i * kMaxStages + slot) * kNMMax * 2;
    if (p.nonfinite[i]) {
      d.status = 5;  // XFLAT_ERR_NONFINITE
      atomicCAS(p.status, 0, 5);
      continue;
    }
    const bool have_moments = !(final_pass && Tab::kAdaptive);
    if (have_moments) {
      double m[NM];
      for (int c = 0; c < NM; ++c) {
        m[c] = fx_read(acc + 2 * c);
        acc[2 * c] = 0ull;
        acc[2 * c + 1] = 0ull;
      }
      const double r = d.rs[slot];
      const double mu = ic.mu_coef / (r * r);
      double lam = 0.0;
      if (ic.matter == kMatterPower) lam = ic.lam_coef * pow(ic.r_ref / r, ic.power);
      for (int c = 0; c < NM; ++c) d.mom[slot][c] = m[c];
      for (int c = 0; c < NCOMP; ++c) {
        d.sc[slot][c] = mu * m[c];
        d.sc[slot][NCOMP + c] = mu * m[NCOMP + c];
      }
      d.sc[slot][NM] = ic.matter == kMatterConst ? ic.lam_const : lam;
    }
    if (!final_pass && !init) continue;
    // ---- step bookkeeping ---------------------------------------------------------------
    if (init) {
      d.stage_evals += Tab::kAdaptive ? 1ull : 0ull;
    } else if (!Tab::kAdaptive) {
      d.parity ^= 1;
      d.accepted += 1;
      d.stage_evals += 4;
      d.n_fixed += 1;
      d.r = (d.n_fixed >= d.n_fixed_total) ? d.r_end : d.r0_fixed + (double)d.n_fixed * d.h_fixed;
      if (d.n_fixed >= d.n_fixed_total) d.done = 1;
      // the final pass reduced the new state's moments at r + h (= stage S radius): stage 1 of
      // the next step
      for (int c = 0; c < NM; ++c) d.mom[1][c] = d.mom[slot][c];
      for (int c = 0; c < Phys::NSC; ++c) d.sc[1][c] = d.sc[slot][c];
    } else {
      const double err = __longlong_as_double((long long)p.errmax[i]);
      p.errmax[i] = 0ull;
      d.err = err;
      d.stage_evals += 6;
      const bool ok = err <= 1.0;
      double fac;
      if (ok) {
        d.r = d.last ? d.r_end : d.r + d.h;
        d.parity ^= 1;
        d.accepted += 1;
        for (int c = 0; c < NM; ++c) d.mom[1][c] = d.mom[7][c];
        for (int c = 0; c < Phys::NSC; ++c) d.sc[1][c] = d.sc[7][c];
        fac = err == 0.0 ? 5.0 : fmin(5.0, fmax(0.2, 0.9 * pow(err, -0.2)));
        if (d.last) d.done = 1;
      } else {
        d.rejected += 1;
        fac = fmax(0.2, 0.9 * pow(err, -0.2));
      }
      d.h = fmin(d.h * fac, ic.h_max);
      if (!d.done && d.h < ic.h_min) {
        d.status = 6;  // XFLAT_ERR_STEP
        atomicCAS(p.status, 0, 6);
        continue;
      }
    }
    if (d.done) continue;
    // ---- geometry of the next step ------------------------------------------------------
    double h;
    if (Tab::kAdaptive) {
      d.last = (d.r + d.h >= d.r_end) ? 1 : 0;
      if (d.last) d.h = d.r_end - d.r;
      h = d.h;
    } else {
      h = d.h_fixed;
    }
    for (int s = 1; s <= Tab::S; ++s) {
      const double rs = (s == 1) ? d.r : __dadd_rn(d.r, __dmul_rn(stage_c<Tab>(s), h));
      d.rs[s] = rs;
      d.xs[s] = ic.R2 / (rs * rs);
    }
  }
}


// ------------------------------------------------------------------------------------------
// Loads that must not hit a stale L1 line: instance dynamics change across barriers.
__device__ __forceinline__ double ldcg(const double* p) { return __ldcg(p); }
__device__ __forceinline__ int ldcg(const int* p) { return __ldcg(p); }

template <typename Real> struct Vec16;
template <> struct Vec16<float> { using T = float4; static constexpr int N = 4; };
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

// Shared-memory view of one piece.
template <typename Real, class Phys>
struct PieceView {
  const Real* cq;       // [kMaxStages][n_jj][2]: cos(theta), 1/cos(theta) at each stage radius
  const Real* dut;      // [n_jj] du_j
  int n_jj;
  __device__ __forceinline__ Real c(int s, int jj) const { return cq[(s * n_jj + jj) * 2]; }
  __device__ __forceinline__ Real q(int s, int jj) const { return cq[(s * n_jj + jj) * 2 + 1]; }
};

// What a pass does (compile time).
enum PassKind : int { kStagePass = 0, kFinalPass = 1, kInitPass = 2 };

template <class Phys, class Tab, typename Real, bool kCF, int kPass, int kKind>
struct PassBody;

// Commutator-form Runge-Kutta (RK4 / DP45) ------------------------------------------------------
template <class Phys, class Tab, typename Real, int kPass, int kKind>
struct PassBody<Phys, Tab, Real, false, kPass, kKind> {
  static constexpr int NC = Phys::NC;
  // number of stage derivatives to rebuild before the stage state of this pass
  static constexpr int kChain = kKind == kInitPass ? 0 : (kKind == kFinalPass ? Tab::S - (Tab::kAdaptive ? 1 : 0) : kPass + 1);
  template <class PS>
  __device__ static inline void beam(const PS& ps, const typename Phys::Consts& C, const typename Phys::Beam& bm,
                                     const PieceView<Real, Phys>& pv, int jj, Real (&y)[NC],
                                     Real (&acc)[Phys::NM], Real& emax, int& bad, bool mixed) {
    Real k[Tab::S + 1][NC];
#pragma unroll
    for (int l = 1; l <= kChain; ++l) {
      Real Y[NC];
#pragma unroll
      for (int i = 0; i < NC; ++i) {
        Real v = y[i];
#pragma unroll
        for (int m = 1; m < l; ++m)
          if (Tab::a(l, m) != 0.0) v += ps.hA[l][m] * k[m][i];
        Y[i] = v;
      }
      Real Kv[NC];
      Phys::K(C, bm, ps.sc[l], pv.q(l, jj), pv.c(l, jj), Kv);
      Phys::f(Kv, Y, k[l]);
    }
    if (kKind == kInitPass) {
      Phys::accum(acc, bm.w, pv.q(1, jj), y);
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
          if (Tab::a(I, m) != 0.0) v += ps.hA[I][m] * k[m][i];
        Y[i] = v;
      }
      if (Tab::kAdaptive && I == Tab::S && mixed) Phys::normalise(Y);
      Phys::accum(acc, bm.w, pv.q(I, jj), Y);
      return;
    }
    // final pass
    Real yn[NC];
#pragma unroll
    for (int i = 0; i < NC; ++i) {
      Real v = y[i];
#pragma unroll
      for (int m = 1; m <= kChain; ++m)
        if (Tab::b(m) != 0.0) v += ps.hB[m] * k[m][i];
      yn[i] = v;
    }
    const Real yn2 = Phys::tnorm2(yn);
    const bool ynok = yn2 <= rbig<Real>();
    if (mixed && ynok) Phys::normalise(yn);
    if (Tab::kAdaptive) {
      if (!(Phys::tnorm2(y) <= rbig<Real>())) bad = 1;     // non-finite input state: fatal
      Real Kv[NC];
      Phys::K(C, bm, ps.sc[Tab::S], pv.q(Tab::S, jj), pv.c(Tab::S, jj), Kv);
      Phys::f(Kv, yn, k[Tab::S]);
      Real e[NC];
#pragma unroll
      for (int i = 0; i < NC; ++i) {
        Real v = 0;
#pragma unroll
        for (int m = 1; m <= Tab::S; ++m)
          if (Tab::e(m) != 0.0) v += ps.hE[m] * k[m][i];
        e[i] = v;
      }
      const Real en = Phys::enorm(e);
      const Real sn = sqrt(fmax(Phys::tnorm2(y), Phys::tnorm2(yn)));
      Real ratio = en / (ps.atol + ps.rtol * sn);
      // a trial step whose stages overflowed the working precision is rejected, not fatal
      if (!(ratio <= rbig<Real>()) || !ynok) ratio = Real(INFINITY);
      emax = fmax(emax, ratio);
    } else {
      Phys::accum(acc, bm.w, pv.q(Tab::S, jj), yn);
    }
#pragma unroll
    for (int i = 0; i < NC; ++i) y[i] = yn[i];
  }
};

// Commutator-free Lie RK4 on Bloch vectors (two flavours) ---------------------------------------
template <class Phys, class Tab, typename Real, int kPass, int kKind>
struct PassBody<Phys, Tab, Real, true, kPass, kKind> {
  static constexpr int NC = 3;
  template <class PS>
  __device__ static inline void beam(const PS& ps, const typename Phys::Consts& C, const typename Phys::Beam& bm,
                                     const PieceView<Real, Phys>& pv, int jj, Real (&y)[NC],
                                     Real (&acc)[Phys::NM], Real& emax, int& bad, bool mixed) {
    if (kKind == kInitPass) {
      Phys::accum(acc, bm.w, pv.q(1, jj), y);
      return;
    }
    const Real h = ps.hB[0];
    Real K1[3], K2[3], K3[3], K4[3], Om[3];
    Phys::K(C, bm, ps.sc[1], pv.q(1, jj), pv.c(1, jj), K1);
    if (kKind == kStagePass && kPass == 0) {
#pragma unroll
      for (int i = 0; i < 3; ++i) Om[i] = Real(0.5) * h * K1[i];
      rotate(Om, y);
      Phys::accum(acc, bm.w, pv.q(2, jj), y);
      return;
    }
    Phys::K(C, bm, ps.sc[2], pv.q(2, jj), pv.c(2, jj), K2);
    if (kKind == kStagePass && kPass == 1) {
#pragma unroll
      for (int i = 0; i < 3; ++i) Om[i] = Real(0.5) * h * K2[i];
      rotate(Om, y);
      Phys::accum(acc, bm.w, pv.q(3, jj), y);
      return;
    }
    Phys::K(C, bm, ps.sc[3], pv.q(3, jj), pv.c(3, jj), K3);
    if (kKind == kStagePass && kPass == 2) {
#pragma unroll
      for (int i = 0; i < 3; ++i) Om[i] = Real(0.5) * h * K1[i];
      rotate(Om, y);
#pragma unroll
      for (int i = 0; i < 3; ++i) Om[i] = h * K3[i] - Real(0.5) * h * K1[i];
      rotate(Om, y);
      Phys::accum(acc, bm.w, pv.q(4, jj), y);
      return;
    }
    Phys::K(C, bm, ps.sc[4], pv.q(4, jj), pv.c(4, jj), K4);
#pragma unroll
    for (int i = 0; i < 3; ++i)
      Om[i] = h * (Real(0.25) * K1[i] + Real(1.0 / 6.0) * (K2[i] + K3[i]) - Real(1.0 / 12.0) * K4[i]);
    rotate(Om, y);
#pragma unroll
    for (int i = 0; i < 3; ++i)
      Om[i] = h * (Real(-1.0 / 12.0) * K1[i] + Real(1.0 / 6.0) * (K2[i] + K3[i]) + Real(0.25) * K4[i]);
    rotate(Om, y);
    if (mixed) Phys::normalise(y);
    Phys::accum(acc, bm.w, pv.q(4, jj), y);
  }
};

// Load the beam constants of (species, j, k).
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

template <typename Real, int NSC>
struct BlockShared {
  Real sc[kMaxStages][NSC];
  Real hA[kMaxStages][kMaxStages];
  Real hB[kMaxStages];
  Real hE[kMaxStages];
  Real Cv[12];
  Real rtol, atol;
  double fx[kNMMax];
  int active;
  int parity;
  int flag;
};

// One pass over all pieces of this block.
template <class Phys, class Tab, typename Real, bool kCF, int kPass, int kKind>
__device__ void run_pass(const KParams& p, BlockShared<Real, Phys::NSC>& bs, unsigned char* dyn_smem) {
  constexpr int NC = Phys::NC, NM = Phys::NM, VN = Vec16<Real>::N;
  using Body = PassBody<Phys, Tab, Real, kCF, kPass, kKind>;
  double* red = reinterpret_cast<double*>(dyn_smem);                 // 32 * NM doubles
  Real* cq = reinterpret_cast<Real*>(red + 32 * kNMMax);             // [kMaxStages][max_jj][2]
  Real* dut = cq + (size_t)kMaxStages * p.max_jj * 2;                 // [max_jj]
  const bool mixed = sizeof(Real) == 4;
  const int slot = kKind == kInitPass ? 1 : (kKind == kStagePass ? kPass + 2 : Tab::S);
  const int b0 = p.blk_piece[blockIdx.x], b1 = p.blk_piece[blockIdx.x + 1];
  for (int pi = b0; pi < b1; ++pi) {
    const Piece pc = p.pieces[pi];
    const InstConst& ic = p.ic[pc.inst];
    const InstDyn* d = p.dyn + pc.inst;
    __syncthreads();
    if (threadIdx.x == 0) {
      bs.active = (ldcg(&d->done) == 0 && ldcg(&d->status) == 0) ? 1 : 0;
      bs.parity = ldcg(&d->parity);
    }
    __syncthreads();
    if (!bs.active) continue;
    // stage constants, step coefficients and geometry tables of this piece
    const double h = Tab::kAdaptive ? ldcg(&d->h) : ldcg(&d->h_fixed);
    for (int t = threadIdx.x; t < kMaxStages * Phys::NSC; t += blockDim.x) {
      const int s = t / Phys::NSC, c = t % Phys::NSC;
      bs.sc[s][c] = (Real)ldcg(&d->sc[s][c]);
    }
    if (threadIdx.x < kMaxStages * kMaxStages) {
      const int i = threadIdx.x / kMaxStages, j = threadIdx.x % kMaxStages;
      if constexpr (!kCF) bs.hA[i][j] = (Real)(h * ((i >= 1 && j >= 1) ? Tab::a(i, j) : 0.0));
    }
    if (threadIdx.x < kMaxStages) {
      const int i = threadIdx.x;
      if constexpr (!kCF) {
        bs.hB[i] = (Real)(h * (i >= 1 ? Tab::b(i) : 0.0));
        bs.hE[i] = (Real)(h * (i >= 1 ? Tab::e(i) : 0.0));
      } else {
        bs.hB[i] = (Real)h;
      }
    }
    if (threadIdx.x == 0) {
      if constexpr (Phys::NC == 3) {
        bs.Cv[0] = (Real)ic.B[0]; bs.Cv[1] = (Real)ic.B[1]; bs.Cv[2] = (Real)ic.B[2];
      } else {
        for (int i = 0; i < 6; ++i) { bs.Cv[i] = (Real)ic.M21[i]; bs.Cv[6 + i] = (Real)ic.M31[i]; }
      }
      bs.rtol = (Real)ic.rtol;
      bs.atol = (Real)ic.atol;
    }
    const int n_jj = pc.n_jj;
    for (int t = threadIdx.x; t < n_jj; t += blockDim.x) {
      const int jj = pc.jj_lo + t;
      const int j = jj >= (int)ic.n_angle ? jj - (int)ic.n_angle : jj;
      dut[t] = (Real)p.du_tab[ic.a_off + j];
    }
    for (int t = threadIdx.x; t < Tab::S * n_jj; t += blockDim.x) {
      const int s = 1 + t / n_jj, tj = t % n_jj;
      const int jj = pc.jj_lo + tj;
      const int j = jj >= (int)ic.n_angle ? jj - (int)ic.n_angle : jj;
      const double c = sqrt(1.0 - p.u_tab[ic.a_off + j] * ldcg(&d->xs[s]));
      cq[(s * n_jj + tj) * 2] = (Real)c;
      cq[(s * n_jj + tj) * 2 + 1] = (Real)(1.0 / c);
    }
    __syncthreads();
    typename Phys::Consts C;
    if constexpr (Phys::NC == 3) {
      C.B[0] = bs.Cv[0]; C.B[1] = bs.Cv[1]; C.B[2] = bs.Cv[2];
    } else {
#pragma unroll
      for (int i = 0; i < 6; ++i) { C.M21[i] = bs.Cv[i]; C.M31[i] = bs.Cv[6 + i]; }
    }
    const PieceView<Real, Phys> pv{cq, dut, n_jj};
    const Real* et = reinterpret_cast<const Real*>(p.etab) + ic.e_off;
    const Real* yin = reinterpret_cast<const Real*>(bs.parity ? p.planeB : p.planeA) + ic.beam_off;
    Real* yout = reinterpret_cast<Real*>(bs.parity ? p.planeA : p.planeB) + ic.beam_off;
    const int ne = (int)ic.n_energy, na = (int)ic.n_angle;
    Real acc[NM];
#pragma unroll
    for (int i = 0; i < NM; ++i) acc[i] = 0;
    Real emax = 0;
    int bad = 0;
    const uint32_t end = pc.start + pc.len;
    for (uint32_t l0 = pc.start + VN * threadIdx.x; l0 < end; l0 += VN * blockDim.x) {
      Real ys[NC][VN];
#pragma unroll
      for (int c = 0; c < NC; ++c) vload(yin + (size_t)c * p.plane_stride + l0, ys[c]);
      int jj = (int)fast_div(l0, ic.div_magic);
      int k = (int)l0 - jj * ne;
#pragma unroll
      for (int v = 0; v < VN; ++v) {
        if (l0 + v < end) {
          const int sigma = jj >= na ? 1 : 0;
          typename Phys::Beam bm;
          load_beam<Real>(et, ne, sigma, k, dut[jj - (int)pc.jj_lo], bm);
          Real y[NC];
#pragma unroll
          for (int c = 0; c < NC; ++c) y[c] = ys[c][v];
          Body::beam(bs, C, bm, pv, jj - (int)pc.jj_lo, y, acc, emax, bad, mixed);
#pragma unroll
          for (int c = 0; c < NC; ++c) ys[c][v] = y[c];
        }
        if (++k == ne) { k = 0; ++jj; }
      }
      if (kKind == kFinalPass) {
#pragma unroll
        for (int c = 0; c < NC; ++c) vstore(yout + (size_t)c * p.plane_stride + l0, ys[c]);
      }
    }
    // reduce this piece into the instance accumulators
    if (kKind == kFinalPass && Tab::kAdaptive) {
      const double em = (emax <= rbig<Real>()) ? (double)emax : __longlong_as_double(0x7ff0000000000000ll);
      const int any_bad = __syncthreads_or(bad);
      const double bmax = block_max(em, red);
      if (threadIdx.x == 0) {
        if (any_bad) atomicExch(&p.nonfinite[pc.inst], 1);
        atomicMax(&p.errmax[pc.inst], (unsigned long long)__double_as_longlong(bmax));
      }
    } else {
      double v[NM];
#pragma unroll
      for (int i = 0; i < NM; ++i) v[i] = (double)acc[i];
      block_sum<NM>(v, red);
      if (threadIdx.x == 0) {
        bool fin = true;
#pragma unroll
        for (int i = 0; i < NM; ++i) { bs.fx[i] = v[i]; fin = fin && (fabs(v[i]) <= 1.7e308); }
        bs.flag = fin ? 1 : 0;
        if (!fin) {
          // adaptive: an overflowing trial step is rejected by the controller; fixed step: fatal
          if (Tab::kAdaptive && kKind == kStagePass)
            atomicMax(&p.errmax[pc.inst], 0x7ff0000000000000ull);
          else
            atomicExch(&p.nonfinite[pc.inst], 1);
        }
      }
      __syncthreads();
      if (bs.flag && threadIdx.x < NM) {
        unsigned long long* a = p.acc + (((size_t)pc.inst * kMaxStages + slot) * kNMMax + threadIdx.x) * 2;
        fx_add(a, bs.fx[threadIdx.x]);
      }
    }
  }
}

template <class Phys, class Tab, typename Real, bool kCF, int kPass>
__device__ __forceinline__ bool pass_and_sync(const KParams& p, BlockShared<Real, Phys::NSC>& bs,
                                              unsigned char* dyn_smem) {
  constexpr bool kFinal = kPass == Tab::kPasses - 1;
  constexpr int kKind = kFinal ? kFinalPass : kStagePass;
  run_pass<Phys, Tab, Real, kCF, kPass, kKind>(p, bs, dyn_smem);
  const bool last = barrier_arrive(p.bar, gridDim.x, p.timeout_ns, p.status, &bs.flag);
  if (last) {
    __threadfence();
    serial_update<Phys, Tab>(p, kFinal ? Tab::S : kPass + 2, kFinal, false);
    __syncthreads();
    if (kFinal && threadIdx.x == 0) {
      int all = 1;
      for (int i = 0; i < p.n_inst; ++i) all &= (p.dyn[i].done || p.dyn[i].status) ? 1 : 0;
      *p.all_done = all;
    }
    barrier_release(p.bar);
  }
  return !barrier_aborted(p.bar, &bs.flag);
}

template <class Phys, class Tab, typename Real, bool kCF, int kPass>
__device__ __forceinline__ bool all_passes(const KParams& p, BlockShared<Real, Phys::NSC>& bs,
                                           unsigned char* dyn_smem) {
  if constexpr (kPass < Tab::kPasses) {
    if (!pass_and_sync<Phys, Tab, Real, kCF, kPass>(p, bs, dyn_smem)) return false;
    return all_passes<Phys, Tab, Real, kCF, kPass + 1>(p, bs, dyn_smem);
  } else {
    return true;
  }
}

template <class Phys, class Tab, typename Real, bool kCF>
__global__ void __launch_bounds__(512) step_kernel(KParams p) {
  extern __shared__ __align__(16) unsigned char dyn_smem[];
  __shared__ BlockShared<Real, Phys::NSC> bs;
  if (p.init_only) {
    run_pass<Phys, Tab, Real, kCF, 0, kInitPass>(p, bs, dyn_smem);
    const bool last = barrier_arrive(p.bar, gridDim.x, p.timeout_ns, p.status, &bs.flag);
    if (last) {
      __threadfence();
      serial_update<Phys, Tab>(p, 1, false, true);
      __syncthreads();
      if (threadIdx.x == 0) {
        int all = 1;
        for (int i = 0; i < p.n_inst; ++i) all &= (p.dyn[i].done || p.dyn[i].status) ? 1 : 0;
        *p.all_done = all;
      }
      barrier_release(p.bar);
    }
    return;
  }
  for (int step = 0; step < p.n_steps; ++step) {
    if (!all_passes<Phys, Tab, Real, kCF, 0>(p, bs, dyn_smem)) return;
    __syncthreads();
    if (threadIdx.x == 0) bs.flag = ldcg(p.all_done);
    __syncthreads();
    if (bs.flag) return;
  }
}

}  // namespace xflat
