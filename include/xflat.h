/*
 * xflat.h -- C ABI of the GB300 bulb-model radial-step solver.
 *
 * The solver advances the flavour density matrices of every neutrino and antineutrino beam of the
 * stationary, spherically symmetric neutrino bulb model (arXiv:1912.10596, Sec. 2):
 *
 *   i cos(theta) d/dr psi     = [H_vac(E) + H_mat(r) + H_nunu(v;r)]   psi        (Eq. eom)
 *   i cos(theta) d/dr psibar  = [H_vac(E) - H_mat(r) - H_nunu^*(v;r)] psibar
 *
 * with H_nunu the angular integral of the flux matrices of all beams (Eq. Hnu, Eq. F), from the
 * initial conditions of Sec. 3.4 (electron flavour (1,0[,0]) at r = R).  A beam is one energy bin
 * (equal-width bins in E) times one emission-angle bin (equal-width bins in u = sin^2 theta_R,
 * Sec. 3.2) times one species (nu, nubar); beams are indexed
 *
 *   b = ((species * n_angle) + j) * n_energy + k,   species 0 = nu, 1 = nubar,
 *
 * energy fastest.  Units: r and R in km, E in MeV, Hamiltonians in 1/km, number luminosities in
 * 1/s.  Every value crossing this boundary is IEEE double, whatever the internal precision.
 *
 * Conventions shared by all entry points
 *  - Every function returns an int status (XFLAT_OK = 0); no C++ exception or abort crosses the ABI.
 *    xflat_last_error() gives a one-line description of the last failure on a handle.
 *  - A handle owns all device memory it allocates; host arrays are caller-owned and copied in or
 *    out during the call; device pointers passed in are borrowed for the duration of the call.
 *  - All device work is enqueued on the CUDA stream given in xflat_config.cuda_stream (NULL = the
 *    legacy default stream); calls that return host data synchronise that stream.
 *  - A handle is not thread-safe: one host thread at a time.
 *  - Requires a GPU of compute capability 10.3 (sm_103a); on anything else xflat_create fails with
 *    XFLAT_ERR_CUDA.  There is no CPU fallback.
 */
#ifndef XFLAT_H
#define XFLAT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define XFLAT_ABI_VERSION 2u

/* ---- status codes ---------------------------------------------------------------------------- */
enum xflat_status {
  XFLAT_OK = 0,
  XFLAT_ERR_INVAL = 1,        /* bad argument (size, range, NULL, layout)                       */
  XFLAT_ERR_NOMEM = 2,        /* a device or host allocation failed                             */
  XFLAT_ERR_CUDA = 3,         /* a CUDA runtime call failed (message in xflat_last_error)       */
  XFLAT_ERR_TIMEOUT = 4,      /* a device-wide barrier exceeded barrier_timeout_ns              */
  XFLAT_ERR_NONFINITE = 5,    /* a NaN or infinity appeared in the state, moments or error norm */
  XFLAT_ERR_STEP = 6,         /* adaptive step size fell below h_min_km                         */
  XFLAT_ERR_STATE = 7,        /* call order violated (e.g. evolve before set_spectra)           */
  XFLAT_ERR_UNSUPPORTED = 8   /* valid request the library does not implement                   */
};

/* ---- configuration enums --------------------------------------------------------------------- */
enum xflat_precision {
  XFLAT_FP64 = 0,             /* every per-beam operation in IEEE double                         */
  XFLAT_MIXED = 1             /* per-beam precession in float, including each beam's moment
                                 contribution w s; the sum of the contributions over beams is
                                 FP64-accurate (per-thread TwoSum pairs, then integer sums across
                                 threads, warps, blocks and the grid: exact and order-free); the
                                 error norm is the exact maximum of the per-beam error ratios with
                                 its square root and the step-size controller in double; |s|
                                 renormalised every step                                          */
};
enum xflat_integrator {
  XFLAT_RK4 = 0,              /* classical 4-stage RK on d(rho)/dr = -i[H,rho]/cos(theta), fixed step */
  XFLAT_DP45 = 1,             /* Dormand-Prince 5(4), FSAL, adaptive (error control below)        */
  XFLAT_LIE_RK4 = 2,          /* commutator-free Lie RK4 whose every update is an exact propagator
                                 exp(-i H dl) of Eq. U (two flavours: the closed form; three: by
                                 the eigen-decomposition of the 3 x 3 generator), fixed step      */
  XFLAT_EXP_MIDPOINT = 3,     /* exponential midpoint rule (Lie-group Runge-Kutta-Munthe-Kaas method
                                 with Runge's midpoint tableau; Sec. 3.4's exact propagator of Eq. U
                                 with a mid-point scheme): y' = exp(-i H(r+h/2, y_half) dl) applied
                                 to y, y_half from an exponential half step; the exponential Euler
                                 step exp(-i H(r, y) dl) is the embedded first-order estimate
                                 (error control as DP45 with the factor 0.9 Err^-1/2); two and
                                 three flavours                                                   */
  XFLAT_LIE_ADAPTIVE = 4      /* adaptive exact propagators: the commutator-free Lie RK4 of
                                 XFLAT_LIE_RK4 with Richardson step-size control -- each attempt
                                 takes one step of h and two of h/2 from the same state, keeps the
                                 two half steps and estimates their error as (y_two - y_full)/15;
                                 error norm, acceptance and controller as DP45 (0.9 Err^-1/5).
                                 Every update is an exact propagator of Eq. U, so the step is set by
                                 how fast the generator changes, not by its size (no explicit
                                 stability limit near R).  11 passes (stage evaluations) per step;
                                 two and three flavours, bulb model (n_phi <= 1)                    */
};
enum xflat_matter {
  XFLAT_MATTER_NONE = 0,
  XFLAT_MATTER_POWER_LAW = 1, /* n_e = Ye rho0 (r_ref/r)^power / m_u                               */
  XFLAT_MATTER_CONSTANT = 2,  /* sqrt(2) G_F n_e = lambda_const_kmi at every r                     */
  XFLAT_MATTER_TABLE = 3      /* sqrt(2) G_F n_e from a table (xflat_set_matter_table): a power law
                                 lambda_i (r/r_i)^p_i on each interval [r_i, r_{i+1}), p_i fixed by
                                 the two end values (a table sampled from rho0 (r_ref/r)^p gives that
                                 profile exactly), the end values outside the table              */
};
enum xflat_geometry {
  XFLAT_GEOMETRY_BULB = 0,    /* the bulb model of Sec. 2: cos theta_b(r) = sqrt(1 - u_j R^2/r^2),
                                 H_nunu = mu(r) (J0 - cos theta_b J1) (Eq. Hnu)                    */
  XFLAT_GEOMETRY_SINGLE_ANGLE = 1, /* single-angle approximation: every beam moves radially
                                 (cos theta = 1 in Eq. eom) and H_nunu = mu(r) f(x) J1 with
                                 f(x) = (1 - sqrt(1 - x))^2 / x, x = R^2/r^2: the geometric factor of
                                 Eq. Hnu integrated over emission uniform in u                      */
  XFLAT_GEOMETRY_HOMOGENEOUS = 2 /* test geometry: every beam radial and H_nunu = mu_const_kmi J1 /
                                 (sum of all per-bin number luminosities), independent of r; the
                                 synchronised-precession limit of the paper's collective term      */
};
enum xflat_layout {
  XFLAT_LAYOUT_MATRIX = 0,    /* [n_beams][n][n] complex double, interleaved (re, im), row major,
                                 the paper's psi psi^dagger (antineutrinos: psibar psibar^dagger) */
  XFLAT_LAYOUT_NATIVE = 1     /* [n_comp][n_beams] double planes of the internal state:
                                 2 flavours n_comp = 3, Bloch vector s of the nu density matrix
                                 P = (1 + s.sigma)/2 and of conj(Pbar) for antineutrinos;
                                 3 flavours n_comp = 9: P00, P11, P22, Re P01, Im P01, Re P02,
                                 Im P02, Re P12, Im P12 of P (nu) and of conj(Pbar) (nubar)     */
};

/* ---- configuration --------------------------------------------------------------------------- */
typedef struct {
  uint32_t abi_version;       /* must be XFLAT_ABI_VERSION                                         */
  uint32_t n_flavor;          /* 2 or 3                                                            */
  uint32_t n_energy;          /* energy bins, >= 1                                                 */
  uint32_t n_angle;           /* emission-angle (u) bins, >= 1                                     */
  uint32_t precision;         /* xflat_precision                                                   */
  uint32_t integrator;        /* xflat_integrator                                                  */
  uint32_t matter_kind;       /* xflat_matter                                                      */
  uint32_t n_phi;             /* 0 or 1: bulb model; >= 2: extended bulb model (Sec. 2, Eq. int-v)
                                 with n_phi equal azimuthal bins phi_p = 2 pi (p + 1/2) / n_phi
                                 around the radial direction, two flavours only.  Beams are then
                                 indexed with a combined angle bin a = j n_phi + p in place of j
                                 (weight du_j / n_phi), n_beams = 2 n_angle n_phi n_energy.       */
  double R_km;                /* neutrino-sphere radius R                                          */
  double E_min_MeV, E_max_MeV;/* energy range, bins of equal width, midpoints                      */
  double dm2_eV2[2];          /* 2 flavours: dm2[0]; 3 flavours: dm2_21, dm2_31 (signed)          */
  double theta[3];            /* 2 flavours: theta[0] = theta_v; 3 flavours: theta12, 13, 23 (rad),
                                 U = R23 R13 R12 with a zero CP phase (real mixing)              */
  double rtol, atol;          /* DP45 error control (see xflat_evolve)                             */
  double h0_km;               /* DP45 first trial step                                             */
  double h_min_km, h_max_km;  /* DP45 step bounds (h_max_km <= 0: unbounded)                       */
  double fixed_dr_km;         /* RK4 / LIE_RK4 target step; n = ceil((r1-r0)/fixed_dr) equal steps */
  double rho0_gcc, r_ref_km, power, Ye;   /* XFLAT_MATTER_POWER_LAW                                */
  double lambda_const_kmi;    /* XFLAT_MATTER_CONSTANT                                             */
  void* cuda_stream;          /* cudaStream_t the handle works on (NULL = default stream)          */
  uint64_t barrier_timeout_ns;/* limit of every device-wide wait (0 = 2 s)                         */
  uint32_t block_size;        /* threads per block: 128, 256 or 512 (0 = library default: 512 for
                                 the mixed two-flavour bulb kernels whose two state buffers fit
                                 the L2, 256 otherwise)                                          */
  uint32_t blocks_per_sm;     /* resident blocks per SM for the persistent grid (0 = occupancy)    */
  uint32_t steps_per_launch;  /* radial steps per persistent launch in xflat_evolve (0 = 64)       */
  uint32_t geometry;          /* xflat_geometry (0 = the bulb model); SINGLE_ANGLE and HOMOGENEOUS
                                 need n_phi <= 1                                                    */
  double mu_const_kmi;        /* XFLAT_GEOMETRY_HOMOGENEOUS: the nu-nu strength mu0 in 1/km       */
} xflat_config;

typedef struct xflat_s* xflat_t;

typedef struct {
  double r_km;                /* current radius of instance 0                                      */
  double h_km;                /* last attempted step                                               */
  double last_err;            /* last DP45 error norm (0 for fixed-step integrators)              */
  uint64_t accepted, rejected;/* steps                                                             */
  uint64_t stage_evals;       /* right-hand-side evaluations per beam (RK stages), incl. rejected  */
  uint64_t beam_stage_updates;/* sum over instances of beams x stage_evals                         */
  uint64_t launches;          /* persistent kernel launches issued                                */
  uint32_t n_beams;           /* beams of instance 0                                               */
  uint32_t n_instances;
  int32_t status;             /* sticky device status (xflat_status) of instance 0                 */
  uint32_t grid_blocks, block_size;
} xflat_stats;

/* ---- lifecycle ------------------------------------------------------------------------------- */

/* Fill *cfg with defaults: 2 flavours, 64 x 32 bins, FP64, RK4, R = 11 km, E in [1, 60] MeV,
 * dm2 = -2.4e-3 eV^2, theta_v = 0.1, no matter, rtol = atol = 1e-9, h0 = 1e-4 km, h_min = 1e-14 km. */
int xflat_default_config(xflat_config* cfg);

/* Create a solver for one bulb-model instance.  Validates cfg (XFLAT_ERR_INVAL on an out-of-range
 * field), allocates the device state (two buffers of n_beams x n_comp values in the working
 * precision), tables and barrier words on the current CUDA device.  *out is set only on success. */
int xflat_create(const xflat_config* cfg, xflat_t* out);

/* Create one solver holding n_inst independent instances (each with its own sizes, mixing,
 * spectra, radius, step size and error control) that advance together in one persistent launch.
 * All instances must share n_flavor, precision and integrator.  Instance i is addressed by the
 * *_inst entry points; the plain entry points address instance 0. */
int xflat_create_batch(const xflat_config* cfgs, uint32_t n_inst, xflat_t* out);

/* Release every resource of the handle (synchronises its stream).  NULL is a no-op. */
int xflat_destroy(xflat_t h);

/* ---- inputs (Sec. 2 flux matrices; Sec. 3.2 discretisation) ----------------------------------- */

/* Per-bin number luminosities N[species][flavor][k] = (L/<E>) f(E_k) dE in 1/s, species 0 = nu,
 * 1 = nubar, flavour 0 = e, then x (2 flavours) or mu, tau (3 flavours; mu and tau must be equal).
 * u_bins / u_weights (host, n_angle each) place the angle bins and weight them; both NULL = equal
 * bins of [0,1] at midpoints with weight 1/n_angle.  Resets the state to the initial condition of
 * Sec. 3.4 at r = R.  XFLAT_ERR_INVAL on non-finite input or u outside [0, 1). */
int xflat_set_spectra(xflat_t h, const double* nnu, const double* u_bins, const double* u_weights);
int xflat_set_spectra_inst(xflat_t h, uint32_t inst, const double* nnu, const double* u_bins,
                           const double* u_weights);

/* Matter profile of instance inst when its matter_kind is XFLAT_MATTER_TABLE (Sec. 2: H_mat with
 * the electron density n_e(r)): n points r_km[i] (strictly increasing, > 0) and
 * lambda_kmi[i] = sqrt(2) G_F n_e(r_i) in 1/km (> 0), host arrays copied in.  Required before the
 * first evolve of such an instance (else XFLAT_ERR_STATE); XFLAT_ERR_STATE for another matter_kind,
 * XFLAT_ERR_INVAL for bad points. */
int xflat_set_matter_table(xflat_t h, uint32_t inst, const double* r_km, const double* lambda_kmi,
                           uint32_t n);

/* Put every beam of every instance back to the initial condition of Sec. 3.4 at radius r0_km. */
int xflat_reset(xflat_t h, double r0_km);

/* ---- evolution (Sec. 3.4: radial integration of Eq. eom) -------------------------------------- */

/* Advance instance 0 (and every other instance, to the same r1) from its current radius to r1_km.
 * r0_km must equal the current radius (set by xflat_reset / xflat_set_rho) to 1e-12 relative,
 * else XFLAT_ERR_STATE.  Fixed-step integrators take n = ceil((r1-r0)/fixed_dr_km) equal steps,
 * step m spanning [r0 + m h, r0 + (m+1) h].  DP45 attempts steps of size h (first h0_km, clipped
 * to end exactly at r1), accepts a step when
 *   Err = max_b ||e_b||_F / (atol + rtol max(||P~_b||_F, ||P~'_b||_F)) <= 1
 * (e_b the embedded error matrix, P~ the traceless part) and continues with
 * h * min(5, max(0.2, 0.9 Err^-1/5)) (at most h after a rejection), clipped to h_max_km.
 * Returns the first device status that is not XFLAT_OK (TIMEOUT, NONFINITE, STEP). */
int xflat_evolve(xflat_t h, double r0_km, double r1_km);

/* Advance every unfinished instance i toward r1_km[i] (host array of n_inst), in one persistent
 * launch per steps_per_launch steps, until all are finished or one fails. */
int xflat_evolve_batch(xflat_t h, const double* r1_km_per_instance);

/* Attempt at most max_steps radial steps of every unfinished instance toward r1_km[i] (NULL: the
 * targets of the previous call) in ONE persistent launch.  When r1_km_per_instance is NULL and the
 * previous call on the handle was also xflat_advance, the call only enqueues the launch (no host
 * synchronisation, no copies), so a loop of advances measures the kernel alone.  *done_out
 * (nullable, host) receives the all-finished flag as last read back from the device, which may lag
 * one call behind; xflat_get_stats gives the exact state after synchronising. */
int xflat_advance(xflat_t h, const double* r1_km_per_instance, uint32_t max_steps, int* done_out);

/* Enqueue n_launches further xflat_advance(h, NULL, max_steps) launches as ONE CUDA graph launch on
 * the handle's stream.  The graph (the persistent launches and the read-back of the status words)
 * is captured on first use for this (n_launches, max_steps) pair and kept by the handle until the
 * pair changes or the handle is destroyed.  The previous call that touched the state must have
 * been xflat_advance or xflat_advance_graph (else XFLAT_ERR_STATE): the graph continues toward the
 * targets set there.  No host synchronisation; *done_out (nullable) as for xflat_advance.
 * XFLAT_ERR_CUDA if the capture fails. */
int xflat_advance_graph(xflat_t h, uint32_t n_launches, uint32_t max_steps, int* done_out);

/* ---- outputs ----------------------------------------------------------------------------------- */

/* Traceless parts of the two beam-independent moments of the current state at the current radius:
 *   J0 = sum_b du_j F_b / cos(theta_b),   J1 = sum_b du_j F_b,
 * F_b the flux matrix of Sec. 2 (Eq. F: Phi_1 = R^2/(2 r^2) J0, Phi_c = R^2/(2 r^2) J1 up to their
 * traces).  J0, J1: caller-owned host arrays of 2 n^2 doubles each (complex n x n, interleaved,
 * row major), units of 1/s.  Computed by the device reduction (deterministic order). */
int xflat_moments(xflat_t h, double* J0, double* J1);
int xflat_moments_inst(xflat_t h, uint32_t inst, double* J0, double* J1);

/* Extended bulb model (n_phi >= 2): the azimuthal moments of the current state,
 *   Jc = sum_b du_a F_b (sin th_b / cos th_b) cos phi_b,   Js = the same with sin phi_b
 * (Eq. F: Phi_sc = R^2/(2 r^2) Jc, Phi_ss = R^2/(2 r^2) Js with the 1/2pi of Eq. int-v), traceless
 * parts, 2 n^2 doubles each as J0 and J1.  XFLAT_ERR_UNSUPPORTED for the bulb model. */
int xflat_moments_phi(xflat_t h, uint32_t inst, double* Jc, double* Js);

/* Copy the state of instance 0 (inst: instance inst) out in the given layout (double).  dst is a
 * host pointer (dst_is_device = 0) or a device pointer on the handle's device (1) holding
 * n_beams x 2 n^2 (MATRIX) or n_comp x n_beams (NATIVE) doubles. */
int xflat_get_rho(xflat_t h, void* dst, int dst_is_device, int layout);
int xflat_get_rho_inst(xflat_t h, uint32_t inst, void* dst, int dst_is_device, int layout);

/* Replace the state of instance 0 (inst) and declare it to be at radius r_km (resume). */
int xflat_set_rho(xflat_t h, const void* src, int src_is_device, int layout, double r_km);
int xflat_set_rho_inst(xflat_t h, uint32_t inst, const void* src, int src_is_device, int layout,
                       double r_km);

/* Electron-flavour survival probability P_ee = |a_e|^2 (Sec. 3.4 validation figure): per beam
 * (nullable host array of n_beams, nu and nubar) and the number-flux weighted mean over nu beams,
 *   Pbar_ee = sum_{j,k} du_j N_nue,k P_ee(nu,j,k) / sum_{j,k} du_j N_nue,k   (nullable). */
int xflat_pee(xflat_t h, double* pee_per_beam, double* pee_mean);
int xflat_pee_inst(xflat_t h, uint32_t inst, double* pee_per_beam, double* pee_mean);

/* Energy spectra of the number flux at the current radius of instance inst (the nu_e flux of the
 * Sec. 3.4 validation figure), summed over angle bins with their weights du_j:
 *   flux[s][a][k] = sum_j du_j [ N[s][e][k] P_ea(s, j, k) + N[s][x][k] (1 - P_ea(s, j, k)) ],
 * s = 0 nu, 1 nubar; a the flavour (e, x or e, mu, tau); P_ea the a-a entry of the density matrix
 * of the beam that started as electron flavour (the other initial flavours, all with spectrum
 * N[s][x], carry 1 - P_ea into flavour a by unitarity).  flux: caller-owned host array of
 * 2 n_flavor n_energy doubles, in the units of N.  At r = R: flux[s][e] = N[s][e] sum_j du_j. */
int xflat_flux_spectra(xflat_t h, uint32_t inst, double* flux);

int xflat_get_stats(xflat_t h, xflat_stats* out);
int xflat_get_stats_inst(xflat_t h, uint32_t inst, xflat_stats* out);

/* ---- adjoint (gradient of the final mean survival probability) -------------------------------- */

/* Discrete adjoint of n_steps fixed RK4 steps (two flavours, FP64) from the initial condition of
 * Sec. 3.4 at r0_km to r1_km, for the objective J = Pbar_ee(r1) of xflat_pee.  The forward pass
 * stores the state every `checkpoint_every` steps and the backward pass recomputes each segment.
 * Outputs (host, nullable):
 *   dJ_dN     [2][n_flavor][n_energy]: dJ / d(per-bin number luminosity N of xflat_set_spectra)
 *   dJ_dtheta : dJ / d(theta_v)
 *   J_out     : the objective itself.
 * Scale-factor gradients follow by the chain rule, e.g. dJ/dlog(L_nue) = sum_k N_e,k dJ_dN[0][0][k]. */
int xflat_adjoint(xflat_t h, double r0_km, double r1_km, uint32_t n_steps, uint32_t checkpoint_every,
                  double* dJ_dN, double* dJ_dtheta, double* J_out);

/* ---- one problem over several GPUs: beam shards --------------------------------------------------
 * The paper splits the angle bins of one problem over MPI ranks and sums the integrals of Eq. F
 * over all ranks at every evaluation of the right-hand side (Sec. 3.3).  A shard handle integrates
 * the beams [beam_lo, beam_hi) of one instance (beam index as above; beam_lo a multiple of 4,
 * beam_hi a multiple of 4 or n_beams) and runs one pass per launch; between passes the caller adds
 * the shards' partial sums (exactly: they are fixed-point integers) and hands the totals back.  A
 * radial integration to r1_km on every rank:
 *   xflat_shard_begin(h, r1_km);
 *   xflat_shard_pass(h, -1); exchange; xflat_shard_serial(h, 1, &done);       -- moments of the state
 *   while (!done) for (p = 0; p < passes; ++p) {
 *     xflat_shard_pass(h, p); exchange;                                       -- exchange = partials,
 *     if (p == passes - 1) xflat_shard_serial(h, 0, &done);                       sum over shards,
 *   }                                                                             set_totals
 * The planes, tables and outputs of a shard handle span the whole instance, but only its own
 * beams are integrated (get_rho / pee / flux on the other beams return the initial state); the
 * moments it reports are those of its own beams.  xflat_evolve / xflat_advance return
 * XFLAT_ERR_STATE on a shard handle.  With the same block decomposition (the shard boundaries on
 * the unsharded handle's block boundaries) the result is bit-identical to the unsharded run. */
int xflat_create_shard(const xflat_config* cfg, uint32_t beam_lo, uint32_t beam_hi, xflat_t* out);
/* passes per radial step of the handle's integrator, and the length of the exchanged word vector */
int xflat_shard_info(xflat_t h, uint32_t* passes_per_step, uint32_t* n_words);
/* set the target radius (as xflat_evolve) without launching anything */
int xflat_shard_begin(xflat_t h, double r1_km);
/* the beam work of pass `pass` (0 .. passes-1) of the current step, or (-1) the moments of the
 * current state, on this shard's beams; enqueued on the handle's stream */
int xflat_shard_pass(xflat_t h, int32_t pass);
/* words [n_words] (host): the last pass's partial moments as 128-bit two's-complement fixed-point
 * integers (lo, hi) per component, then the bits of its error maximum (a non-negative double; the
 * total is the maximum over shards) and its non-finite flag (the total is the logical or).
 * Synchronises the stream. */
int xflat_shard_partials(xflat_t h, int64_t* words);
/* the totals over all shards, same layout, in place of this shard's partials */
int xflat_shard_set_totals(xflat_t h, const int64_t* words);
/* the serial section after the moment pass (after_moment_pass = 1) or after a step's final pass
 * (0): stage constants, step-size control, the next step's geometry.  *done_out (nullable): every
 * target reached.  Synchronises the stream; returns the device status. */
int xflat_shard_serial(xflat_t h, int32_t after_moment_pass, int* done_out);

/* ---- allocation-free moments (the paper has no counterpart: an addition for callers) ------------ */

#define XFLAT_NOALLOC_MAX_ANGLES 4096u

/* The two moments J0, J1 of xflat_moments for a two-flavour state supplied by the caller, computed
 * without allocating any memory: for callers that cannot call cudaMalloc at that point -- a host
 * framework that owns the device memory pool through its own allocator, or a time-critical loop
 * that must not stall, since cudaMalloc/cudaFree can synchronise the device and can fail when
 * memory is short.  No handle is needed and nothing is allocated: the inputs and the output are
 * caller-owned device memory, and the only scratch (two rows of six doubles per angle bin and a
 * counter, 393 KB in all) is a fixed array that every GPU which loads the library holds until the
 * process exits.
 *   d_state   [3][2 n_angle n_energy] double: Bloch planes in XFLAT_LAYOUT_NATIVE order (beam
 *             index as above; antineutrino beams hold the vector of conj(Pbar))
 *   d_g       [2][n_energy] double: signed per-bin weights, nu: N_e,k - N_x,k; nubar:
 *             -(Nbar_e,k - Nbar_x,k), in 1/s
 *   d_u, d_du [n_angle] double: angle-bin positions u_j in [0, 1) and weights du_j
 *   R_km, r_km: neutrino-sphere radius and the radius at which cos(theta) is evaluated (r >= R)
 *   d_J       [6] double out: Bloch vectors j0 then j1, with J = (1/2) j.sigma, units of 1/s
 *   cuda_stream: cudaStream_t for the work (NULL = default stream)
 * Returns XFLAT_ERR_INVAL for NULL pointers, empty sizes, r < R or n_angle >
 * XFLAT_NOALLOC_MAX_ANGLES (the scratch has no room for more rows), XFLAT_ERR_CUDA if a launch
 * fails.  The work is only enqueued: synchronise the stream before reading d_J.
 * The first call on a device (with that device current) looks up the device address of the
 * scratch array; make that first call before any stream capture.  Every call on a device shares
 * the one scratch array: calls whose work overlaps on the GPU (other streams, other host threads)
 * race and give wrong results; serialise them. */
int xflat_moments_2f_noalloc(const double* d_state, uint32_t n_energy, uint32_t n_angle,
                             const double* d_g, const double* d_u, const double* d_du, double R_km,
                             double r_km, double* d_J, void* cuda_stream);

/* ---- diagnostics ------------------------------------------------------------------------------- */

const char* xflat_status_string(int status);
const char* xflat_last_error(xflat_t h);

/* Test hook: every device-wide barrier of the next launch waits for `extra` more arrivals than
 * there are blocks, so it cannot complete; every block gives up after barrier_timeout_ns and the
 * call returns XFLAT_ERR_TIMEOUT with the context intact.  0 restores normal operation. */
int xflat_debug_barrier_extra(xflat_t h, uint32_t extra);

/* Test hook for the cleanup paths: the nth device or pinned-host allocation the library makes after
 * this call fails as if memory were exhausted (process-wide, once); 0 disarms.  The call that made
 * the allocation returns XFLAT_ERR_NOMEM or XFLAT_ERR_CUDA after freeing what it had allocated; a
 * handle that existed before stays usable.  Returns XFLAT_OK. */
int xflat_debug_fail_alloc(uint32_t nth);

/* Pass trace (profiling aid).  host_out == NULL: arm tracing of the first n_passes passes of every
 * following step launch (n_passes = 0 disarms; the handle allocates n_passes x grid x 4 u64 of
 * device memory).  host_out != NULL: synchronise and copy the trace out: for pass i and block b,
 * host_out[(i*grid + b)*4 + 0..3] = %globaltimer (ns) at the pass start, after the block's beams and
 * reduction, after the device-wide barrier let it go, and 1 if the block arrived last (then the
 * third stamp is its arrival).  *grid_out (nullable) receives the number of blocks. */
int xflat_debug_trace(xflat_t h, uint32_t n_passes, uint64_t* host_out, uint32_t* grid_out);

#ifdef __cplusplus
}
#endif
#endif /* XFLAT_H */
