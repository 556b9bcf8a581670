/*
 * qcams.h - C ABI of the GB300 quasi-classical trajectory (QCT) library.
 *
 * The library integrates very many independent atom-diatom trajectories
 * A + BC -> products with the QCT method of Koots & Perez-Rios, "PyQCAMS:
 * Python Quasi-Classical Atom-Molecule Scattering" (Comput. Phys. Commun.),
 * one trajectory per CUDA thread on sm_103a:
 *   - initial states from Bohr-Sommerfeld (v, j) levels with random
 *     orientation and vibrational phase (Sec. 2.1, Eqs. 5-7);
 *   - Hamilton's equations in Jacobi coordinates (Sec. 2, Eqs. 2-4) under
 *     pairwise Morse / generalized Lennard-Jones / Buckingham potentials
 *     (Sec. 3.2), integrated by the Dormand-Prince 5(4) pair with a per-lane
 *     adaptive step (Sec. 3.2, SciPy's RK45);
 *   - product analysis: bound-pair criterion, j', v', Gaussian binning
 *     (Sec. 2.2, Eqs. 8-11);
 *   - opacity, Monte-Carlo error and cross sections (Sec. 2.3, Eqs. 12-16;
 *     Sec. 4, Eq. 18).
 *
 * Conventions shared by every entry point:
 *   - Units: atomic units (hbar = 1; masses in electron masses; energies in
 *     hartree; lengths in bohr; time in hbar/hartree).
 *   - Memory: every array pointer is caller-owned.  "device" arrays must be
 *     CUDA device (or managed) memory of the current device; "host" arrays
 *     are ordinary host memory.  The library keeps only a small per-device
 *     context (level table, potential shape table, work counters), created
 *     on first use with cudaMalloc and released by qcams_shutdown(); make
 *     the first call on a device before capturing any of its calls into a
 *     CUDA graph.  Calls that use the context on one device (qcams_levels,
 *     qcams_init_states, qcams_run_batch, qcams_analyze, qcams_autotune,
 *     qcams_last_run_stats) share it: serialise them on one stream.
 *   - Streams: `cuda_stream` is a cudaStream_t (NULL = legacy default
 *     stream).  Calls only enqueue work on it and return without waiting,
 *     except where a function states that it synchronises.
 *   - Errors: functions return a qcams_status (0 = OK, negative = error); no
 *     exception crosses the ABI.  Argument errors are detected before any
 *     work is enqueued.  Per-trajectory failures do not fail a call: they
 *     are reported in the lane status array.
 *   - Ordering: calls that share a batch must be ordered on one stream.
 */
#ifndef QCAMS_H
#define QCAMS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define QCAMS_ABI_VERSION 1

/* ---------------------------------------------------------------------- */
/* Status codes.                                                           */
/* ---------------------------------------------------------------------- */
typedef enum {
  QCAMS_OK = 0,
  QCAMS_E_INVALID = -1,   /* bad argument (null pointer, size, parameter)  */
  QCAMS_E_NO_LEVEL = -2,  /* a requested (v, j) level does not exist       */
  QCAMS_E_CUDA = -3,      /* a CUDA runtime call failed                    */
  QCAMS_E_CAPACITY = -4,  /* a size exceeds a documented library limit     */
  QCAMS_E_TIMEOUT = -5,   /* a bounded device wait gave up                 */
  QCAMS_E_NODEVICE = -6   /* no CUDA device of compute capability 10.3     */
} qcams_status;

/* Human-readable text for a status code (static storage, never NULL). */
const char* qcams_status_string(int code);

/* Library limits. */
#define QCAMS_MAX_SYS 4    /* systems per call                           */
#define QCAMS_V_MAX 63     /* largest initial v served by the level table */
#define QCAMS_J_MAX 255    /* largest initial j served by the level table */
#define QCAMS_LJ_MAX_POW 32 /* LJ exponents are integers 3 <= n < m <= 32  */

/* ---------------------------------------------------------------------- */
/* Potentials and systems (Sec. 3.2 "Main Code", items 1-3).               */
/* ---------------------------------------------------------------------- */
typedef enum {
  QCAMS_MORSE = 0, /* p = {De, re, alpha}:  V = De (1 - e^{-alpha (r-re)})^2 - De          */
  QCAMS_LJ = 1,    /* p = {m, n, Cm, Cn, r_scale}: V = Cm / r^m - Cn / r^n, integers m > n */
  QCAMS_BUCK = 2   /* p = {A, B, C6, r_max_guess}: V = A e^{-B r} - C6 / r^6               */
} qcams_pot_kind;

typedef struct {
  int32_t kind;   /* qcams_pot_kind */
  int32_t pad;
  double p[5];    /* parameters as listed for `kind`; unused entries 0.
                     LJ r_scale: a length near the well (the paper's "re
                     guess"), used to bound root searches.  Buckingham
                     r_max_guess: a length near the short-range maximum
                     (the paper's "max").  Morse pairs need alpha re < 700
                     and Buckingham pairs A B < e^700 (QCAMS_E_INVALID
                     otherwise): e^{alpha (re - r)} and A B e^{-B r} stay
                     finite down to r = 0. */
} qcams_pair;

typedef struct {
  double mass[3];       /* atoms A, B, C (electron masses); AB is the initial
                           molecule, C the projectile (Sec. 3.1) */
  qcams_pair pair[3];   /* potentials of the pairs AB, BC, CA */
} qcams_system;

/* Pair specification kinds for qcams_system_setup (input convenience). */
typedef enum {
  QCAMS_SPEC_MORSE = 0,    /* {De, re, alpha}                              */
  QCAMS_SPEC_LJ = 1,       /* {m, n, Cm, Cn, r_scale}                      */
  QCAMS_SPEC_BUCK = 2,     /* {A, B, C6, r_max_guess}                      */
  QCAMS_SPEC_LJ_FIT = 3,   /* {m, n, De, re}: Cm, Cn fitted so that V has
                              its minimum -De at re                        */
  QCAMS_SPEC_MORSE_WE = 4  /* {De, re, omega_e}: alpha = omega_e sqrt(mu/2De)
                              with mu the pair's reduced mass (the paper's
                              input form, Sec. 3.1 listing)               */
} qcams_spec_kind;

/*
 * Build a qcams_system from masses in unified atomic mass units
 * (1 u = 1822.888486209 m_e) and three pair specs (AB, BC, CA), each
 * spec[k][0..4] interpreted per kind[k].  Host-only, synchronous, no GPU
 * work.  Returns QCAMS_E_INVALID for a non-positive mass, an unknown kind
 * or parameters outside the limits checked by qcams_init_states.
 */
int qcams_system_setup(const double mass_u[3], const int32_t kind[3],
                       const double spec[3][5], qcams_system* out);

/* ---------------------------------------------------------------------- */
/* Integration parameters (Sec. 3.1 "int_params", Sec. 3.2).               */
/* ---------------------------------------------------------------------- */
typedef struct {
  double rtol, atol;   /* local error tolerances of the adaptive step */
  double r_stop;       /* stop once the largest pair distance exceeds
                          r_stop while the atom-molecule distance grows */
  double t_stop;       /* stop once t >= t_stop * R / v_rel (R, v_rel the
                          initial atom-molecule distance and speed) */
  double h_fixed;      /* step size when fixed_step = 1 */
  double gb_sigma;     /* Gaussian-binning width (Eq. 11); 0 selects
                          0.1 / (2 sqrt(2 ln 2)) (FWHM 0.1) */
  int64_t max_steps;   /* adaptive: accepted + rejected step cap per lane
                          (lane fails with FAIL_MAXSTEPS); fixed-step: the
                          exact number of steps taken */
  int32_t fixed_step;  /* 1 = constant step h_fixed, no error control, no
                          stop test (used to test the integrator) */
  int32_t precision;   /* 64 = FP64 integrator; 32 = FP32 integrator with
                          compensated (Kahan) state updates */
  int32_t persistent;  /* 1 = persistent refill-queue launch (finished lanes
                          take the next trajectory from a device counter);
                          0 = one thread per trajectory;
                          2 = three lanes per trajectory, 3 = six lanes
                          per trajectory (FP64 adaptive steps only, else
                          QCAMS_E_INVALID; block and blocks_per_sm are not
                          used): a step takes about 2.8x (3.4x) fewer
                          warp-wide FP64 instructions, for batches too
                          small to fill the GPU (below ~10,000
                          trajectories); a warp holds 10 (5) trajectories
                          instead of 32 */
  int32_t block;       /* threads per block (0 = 128) */
  int32_t blocks_per_sm; /* resident blocks per SM the integrator variant is
                            compiled for (its __launch_bounds__ minimum, which
                            caps registers per thread; 0 = 1).  Supported
                            (block, blocks_per_sm): (128,1) (64,1) (128,3)
                            (64,6) (64,7) (256,1); qcams_autotune picks one.
                            The persistent grid is the resulting occupancy
                            times the SM count. */
  int32_t pad;
} qcams_integ;

/* Lane status values (uint8 array qcams_batch.status). */
enum {
  QCAMS_LANE_READY = 0,         /* initialised, not yet integrated          */
  QCAMS_LANE_RUNNING = 1,       /* integrated part way (fixed-step mode)    */
  QCAMS_LANE_DONE_RSTOP = 2,    /* stopped by the r_stop rule               */
  QCAMS_LANE_DONE_TMAX = 3,     /* stopped at t_max (analysed anyway)       */
  QCAMS_LANE_FAIL_MAXSTEPS = 4, /* step cap reached                         */
  QCAMS_LANE_FAIL_HMIN = 5,     /* step size fell below 10 ulp(t)           */
  QCAMS_LANE_FAIL_NAN = 6,      /* non-finite error norm                    */
  QCAMS_LANE_FAIL_COLLAPSE = 7, /* a Buckingham pair fell inside its
                                   short-range maximum                      */
  QCAMS_LANE_NO_LEVEL = 8,      /* (v, j) has no bound level or exceeds the
                                   level table limits                       */
  QCAMS_LANE_INVALID = 9        /* bad lane input (E <= 0, R <= b, bad sys) */
};

/* Outcome classes (uint8 array qcams_batch.cls; Sec. 2.2 product list). */
enum {
  QCAMS_CLS_Q = 0,     /* AB(v') + C: quenching / inelastic                 */
  QCAMS_CLS_R_AC = 1,  /* AC + B (pair CA bound): reaction n_r1            */
  QCAMS_CLS_R_BC = 2,  /* BC + A (pair BC bound): reaction n_r2            */
  QCAMS_CLS_D = 3,     /* A + B + C: dissociation                          */
  QCAMS_CLS_AMBIG = 4, /* more than one pair bound (unfinished complex)    */
  QCAMS_CLS_FAIL = 5,  /* the lane failed (status FAIL_*, NO_LEVEL, ...)   */
  QCAMS_N_CLS = 6
};

/*
 * Structure-of-arrays batch of n trajectories.  Every pointer is caller-
 * owned DEVICE memory of n elements unless marked optional (may be NULL).
 * State layout: y[0..2] = rho1 (x,y,z), y[3..5] = rho2, y[6..8] = P1,
 * y[9..11] = P2; rho1 = r_B - r_A, rho2 = r_C - (centre of mass of AB),
 * P1, P2 their conjugate momenta (Sec. 2, Eq. 2).
 */
typedef struct {
  int64_t n;
  /* per-lane inputs */
  const int32_t* sys_id;   /* system index in [0, n_sys) */
  const int32_t* cell;     /* histogram cell (read by qcams_reduce_xsec) */
  const double* isw;       /* optional: importance-sampling weight (reduce) */
  /* state (written by qcams_init_states, advanced by qcams_run_batch) */
  double* y[12];
  double* t;               /* time */
  double* h;               /* next step size (0 = choose a starting step) */
  double* t_scale;         /* R / v_rel; t_max = t_stop * t_scale */
  double* E0;              /* total energy at t = 0 (Eq. 2) */
  double* Ecol;            /* collision energy (copied by init) */
  double* u[4];            /* optional outputs of init: the uniforms behind
                              cos(theta) = 2u0-1, phi = 2 pi u1,
                              eta = 2 pi u2, chi = u3 */
  uint8_t* status;         /* QCAMS_LANE_* */
  /* outputs of the run (product analysis) */
  uint8_t* cls;            /* QCAMS_CLS_* */
  int32_t* nsteps;         /* accepted steps */
  int32_t* nrej;           /* rejected steps */
  double* dE;              /* H(final) - E0 */
  double* vprime;          /* continuous v' of the bound pair (Eq. 10) */
  double* jprime;          /* continuous j' (Eq. 9) */
  double* gbw;             /* Gaussian-binning weight W(v', v_t) (Eq. 11) */
  int16_t* vt;             /* v_t = nearest integer to v' (>= 0) */
  int16_t* jt;             /* nearest integer to j' */
} qcams_batch;

/* ---------------------------------------------------------------------- */
/* Entry points of the hot path.                                           */
/* ---------------------------------------------------------------------- */

/*
 * Bohr-Sommerfeld levels (Sec. 2.1: E_int and tau; the quantisation rule of
 * Eq. 10 with v' = v): for each request k, the level (v[k], j[k]) of pair AB
 * of system sys[sys_id[k]].  Host arrays in and out, n_levels <= 65536;
 * out[k] = {E, r_minus, r_plus, tau, ok}: ok = 1 if the level exists (its
 * energy lies below the top of the effective potential's outer barrier, or
 * below 0 for j = 0).  Synchronises the stream.  Returns QCAMS_E_NO_LEVEL
 * if any level is missing (all existing levels are still written).
 */
typedef struct { double E, r_minus, r_plus, tau; int32_t ok, pad; } qcams_level;
int qcams_levels(const qcams_system* sys, int32_t n_sys, const int32_t* sys_id,
                 const int32_t* v, const int32_t* j, int32_t n_levels,
                 qcams_level* out, void* cuda_stream);

/*
 * Initial conditions (Sec. 2.1, Eqs. 5-6).  For each lane i (device arrays
 * E_col, b, v, j of n = batch->n elements): the level (v_i, j_i) of system
 * batch->sys_id[i] is solved on the device (once per distinct level); the
 * molecule is placed at its outer turning point r+ with orientation
 * (theta, phi) and rotation-plane angle eta; the atom starts at distance
 * R = R0 + chi P2 tau / mu123 with impact parameter b along +y and momentum
 * P2 = sqrt(2 mu123 E_col) along +z.  The uniforms come from Philox4x32-10
 * with key = seed and counter = (id_offset + i, 0, 0), u = (word + 1/2) 2^-32,
 * unless u_in is given: then u_in[k][i] (device, 4 arrays of n) are used
 * (importance sampling).  Writes y, t = 0, h = 0, t_scale, E0, Ecol,
 * status (READY, NO_LEVEL or INVALID) and, if non-NULL, u[k].
 * Limits: 1 <= n_sys <= QCAMS_MAX_SYS (more: QCAMS_E_CAPACITY, as for every
 * entry point taking a system list); R0 > 0.  Lanes with v > QCAMS_V_MAX
 * or j > QCAMS_J_MAX get NO_LEVEL.  Asynchronous.
 */
int qcams_init_states(const qcams_system* sys, int32_t n_sys, const double* E_col,
                      const double* b, const int32_t* v, const int32_t* j, double R0,
                      uint64_t seed, uint64_t id_offset, const double* const* u_in,
                      qcams_batch* batch, void* cuda_stream);

/*
 * Integrate and analyse (Sec. 2, Eqs. 3-4; Sec. 3.2; Sec. 2.2).  Every lane
 * whose status is READY or RUNNING is advanced by the Dormand-Prince 5(4)
 * method from (t, y, h) until a stop rule fires, then the products are
 * classified: per pair the internal energy E_ab and angular momentum L^2,
 * bound iff E_ab < V_eff(r_0) at the outer maximum r_0 of the effective
 * potential (0 when L = 0) with the pair inside r_0; exactly one bound pair
 * gives Q / R_AC / R_BC, none gives D, more than one AMBIG; j' from L^2,
 * v' from the action integral, v_t, j_t and the Gaussian weight W.  Writes
 * y, t, h, status, nsteps, nrej and the outputs; failed lanes get cls FAIL.
 * In fixed-step mode exactly max_steps steps of h_fixed are taken, the
 * status becomes RUNNING and no analysis is done.  Asynchronous.
 */
int qcams_run_batch(const qcams_system* sys, int32_t n_sys, const qcams_integ* integ,
                    qcams_batch* batch, void* cuda_stream);

/*
 * Product analysis alone (Sec. 2.2) for lanes whose status is DONE_RSTOP or
 * DONE_TMAX (other lanes get cls FAIL): same outputs as qcams_run_batch.
 * Asynchronous.
 */
int qcams_analyze(const qcams_system* sys, int32_t n_sys, const qcams_integ* integ,
                  qcams_batch* batch, void* cuda_stream);

/*
 * Histogram record per cell (int64, QCAMS_H_STRIDE entries, all counts
 * exact integers; weighted sums in fixed point, value * 2^32 rounded to
 * nearest, so that any summation order gives the same bits):
 *   [QCAMS_H_COUNT + k]   lanes of class k (k < 6); [+6] all lanes; [+7] 0
 *   [QCAMS_H_VT + 64 c + v]   class c in {Q, R_AC, R_BC}: lanes with v_t = v
 *                          (v = 63 collects v_t >= 63)
 *   [QCAMS_H_JT + 256 c + j]  same for j_t (255 collects j_t >= 255)
 *   [QCAMS_H_GB + 64 c + v]   sum of Gaussian weights W (Eq. 11), fixed point
 *   [QCAMS_H_W + k], [QCAMS_H_W2 + k]  sums of isw and isw^2 (1 if isw is NULL)
 */
#define QCAMS_H_COUNT 0
#define QCAMS_H_VT 8
#define QCAMS_H_JT 200
#define QCAMS_H_GB 968
#define QCAMS_H_W 1160
#define QCAMS_H_W2 1168
#define QCAMS_H_STRIDE 1176
#define QCAMS_XSEC_ENTRIES 7

typedef struct {
  int32_t n_cells;      /* cells referenced by batch->cell, <= 65536 */
  int32_t n_groups;     /* groups (one cross section each), may be 0 */
  const double* b;      /* host [n_cells]: impact parameter of the cell */
  const double* w;      /* host [n_cells]: quadrature weight of the cell */
  const int32_t* group; /* host [n_cells]: group of the cell (-1 = none) */
  int32_t weighted;     /* 1 = importance-weighted estimator (uses isw) */
  int32_t pad;
} qcams_cells;

/*
 * Reduce outcomes to histograms and cross sections (Sec. 2.3, Eqs. 12-16;
 * Sec. 4, Eq. 18).  Device kernel: block-level shared-memory histograms of
 * the lanes' (cls, v_t, j_t, W, isw) per cell, flushed with int64 atomics
 * into hist_out (device, n_cells * QCAMS_H_STRIDE int64, zeroed by this
 * call).  Lanes with a cell outside [0, n_cells) are ignored.
 * If xsec_out (host) is non-NULL the call synchronises the stream, copies
 * the histograms back and writes, in doubles, with E = QCAMS_XSEC_ENTRIES
 * entries per cell and per group (k = 0..5 the classes, k = 6 the reactive
 * total R_AC + R_BC):
 *   per cell c, entry k:  xsec_out[2E c + 2 k] = P_k = N_k / N,
 *                         xsec_out[2E c + 2 k + 1] = delta_k
 *                         = sqrt(N_k)/N sqrt((N - N_k)/N)   (Eq. 16),
 *     with N the lanes of classes Q, R_AC, R_BC, D, AMBIG (failures are
 *     excluded); weighted mode: P_k = sum(isw 1_k)/N and its sample error;
 *   then per group g: xsec_out[2E n_cells + 2E g + 2 k] = sigma_k
 *                         = 2 pi sum_{c in g} w_c b_c P_k(c),
 *     [.. + 1] = 2 pi sqrt(sum (w_c b_c delta_k(c))^2).
 * (Eq. 18 prints the prefactor 8 pi^2; the 8 pi^2 of the angular measure
 * is already divided out of P, leaving 2 pi int P b db.)
 */
int qcams_reduce_xsec(const qcams_batch* batch, const qcams_cells* cells,
                      int64_t* hist_out, double* xsec_out, void* cuda_stream);

/*
 * Cross sections from histograms already on the host (Sec. 2.3, Eqs. 13-16;
 * Sec. 4, Eq. 18): the same per-cell opacities, errors and per-group
 * sigma / SE as qcams_reduce_xsec writes to xsec_out, computed from a host
 * copy of the histogram records hist[cells->n_cells][QCAMS_H_STRIDE] (for
 * example the int64 sum of several shards' histograms, which is exact).
 * Host-only and synchronous: no device, no stream.  Same limits as
 * qcams_reduce_xsec; cells->b, cells->w (and cells->group if n_groups > 0)
 * are required.
 */
int qcams_xsec_from_hist(const int64_t* hist, const qcams_cells* cells, double* xsec_out);

/*
 * qcams_run_batch without any device allocation.  The paper has no
 * counterpart: this is a deployment variant for callers that cannot call
 * cudaMalloc (an application whose device memory all comes from its own pool
 * or a fixed budget, or that must not let a library allocation synchronise
 * the device in the middle of its stream work).  Same arguments, outputs and
 * per-lane semantics as qcams_run_batch.  Its scratch (the potential shape
 * table and the work counters) lives in one static device array of
 * QCAMS_NOALLOC_SCRATCH_BYTES bytes that every GPU which loads the library
 * holds until the process exits.
 *   - The first call on a device looks up that array's device address
 *     (cudaGetSymbolAddress, with the device current); make this first call
 *     before any stream capture.  The address is kept until qcams_shutdown
 *     on that device: a caller that resets the device (cudaDeviceReset)
 *     calls qcams_shutdown first.
 *   - Calls on one device share the array and it keeps the last call's
 *     contents (each call rewrites the shape table and clears the counters
 *     it uses), so calls that overlap on the GPU race: serialise them on one
 *     stream.
 *   - Returns QCAMS_E_CAPACITY if n_sys > QCAMS_NOALLOC_MAX_SYS.  It calls
 *     no cudaMalloc / cudaFree and no allocating library routine, and does
 *     not update the statistics read by qcams_last_run_stats.
 */
#define QCAMS_NOALLOC_SCRATCH_BYTES 1024
#define QCAMS_NOALLOC_MAX_SYS 4
int qcams_run_batch_noalloc(const qcams_system* sys, int32_t n_sys, const qcams_integ* integ,
                            qcams_batch* batch, void* cuda_stream);

/*
 * Launch autotuner for the FP64 integrator (the paper has no counterpart;
 * it sizes the GPU launch).  `sample` is an initialised batch (device SoA,
 * status READY) representative of the workload, ideally the workload
 * itself when it is small; the integrator runs on it, from the same saved
 * initial state, with at most `max_attempts` step attempts per lane, once
 * for every supported (block, blocks_per_sm) variant of the persistent
 * launch and, when the sample has no more lanes than one warp per SM
 * sub-partition (SM count x 128) or max_attempts is not below
 * integ->max_steps (an uncapped run), once for each lane-group launch
 * (persistent = 2 and 3, one warp per block); the attempted lane-steps per
 * second are measured with CUDA events.  (A larger capped sample cannot
 * show the lane-group kernels' tails: their warps run until their longest
 * trajectory ends, without refill.)  The sample's state is restored afterwards.  results
 * (host, room for QCAMS_TUNE_MAX_VARIANTS entries) receives one entry per
 * launch, *n_results their number, and *best a copy of *integ with the
 * fastest launch (its persistent, block and blocks_per_sm).  Persistent
 * shapes within 2 % of the fastest persistent shape count as a tie, which
 * goes to the smallest block (then the fewest blocks per SM); a lane-group
 * launch is chosen only if it is strictly the fastest.  Synchronous;
 * allocates a temporary copy of the sample state (~121 bytes per lane) with
 * cudaMallocAsync.
 */
#define QCAMS_TUNE_MAX_VARIANTS 16
typedef struct {
  int32_t block, blocks_per_sm;  /* the variant */
  int32_t regs;                  /* registers per thread */
  int32_t resident_blocks;       /* occupancy: blocks per SM */
  int32_t persistent;            /* launch mode: 1 persistent, 2 / 3 lane groups */
  int32_t pad;
  double ms;                     /* integrator time on the sample */
  double lane_steps_per_s;       /* attempted lane-steps per second */
} qcams_tune_result;
int qcams_autotune(const qcams_system* sys, int32_t n_sys, const qcams_integ* integ,
                   qcams_batch* sample, int64_t max_attempts, qcams_tune_result* results,
                   int32_t* n_results, qcams_integ* best, void* cuda_stream);

/* ---------------------------------------------------------------------- */
/* Learned importance-sampling proposal (the outcome study's extension:    */
/* the sampled trajectories are still integrated exactly; the proposal     */
/* only reweights where in (b^2, cos theta, phi, eta, chi) they are drawn). */
/* ---------------------------------------------------------------------- */

/*
 * MLP 8 -> 64 -> 64 -> 64 -> 4 with SiLU (z sigmoid(z)) hidden activations
 * and softmax outputs over (Q, R_AC, R_BC, D).  Inputs, in order: E_col, b,
 * v, j, theta, phi, chi, eta, standardised with x_mean / x_std.  FP32 master
 * parameters, layout (row-major): W1[64][8] b1[64] W2[64][64] b2[64]
 * W3[64][64] b3[64] W4[4][64] b4[4].  Matrix products run on the tensor
 * cores in BF16 (weights and activations rounded to BF16) with FP32
 * accumulation; biases, activations, softmax and Adam are FP32.
 * All pointers are caller-owned device arrays of QCAMS_MLP_NPARAMS elements.
 */
#define QCAMS_MLP_NPARAMS 9156
typedef struct {
  float* params;        /* FP32 master parameters */
  float* adam_m;        /* Adam first moments */
  float* adam_v;        /* Adam second moments */
  float* grad;          /* gradient of the last train / grad call */
  uint16_t* params_bf16;/* BF16 copy used by the tensor-core kernels */
  float x_mean[8];      /* input standardisation (host values) */
  float x_std[8];
  int64_t step;         /* Adam steps taken */
} qcams_mlp;

/* Parameters W ~ U(-1/sqrt(fan_in), 1/sqrt(fan_in)) from Philox4x32-10
 * (key = seed, counter words (index, 0, 3, 0), first output word), biases 0,
 * moments 0, step 0, standardisation = identity.  Asynchronous. */
int qcams_mlp_init(qcams_mlp* m, uint64_t seed, void* cuda_stream);
/* Refresh params_bf16 from params (after the caller writes params). */
int qcams_mlp_sync(const qcams_mlp* m, void* cuda_stream);
/* Network inputs of initialised lanes: x[i] = (E_col, b, v, j, theta, phi,
 * chi, eta) from the lane inputs and the uniforms batch->u written by
 * qcams_init_states (theta = acos(2 u0 - 1), phi = 2 pi u1, eta = 2 pi u2,
 * chi = u3).  x: device float [n][8].  Asynchronous. */
int qcams_mlp_features(const qcams_batch* batch, const double* E_col, const double* b,
                       const int32_t* v, const int32_t* j, float* x, void* cuda_stream);
/* Set x_mean / x_std to the mean and standard deviation of x[n][8]
 * (device); synchronises. */
int qcams_mlp_fit_standardizer(qcams_mlp* m, const float* x, int64_t n, void* cuda_stream);
/* Softmax cross-entropy summed over the n samples and divided by n, with
 * targets the outcome classes cls[n] as qcams_run_batch writes them (device
 * uint8: Q, R_AC, R_BC, D = 0..3; AMBIG and FAIL samples contribute
 * nothing), and its gradient into m->grad; *loss_out (device float,
 * optional) receives the loss.  Asynchronous. */
int qcams_mlp_grad(const qcams_mlp* m, const float* x, const uint8_t* cls, int64_t n,
                   float* loss_out, void* cuda_stream);
/* qcams_mlp_grad followed by one Adam step (beta1 0.9, beta2 0.999,
 * eps 1e-8, bias-corrected) with learning rate lr; increments m->step. */
int qcams_mlp_train_step(qcams_mlp* m, const float* x, const uint8_t* cls, int64_t n,
                         float lr, float* loss_out, void* cuda_stream);
/*
 * `steps` minibatch Adam steps on the samples (x[n][8], cls[n]) as
 * qcams_mlp_train_step takes them, all on the device: before each step the
 * batch row indices idx[0..batch) (caller-owned device int64 scratch) are
 * drawn uniformly on [0, n) with replacement (Philox4x32-10, key = seed,
 * counter (i, step_lo, step_hi, 4) with step = m->step before the update;
 * index = high 64 bits of (w1:w0) * n), the gradient is taken over the
 * gathered rows and Adam updates the parameters.  losses (device float
 * [steps], optional) receives each step's minibatch loss.  On return idx
 * holds the last step's indices.  Asynchronous; capturable in a graph.
 */
int qcams_mlp_train(qcams_mlp* m, const float* x, const uint8_t* cls, int64_t n, int64_t steps,
                    int32_t batch, float lr, uint64_t seed, int64_t* idx, float* losses,
                    void* cuda_stream);
/* Class probabilities probs[n][4] (device float) for inputs x[n][8]. */
int qcams_mlp_infer(const qcams_mlp* m, const float* x, int64_t n, float* probs,
                    void* cuda_stream);

/*
 * Proposal over one (E_col, v, j): an n_b2 x n_cth x n_phi x n_eta x n_chi
 * grid of equal-measure cells in (b^2 in [0, b2_max], cos theta, phi, eta,
 * chi); cell index ((((i_b2 n_cth + i_cth) n_phi + i_phi) n_eta + i_eta)
 * n_chi + i_chi).  q_c = alpha / N + (1 - alpha) g_c / sum g with
 * g_c = sqrt(eps + p_R(centre of c)), p_R = P(R_AC) + P(R_BC) from the MLP
 * (defensive mixture: q_c >= alpha / N, so every weight is <= 1 / alpha).
 * q (device double [N]); qfix (device int64 [N]) = round(q 2^40) and
 * cdf (device int64 [N]) its inclusive prefix sums: sampling uses the exact
 * integer distribution qfix / cdf[N-1].  N <= 2^22 (more: QCAMS_E_CAPACITY).
 * Asynchronous.
 */
typedef struct {
  double E_col;
  int32_t v, j;
  int32_t n_b2, n_cth, n_phi, n_eta, n_chi, pad;
  double b2_max, eps, alpha;
} qcams_proposal_spec;
int qcams_build_proposal(const qcams_mlp* m, const qcams_proposal_spec* spec, double* q,
                         int64_t* qfix, int64_t* cdf, void* cuda_stream);
/*
 * Draw n lanes from the proposal: for lane i, Philox4x32-10 with key = seed
 * and counter words (id_lo, id_hi, 1, 0) then (id_lo, id_hi, 2, 0), id =
 * id_offset + i, gives u_0..u_7 = (word + 1/2) 2^-32; cell c = first index
 * with cdf[c] > floor(u_0 cdf[N-1]) (computed exactly in integers); inside c: b^2 = b2_max (i_b2 + u_1)/n_b2, cos theta
 * = 2 (i_cth + u_2)/n_cth - 1, phi / 2 pi = (i_phi + u_3)/n_phi, eta / 2 pi
 * = (i_eta + u_4)/n_eta, chi = (i_chi + u_5)/n_chi.  Outputs (device):
 * b[n], u_out[0..3][n] = the uniforms qcams_init_states takes as u_in,
 * w[n] = (cdf[N-1] / N) / qfix[c] (the likelihood ratio), cell[n].
 */
int qcams_sample_proposal(const qcams_proposal_spec* spec, const int64_t* qfix,
                          const int64_t* cdf, int64_t n, uint64_t seed, uint64_t id_offset,
                          double* b, double* const* u_out, double* w, int32_t* cell,
                          void* cuda_stream);

/* ---------------------------------------------------------------------- */
/* Reports derived from cross sections and histograms (host, synchronous). */
/* ---------------------------------------------------------------------- */

/*
 * Rate constants k(E) = sigma(E) sqrt(2 E / mu123) (Sec. 4, Eq. 19, with the
 * atom-molecule reduced mass mu123 for mu) and their standard errors, for n
 * collision energies: host arrays sigma, sigma_se, E_col in; k, k_se out.
 */
int qcams_rate_constants(const double* sigma, const double* sigma_se, const double* E_col,
                         int32_t n, double mu123, double* k, double* k_se);

/*
 * Gaussian-binned product vibrational distributions (Sec. 2.3, Eqs. 14-15)
 * over the cells cell_ids[n_sel] of a host copy of the histograms
 * hist[n_cells][QCAMS_H_STRIDE]: with S_c(v) the summed Gaussian weights of
 * channel c in {Q, R_AC, R_BC} at v_t = v and N_D the dissociations,
 * W = sum_v (S_Q(v) + S_RAC(v) + S_RBC(v)) + N_D and
 * out[64 c + v] = S_c(v) / W (out: host double [3][64]; v = 63 collects
 * v_t >= 63).  *W_out (optional) receives W.  Returns QCAMS_E_INVALID for
 * an empty selection or W = 0.
 */
int qcams_gb_distribution(const int64_t* hist, int32_t n_cells, const int32_t* cell_ids,
                          int32_t n_sel, double* out, double* W_out);

/* ---------------------------------------------------------------------- */
/* Measurement and housekeeping.                                           */
/* ---------------------------------------------------------------------- */

/*
 * Statistics of the last qcams_run_batch on this device, read back
 * synchronously (the call synchronises `cuda_stream`): rhs = right-hand-side
 * evaluations and steps = attempted steps, summed over lanes; integrate_ms
 * and analyze_ms = durations of the integrator and analysis kernels measured
 * with CUDA events recorded on the launching stream around each launch.
 */
typedef struct {
  int64_t rhs, steps;
  double integrate_ms, analyze_ms;
} qcams_run_stats;
int qcams_last_run_stats(qcams_run_stats* out, void* cuda_stream);

/*
 * Arithmetic-peak microbenchmark: runs a register-resident chain of
 * fused multiply-adds (precision 64 = DFMA, 32 = FFMA) over the whole GPU
 * and returns the achieved FLOP/s (FMA = 2 FLOP).  Synchronous.
 */
int qcams_fma_peak(int32_t precision, double* flops_per_s, void* cuda_stream);

/* Device properties used for launch shapes: SM count and CC. */
int qcams_device_info(int32_t* sm_count, int32_t* cc_major, int32_t* cc_minor);

/* Release the per-device context of the current device. */
int qcams_shutdown(void);

#ifdef __cplusplus
}
#endif

#endif /* QCAMS_H */
