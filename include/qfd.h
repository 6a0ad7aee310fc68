/*
 * qfd.h - C ABI of the GB300 imaginary-time Schroedinger solver with FFT
 * kinetic terms (arXiv:2006.16935, "quantumfdtd v3").
 *
 * The library evolves a wave-function psi on an N^3 periodic lattice with
 * spacing A by the imaginary-time step of Sec. 2.2, Eq. (iter_proced):
 *
 *     psi(tau + dtau) = A psi(tau) - B dtau H_K psi(tau),
 *     A = (1 - dtau V/2) / (1 + dtau V/2),   B = 1 / (1 + dtau V/2),
 *
 * where H_K is one of the FFT kinetic terms of Sec. 2.1, Eqs. (HK1)-(HK3),
 * applied as (1/N^3) IFFT[T(k) FFT[psi]] with the unnormalised transforms of
 * Sec. 2.1 and the momenta k_l of Eq. (eigenmodes).  Every SNAPUPDATE-like
 * cadence (`ortho_every` steps, Sec. 5.1) the state is parity projected
 * (Eq. (parity)), Gram-Schmidt deflated against the lower states and
 * normalised to sum |psi|^2 = 1; every `check_every` steps the Rayleigh
 * energy <psi|H_K + V|psi>/<psi|psi> is taken, and a solve stops once two
 * successive energies agree to |dE| <= tol |E| (TOLERANCE, Sec. 5.1).
 *
 * Conventions for every entry point:
 *  - Lattice arrays are row-major [x][y][z] (z fastest), N^3 sites, indexed
 *    with 64-bit integers.  Complex arrays are interleaved (re, im) doubles.
 *  - Pointers flagged `on_device` = 1 are CUDA device pointers of the current
 *    device, otherwise host pointers (pinned host memory makes copies async).
 *    Caller buffers are only read or written during the call; the library
 *    copies inputs and owns all of its device memory.
 *  - All work is ordered on the plan's CUDA stream (`qfd_params.stream`, or a
 *    stream the plan creates).  Calls that return values to the host
 *    synchronise that stream before returning.
 *  - Every call returns a qfd_status; nothing aborts.  After an error,
 *    qfd_last_error() describes it.  A plan is used by one host thread at a time.
 *  - Supported lattices: N in {8, 16, 32, 64, 96, 128, 192, 256, 512, 1024}
 *    (powers of two, and 96 = 3 * 32, 192 = 3 * 64 with one radix-12 stage).
 */
#ifndef QFD_H
#define QFD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct qfd_plan_s* qfd_plan_t;

typedef enum {
  QFD_OK = 0,
  QFD_ERR_ARG = -1,           /* invalid argument or unsupported size */
  QFD_ERR_OOM = -2,           /* device allocation failed */
  QFD_ERR_UNSTABLE_DT = -3,   /* dtau * max T(k) >= 2, or 1 + dtau V/2 <= 0 somewhere */
  QFD_ERR_DIVERGED = -4,      /* energy or norm became non-finite */
  QFD_ERR_TIMEOUT = -5,       /* a bounded wait ran out: the server's period watchdog (qfd_server_set_timeout), or the
                                 TMA-staged pass A giving up on its tile copies (see qfd_set_tuning) */
  QFD_ERR_CUDA = -6,          /* a CUDA call failed */
  QFD_ERR_NOT_CONVERGED = -7, /* max_steps reached before the tolerance */
  QFD_ERR_STATE = -8          /* call out of order (e.g. stepping before a potential is set) */
} qfd_status;

/* Kinetic terms, numbered as the paper's KINTERM (Sec. 5.1).  QFD_KIN_FDTD is
 * H_K(0) of Sec. 2.1, Eq. (HK0): the finite-difference Laplacian with
 * Dirichlet boundaries (psi = 0 outside the lattice; every lattice site
 * evolves), normalised as its momentum-space form, Eq.
 * (HK0_momentum_space_1): H_K(0) psi = -(1/(2 M A^2)) sum over the three axes
 * of [psi(x + e) + psi(x - e) - 2 psi(x)].  (The printed position-space form
 * carries an extra factor 1/2.)  Its box is symmetric about the off-grid
 * centre, so parity work with it should use QFD_CENTRE_OFFGRID.  The FFT
 * terms use periodic boundaries. */
enum { QFD_KIN_FDTD = 0, QFD_KIN_P2 = 1, QFD_KIN_SIN2 = 2, QFD_KIN_REL = 3 };
/* Arithmetic of the steps (reductions end in FP64 in all of them):
 *  QFD_C128          complex128 storage, native FP64 arithmetic;
 *  QFD_C64           complex64 storage and FP32 arithmetic;
 *  QFD_C64_REFINE    complex64 bulk to tol_bulk, then QFD_C128 steps of the
 *                    same iteration to tol;
 *  QFD_DF64          16 bytes per site like complex128, each real held as an
 *                    unevaluated sum hi + lo of two FP32 numbers and all
 *                    arithmetic done on the FP32 pipe with error-free
 *                    transformations (relative rounding about 2^-46 per
 *                    operation, about 2^-48 for stored values);
 *  QFD_C64_REFINE_DF complex64 bulk, then QFD_DF64 refinement. */
/* (QFD_C128 and QFD_C64_REFINE keep the numbers 0 and 1 of the two forms the
 * method statement names: plain FP64 and complex64 with an FP64 refinement.) */
enum { QFD_C128 = 0, QFD_C64_REFINE = 1, QFD_C64 = 2, QFD_DF64 = 3, QFD_C64_REFINE_DF = 4 };
/* Parity projection of a state (Eq. (parity)): none, P+, P-. */
enum { QFD_PAR_NONE = 0, QFD_PAR_EVEN = 1, QFD_PAR_ODD = -1 };
/* Potential centre (Sec. 1.3 / 5.3): the grid site (N/2, N/2, N/2) with the
 * reflection x -> (N - x) mod N, or the paper's off-grid point (N-1)/2 with
 * x -> N - 1 - x. */
enum { QFD_CENTRE_GRID = 0, QFD_CENTRE_OFFGRID = 1 };
/* Analytic potentials of qfd_fill_potential (r = A |x - centre|):
 *  ZERO      V = 0
 *  HO        V = c0 r^2 / 2                       (harmonic oscillator, Sec. 5.3 item 4)
 *  CORNELL   V = -c0 / r + c1 r, r >= A/2          (Cornell, Sec. 5.3 item 6, no string breaking)
 *  COULOMB   V = -1 / r, r >= A/2                  (Sec. 5.3 item 2)
 *  SOFTCOUL  V = -1 / sqrt(r^2 + c0)               (softened Coulomb) */
enum { QFD_POT_ZERO = 0, QFD_POT_HO = 1, QFD_POT_CORNELL = 2, QFD_POT_COULOMB = 3, QFD_POT_SOFTCOUL = 4 };

/* Stop rules, applied after every energy check (every check_every steps) with
 * D_k = E_k - E_(k-1):
 *  PAPER  |D_k| <= tol |E_k|  (TOLERANCE of Sec. 5.1).
 *  TAIL   PAPER, and the change still to come is bounded as well: either
 *         |D_k| <= 1e-3 tol |E_k|, or D_k, D_(k-1), D_(k-2) share one sign, the
 *         ratio r = D_k / D_(k-1) is below 1 and not below 0.9 D_(k-1)/D_(k-2),
 *         and the geometric tail |D_k| r / (1 - r) <= tol |E_k|.  The update
 *         of Sec. 2.2 is not a symmetric operator, so the energy can fall
 *         below its limit and creep back: PAPER then stops near the turn, up to
 *         tens of tol away from the limit; TAIL does not.  Not in the paper.
 * A complex64 bulk phase always uses PAPER with tol_bulk and additionally
 * stops once its energy rises after the third check. */
enum { QFD_STOP_PAPER = 0, QFD_STOP_TAIL = 1 };

typedef struct {
  int64_t n;            /* lattice points per axis (NUM): 8, 16, 32, 64, 96, 128, 192, 256, 512 or 1024 */
  double a;             /* lattice spacing A (> 0) */
  double mass;          /* mass M (> 0) */
  double dtau;          /* imaginary time step EPS (> 0) */
  int32_t kinetic;      /* QFD_KIN_* */
  int32_t rest_mass;    /* HK3 only: 1 keeps sqrt(p^2 + M^2) of Eq. (HK3); 0 subtracts M */
  int32_t nstates;      /* capacity of the state stack (1..8) */
  int32_t precision;    /* QFD_C128, QFD_C64, QFD_C64_REFINE, QFD_DF64 or QFD_C64_REFINE_DF */
  int32_t ortho_every;  /* steps between parity / Gram-Schmidt / normalisation (>= 1) */
  int32_t check_every;  /* steps between energy checks in qfd_solve_states (>= 1) */
  int32_t centre;       /* QFD_CENTRE_* */
  int32_t stop_rule;    /* QFD_STOP_PAPER or QFD_STOP_TAIL (the final phase's stop rule) */
  int64_t max_steps;    /* per state (per phase for QFD_C64_REFINE) */
  double tol;           /* relative energy tolerance of the final phase (< 0: run max_steps) */
  double tol_bulk;      /* relative energy tolerance of the complex64 bulk phase */
  void* stream;         /* cudaStream_t to order all work on, or NULL for a plan-owned stream */
} qfd_params;

/* Creates a plan: checks the parameters, allocates every device buffer
 * (state stack, one work lattice, potential and update coefficients,
 * twiddles and per-axis kinetic tables) and rejects an unstable time step:
 * dtau * max_k T(k) >= 2 gives QFD_ERR_UNSTABLE_DT (the highest mode of the
 * update would not decay).  Sections 2.1-2.2. *out is NULL on failure. */
qfd_status qfd_plan(const qfd_params* params, qfd_plan_t* out);

/* Releases the plan and its device memory (NULL is ignored).  Library
 * bookkeeping: no counterpart in the paper. */
void qfd_destroy(qfd_plan_t plan);

/* Message of the last error on `plan` (or of the last failed qfd_plan call of
 * this thread when plan is NULL).  Owned by the library.  Library
 * bookkeeping: no counterpart in the paper. */
const char* qfd_last_error(qfd_plan_t plan);

/* Copies a real potential V (N^3 doubles, [x][y][z]) and derives the update
 * coefficients A, B of Sec. 2.2 on the device.  V_b = V, V_s = 0 (Sec. 5.1).
 * QFD_ERR_UNSTABLE_DT if 1 + dtau V / 2 <= 0 or V is non-finite somewhere. */
qfd_status qfd_set_potential(qfd_plan_t plan, const double* V, int on_device);

/* Fills one of the QFD_POT_* potentials on the device (coefficients c0, c1 as
 * listed at the enum; ncoeffs of them are read), then derives A, B as
 * qfd_set_potential does. */
qfd_status qfd_fill_potential(qfd_plan_t plan, int kind, const double* coeffs, int ncoeffs);

/* Adds a smooth Gaussian random field to the plan's potential (the seeded
 * stand-in for the paper's file-based potentials, Sec. 5.3): white noise
 * (per site the two counter-mode uniforms u0, u1 of qfd_fill_psi_uniform's
 * generator under `seed`, through Box-Muller: sqrt(-2 ln(1 - u0)) cos(2 pi u1)),
 * filtered by exp(-k^2 corr^2 / 2) (corr in lattice units, at most 21; done
 * as three periodic real-space Gaussian convolutions, which differ from the
 * momentum-space filter by aliasing of order exp(-pi^2 corr^2 / 2), below
 * 1e-16 for corr >= 2.8), then shifted and scaled
 * to mean 0 and standard deviation `amplitude` over the lattice, and added to
 * V; the update coefficients are derived again.  Uses the work lattice as
 * scratch.  Needs a potential set first. */
qfd_status qfd_add_random_field(qfd_plan_t plan, uint64_t seed, double corr, double amplitude);

/* Copies the potential V the plan holds (N^3 doubles) into the caller's buffer. */
qfd_status qfd_get_potential(qfd_plan_t plan, double* V, int on_device);

/* Copies state `state` in (interleaved complex128, N^3 sites) and resets its
 * step counter: the paper's initial condition read from stored wave-functions
 * (INITCONDTYPE 0, Sec. 5.2), here from a caller's buffer instead of files.
 * Complex64 and double-float plans round the values to their representation.
 * Non-finite values are copied as they are: a later solve reports them as
 * QFD_ERR_DIVERGED at its first energy check. */
qfd_status qfd_set_psi(qfd_plan_t plan, int state, const double* psi, int on_device);

/* Fills state `state` on the device with Re, Im i.i.d. U[-1, 1) from the
 * counter-based SplitMix64 stream: value(site, part) = 2 u - 1 with
 * u = (splitmix64(seed * 0x9E3779B97F4A7C15 ^ (2 site + part)) >> 11) 2^-53
 * (part 0 = Re, 1 = Im); resets the step counter. */
qfd_status qfd_fill_psi_uniform(qfd_plan_t plan, int state, uint64_t seed);

/* Copies state `state` out (interleaved complex128) into the caller's buffer:
 * the wave-function output of the paper (SAVEWAVEFNCS, Sec. 5.1: the full 3D
 * wave-functions at the end of a run), into memory instead of files.  A
 * pending normalisation factor is applied first. */
qfd_status qfd_get_psi(qfd_plan_t plan, int state, double* out, int on_device);

/* Observables of `state` in lattice units, d = x - centre per axis (FP64):
 * out[0] sum |psi|^2; out[1] the same over the effective volume of Sec. 2.3
 * (sites with |d_l| <= (1 - min_sep_edge) N / 2 on every axis); out[2] the
 * box-normalised average radius <rho>_box of Eq. (box_normalization);
 * out[3] <rho^2>, out[4..6] <x>, <y>, <z> over the full lattice (the UPDATE
 * observables of Sec. 5.1); out[7], out[8] the box-normalised weights of the
 * parity projections P+ and P- (Sec. 2.4, they sum to 1); out[9..11] those of
 * the axis projections P-_{e_k}, k = 1, 2, 3, of Eq. (parity_axis) (odd under
 * the reflection of axis k, even under that of the two others; normalised as
 * projectors, 1/4 of the bracket).  The first nout (<= 12) values are
 * written; 0 <= min_sep_edge < 1. */
qfd_status qfd_observables(qfd_plan_t plan, int state, double min_sep_edge, double* out, int nout);

/* Parity sector applied to `state` at every cadence (QFD_PAR_*). */
qfd_status qfd_set_parity(qfd_plan_t plan, int state, int parity);

/* Advances `state` by nsteps steps of Eq. (iter_proced).  After every step t
 * of the state's counter with t % ortho_every == 0 the state is parity
 * projected, Gram-Schmidt deflated against states 0..state-1 (which must be
 * normalised) and normalised.  Steps in the plan's current arithmetic
 * (complex64 for QFD_C64 and, before a refinement, QFD_C64_REFINE). */
qfd_status qfd_step(qfd_plan_t plan, int state, int64_t nsteps);

/* Largest number of lattices one qfd_step_batch call steps together. */
#define QFD_MAX_BATCH 32

/* qfd_step for several plans at once: advances states[i] of plans[i] by
 * nsteps steps of Eq. (iter_proced) (Sec. 2.2, with the FFT kinetic terms of
 * Sec. 2.1), i < count, with exactly the operations qfd_step applies to each.
 * Each pass of a step (the y transforms, the z pass with T(k), the update
 * with the x transforms) is one launch over all the lattices; the cadence
 * (projection, deflation, normalisation) runs per plan.  There is no
 * counterpart in the paper, whose code steps one lattice.
 *   plans, states  arrays of `count` entries, 1 <= count <= QFD_MAX_BATCH;
 *                  the plans are distinct, have the same n, the same current
 *                  arithmetic and FFT kinetic terms (kinetic 1..3), and a
 *                  potential; their parameters may differ otherwise.
 *   nsteps         >= 0.
 * Kernels and launch shapes: qfd_step runs the same step kernels over a batch
 * of one lattice, so with the same launch shapes every plan's state is
 * bit-identical to what qfd_step gives it.  The batch takes plans[0]'s launch
 * shapes (qfd_autotune / qfd_set_tuning; the choice depends only on n and the
 * arithmetic).
 * Streams: the work runs on plans[0]'s stream; each other plan's stream is
 * ordered before it and after it with events, and the call returns after
 * every plan's work has completed (as qfd_step does).
 * Errors: QFD_ERR_ARG for a null array, a count out of range, a repeated
 * plan, a state index out of range, n > 256, or plans that differ in n,
 * arithmetic or kinetic kind (message in qfd_last_error of plans[0], or of NULL when plans
 * is NULL or count is out of range); QFD_ERR_STATE for a plan without a
 * potential; a launch error as QFD_ERR_CUDA.  Nothing is stepped when an
 * argument is rejected.  After a failure inside the loop every plan's state,
 * work lattice and step counter still agree with each other, but the number
 * of steps taken, and whether the last step's cadence ran, are unspecified. */
qfd_status qfd_step_batch(const qfd_plan_t* plans, const int* states, int count, int64_t nsteps);

/* Rayleigh energy <psi|H_K + V|psi> / <psi|psi> of `state` (FP64 sums;
 * <psi|H_K|psi> by Parseval, (1/N^3) sum_k T(k) |FFT psi|^2) and its squared
 * norm sum |psi|^2.  Either output may be NULL. */
qfd_status qfd_energy(qfd_plan_t plan, int state, double* E, double* norm2);

/* Solves states 0..nstates-1 in turn from their current contents: state i is
 * parity projected with parity[i] (parity may be NULL), deflated against the
 * converged states 0..i-1, stepped until the relative energy change between
 * two checks is <= tol (or max_steps), and left normalised.  For
 * QFD_C64_REFINE / QFD_C64_REFINE_DF each state first runs in complex64 to
 * tol_bulk (or until its energy rises between two checks after the third
 * one: FP32 rounding then dominates the decay), then in the FP64-class
 * arithmetic to tol.  E_out[i] receives the final energy and steps_out[i]
 * the total number of steps (both may be NULL).  Returns
 * QFD_ERR_NOT_CONVERGED (outputs still filled) if a state reached
 * max_steps, QFD_ERR_DIVERGED on a non-finite energy. */
qfd_status qfd_solve_states(qfd_plan_t plan, int nstates, const int* parity, double* E_out, int64_t* steps_out);

/* Excited states by the paper's snapshot overlaps (Sec. 2.2: the snapshots
 * kept at every SNAPUPDATE): one evolution of state 0 from its stored initial
 * state, with parity `parity` and the plan's tol / max_steps / stop rule,
 * keeping normalised snapshots every snap_every steps (a positive multiple of
 * ortho_every).  The ground state is the final state; excited state k
 * (1 <= k < nout) is the k-th latest snapshot taken before the end, parity
 * projected, Gram-Schmidt deflated against states 0..k-1 and normalised, in
 * state slot k.  E_out[0..nout-1] receives the Rayleigh energies and
 * *steps_out the evolution's steps.  nout is 1..3; the plan needs nout + 1
 * state slots (snapshot buffers) for nout > 1 and a single-arithmetic
 * precision (QFD_C128, QFD_C64, QFD_DF64).  QFD_ERR_STATE when fewer
 * snapshots than excited states were taken.  How well the excited states are
 * separated depends on the snapshot spacing against the inverse level gaps,
 * as the paper discusses; the per-state Gram-Schmidt solve of
 * qfd_solve_states converges each state instead. */
qfd_status qfd_snapshot_states(qfd_plan_t plan, int nout, int parity, int64_t snap_every, double* E_out,
                               int64_t* steps_out);

/* Launch-shape and radix-schedule autotuner (a tuning of this implementation;
 * the paper has no counterpart).  For every arithmetic the plan uses, times
 * the y passes with tiles of the default width and of twice that width, the
 * z pass with one and with two line groups per CTA, for complex64 at
 * n = 128..1024 also both passes with the two-stage radix schedule (radix
 * 16.8, 16.16, 32.16 or 32.32 with 16 or 32 elements per thread: one
 * shared-memory exchange per transform instead of two or three), and (once a
 * potential is set, FFT kinetic terms) pass A with tiles of the default width,
 * of half of it at two CTAs per SM, and (complex64, n = 256..1024) the
 * TMA-staged persistent kernel, on the work lattice and the spare state
 * lattice (5 launches each after 2 warm-ups), and keeps the fastest of each
 * for later launches.  Tilings do not change the arithmetic of a line;
 * the radix schedule changes the order of the operations of a transform.
 * Results agree to rounding whatever is chosen (complex128 / complex64
 * kernels may also differ in where the compiler fuses a multiply-add;
 * double-float tilings are bit-identical).  ms_out (NULL or 27 doubles): per
 * policy (0 complex128, 1 complex64, 2 double-float) the median times of
 * y-default, y-wide, y-two-stage, z-1, z-2, z-two-stage, x-default, x-half,
 * x-TMA in ms (NaN where not timed).  Synchronises; the work lattice is recomputed at
 * the next step. */
qfd_status qfd_autotune(qfd_plan_t plan, double* ms_out);

/* Sets the launch shapes of one policy (0 complex128, 1 complex64, 2
 * double-float) by hand: y_variant 0 default width, 1 twice it, 2 the
 * two-stage radix schedule; z_variant -1 the policy's default grouping, 0 one
 * line group, 1 two, 2 the two-stage radix schedule; x_variant 0 pass A's
 * default tile width, 1 half of it (two CTAs per SM), 2 the TMA-staged
 * persistent pass A.  The two-stage schedule exists for complex64 at
 * n = 128..1024 and the TMA pass A for complex64 at n = 256..1024 (when the
 * plan could build its tensor maps, qfd_has_tma); elsewhere 2 runs the default.
 *
 * The TMA-staged pass A runs one persistent CTA per SM; the Tensor Memory
 * Accelerator copies the next tile's W, psi and V (2D tensor maps of the
 * plan's lattices, boxes of 16, 8 or 4 sites by 256 rows) into shared memory
 * while the current tile is transformed.  Its waits for those copies are
 * bounded (about a second); when one runs out the kernel stops, the plan's
 * error flag is set, and the next synchronising call (qfd_step, an energy,
 * a solve's check) returns QFD_ERR_TIMEOUT.  The partial sums of a CTA cover
 * several tiles, so sums and energies agree with the other widths to
 * rounding. */
qfd_status qfd_set_tuning(qfd_plan_t plan, int policy, int y_variant, int z_variant, int x_variant);

/* Whether the plan holds the tensor maps of the TMA-staged pass A (1) or not (0). */
int qfd_has_tma(qfd_plan_t plan);

/* Test switch of the TMA-staged pass A (no counterpart in the paper):
 * arm_without_copies = 1 arms its barriers without issuing any copy, so that
 * every bounded wait runs out and the step reports QFD_ERR_TIMEOUT with no
 * copy in flight; 0 restores normal operation.  The lattice contents are
 * then undefined: set the states again. */
qfd_status qfd_set_tma_test(qfd_plan_t plan, int arm_without_copies);

/* Replaces the plan's max_steps, tol and tol_bulk (same meaning as in
 * qfd_params) for later qfd_solve_states calls. */
qfd_status qfd_set_limits(qfd_plan_t plan, int64_t max_steps, double tol, double tol_bulk);

/* Per-state statistics of the last qfd_solve_states: steps spent in
 * complex64 and complex128 and the energy at the end of the complex64 phase
 * (NaN if none).  Any output may be NULL. */
qfd_status qfd_get_stats(qfd_plan_t plan, int state, int64_t* steps_c64, int64_t* steps_c128, double* e_bulk);

/* Energy history of `state` in its last qfd_solve_states (the SAVEDECAY table
 * of Sec. 5.1): for every check, the step count within its phase and the
 * energy; the complex64 checks of a mixed solve come first.  Copies at most
 * `capacity` entries into steps[] and E[] and sets *count to the total. */
qfd_status qfd_get_history(qfd_plan_t plan, int state, int64_t* steps, double* E, int capacity, int* count);

/* The decay-rate energy estimator at the last check of `state` in a solve:
 * (1 - lambda) / dtau, with lambda the per-step norm ratio over the k steps
 * since the last normalisation (k = ortho_every at a cadence step), from the
 * squared norm N2 after those steps and the cadence's projections:
 * lambda = N2^(1/(2k)).  The state decays as exp(-E tau) under Eq.
 * (iter_proced), so at the fixed point this is the eigenvalue of the update
 * (Sec. 2.2), next to the Rayleigh energy of qfd_energy.  NaN before the
 * first check. */
qfd_status qfd_get_decay(qfd_plan_t plan, int state, double* e_decay);

/* Kernel timing: when enabled, every kernel launch of the plan is bracketed
 * by CUDA events on the plan's stream.  qfd_timing_query synchronises and
 * returns, for the pass kind (0 update-x, 1 forward-y, 2 z kinetic,
 * 3 inverse-y, 4 forward-x, 5 GS overlaps, 6 GS apply, 7 reductions,
 * 8 other), the number of launches and their summed duration in ms since the
 * last reset.  qfd_launch_count returns all kernel launches since the reset. */
qfd_status qfd_timing_enable(qfd_plan_t plan, int enable);
qfd_status qfd_timing_reset(qfd_plan_t plan);
qfd_status qfd_timing_query(qfd_plan_t plan, int kind, int64_t* launches, double* total_ms);
int64_t qfd_launch_count(qfd_plan_t plan);

/* Measured FMA issue rate of one vector pipe of the current device, in
 * TFLOP/s (2 flops per FMA): fp64 = 1 the FP64 pipe, 0 the FP32 pipe.  A
 * measurement utility with no counterpart in the paper: it is the roofline
 * denominator of the passes bound by vector arithmetic instead of HBM (the
 * complex128 transforms; no tensor cores are used).  Every thread of a grid
 * of 8 CTAs of 256 threads per SM runs 8 independent FMA chains; one warm-up
 * launch, then the best of five timed with CUDA events on the legacy default
 * stream (about 0.1 s each).  Allocates and frees a small device buffer and
 * synchronises. */
qfd_status qfd_fma_rate(int fp64, double* tflops);

/* Rayleigh energy <psi|H_K + V|psi> / <psi|psi> and sum |psi|^2 of a lattice
 * that lives in the caller's device memory, computed in FP64 without
 * allocating any device memory.  There is no counterpart in the paper: this
 * entry point exists for callers that cannot allocate device memory (for
 * example a serving process that gives its whole memory budget to its own
 * pool up front, or a latency-critical path where a cudaMalloc could fail or
 * stall).  Its scratch (work lattice, partial sums, tables) is one static
 * device array of about 33 MiB that every GPU loading this library holds
 * until exit; it bounds the lattice to n <= 128 (QFD_ERR_ARG above that).
 * psi: device, interleaved complex128, n^3 sites [x][y][z], read only; V:
 * device, n^3 doubles, read only; a, mass, rest_mass as in qfd_params;
 * kinetic: one of the FFT kinetic terms 1..3 (Eqs. HK1-HK3) only, since
 * H_K(0) has no Parseval form (QFD_ERR_ARG for 0); stream: cudaStream_t or
 * NULL.  E and norm2 are host outputs (either may be NULL); the call
 * synchronises the stream.  The array is shared by every call and keeps the
 * last call's contents; calls that overlap on the GPU race on it.  The first
 * call on a device looks up the array's device address (with that device
 * current) and keeps it for the process; make that first call before any
 * stream capture.  A cudaDeviceReset destroys the array with the context, so
 * after one this entry point must not be called again on that device in the
 * same process. */
qfd_status qfd_energy_noalloc(const double* psi, const double* V, int64_t n, double a, double mass, int kinetic,
                              int rest_mass, void* stream, double* E, double* norm2);

/* Device bytes a plan with these parameters allocates (used for admission by
 * budget). */
size_t qfd_plan_bytes(const qfd_params* params);

/* ------------------------------------------------------------- server ----
 * Continuous batching of solve requests (a serving form of the method; the
 * paper has a single solve per run).  Requests wait in FIFO order and are
 * admitted while the device bytes of the admitted requests (qfd_plan_bytes)
 * stay within hbm_budget_bytes; each admitted request owns a plan on its own
 * stream (priority rising as the lattice shrinks), so requests overlap on the
 * device and each advances at its own pace.  qfd_server_poll admits what
 * fits, queues one period (check_every steps and an energy check, exactly as
 * qfd_solve_states runs them) for every admitted request with none queued,
 * blocks until at least one queued period has ended, applies the stop rule of
 * each request whose period ended, moves it to its next phase or state, and
 * returns the results of the requests that finished.  From the second period
 * of a phase on, a request's period is captured once as a CUDA graph and
 * replayed.  A request's numbers are the same alone and in any mix.
 *
 * Cohort mode (cohorts = 1): admitted requests of one lattice size share a
 * stream in cohorts of up to QFD_MAX_BATCH and advance together, one period of
 * every member per cohort period, each pass of each step one launch over the
 * members of one arithmetic (the lockstep batches of qfd_step_batch, with the
 * energy checks batched too); the cadence and the stop rule stay per request.
 * Once no member is in the first period of a phase, a cohort period is
 * captured as one CUDA graph and replayed while the members and their states
 * and phases are unchanged.  Stream priority rises as the lattice shrinks, as
 * for single requests.  The step kernels are the same as a lone plan's, so a
 * request's numbers are bit-identical in a cohort, alone, without cohorts and
 * through qfd_solve_states. */
typedef struct qfd_server_s* qfd_server_t;

typedef struct {
  double hbm_budget_bytes; /* admission budget (device bytes of admitted requests) */
  int32_t max_active;      /* at most this many requests at once (0: no limit) */
  int32_t check_every;     /* steps per period; a multiple of ortho_every */
  int32_t ortho_every;     /* projection / normalisation cadence of every request */
  int32_t use_graphs;      /* 1: capture a request's period once per phase and replay it */
  void* stream;            /* cudaStream_t whose queued work admitted requests follow, or NULL */
  int32_t cohorts;         /* 1: lockstep cohorts of requests of one size (see above); 0: a stream per request */
  int32_t autotune;        /* 1: the first request of each lattice size and precision runs qfd_autotune
                              on its plan, and every later one of that kind takes the same launch
                              shapes (so requests of one kind still give the same numbers in any
                              mix within the server's life); 0: default shapes */
} qfd_server_params;

typedef struct {
  int64_t n;               /* lattice as in qfd_params */
  double a, mass, dtau;
  int32_t kinetic, rest_mass;
  int32_t nstates;         /* 1..8 states, solved in turn with Gram-Schmidt */
  int32_t precision;       /* QFD_C128, QFD_C64, QFD_DF64, QFD_C64_REFINE, QFD_C64_REFINE_DF */
  int32_t potential;       /* QFD_POT_* with coefficients pot_coeffs[0..1] */
  int32_t stop_rule;       /* QFD_STOP_* */
  double pot_coeffs[2];
  int32_t centre;
  int32_t parity[8];       /* per state */
  uint64_t seed;           /* state i starts from qfd_fill_psi_uniform(seed + i) */
  int64_t max_steps;       /* per state and phase */
  double tol, tol_bulk;
  double grf_amplitude;    /* > 0: add qfd_add_random_field(grf_seed, grf_corr, grf_amplitude) */
  double grf_corr;
  uint64_t grf_seed;
} qfd_request;

typedef struct {
  int64_t id;
  int32_t status;          /* QFD_OK, QFD_ERR_NOT_CONVERGED, or the error that ended it */
  int32_t nstates;
  double energy[8];        /* final energy per state */
  int64_t steps[8];        /* steps per state (all phases) */
  int64_t steps_c64[8];    /* of which complex64 bulk steps */
  double t_submit, t_admit, t_done; /* seconds on the server clock */
} qfd_result;

qfd_status qfd_server_create(const qfd_server_params* params, qfd_server_t* out);
void qfd_server_destroy(qfd_server_t server);
const char* qfd_server_last_error(qfd_server_t server);
double qfd_server_clock(qfd_server_t server);
qfd_status qfd_server_submit(qfd_server_t server, const qfd_request* request, int64_t* id);
/* One scheduling round (see above); up to `capacity` finished results are
 * written to out, the rest stay for the next call. */
qfd_status qfd_server_poll(qfd_server_t server, qfd_result* out, int capacity, int* count);
/* Watchdog on the periods in flight (a serving safeguard; the paper has no
 * counterpart): a period still unfinished `seconds` after it was queued (time
 * spent waiting behind other requests' work counts) ends its request with
 * QFD_ERR_TIMEOUT in its qfd_result; the work already queued for it still
 * runs to its end on the device before its memory is released, and the other
 * requests go on.  0 (the default) turns the watchdog off.  QFD_ERR_ARG for a
 * negative or non-finite value. */
qfd_status qfd_server_set_timeout(qfd_server_t server, double seconds);
/* Kernel launches the server has queued so far: direct launches plus the
 * launches held by every replayed CUDA graph (server instrumentation; no
 * counterpart in the paper). */
qfd_status qfd_server_kernels(qfd_server_t server, int64_t* kernels);
qfd_status qfd_server_stats(qfd_server_t server, int* waiting, int* active, double* used_bytes, int64_t* periods,
                            int64_t* graph_replays, int64_t* graph_captures);

/* The plan's CUDA stream (cudaStream_t) for event recording by the caller. */
void* qfd_get_stream(qfd_plan_t plan);

/* Blocks until all work queued on the plan's stream has finished. */
qfd_status qfd_sync(qfd_plan_t plan);

#ifdef __cplusplus
}
#endif

#endif /* QFD_H */
