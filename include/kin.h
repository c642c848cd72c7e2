/*
 * kin — batched Radau IIA integration of constant-pressure reactor states on
 * NVIDIA GB300 (sm_103a).  C ABI of libkin.so.
 *
 * What is computed (Curtis, Niemeyer & Sung, "An investigation of GPU-based
 * stiff chemical kinetics integration methods"): each state (T, P, Y) is an
 * independent initial-value problem of the constant-pressure,
 * mass-fraction-based reactor (Sec. 2.1), advanced over one global time step
 * dt with the three-stage, fifth-order Radau IIA method, adaptive internal
 * steps under atol/rtol and per-IVP Jacobian reuse (Sec. 2.1), with an
 * analytical Jacobian or a CVODE-style finite-difference one (Sec. 2.1,
 * Sec. 3.4).  Source terms: reversible Arrhenius, third-body and Troe
 * falloff reactions, reverse rates from NASA-7 thermodynamics.
 *
 * Conventions for every entry point:
 *   - Units are SI with kmol: T in K, P in Pa, W in kg/kmol, Arrhenius A in
 *     (m^3/kmol)^(order-1)/s, activation temperatures Theta = Ea/R in K.
 *   - States are stored species-major (structure of arrays): Y[k*n + i] is
 *     the mass fraction of species k in state i; T[i], P[i].  All ns mass
 *     fractions are stored; the last species is inert and, on output, equals
 *     1 minus the sum of the others.
 *   - "dev" pointers are CUDA device pointers owned by the caller; "host"
 *     pointers are host memory owned by the caller.  The library owns the
 *     mechanism tables, its workspace and its counters.
 *   - Functions taking a stream are asynchronous on that stream (NULL = the
 *     legacy default stream); results are valid after the stream
 *     synchronises.  A kin_mech is used by one stream at a time.
 *   - Errors: every function returns a kin_status.  Argument errors and CUDA
 *     errors are reported at call time and leave outputs unspecified.
 *     Per-state numerical failures are not call errors: they are written to
 *     the optional status array, and the failed state keeps its last
 *     accepted values (a failing IVP keeps its solution, Sec. 1).
 */
#ifndef KIN_H
#define KIN_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  KIN_OK = 0,
  KIN_ERR_INVALID_ARG = 1,
  KIN_ERR_CUDA = 2,
  KIN_ERR_NOMEM = 3,
  KIN_ERR_MECH = 4,
  KIN_ERR_STATE_FAILED = 5,
  KIN_ERR_UNSUPPORTED = 6
} kin_status;

/* per-state status codes written to the status array */
enum {
  KIN_STATE_OK = 0,
  KIN_STATE_MAX_STEPS = 1,   /* internal step limit reached */
  KIN_STATE_H_UNDERFLOW = 2, /* internal step below round-off of t (a final step
                                that short instead ends the integration at dt) */
  KIN_STATE_SINGULAR = 3,    /* iteration matrix singular 5 times in a row */
  KIN_STATE_NONFINITE = 4,   /* non-finite right-hand side or Jacobian */
  KIN_STATE_NEWTON_FIXED = 5 /* kin_options.h_fixed: Newton failed at the fixed step */
};

/* maximum number of species (N = ns unknowns per state) */
#define KIN_MAX_SPECIES 64

/* Mechanism description: plain host arrays, copied by kin_mech_create.
 *   W     [ns]      molar masses
 *   nasa  [ns*17]   T_low, T_mid, T_high, 7 coefficients for T < T_mid,
 *                   7 for T >= T_mid (NASA-7: cp/R, h/RT, s/R polynomials)
 *   reac  [nr*3]    species index of each reactant slot, -1 = empty slot
 *                   (a species listed twice has coefficient 2)
 *   prod  [nr*3]    same for products
 *   arrh  [nr*3]    A, b, Theta of k = A T^b exp(-Theta/T) (k_inf for Troe)
 *   rtype [nr]      0 elementary, 1 third body, 2 Troe falloff
 *   eff   [nr*ns]   collision efficiencies (used by types 1 and 2; 1 = default)
 *   fall  [nr*7]    type 2: k0 A, k0 b, k0 Theta, Troe a, T***, T*, T**
 * The last species (ns-1) must take part in no reaction (it may collide). */
typedef struct {
  int32_t ns, nr;
  const double *W;
  const double *nasa;
  const int32_t *reac;
  const int32_t *prod;
  const double *arrh;
  const int32_t *rtype;
  const double *eff;
  const double *fall;
} kin_mech_desc;

typedef struct kin_mech kin_mech;

/* Kernel layouts. */
enum {
  KIN_LAYOUT_PLAIN = 0, /* one state per thread, nested step/Newton loops: the
                           paper's GPU organisation (Sec. 1, Sec. 3.3) */
  KIN_LAYOUT_QUEUE = 1  /* one state per thread in a persistent launch: every
                           loop trip is one step attempt per lane, and a lane
                           whose state is done takes the next one from an
                           atomic work queue (answers the warp divergence of
                           Sec. 3.3: no lane waits for the slowest state) */,
  KIN_LAYOUT_WARP = 2,  /* one state per group of kin_options.lanes lanes
                           (a whole warp: ns <= 63; 4, 8 or 16 lanes:
                           ns <= 15): vectors over the group's lanes, Newton
                           matrices in shared memory, group-cooperative LU
                           and solves, rates in parallel over reactions;
                           groups pop states from the atomic queue (the
                           per-block strategy of Sec. 3.3) */
  KIN_LAYOUT_AUTO = 3   /* the library chooses at each call: the launch
                           configuration kin_autotune last found for this
                           mechanism with the same matrix precision, Jacobian
                           kind and decade of dt (of the tuned batch sizes,
                           the one nearest to n in log2), else PLAIN with 64
                           threads for ns <= 16 and WARP with 32 lanes beyond
                           (the per-thread matrices no longer fit on chip);
                           with h_fixed > 0, where WARP is not available,
                           PLAIN.  kin_resolve_options shows the choice. */
};

/* Integration options.  kin_options_default fills the defaults. */
typedef struct {
  int32_t layout;        /* KIN_LAYOUT_*                                   (3) */
  int32_t lu_fp32;       /* 1: Jacobian storage, factorisation and solves of
                            the Newton matrices in FP32 (rates, residuals,
                            stage update, error estimate stay FP64)       (0) */
  int32_t jac_fd;        /* 1: CVODE-style one-sided difference Jacobian   (0) */
  int32_t max_steps;     /* internal step limit per state             (100000) */
  int32_t nit;           /* Newton iterations per step                     (7) */
  int32_t block;         /* threads per block; 0 = library choice          (0) */
  int32_t grid_per_sm;   /* QUEUE: resident blocks per SM; 0 = occupancy   (0) */
  int32_t transform_tol; /* 1: rtol' = 0.1 rtol^(2/3), atol' = rtol' atol/rtol (1) */
  int32_t queue_refill;  /* QUEUE: a warp refills once at least this many of its
                            lanes are idle (1..32), taking that many states
                            with one atomic; 0 = 1                         (0) */
  int32_t stop_after;    /* > 0: end a state after this many accepted steps
                            (it is returned at the time reached, status 0);
                            used to collect first steps for training     (0) */
  const double *h0;      /* dev [n] first internal step per state, or NULL  */
  const double *z0;      /* dev [3*ns][n] first-step stage guesses, or NULL */
  double *h_first;       /* dev [n] out: first accepted step, or NULL       */
  double *z_first;       /* dev [3*ns][n] out: converged first-step stages  */
  const int32_t *order;  /* dev [n] slot -> state permutation (for example from
                            kin_order_states), or NULL for the identity.
                            Slot i integrates state order[i]; indices of Y,
                            T, P, status, counters, h0, z0, h_first, z_first
                            are state indices.  Entries outside [0, n) are
                            skipped and make kin_get_stats return
                            KIN_ERR_INVALID_ARG; a repeated entry integrates
                            that state twice and leaves another untouched.
                            n <= 2^31 - 1 with an order.              (NULL) */
  int32_t lanes;         /* KIN_LAYOUT_WARP: lanes per state, 4, 8, 16 or 32
                            (0 = 32).  4, 8 and 16 hold at most 15 species
                            and place 32/lanes states in each warp      (0) */
  double h_fixed;        /* > 0: constant internal step h_fixed (the last step
                            clipped onto dt; x + 1.0001 h >= dt ends it),
                            every step accepted, a fresh Jacobian every step,
                            Newton iterated until it converges, diverges or
                            reaches nit (no slow-contraction exit); the error
                            estimate is still computed.  For
                            convergence studies (Sec. 2.3).  PLAIN and QUEUE
                            layouts only; a Newton failure ends the state
                            with KIN_STATE_NEWTON_FIXED                 (0) */
  int32_t order_by;      /* kin_integrate_host only: 1 = order the states by
                            the starting-step heuristic (kin_order_states) in
                            the entry's own device buffers before integrating;
                            0 = none.  kin_integrate_ex takes an explicit
                            order instead and rejects a nonzero value    (0) */
} kin_options;

/* Per-state counters written by kin_integrate_ex when counters != NULL:
 * counters[c*n + i] for c in this order. */
enum {
  KIN_CNT_NSTEP = 0, KIN_CNT_NACCPT, KIN_CNT_NREJCT, KIN_CNT_NFCN, KIN_CNT_NJAC,
  KIN_CNT_NDEC, KIN_CNT_NSOL, KIN_CNT_STATUS, KIN_NCOUNTERS
};

/* Fill *opt with the defaults shown above.  Returns KIN_ERR_INVALID_ARG for NULL. */
int kin_options_default(kin_options *opt);

/* Copy a mechanism description to the device and build its tables
 * (Sec. 2.1: source terms and Jacobian of the chosen model).  *out receives a
 * handle to free with kin_destroy.  Errors: KIN_ERR_INVALID_ARG (NULL or
 * ns outside [2, KIN_MAX_SPECIES], nr < 1), KIN_ERR_MECH (a slot index out
 * of range, an inert species that reacts, a non-positive molar mass or
 * temperature bound), KIN_ERR_NOMEM / KIN_ERR_CUDA (device allocation). */
int kin_mech_create(const kin_mech_desc *desc, kin_mech **out);

/* Free a mechanism and its workspace.  NULL is ignored.  The caller must not
 * have work in flight on the mechanism. */
void kin_destroy(kin_mech *m);

/* Advance n independent states over one global step dt (Sec. 2.1, Sec. 3):
 * Y dev [ns][n] in/out, T dev [n] in/out, P dev [n] (constant).  Radau IIA
 * with rtol/atol (the paper uses rtol 1e-6, atol 1e-10) and the default
 * options.  n = 0 is a no-op.  Errors: KIN_ERR_INVALID_ARG for NULL
 * pointers with n > 0, n < 0, dt <= 0 or non-positive tolerances;
 * KIN_ERR_CUDA if a launch fails. */
int kin_integrate(kin_mech *m, double *Y, double *T, const double *P, int64_t n, double dt,
                  double rtol, double atol, void *stream);

/* kin_integrate with options (NULL = defaults) and optional per-state
 * outputs: status dev [n] (KIN_STATE_*), counters dev [KIN_NCOUNTERS][n]
 * (statistics and the internal step counts d_i of Sec. 3.3). */
int kin_integrate_ex(kin_mech *m, double *Y, double *T, const double *P, int64_t n, double dt,
                     double rtol, double atol, const kin_options *opt, int32_t *status,
                     int32_t *counters, void *stream);

/* The same integration from HOST buffers: the library copies the inputs to
 * device buffers it owns, integrates, copies Y and T back and synchronises
 * the stream before returning (the paper's timing includes these copies,
 * Sec. 3).  Y host [ns][n], T host [n] in/out; P host [n]; status and
 * counters host or NULL.  Device pointers inside opt are not allowed
 * (KIN_ERR_INVALID_ARG).  Pinned host memory gives asynchronous copies. */
int kin_integrate_host(kin_mech *m, double *Y, double *T, const double *P, int64_t n, double dt,
                       double rtol, double atol, const kin_options *opt, int32_t *status,
                       int32_t *counters, void *stream);

/* Autotuner: time candidate launch configurations on the caller's states
 * (Y, T, P dev, n states; copied, the inputs are not modified) and return the
 * fastest in *best.  The result is also kept in the mechanism's tuning cache
 * (keyed on the matrix precision, the Jacobian kind, the decade of dt and
 * log2 n; at most 64 entries, a repeated key replaced), which
 * KIN_LAYOUT_AUTO consults.  Candidates for ns <= 15: PLAIN with 64 and 32 threads
 * per block; QUEUE with 64 threads and refill batches 1, 4, 8, 16, 32; QUEUE
 * with 32 threads and refill 1; WARP with 32, 16, 8 and 4 lanes per state
 * (12 in all; the first max_candidates are timed).  ns = 16 drops the
 * grouped WARP forms (9).  For ns > 16 the per-thread matrices do not fit
 * on chip and WARP (32 lanes) is returned without timing.  The other option fields (precision,
 * Jacobian, limits; h0/z0 must be NULL) come from base (NULL = defaults).
 * Once a WARP candidate takes over twice the best time so far, the WARP
 * candidates after it (smaller lane groups) are skipped.
 * seconds: host [max_candidates] or NULL, each candidate's device time in
 * that order, -1 for a skipped one (entries past the candidates are not
 * written).  Allocates
 * and frees temporary device copies of the states.  Synchronises the
 * stream. */
int kin_autotune(kin_mech *m, const double *Y, const double *T, const double *P, int64_t n,
                 double dt, double rtol, double atol, const kin_options *base, kin_options *best,
                 double *seconds, int32_t max_candidates, void *stream);

/* The launch configuration kin_integrate_ex would use for a batch of n
 * states over dt with the options opt (NULL = defaults): *out = opt with
 * KIN_LAYOUT_AUTO replaced by the chosen layout, block, queue_refill and
 * lanes (other layouts are returned unchanged).  Host only; runs nothing on
 * the GPU.  Errors: KIN_ERR_INVALID_ARG for NULL m or out, n < 0, dt <= 0. */
int kin_resolve_options(kin_mech *m, int64_t n, double dt, const kin_options *opt,
                        kin_options *out);

/* Totals of the last kin_integrate* call on this mechanism, reduced on the
 * device: out[0..6] = sums of the KIN_CNT_* counters 0..6, out[7] = number of
 * failed states, out[8] = largest per-state step count.  Synchronises the
 * mechanism's last stream.  Returns KIN_ERR_INVALID_ARG when the call's
 * kin_options.order held entries outside [0, n) (those slots were skipped),
 * else KIN_ERR_STATE_FAILED when out[7] > 0. */
int kin_get_stats(kin_mech *m, int64_t *out);

/* Stiffness-ordered batching.  The paper names warp divergence from differing
 * internal step counts as the main limit of the per-thread integrator
 * (Sec. 3.3, Sec. 4.2); grouping states of similar stiffness in a warp
 * reduces it.  Writes to order (dev [n]) a permutation of 0..n-1 that sorts
 * key (dev [n]) ascending, stiffest states first, by a counting sort into
 * 4096 equal-width bins between the smallest and largest finite key (-inf
 * first, +inf and NaN last; the order within a bin is unspecified, and the
 * integration of a state does not depend on its slot).
 *   key_mode KIN_KEY_STEP_HEURISTIC: the library first writes into key the
 *     natural log of the starting-step heuristic 0.01 d0/d1 (weighted RMS
 *     norms of y and f(y), tolerances transformed as in the integrator): one
 *     right-hand side per state from Y, T, P (dev, as kin_integrate); a state
 *     whose rates are not finite gets -inf.
 *   key_mode KIN_KEY_GIVEN: key is read as given; Y, T, P, rtol and atol
 *     are not used and may be NULL/0.
 *   key_mode KIN_KEY_GIVEN_LOG: as KIN_KEY_GIVEN, sorted by the natural log
 *     of a positive key (for example the predictor's h0 from
 *     kin_mlp_predict); a zero key goes first and a negative one last.
 * n <= 2^31 - 1.  Asynchronous on stream; uses a workspace owned by the
 * mechanism, so calls on one kin_mech must not overlap. */
enum { KIN_KEY_GIVEN = 0, KIN_KEY_STEP_HEURISTIC = 1, KIN_KEY_GIVEN_LOG = 2 };
int kin_order_states(kin_mech *m, const double *Y, const double *T, const double *P, int64_t n,
                     double rtol, double atol, int32_t key_mode, double *key, int32_t *order,
                     void *stream);

/* Source terms f(y) for n states (y = [T, Y_0..Y_{ns-2}], N = ns):
 * y dev [N][n], P dev [n], f dev [N][n] out.  Unit-level entry of the
 * right-hand side every Radau stage evaluates (Sec. 2.1). */
int kin_rhs(kin_mech *m, const double *y, const double *P, int64_t n, double *f, void *stream);

/* Jacobian df/dy for n states: J dev [N*N][n] out, entry (r, c) at
 * J[(r*N + c)*n + i].  fd = 0: analytical (Sec. 2.1); fd = 1: the one-sided
 * difference quotient with the CVODE increment rule, which also needs
 * h (the internal step) and scal dev [N][n] (error weights 1/w). */
int kin_jacobian(kin_mech *m, const double *y, const double *P, int64_t n, int32_t fd, double h,
                 const double *scal, double *J, void *stream);

/* Size of the device array kin_integrate_static works in: 64 KiB for the
 * mechanism tables plus 256 B of counters. */
#define KIN_STATIC_SCRATCH_BYTES (64 * 1024 + 256)

/* kin_integrate with the default options for callers that cannot allocate
 * device memory: no cudaMalloc, cudaFree or allocating library call is made.
 * Such callers run inside a host framework whose own allocator owns (and may
 * have reserved) all device memory, or in a loop that must not allocate once
 * running.  The mechanism is passed as its host description; its tables and
 * the kernel's counters go to a fixed device array inside libkin
 * (KIN_STATIC_SCRATCH_BYTES, held by every GPU that loads the library until
 * the process exits) instead of a kin_mech's workspace.  The paper has no
 * counterpart.  Y, T, P and status are as for kin_integrate_ex (dev
 * pointers).
 *   - Kernel: one state per thread (PLAIN), FP64 Newton matrices, whatever
 *     the mechanism size: the state-per-warp layout needs a per-mechanism
 *     workspace.  It serves mechanisms of up to 16 species at the thread
 *     layouts' speed; larger ones are integrated correctly but far more
 *     slowly than kin_integrate_ex would (its 64-species per-thread kernel).
 *   - Set-up: the first call on a device looks up the array's device
 *     address.  The first launch of an integration kernel on a device can
 *     also make the CUDA driver reserve local memory for the kernel's
 *     per-thread frame times the device's resident threads (gigabytes for
 *     these kernels); a host whose allocator reserves all device memory
 *     should make one call, on any small batch, before it does.
 *   - Not capturable: the tables are uploaded from host memory the call
 *     frees, so a call on a stream that is being captured into a CUDA graph
 *     returns KIN_ERR_UNSUPPORTED and issues nothing.
 *   - Sharing: every call uses the same array, rewrites the tables and
 *     clears the counters before its launch; calls whose GPU work overlaps
 *     (on different streams) race on it and must not be issued.  The
 *     per-state status is the only diagnostic: kin_get_stats cannot see a
 *     static call's totals, and the array's contents after a call are
 *     unspecified.
 * Errors: as kin_integrate, plus KIN_ERR_UNSUPPORTED when the mechanism's
 * tables exceed 64 KiB or the stream is capturing. */
int kin_integrate_static(const kin_mech_desc *desc, double *Y, double *T, const double *P,
                         int64_t n, double dt, double rtol, double atol, int32_t *status,
                         void *stream);

/* The exponential the rate kernels use (Tang's table-driven method, accurate
 * to about 1 ulp for |x| < 700, the library exp beyond): y[i] = exp(x[i]) for
 * x, y dev [n].  Unit-level entry for testing; needs a mechanism only for
 * its 2^(j/256) table. */
int kin_exp(kin_mech *m, const double *x, double *y, int64_t n, void *stream);

/* Radau IIA constants the kernels use, computed by the library from closed
 * forms (Hairer & Wanner IV.5, IV.8; the method of Sec. 2.1):
 * out[0..2] c, [3..5] gamma, alpha, beta (eigenvalues of A^-1),
 * [6..14] T row-major, [15..23] T^-1, [24..26] error weights d_i
 * (the estimate is (gamma/h I - J)^-1 (f0 + sum d_i z_i / h)).  len >= 27.
 * Needs no GPU. */
int kin_radau_constants(double *out, int32_t len);

/* ---------------------------------------------------------------------------
 * Concentration-based form with a sparse LU (Sec. 3.3 and Sec. 4: the paper
 * proposes reformulating the kinetics in species concentrations so that the
 * Jacobian is sparse and the Newton matrices admit a sparse factorisation).
 * Each state is integrated in phi = [T, V, n_0 .. n_{ns-2}] per unit mass of
 * mixture at constant pressure: the volume and the moles of every species
 * but the last (the inert bath gas, whose moles close P V = n Ru T):
 *   dn_k/dt = V wdot_k,  dT/dt = -sum_k H_k wdot_k / sum_k C_k Cp_k,
 *   dV/dt = V (Ru T / P sum_k wdot_k + (dT/dt) / T),  C_k = n_k / V.
 * The Jacobian couples two species only through a reaction both take part
 * in, or a collision efficiency that differs from the bath gas's; the T and
 * V rows and columns are full.  Radau IIA is the same method as
 * kin_integrate's, with rtol/atol weighing phi; inputs and outputs are mass
 * fractions (n_k = Y_k / W_k, V = 1 / rho on entry; Y_k = W_k n_k over the
 * mixture's mass on exit), so the results are those of the same reactor
 * integrated to the same tolerances in other variables.
 * ------------------------------------------------------------------------- */
typedef struct kin_conc kin_conc;

/* Symbolic analysis only (host; no GPU): the elimination order and the
 * filled pattern kin_conc_create would use.  The species are ordered by
 * minimum degree of the symmetric species structure (ties to the lower
 * index), T and V last; the LU takes its pivots in that order, without
 * pivoting.  var host [ns+1] or NULL: var[g] = the phi index (0 T, 1 V,
 * 2 + k species k) at elimination position g.  pattern host [(ns+1)^2] or
 * NULL: 1 where L + U (diagonal included) may be non-zero, row-major in
 * elimination order.  counts host [4] or NULL: non-zeros of J's pattern,
 * non-zeros of L + U, operations of one real factorisation over the pattern
 * (a division and the multiplier products per pivot, 2 per update) and of
 * one real solve (2 per off-diagonal entry and N divisions).  Errors:
 * KIN_ERR_INVALID_ARG (NULL desc or arrays, ns outside [2, KIN_MAX_SPECIES],
 * nr < 1), KIN_ERR_MECH (a slot out of range, the last species reacting),
 * KIN_ERR_UNSUPPORTED (the last species has a non-default collision
 * efficiency, which would couple every species). */
int kin_conc_analyse(const kin_mech_desc *desc, int32_t *var, uint8_t *pattern,
                     int64_t *counts);

/* Build the device tables and the sparse structure of a mechanism for the
 * concentration-based form on the current device; *out receives a handle to
 * free with kin_conc_destroy.  Errors: those of kin_mech_create and
 * kin_conc_analyse, and KIN_ERR_UNSUPPORTED for ns > 63. */
int kin_conc_create(const kin_mech_desc *desc, kin_conc **out);

/* Free a plan and its workspace (NULL is ignored; no work may be in flight). */
void kin_conc_destroy(kin_conc *c);

/* kin_integrate_ex in the concentration-based form: Y dev [ns][n] in/out,
 * T dev [n] in/out, P dev [n].  One state per warp (32 lanes), Newton
 * matrices dense in shared memory or a global slot as in KIN_LAYOUT_WARP but
 * factorised and solved over the sparse pattern.  Options (NULL = defaults):
 * layout WARP or AUTO, lanes 0 or 32, analytical Jacobian, no h_fixed, no z0
 * or z_first (KIN_ERR_UNSUPPORTED otherwise); lu_fp32, max_steps, nit,
 * transform_tol, stop_after, h0, h_first and order as kin_integrate_ex.  A
 * zero pivot counts as a singular matrix (KIN_STATE_SINGULAR after 5 in a
 * row).  status and counters as kin_integrate_ex.  Asynchronous on stream;
 * calls on one kin_conc must not overlap. */
int kin_integrate_conc(kin_conc *c, double *Y, double *T, const double *P, int64_t n, double dt,
                       double rtol, double atol, const kin_options *opt, int32_t *status,
                       int32_t *counters, void *stream);

/* Totals of the last kin_integrate_conc call, as kin_get_stats. */
int kin_conc_get_stats(kin_conc *c, int64_t *out);

/* ---------------------------------------------------------------------------
 * exprb43: the fourth-order exponential Rosenbrock method the paper runs
 * beside Radau IIA (Sec. 2.1, Table of solvers; Sec. 3.1), for the same
 * mass-fraction reactor and analytical Jacobian.  With g(u) = F(u) - J_n u
 * and D_i = g(U_i) - g(u_n):
 *   U2 = u_n + h/2 phi1(h/2 J) F(u_n),  U3 = u_n + h phi1(h J) (F(u_n) + D2),
 *   u_{n+1} = u_n + h phi1(h J) F(u_n) + h (16 phi3 - 48 phi4)(h J) D2
 *             + h (-2 phi3 + 12 phi4)(h J) D3,
 * with the embedded third-order solution (16 phi3 D2 - 2 phi3 D3) for the
 * step-size control (Hairer-Norsett-Wanner: weights atol + rtol max(|u_n|,
 * |u_{n+1}|), h min(5, max(0.2, 0.9 err^-1/4)), no growth right after a
 * rejection; a non-finite stage halves h).  J_n is evaluated at every new
 * point.  The phi-function products come from one Krylov space per vector
 * (Arnoldi), grown until Saad's leading error term of every product taken
 * from it is at most kappa in the step's error weights (kappa = 0: the
 * whole space), and phi_k of the small Hessenberg matrix from the
 * exponential of an augmented matrix (scaling and squaring, Pade (6,6)).
 * One state per warp; ns <= 57.
 * ------------------------------------------------------------------------- */
typedef struct kin_exprb kin_exprb;

/* Build the tables and the per-warp workspace (basis, Hessenberg and
 * matrix-function work, about 8 (ns+7)^2 doubles per resident warp) on the
 * current device.  Errors: those of kin_mech_create; KIN_ERR_UNSUPPORTED
 * for ns > 57. */
int kin_exprb_create(const kin_mech_desc *desc, kin_exprb **out);

/* Free (NULL is ignored; no work may be in flight). */
void kin_exprb_destroy(kin_exprb *x);

/* Advance n states over dt: Y dev [ns][n], T dev [n] in/out, P dev [n];
 * tolerances as given (no transform); kappa >= 0 the Krylov tolerance;
 * h0 dev [n] first steps or NULL (the starting-step heuristic); max_steps
 * >= 1 per state.  status dev [n] (KIN_STATE_OK, _MAX_STEPS, _H_UNDERFLOW,
 * _NONFINITE) and counters dev [8][n] or NULL: steps, accepted, rejected,
 * right-hand sides, Jacobians, Krylov spaces built, their summed dimension,
 * status.  Errors: KIN_ERR_INVALID_ARG (NULL with n > 0, n < 0, dt, rtol or
 * atol not positive, kappa negative, max_steps < 1, another device).
 * Asynchronous on stream; calls on one kin_exprb must not overlap. */
int kin_integrate_exprb(kin_exprb *x, double *Y, double *T, const double *P, int64_t n,
                        double dt, double rtol, double atol, double kappa, const double *h0,
                        int32_t max_steps, int32_t *status, int32_t *counters, void *stream);

/* Totals of the last kin_integrate_exprb call in the counters' order (0..6),
 * failed states (7) and the largest step count (8); KIN_ERR_STATE_FAILED
 * when a state failed. */
int kin_exprb_get_stats(kin_exprb *x, int64_t *out);

/* The matrix functions the Krylov products use, as a unit-level entry for
 * testing: out[i*p + k-1] = (phi_k(tau H) e1)_i for k = 1..p, i < m, H dev
 * [m*m] row-major, out dev [m*p]; 1 <= m <= ns, 1 <= p <= 5.  Runs on one
 * warp in the first workspace slot (no integration may be in flight).
 * KIN_ERR_INVALID_ARG outside those ranges; NaN when the Pade denominator is
 * singular or tau H is not finite. */
int kin_exprb_phi(kin_exprb *x, const double *H, int32_t m, int32_t p, double tau, double *out,
                  void *stream);

/* The right-hand side and analytical Jacobian exprb43 evaluates (those of the
 * state-per-warp kernels), as a unit-level entry for testing: y dev [N][n]
 * (N = ns, y = [T, Y_0..Y_{ns-2}]), P dev [n]; f dev [N][n] from the
 * evaluation that assembles J, f_rates dev [N][n] from the rate-only
 * evaluation, J dev [N*N][n] with entry (r, c) at J[(r*N + c)*n + i].  No
 * integration may be in flight on x. */
int kin_exprb_chem(kin_exprb *x, const double *y, const double *P, int64_t n, double *f,
                   double *f_rates, double *J, void *stream);

/* ---------------------------------------------------------------------------
 * Step/guess predictor (the learned part; the paper has no counterpart).
 * An MLP x (din) -> 3 x [Linear(width) -> SiLU] -> Linear(dout) trained on
 * first steps the integrator itself produced, predicting the first internal
 * step (log h0) and the first step's Newton starting stages (3 N values),
 * which kin_options.h0 / .z0 feed back to the integrator.  Radau keeps its
 * error test and step control, so only rejected steps and Newton iterations
 * can change.  precision 0: BF16 tensor-core GEMMs with FP32 accumulation,
 * BF16 activations between layers, FP32 master weights and Adam; 1: FP32
 * everywhere (a check mode).  Matrices are row-major [rows][features], FP32,
 * device pointers unless stated.  Calls on one kin_mlp are stream-ordered
 * (one stream at a time).
 * ------------------------------------------------------------------------- */
typedef struct kin_mlp kin_mlp;

/* Create with seeded He-uniform weights and zero biases.  KIN_ERR_INVALID_ARG
 * for sizes out of [1, 4096] (width >= 8) or an unknown precision. */
int kin_mlp_create(int32_t din, int32_t width, int32_t dout, int32_t precision, uint64_t seed,
                   kin_mlp **out);
void kin_mlp_destroy(kin_mlp *net);
/* Parameter count of the layout W0 [din][width], b0, W1, b1, W2, b2,
 * W3 [width][dout], b3 used by get/set (host arrays); -1 for NULL. */
int64_t kin_mlp_num_params(const kin_mlp *net);
int kin_mlp_get_params(kin_mlp *net, float *host, int64_t len);
/* set also resets the optimiser state */
int kin_mlp_set_params(kin_mlp *net, const float *host, int64_t len);
/* Y [M][dout] = net(X [M][din]). */
int kin_mlp_forward(kin_mlp *net, const float *X, float *Y, int64_t M, void *stream);
/* Gradient of the mean squared error over X [M][din], targets T [M][dout]:
 * grad_out dev [num_params] (same layout as get/set) or NULL, loss_out dev
 * scalar or NULL.  Synchronises the stream when grad_out is given. */
int kin_mlp_grad(kin_mlp *net, const float *X, const float *T, int64_t M, float *grad_out,
                 float *loss_out, void *stream);
/* One Adam step (beta 0.9 / 0.999, eps 1e-8, bias-corrected) on a minibatch. */
int kin_mlp_train_step(kin_mlp *net, const float *X, const float *T, int64_t M, float lr,
                       float *loss_out, void *stream);
/* The same step on the minibatch rows[0..M) (dev int32) of a training set
 * X dev [R][din], T dev [R][dout]: the library gathers the rows itself.  An
 * index outside [0, R) contributes a zero row.  The gather buffers belong to
 * the network and grow with M. */
int kin_mlp_train_step_rows(kin_mlp *net, const float *X, const float *T, int64_t R,
                            const int32_t *rows, int64_t M, float lr, float *loss_out,
                            void *stream);
/* Column means and standard deviations (floored at 1e-12) of X [M][d]. */
int kin_moments(const float *X, int64_t M, int32_t d, float *mean, float *stdv, void *stream);
/* Network inputs for n states (Y dev [ns][n], T, P dev [n], all FP64):
 * X [n][3 + ns] = [ln T, ln P, ln dt, log10(max(Y_k, 1e-12))], standardised
 * with mean/stdv [3 + ns] unless both are NULL. */
int kin_mlp_features(int32_t ns, const double *Y, const double *T, const double *P, int64_t n,
                     double dt, const float *mean, const float *stdv, float *X, void *stream);
/* Training targets [n][1 + nz] = [ln h, z_0..z_{nz-1}] from the integrator's
 * first-step outputs h dev [n], z dev [nz][n] (kin_options.h_first /
 * .z_first), standardised with mean/stdv [1 + nz] unless both are NULL. */
int kin_mlp_targets(int32_t nz, const double *h, const double *z, int64_t n, const float *mean,
                    const float *stdv, float *tgt, void *stream);
/* Features -> network -> h0 dev [n] (exp of the de-standardised output 0,
 * clipped to [1e-14, dt]) and z0 dev [3 ns][n] (outputs 1..3 ns) for
 * kin_options.h0 / .z0; either output may be NULL.  The net must have
 * din = 3 + ns and dout = 1 + 3 ns. */
int kin_mlp_predict(kin_mlp *net, int32_t ns, const double *Y, const double *T, const double *P,
                    int64_t n, double dt, const float *in_mean, const float *in_std,
                    const float *out_mean, const float *out_std, double *h0, double *z0,
                    void *stream);

/* Message for a kin_status. */
const char *kin_status_string(int status);

#ifdef __cplusplus
}
#endif
#endif
