/*
 * FP64 CPU oracle for batched Radau IIA integration of constant-pressure
 * reactor states.  TEST INFRASTRUCTURE ONLY: only the test-suite, the smoke
 * check and the benchmark's CPU-baseline leg may load it.  It shares no code
 * with the CUDA path and is written for obviousness, not speed: naive loops,
 * dense matrices, no blocking, no fusion.
 *
 * What it computes (paper: Curtis, Niemeyer & Sung, "An investigation of
 * GPU-based stiff chemical kinetics integration methods"):
 *   - the constant-pressure, mass-fraction-based reactor ODE with source terms
 *     and an analytical Jacobian (Sec. 2.1, the formulation the paper takes
 *     from pyJac);
 *   - a one-sided finite-difference Jacobian in the style of CVODE (Sec. 2.1,
 *     Sec. 3.4);
 *   - the three-stage, fifth-order Radau IIA method with its built-in
 *     step-size control and Jacobian reuse (Sec. 2.1, Table "solvers"), with
 *     atol/rtol as in Sec. 2.1;
 *   - per-state statistics (internal step counts d_i, Sec. 3.3).
 *
 *   - the concentration-based (extensive, moles) form of the same reactor,
 *     whose Jacobian is sparse (Sec. 3.3, Sec. 4): chem.c, orc_rhs_conc.
 *
 * State vector: y = [T, Y_0 .. Y_{ns-2}], N = ns; the last species is inert
 * and its mass fraction is 1 - sum of the others.  Units: SI with kmol.  The
 * concentration-based form's state is phi = [T, V, n_0 .. n_{ns-2}] per unit
 * mass (N = ns + 1).
 */
#ifndef KIN_ORACLE_H
#define KIN_ORACLE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ORC_RU 8314.46261815324 /* J/(kmol K) */
#define ORC_PATM 101325.0       /* Pa */

typedef struct {
  int ns, nr;
  const double *W;     /* [ns] kg/kmol */
  const double *nasa;  /* [ns*17] T_low, T_mid, T_high, low a1..a7, high a1..a7 */
  const int32_t *reac; /* [nr*3] species index per slot, -1 empty */
  const int32_t *prod; /* [nr*3] */
  const double *arrh;  /* [nr*3] A (SI), b, Theta (K); k_inf for Troe */
  const int32_t *rtype;/* [nr] 0 elementary, 1 third-body, 2 Troe */
  const double *eff;   /* [nr*ns] third-body efficiencies */
  const double *fall;  /* [nr*7] k0 A, k0 b, k0 Theta, a, T3, T1, T2 */
} orc_mech;

/* Radau options; see radau.c for the meaning of each. */
typedef struct {
  double rtol, atol;   /* user tolerances */
  int transform_tol;   /* 1: rtol' = 0.1 rtol^(2/3), atol' = rtol' atol / rtol */
  int nit;             /* maximum simplified-Newton iterations per step */
  double h0;           /* first internal step; <= 0 selects the heuristic */
  double hfixed;       /* > 0: constant internal step, no error control */
  int max_steps;       /* limit on attempted steps */
  int jac_kind;        /* 0 analytical, 1 finite difference */
  const double *z0;    /* optional first-step stage guess [3*N] or NULL */
  double *z_first_out; /* optional [3*N]: stage increments of the first accepted step */
  int form;            /* batch driver: 0 mass fractions, 1 concentration-based (moles) */
  const double *atol_scale; /* optional [N]: component i's absolute tolerance is
                               atol * atol_scale[i] (NULL: atol for all) */
} orc_opts;

typedef struct {
  int32_t nstep, naccpt, nrejct, nfcn, njac, ndec, nsol, status;
  double h_first;      /* first accepted internal step */
  double h_last;       /* step size proposed after the last accepted step */
  double err_last;     /* scaled error estimate of the last accepted step */
} orc_stats;

/* per-state status codes */
#define ORC_OK 0
#define ORC_MAX_STEPS 1
#define ORC_H_UNDERFLOW 2
#define ORC_SINGULAR 3
#define ORC_NONFINITE 4
#define ORC_NEWTON_FIXED 5 /* Newton failed at a fixed step: no smaller step to retry */

typedef int (*orc_rhs_fn)(void *ctx, double t, const double *y, double *f);
typedef int (*orc_jac_fn)(void *ctx, double t, const double *y, const double *f0,
                          double h, const double *scal, double *J);

/* chem.c */
void orc_thermo(const orc_mech *m, double T, double *cp_R, double *h_RT, double *s_R);
int orc_rhs(const orc_mech *m, double P, const double *y, double *f);
int orc_jac(const orc_mech *m, double P, const double *y, double *J);
int orc_jac_fd(const orc_mech *m, double P, const double *y, const double *f0,
               double h, const double *scal, double *J);
void orc_rate_constants(const orc_mech *m, double T, const double *C,
                        double *kf_eff, double *kr_eff);
void orc_wdot(const orc_mech *m, double T, double P, const double *Yfull, double *wdot);
int orc_rhs_conc(const orc_mech *m, double P, const double *phi, double *f);
int orc_jac_conc(const orc_mech *m, double P, const double *phi, double *J);

/* linalg.c */
int orc_lu_real(int n, double *a, int32_t *ipiv);
void orc_lu_solve_real(int n, const double *lu, const int32_t *ipiv, double *b);
int orc_lu_cplx(int n, double *a_re_im, int32_t *ipiv);
void orc_lu_solve_cplx(int n, const double *lu_re_im, const int32_t *ipiv, double *b_re_im);

/* radau.c */
typedef struct {
  double c[3], A[9], b[3];
  double gamma, alpha, beta;  /* eigenvalues of A^-1: gamma, alpha +- i beta */
  double T[9], TI[9];         /* T^-1 A^-1 T = [[gamma,0,0],[0,alpha,-beta],[0,beta,alpha]] */
  double e[3];                /* error-estimate weights on the stage increments */
  double gamma0;              /* weight of h f(y_n) in the embedded formula */
} orc_tableau;
void orc_radau_tableau(orc_tableau *tb);
int orc_radau(int n, orc_rhs_fn f, orc_jac_fn jac, void *ctx, double t0, double t1,
              double *y, const orc_opts *o, orc_stats *st);
double orc_initial_step(int n, orc_rhs_fn f, void *ctx, double t0, double t1,
                        const double *y, const double *f0, double rtol, double atol, int *nfcn);
int orc_fd_jacobian(int n, orc_rhs_fn f, void *ctx, double t, const double *y, const double *f0,
                    double h, const double *scal, double *J);

/* batch.c */
int orc_integrate_batch(const orc_mech *m, int64_t n, double *Y, double *T, const double *P,
                        double dt, const orc_opts *o, int32_t *status, int32_t *counters,
                        int nthreads);
int orc_num_threads(void);

#ifdef __cplusplus
}
#endif
#endif
