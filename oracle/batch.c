/*
 * Oracle batch driver: integrates independent reactor states over one global
 * step dt.  TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * Each state is its own IVP (Sec. 1, Sec. 3: one IVP per condition).  The
 * CPU runs parallelise per condition with OpenMP, one state per thread, as
 * the paper's CPU solvers do (Sec. 3); results do not depend on the thread
 * count.  A state whose integration fails keeps its last accepted values.
 *
 * Layout: Y is species-major [ns][n] (SoA), T and P are [n].  counters is
 * [n][8]: nstep, naccpt, nrejct, nfcn, njac, ndec, nsol, status.
 *
 * With o->form = 1 each state is integrated in the concentration-based form
 * (chem.c): per unit mass, n_k = Y_k / W_k and V = Ru T sum_k (Y_k / W_k) / P
 * on entry, with the moles' absolute tolerance atol / W_k (T's and V's atol); on exit the bath gas's moles close the ideal-gas law and the
 * mass fractions are W_k n_k over the mixture's mass sum_k W_k n_k.
 */
#include <stdlib.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#include "oracle.h"

typedef struct {
  const orc_mech *m;
  double P;
  int jac_kind;
} kin_ctx;

static int conc_rhs(void *c, double t, const double *y, double *f) {
  (void)t;
  kin_ctx *k = (kin_ctx *)c;
  return orc_rhs_conc(k->m, k->P, y, f);
}

static int conc_jac(void *c, double t, const double *y, const double *f0, double h,
                    const double *scal, double *J) {
  (void)t;
  kin_ctx *k = (kin_ctx *)c;
  if (k->jac_kind == 1)
    return orc_fd_jacobian(k->m->ns + 1, conc_rhs, c, 0.0, y, f0, h, scal, J);
  return orc_jac_conc(k->m, k->P, y, J);
}

/* one state in the concentration-based form; Yi strided by n */
static void integrate_conc(const orc_mech *m, double *Yi, int64_t n, double *Ti, double P,
                           double dt, const orc_opts *o, orc_stats *st) {
  int ns = m->ns, in = ns - 1;
  double *phi = malloc(sizeof(double) * (ns + 1));
  double S = 0.0;
  for (int k = 0; k < ns; ++k) S += Yi[(size_t)k * n] / m->W[k];
  phi[0] = *Ti;
  phi[1] = ORC_RU * *Ti * S / P;
  for (int k = 0; k < in; ++k) phi[2 + k] = Yi[(size_t)k * n] / m->W[k];
  /* the moles' absolute tolerance is atol / W_k, so a mole error weighs as
   * the mass-fraction error W_k dn_k does in the mass-fraction form */
  double *aw = malloc(sizeof(double) * (ns + 1));
  aw[0] = aw[1] = 1.0;
  for (int k = 0; k < in; ++k) aw[2 + k] = 1.0 / m->W[k];
  orc_opts oc = *o;
  oc.atol_scale = aw;
  kin_ctx ctx = {m, P, o->jac_kind};
  orc_radau(ns + 1, conc_rhs, conc_jac, &ctx, 0.0, dt, phi, &oc, st);
  free(aw);
  double T = phi[0], V = phi[1], nin = P * V / (ORC_RU * T), mass = 0.0;
  for (int k = 0; k < in; ++k) {
    nin -= phi[2 + k];
    mass += m->W[k] * phi[2 + k];
  }
  mass += m->W[in] * nin;
  *Ti = T;
  for (int k = 0; k < in; ++k) Yi[(size_t)k * n] = m->W[k] * phi[2 + k] / mass;
  Yi[(size_t)in * n] = m->W[in] * nin / mass;
  free(phi);
}

static int kin_rhs(void *c, double t, const double *y, double *f) {
  (void)t;
  kin_ctx *k = (kin_ctx *)c;
  return orc_rhs(k->m, k->P, y, f);
}

static int kin_jac(void *c, double t, const double *y, const double *f0, double h,
                   const double *scal, double *J) {
  (void)t;
  kin_ctx *k = (kin_ctx *)c;
  if (k->jac_kind == 1) return orc_jac_fd(k->m, k->P, y, f0, h, scal, J);
  return orc_jac(k->m, k->P, y, J);
}

/* one state in the mass-fraction form; Yi strided by n */
static void integrate_massfrac(const orc_mech *m, double *Yi, int64_t n, double *Ti, double P,
                               double dt, const orc_opts *o, orc_stats *st) {
  int ns = m->ns;
  double *y = malloc(sizeof(double) * ns);
  y[0] = *Ti;
  for (int k = 0; k < ns - 1; ++k) y[1 + k] = Yi[(size_t)k * n];
  kin_ctx ctx = {m, P, o->jac_kind};
  orc_radau(ns, kin_rhs, kin_jac, &ctx, 0.0, dt, y, o, st);
  *Ti = y[0];
  double sum = 0.0;
  for (int k = 0; k < ns - 1; ++k) {
    Yi[(size_t)k * n] = y[1 + k];
    sum += y[1 + k];
  }
  Yi[(size_t)(ns - 1) * n] = 1.0 - sum;
  free(y);
}

int orc_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

int orc_integrate_batch(const orc_mech *m, int64_t n, double *Y, double *T, const double *P,
                        double dt, const orc_opts *o, int32_t *status, int32_t *counters,
                        int nthreads) {
  int nfail = 0;
  if (nthreads <= 0) nthreads = orc_num_threads();
#pragma omp parallel for schedule(dynamic, 16) num_threads(nthreads) reduction(+ : nfail)
  for (int64_t i = 0; i < n; ++i) {
    orc_stats st;
    if (o->form == 1)
      integrate_conc(m, Y + i, n, T + i, P[i], dt, o, &st);
    else
      integrate_massfrac(m, Y + i, n, T + i, P[i], dt, o, &st);
    if (status) status[i] = st.status;
    if (counters) {
      int32_t *c = counters + 8 * i;
      c[0] = st.nstep;
      c[1] = st.naccpt;
      c[2] = st.nrejct;
      c[3] = st.nfcn;
      c[4] = st.njac;
      c[5] = st.ndec;
      c[6] = st.nsol;
      c[7] = st.status;
    }
    nfail += (st.status != ORC_OK);
  }
  return nfail;
}
