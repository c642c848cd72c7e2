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
  int ns = m->ns;
  int nfail = 0;
  if (nthreads <= 0) nthreads = orc_num_threads();
#pragma omp parallel for schedule(dynamic, 16) num_threads(nthreads) reduction(+ : nfail)
  for (int64_t i = 0; i < n; ++i) {
    double *y = malloc(sizeof(double) * ns);
    y[0] = T[i];
    for (int k = 0; k < ns - 1; ++k) y[1 + k] = Y[(size_t)k * n + i];
    kin_ctx ctx = {m, P[i], o->jac_kind};
    orc_stats st;
    orc_radau(ns, kin_rhs, kin_jac, &ctx, 0.0, dt, y, o, &st);
    T[i] = y[0];
    double sum = 0.0;
    for (int k = 0; k < ns - 1; ++k) {
      Y[(size_t)k * n + i] = y[1 + k];
      sum += y[1 + k];
    }
    Y[(size_t)(ns - 1) * n + i] = 1.0 - sum;
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
    free(y);
  }
  return nfail;
}
