/*
 * Oracle dense linear algebra: LU factorisation with partial pivoting and the
 * matching solves, real and complex.  TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * The paper's GPU Radau needs "specialized implementations of several BLAS
 * and LAPACK methods, mostly related to LU factorization" (Sec. 2.1).  This is
 * the plain right-looking Doolittle elimination with row interchanges; the
 * pivot is the first row holding the largest |a| (real) or |Re a| + |Im a|
 * (complex), the LAPACK i?amax convention.  Matrices are row-major; complex
 * entries are stored as interleaved (re, im) pairs.
 */
#include <complex.h>
#include <math.h>

#include "oracle.h"

/* Returns 0, or k+1 when column k has no nonzero pivot. */
int orc_lu_real(int n, double *a, int32_t *ipiv) {
  for (int k = 0; k < n; ++k) {
    int p = k;
    for (int i = k + 1; i < n; ++i)
      if (fabs(a[(size_t)i * n + k]) > fabs(a[(size_t)p * n + k])) p = i;
    ipiv[k] = p;
    if (a[(size_t)p * n + k] == 0.0) return k + 1;
    if (p != k)
      for (int j = 0; j < n; ++j) {
        double t = a[(size_t)k * n + j];
        a[(size_t)k * n + j] = a[(size_t)p * n + j];
        a[(size_t)p * n + j] = t;
      }
    for (int i = k + 1; i < n; ++i) {
      double l = a[(size_t)i * n + k] / a[(size_t)k * n + k];
      a[(size_t)i * n + k] = l;
      for (int j = k + 1; j < n; ++j) a[(size_t)i * n + j] -= l * a[(size_t)k * n + j];
    }
  }
  return 0;
}

void orc_lu_solve_real(int n, const double *lu, const int32_t *ipiv, double *b) {
  for (int k = 0; k < n; ++k) {
    int p = ipiv[k];
    if (p != k) {
      double t = b[k];
      b[k] = b[p];
      b[p] = t;
    }
  }
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < i; ++j) b[i] -= lu[(size_t)i * n + j] * b[j];
  for (int i = n - 1; i >= 0; --i) {
    for (int j = i + 1; j < n; ++j) b[i] -= lu[(size_t)i * n + j] * b[j];
    b[i] /= lu[(size_t)i * n + i];
  }
}

static double cabs1(double complex z) { return fabs(creal(z)) + fabs(cimag(z)); }

int orc_lu_cplx(int n, double *a_re_im, int32_t *ipiv) {
  double complex *a = (double complex *)a_re_im;
  for (int k = 0; k < n; ++k) {
    int p = k;
    for (int i = k + 1; i < n; ++i)
      if (cabs1(a[(size_t)i * n + k]) > cabs1(a[(size_t)p * n + k])) p = i;
    ipiv[k] = p;
    if (cabs1(a[(size_t)p * n + k]) == 0.0) return k + 1;
    if (p != k)
      for (int j = 0; j < n; ++j) {
        double complex t = a[(size_t)k * n + j];
        a[(size_t)k * n + j] = a[(size_t)p * n + j];
        a[(size_t)p * n + j] = t;
      }
    for (int i = k + 1; i < n; ++i) {
      double complex l = a[(size_t)i * n + k] / a[(size_t)k * n + k];
      a[(size_t)i * n + k] = l;
      for (int j = k + 1; j < n; ++j) a[(size_t)i * n + j] -= l * a[(size_t)k * n + j];
    }
  }
  return 0;
}

void orc_lu_solve_cplx(int n, const double *lu_re_im, const int32_t *ipiv, double *b_re_im) {
  const double complex *lu = (const double complex *)lu_re_im;
  double complex *b = (double complex *)b_re_im;
  for (int k = 0; k < n; ++k) {
    int p = ipiv[k];
    if (p != k) {
      double complex t = b[k];
      b[k] = b[p];
      b[p] = t;
    }
  }
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < i; ++j) b[i] -= lu[(size_t)i * n + j] * b[j];
  for (int i = n - 1; i >= 0; --i) {
    for (int j = i + 1; j < n; ++j) b[i] -= lu[(size_t)i * n + j] * b[j];
    b[i] /= lu[(size_t)i * n + i];
  }
}
