// exprb43 with Krylov phi-function products (kin_exprb_* of the C ABI): the
// fourth-order exponential Rosenbrock method the paper compares with Radau
// IIA (Sec. 2.1, Table of solvers; Sec. 3.1), one state per warp.
//
// Scheme (Hochbruck, Ostermann & Schweitzer), g(u) = F(u) - J_n u,
// D_i = g(U_i) - g(u_n):
//   U2 = u_n + h/2 phi1(h/2 J) F(u_n)
//   U3 = u_n + h phi1(h J) F(u_n) + h phi1(h J) D2
//   u_{n+1} = u_n + h phi1(h J) F(u_n) + h (16 phi3 - 48 phi4)(h J) D2
//             + h (-2 phi3 + 12 phi4)(h J) D3
//   embedded (order 3): 16 phi3 for D2 and -2 phi3 for D3.
// J_n is the analytical Jacobian at u_n (once per accepted point).  Each of
// F(u_n), D2 and D3 spans its own Krylov space (Arnoldi, modified
// Gram-Schmidt, in the inner product of the step's error weights D: on
// D^-1 J D, which keeps the Hessenberg matrix as well scaled as the
// chemistry's time scales; vectors over the warp's lanes as in the Radau
// WARP layout, the basis and the Hessenberg matrix in the warp's global
// slot); its
// dimension grows until Saad's leading error term of every product taken
// from it, h beta (h h_{m+1,m}) c_k |e_m^T phi_{k+1}(h H_m) e1| in the
// step's error weights, is at most kappa, or the space is exhausted.
// phi_1..phi_p(tau H_m) e1 are columns of the exponential of the augmented
// matrix [[tau H_m, e1, 0], [0, 0, I], [0, 0, 0]], computed by scaling and
// squaring with the (6,6) Pade approximant and a partial-pivoting LU.  (The
// paper uses a (10,10) Caratheodory-Fejer rational approximant of exp on
// the negative real axis instead; scaling and squaring holds for any
// spectrum, including the positive eigenvalues of igniting states.)  Step
// size control: Hairer-Norsett-Wanner on the embedded difference.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <vector>

#include "../../include/kin.h"
#include "kin_internal.h"
#include "kin_warp.cuh"

using namespace kin;

namespace {

constexpr int XL = 32;
using XG = Grp<XL>;
constexpr int XWR = XG::WR;
using XV = WVecT<XWR>;
constexpr int XKP = 5;  // augmented columns: phi_1 .. phi_5

// Pade (6,6) coefficients of exp: c_j = (12 - j)! 6! / (12! j! (6 - j)!)
__device__ __constant__ double PADE6[7] = {1.0,        0.5,          5.0 / 44.0,    1.0 / 66.0,
                                           1.0 / 792.0, 1.0 / 15840.0, 1.0 / 665280.0};

// per-warp workspace in global memory (after the Jacobian slot)
struct XWork {
  double *V;   // basis: vector j at V + j * N, j <= N
  double *H;   // Hessenberg, (N + 1) x N, H[i * N + j]
  double *X, *X2, *X4, *U, *W, *R, *Tm;  // S x S, row-major, ld S
  double *vt;  // S: solve scratch
  double *vd;  // N: a vector handed to the matrix-vector product
  int *ip;     // S pivots
  int S;
};

__host__ __device__ inline int xS(int N) { return (N + XKP + 2) & ~1; }
__host__ __device__ inline size_t xslot_doubles(int N) {
  const size_t S = (size_t)xS(N);
  size_t d = (size_t)warp_slot_mats(sizeof(double)) * N * (N + 1);  // J, E2r, E2i
  d += 2 * (size_t)(N + 1) * N + 7 * S * S + S + (size_t)N + S;     // V, H, 7 matrices, vt, vd, ip
  return (d + 31) / 32 * 32;
}

__device__ XWork carve_xwork(double *slot, int N) {
  XWork w;
  w.S = xS(N);
  double *p = slot + (size_t)warp_slot_mats(sizeof(double)) * N * (N + 1);
  w.V = p;
  p += (size_t)(N + 1) * N;
  w.H = p;
  p += (size_t)(N + 1) * N;
  const size_t SS = (size_t)w.S * w.S;
  w.X = p;
  w.X2 = p + SS;
  w.X4 = p + 2 * SS;
  w.U = p + 3 * SS;
  w.W = p + 4 * SS;
  w.R = p + 5 * SS;
  w.Tm = p + 6 * SS;
  p += 7 * SS;
  w.vt = p;
  p += w.S;
  w.vd = p;
  p += N;
  w.ip = reinterpret_cast<int *>(p);
  return w;
}

__device__ __forceinline__ double xdot(int N, const XV &a, const XV &b) {
  double s = 0.0;
#pragma unroll
  for (int r = 0; r < XWR; ++r)
    if (XG::lane() + XL * r < N) s += a.v[r] * b.v[r];
  return XG::sum(s);
}

__device__ __forceinline__ double xwrms(int N, const XV &a, const XV &sc) {
  double s = 0.0;
#pragma unroll
  for (int r = 0; r < XWR; ++r)
    if (XG::lane() + XL * r < N) {
      const double q = a.v[r] / sc.v[r];
      s += q * q;
    }
  return sqrt(XG::sum(s) / N);
}

__device__ __forceinline__ void xload(int N, const double *p, XV &x) {
#pragma unroll
  for (int r = 0; r < XWR; ++r) {
    const int g = XG::lane() + XL * r;
    x.v[r] = g < N ? p[g] : 0.0;
  }
}

__device__ __forceinline__ void xstore(int N, double *p, const XV &x) {
#pragma unroll
  for (int r = 0; r < XWR; ++r) {
    const int g = XG::lane() + XL * r;
    if (g < N) p[g] = x.v[r];
  }
}

// y = J x, J row-major (ld) and x in global memory
__device__ void xmatvec(int N, int ld, const double *J, const double *x, XV &y) {
#pragma unroll
  for (int r = 0; r < XWR; ++r) {
    const int g = XG::lane() + XL * r;
    double s = 0.0;
    if (g < N)
      for (int c = 0; c < N; ++c) s += J[g * ld + c] * x[c];
    y.v[r] = s;
  }
}

// C = A B for s x s matrices (ld S)
__device__ void xmatmul(int s, int S, const double *A, const double *B, double *C) {
  for (int e = XG::lane(); e < s * s; e += XL) {
    const int i = e / s, j = e % s;
    double acc = 0.0;
    for (int k = 0; k < s; ++k) acc += A[i * S + k] * B[k * S + j];
    C[i * S + j] = acc;
  }
  XG::sync();
}

// exp(w.X) (s x s) by scaling and squaring with the (6,6) Pade approximant;
// returns the result's matrix (w.R or w.Tm), or nullptr when the
// denominator is singular or the norm is not finite
__device__ const double *xexpm(int s, const XWork &w) {
  const int S = w.S, lane = XG::lane();
  double nrm = 0.0;
  for (int c = lane; c < s; c += XL) {
    double cs = 0.0;
    for (int i = 0; i < s; ++i) cs += fabs(w.X[i * S + c]);
    nrm = fmax(nrm, cs);
  }
#pragma unroll
  for (int o = XL / 2; o > 0; o >>= 1) nrm = fmax(nrm, __shfl_xor_sync(XG::mask(), nrm, o, XL));
  if (!isfinite(nrm)) return nullptr;
  int sq = 0;
  while (nrm > 0.25 && sq < 1100) {  // ||X / 2^sq||_1 <= 1/4 (finite norms stop well before)
    nrm *= 0.5;
    ++sq;
  }
  const double sc = ldexp(1.0, -sq);
  for (int e = lane; e < s * s; e += XL) w.X[(e / s) * S + e % s] *= sc;
  XG::sync();
  xmatmul(s, S, w.X, w.X, w.X2);
  xmatmul(s, S, w.X2, w.X2, w.X4);
  // W = c1 I + c3 X2 + c5 X4, U = X W
  for (int e = lane; e < s * s; e += XL) {
    const int i = e / s, j = e % s, q = i * S + j;
    w.W[q] = PADE6[3] * w.X2[q] + PADE6[5] * w.X4[q] + (i == j ? PADE6[1] : 0.0);
  }
  XG::sync();
  xmatmul(s, S, w.X, w.W, w.U);
  xmatmul(s, S, w.X2, w.X4, w.Tm);  // X6
  // V = c0 I + c2 X2 + c4 X4 + c6 X6; numerator V + U (R), denominator V - U (W)
  for (int e = lane; e < s * s; e += XL) {
    const int i = e / s, j = e % s, q = i * S + j;
    const double v = PADE6[2] * w.X2[q] + PADE6[4] * w.X4[q] + PADE6[6] * w.Tm[q] +
                     (i == j ? PADE6[0] : 0.0);
    w.R[q] = v + w.U[q];
    w.W[q] = v - w.U[q];
  }
  XG::sync();
  if (warp_lu_real<XL, double>(s, S, w.W, w.ip)) return nullptr;
  for (int c = 0; c < s; ++c) {  // Tm = W^-1 R, column by column
    XV x;
#pragma unroll
    for (int r = 0; r < XWR; ++r) {
      const int g = lane + XL * r;
      x.v[r] = g < s ? w.R[g * S + c] : 0.0;
    }
    warp_solve_real<XL, double>(s, S, w.W, w.ip, w.vt, x);
#pragma unroll
    for (int r = 0; r < XWR; ++r) {
      const int g = lane + XL * r;
      if (g < s) w.Tm[g * S + c] = x.v[r];
    }
  }
  XG::sync();
  double *a = w.Tm, *b = w.R;
  for (int i = 0; i < sq; ++i) {
    xmatmul(s, S, a, a, b);
    double *t = a;
    a = b;
    b = t;
  }
  return a;
}

// phi_1 .. phi_p (tau H_m) e1: the exponential of the augmented matrix;
// phi_k is column m + k - 1 (rows 0 .. m-1) of the returned matrix
__device__ const double *xphi(int N, int m, int p, double tau, const XWork &w) {
  const int s = m + p, S = w.S;
  for (int e = XG::lane(); e < s * s; e += XL) {
    const int i = e / s, j = e % s;
    double v = 0.0;
    if (i < m && j < m && i <= j + 1)  // upper Hessenberg: Arnoldi writes no other entry
      v = tau * w.H[i * N + j];
    else if (i == 0 && j == m)
      v = 1.0;
    else if (i >= m && j == i + 1)
      v = 1.0;
    w.X[i * S + j] = v;
  }
  XG::sync();
  return xexpm(s, w);
}

// D beta V_m phi_k e1 with phi_k read from the exponential E (column m+k-1)
__device__ void xproduct(int N, int m, double beta, const XWork &w, const double *E, int k,
                         const XV &scal, XV &out) {
  const int S = w.S;
#pragma unroll
  for (int r = 0; r < XWR; ++r) {
    const int g = XG::lane() + XL * r;
    double s = 0.0;
    if (g < N)
      for (int i = 0; i < m; ++i) s += w.V[i * N + g] * E[i * S + m + k - 1];
    out.v[r] = scal.v[r] * (beta * s);
  }
}

struct XProducts {
  int np, kmax;
  int k[3];
  double c[3];
};

// Arnoldi in the error-weighted inner product (on D^-1 J D from D^-1 v,
// D = diag(scal)) with the stopping rule; returns m (0 for v = 0), -1 when
// a matrix function failed; beta out
__device__ int xarnoldi(int N, int ld, const double *J, const XV &v, double h,
                        const XProducts &pr, const XV &scal, double kappa, const XWork &w,
                        double &beta) {
  const int lane = XG::lane();
  XV q;
#pragma unroll
  for (int r = 0; r < XWR; ++r) q.v[r] = v.v[r] / scal.v[r];  // D^-1 v
  beta = sqrt(xdot(N, q, q));
  if (beta == 0.0) return 0;
#pragma unroll
  for (int r = 0; r < XWR; ++r) q.v[r] = q.v[r] / beta;
  xstore(N, w.V, q);
  XG::sync();
  for (int j = 0; j < N; ++j) {
    XV x;
    xload(N, w.V + (size_t)j * N, x);  // D^-1 J D v_j: the product of J with D v_j
#pragma unroll
    for (int r = 0; r < XWR; ++r) x.v[r] *= scal.v[r];
    xstore(N, w.vd, x);
    XG::sync();
    xmatvec(N, ld, J, w.vd, x);
#pragma unroll
    for (int r = 0; r < XWR; ++r) x.v[r] = x.v[r] / scal.v[r];
    XG::sync();
    const double nw = sqrt(xdot(N, x, x));
    for (int i = 0; i <= j; ++i) {  // modified Gram-Schmidt
      XV vi;
      xload(N, w.V + (size_t)i * N, vi);
      const double hij = xdot(N, vi, x);
#pragma unroll
      for (int r = 0; r < XWR; ++r) x.v[r] -= hij * vi.v[r];
      if (lane == 0) w.H[i * N + j] = hij;
    }
    const double hn = sqrt(xdot(N, x, x));
    if (lane == 0) w.H[(j + 1) * N + j] = hn;
    const int m = j + 1;
    if (hn <= 1e-13 * nw || m == N) {
      XG::sync();
      return m;
    }
#pragma unroll
    for (int r = 0; r < XWR; ++r) x.v[r] = x.v[r] / hn;
    xstore(N, w.V + (size_t)(j + 1) * N, x);
    XG::sync();
    const double *E = xphi(N, m, pr.kmax + 1, h, w);
    // a failed matrix function or a non-finite entry gives no estimate: keep growing
    double lead = E ? 0.0 : NAN;
    if (E)
      for (int t = 0; t < pr.np; ++t) {
        const double v = pr.c[t] * fabs(E[(m - 1) * w.S + m + pr.k[t]]);  // phi_{k+1}
        lead = isnan(v) || isnan(lead) ? NAN : fmax(lead, v);
      }
    // v_{m+1} has unit 2-norm in the scaled space: weighted RMS 1/sqrt(N)
    const double est = h * beta * (h * hn) * lead / sqrt((double)N);
    XG::sync();
    if (est <= kappa) return m;
  }
  return N;
}

struct XParams {
  double rtol, atol, dt, kappa;
  int max_steps;
  int64_t n;
  const double *h0;
};

// D = F(U) - F(u) - J (U - u)
__device__ void xremainder(int N, int ld, const double *J, const XV &U, const XV &u,
                           const XV &FU, const XV &Fu, const XWork &w, XV &D) {
  XV d;
#pragma unroll
  for (int r = 0; r < XWR; ++r) d.v[r] = U.v[r] - u.v[r];
  xstore(N, w.vd, d);
  XG::sync();
  XV Jd;
  xmatvec(N, ld, J, w.vd, Jd);
#pragma unroll
  for (int r = 0; r < XWR; ++r) D.v[r] = FU.v[r] - Fu.v[r] - Jd.v[r];
  XG::sync();
}

// one attempt: 0 done (unew, uhat), 1 a stage was not finite, 2 a matrix
// function failed
__device__ int xstep(const MechView &m, const WarpBuf<double> &b, double P, const XWork &w,
                     const XV &y, const XV &fy, double h, const XV &scal, double kappa, XV &unew,
                     XV &uhat, int &nf, int &kdim) {
  const int N = m.ns, ld = b.ld;
  const double *J = b.J;
  const XProducts PF = {1, 1, {1, 0, 0}, {1.0, 0.0, 0.0}};
  const XProducts PD2 = {3, 4, {1, 3, 4}, {1.0, 16.0, 48.0}};
  const XProducts PD3 = {2, 4, {3, 4, 0}, {2.0, 12.0, 0.0}};
  nf = 0;
  kdim = 0;
  double beta;
  XV half, full, U, F, D, q1, q3, q4, r3, r4;
  int mk = xarnoldi(N, ld, J, fy, h, PF, scal, kappa, w, beta);
  if (mk < 0) return 2;
  kdim += mk;
  if (mk == 0) {
#pragma unroll
    for (int r = 0; r < XWR; ++r) half.v[r] = full.v[r] = 0.0;
  } else {
    const double *E = xphi(N, mk, 1, 0.5 * h, w);
    if (!E) return 2;
    xproduct(N, mk, beta, w, E, 1, scal, half);
    XG::sync();
    E = xphi(N, mk, 1, h, w);
    if (!E) return 2;
    xproduct(N, mk, beta, w, E, 1, scal, full);
    XG::sync();
  }
#pragma unroll
  for (int r = 0; r < XWR; ++r) U.v[r] = y.v[r] + 0.5 * h * half.v[r];
  nf++;
  if (warp_chem<XL, double>(m, b, P, U, F, false)) return 1;
  xremainder(N, ld, J, U, y, F, fy, w, D);
  mk = xarnoldi(N, ld, J, D, h, PD2, scal, kappa, w, beta);
  if (mk < 0) return 2;
  kdim += mk;
  if (mk == 0) {
#pragma unroll
    for (int r = 0; r < XWR; ++r) q1.v[r] = q3.v[r] = q4.v[r] = 0.0;
  } else {
    const double *E = xphi(N, mk, 4, h, w);
    if (!E) return 2;
    xproduct(N, mk, beta, w, E, 1, scal, q1);
    xproduct(N, mk, beta, w, E, 3, scal, q3);
    xproduct(N, mk, beta, w, E, 4, scal, q4);
    XG::sync();
  }
#pragma unroll
  for (int r = 0; r < XWR; ++r) U.v[r] = y.v[r] + h * full.v[r] + h * q1.v[r];
  nf++;
  if (warp_chem<XL, double>(m, b, P, U, F, false)) return 1;
  xremainder(N, ld, J, U, y, F, fy, w, D);
  mk = xarnoldi(N, ld, J, D, h, PD3, scal, kappa, w, beta);
  if (mk < 0) return 2;
  kdim += mk;
  if (mk == 0) {
#pragma unroll
    for (int r = 0; r < XWR; ++r) r3.v[r] = r4.v[r] = 0.0;
  } else {
    const double *E = xphi(N, mk, 4, h, w);
    if (!E) return 2;
    xproduct(N, mk, beta, w, E, 3, scal, r3);
    xproduct(N, mk, beta, w, E, 4, scal, r4);
    XG::sync();
  }
#pragma unroll
  for (int r = 0; r < XWR; ++r) {
    const double base = y.v[r] + h * full.v[r];
    unew.v[r] = base + h * (16.0 * q3.v[r] - 48.0 * q4.v[r]) + h * (-2.0 * r3.v[r] + 12.0 * r4.v[r]);
    uhat.v[r] = base + h * (16.0 * q3.v[r]) + h * (-2.0 * r3.v[r]);
  }
  return 0;
}

struct XCount {
  int nstep, naccpt, nrejct, nfcn, njac, narn, kdim, status;
};

// One state from y (in: [T, Y_0 .. Y_{ns-2}], out: the state at dt or at
// its last accepted point).
__device__ XCount xintegrate(const MechView &m, const WarpBuf<double> &b, double P,
                             const XWork &w, const XParams &p, int64_t idx, XV &y) {
  const int N = m.ns;
  XCount c = {0, 0, 0, 0, 0, 0, 0, 0};
  XV fy, scal, unew, uhat;
  c.nfcn = 1;
  c.njac = 1;
  if (warp_chem<XL, double>(m, b, P, y, fy, true)) {
    c.status = 4;
    return c;
  }
#pragma unroll
  for (int r = 0; r < XWR; ++r) scal.v[r] = p.atol + p.rtol * fabs(y.v[r]);
  double h;
  if (p.h0) {
    h = p.h0[idx];
  } else {  // starting step (Hairer-Norsett-Wanner Vol. I, II.4), order 4
    const double d0 = xwrms(N, y, scal), d1 = xwrms(N, fy, scal);
    double h0 = (d0 < 1e-5 || d1 < 1e-5) ? 1e-6 : 0.01 * d0 / d1;
    h0 = fmin(h0, p.dt);
    XV u, fu;
#pragma unroll
    for (int r = 0; r < XWR; ++r) u.v[r] = y.v[r] + h0 * fy.v[r];
    const int rc = warp_chem<XL, double>(m, b, P, u, fu, false);
    c.nfcn++;
    if (rc) {
      h = 0.01 * h0;
    } else {
      XV df;
#pragma unroll
      for (int r = 0; r < XWR; ++r) df.v[r] = fu.v[r] - fy.v[r];
      const double d2 = xwrms(N, df, scal) / h0;
      const double dm = fmax(d1, d2);
      const double h1 = (dm <= 1e-15) ? fmax(1e-6, h0 * 1e-3) : pow(0.01 / dm, 0.25);
      h = fmin(100.0 * h0, h1);
    }
    h = fmin(h, p.dt);
  }
  double x = 0.0, facmax = 5.0;
  bool last = false;
  for (;;) {
    if (c.nstep >= p.max_steps) {
      c.status = 1;
      return c;
    }
    if (0.1 * fabs(h) <= fabs(x) * 1e-16) {
      c.status = 2;
      return c;
    }
    if (x + 1.0001 * h >= p.dt) {
      h = p.dt - x;
      last = true;
    }
    c.nstep++;
#pragma unroll
    for (int r = 0; r < XWR; ++r) scal.v[r] = p.atol + p.rtol * fabs(y.v[r]);
    int nf = 0, kd = 0;
    const int rc = xstep(m, b, P, w, y, fy, h, scal, p.kappa, unew, uhat, nf, kd);
    c.nfcn += nf;
    c.narn += 3;
    c.kdim += kd;
    if (rc == 1) {
      c.nrejct++;
      h *= 0.5;
      last = false;
      facmax = 1.0;
      continue;
    }
    XV d, sc;
#pragma unroll
    for (int r = 0; r < XWR; ++r) {
      d.v[r] = unew.v[r] - uhat.v[r];
      sc.v[r] = p.atol + p.rtol * fmax(fabs(y.v[r]), fabs(unew.v[r]));
    }
    // a matrix function that failed, or a non-finite estimate: rejected with
    // the smallest factor
    const double e = rc == 2 ? INFINITY : xwrms(N, d, sc);
    const double err = isfinite(e) ? fmax(e, 1e-10) : INFINITY;
    const double fac = isfinite(err) ? 0.9 * pow(err, -0.25) : 0.0;
    if (err <= 1.0) {
      x = last ? p.dt : x + h;
      y = unew;
      c.naccpt++;
      if (last) return c;
      c.nfcn++;
      c.njac++;
      if (warp_chem<XL, double>(m, b, P, y, fy, true)) {
        c.status = 4;
        return c;
      }
      h = h * fmin(facmax, fmax(0.2, fac));
      facmax = 5.0;
    } else {
      c.nrejct++;
      h = h * fmax(0.2, fac);
      facmax = 1.0;
      last = false;
    }
  }
}

struct XArgs {
  MechLayout L;
  const double *tab;
  const int *itab;
  double *Y, *T;
  const double *P;
  int32_t *status, *counters;
  unsigned long long *totals;
  XParams p;
  double *scratch;
  int64_t slots;
};

__global__ void __launch_bounds__(256) k_integrate_exprb(XArgs a) {
  extern __shared__ double smem[];
  const MechView m = make_view(a.L, a.tab, a.itab);
  const int N = m.ns, lane = XG::lane(), grp = (int)(threadIdx.x / XL);
  const int64_t n = a.p.n;
  char *base = reinterpret_cast<char *>(smem) + (size_t)grp * warp_buf_bytes(N, m.nr, sizeof(double));
  const int64_t slot = (int64_t)blockIdx.x * (blockDim.x / XL) + grp;  // < slots (launch)
  double *gs = a.scratch + slot * (int64_t)xslot_doubles(N);
  const WarpBuf<double> b = carve_warp_buf<double>(base, N, m.nr, gs);
  const XWork w = carve_xwork(gs, N);
  unsigned long long *queue = a.totals + 9;
  for (;;) {
    unsigned long long t = 0;
    if (lane == 0) t = atomicAdd(queue, 1ull);
    t = XG::bcast(t, 0);
    if (t >= (unsigned long long)n) break;
    const int64_t idx = (int64_t)t;
    const double P = a.P[idx];
    XV y;
#pragma unroll
    for (int r = 0; r < XWR; ++r) {
      const int g = lane + XL * r;
      y.v[r] = (g == 0) ? a.T[idx] : (g < N ? a.Y[(int64_t)(g - 1) * n + idx] : 0.0);
    }
    const XCount c = xintegrate(m, b, P, w, a.p, idx, y);
    double sum = 0.0;
#pragma unroll
    for (int r = 0; r < XWR; ++r) {
      const int g = lane + XL * r;
      if (g == 0) a.T[idx] = y.v[r];
      if (g >= 1 && g < N) {
        a.Y[(int64_t)(g - 1) * n + idx] = y.v[r];
        sum += y.v[r];
      }
    }
    sum = XG::sum(sum);
    if (lane == 0) {
      a.Y[(int64_t)(N - 1) * n + idx] = 1.0 - sum;
      if (a.status) a.status[idx] = c.status;
      if (a.counters) {
        const int32_t cc[8] = {c.nstep, c.naccpt, c.nrejct, c.nfcn, c.njac, c.narn, c.kdim,
                               c.status};
        for (int q = 0; q < 8; ++q) a.counters[(int64_t)q * n + idx] = cc[q];
      }
      const unsigned long long c7[7] = {
          (unsigned long long)c.nstep, (unsigned long long)c.naccpt, (unsigned long long)c.nrejct,
          (unsigned long long)c.nfcn,  (unsigned long long)c.njac,   (unsigned long long)c.narn,
          (unsigned long long)c.kdim};
      for (int q = 0; q < 7; ++q) atomicAdd(a.totals + q, c7[q]);
      if (c.status) atomicAdd(a.totals + 7, 1ull);
      atomicMax(a.totals + 8, (unsigned long long)c.nstep);
    }
    XG::sync();
  }
}

// unit entry: phi_1..phi_p (tau H) e1 of one m x m matrix, on one warp
__global__ void k_exprb_phi(const double *H, int m, int p, double tau, double *out,
                            double *scratch, int N) {
  XWork w = carve_xwork(scratch, N);
  for (int e = threadIdx.x; e < m * m; e += XL) w.H[(e / m) * N + e % m] = H[e];
  XG::sync();
  const double *E = xphi(N, m, p, tau, w);
  for (int e = threadIdx.x; e < m * p; e += XL)
    out[e] = E ? E[(e / p) * w.S + m + e % p] : NAN;  // out[i * p + k - 1] = phi_k[i]
}

// unit entry: the right-hand side (with and without the Jacobian's assembly)
// and the analytical Jacobian the method uses, one state per warp
__global__ void k_exprb_chem(MechLayout L, const double *tab, const int *itab, const double *y,
                             const double *P, int64_t n, double *f, double *f2, double *J,
                             double *scratch, int64_t slots) {
  extern __shared__ double smem[];
  const MechView m = make_view(L, tab, itab);
  const int N = m.ns, lane = XG::lane(), grp = (int)(threadIdx.x / XL);
  const int64_t slot = (int64_t)blockIdx.x * (blockDim.x / XL) + grp;
  if (slot >= slots) return;
  char *base = reinterpret_cast<char *>(smem) + (size_t)grp * warp_buf_bytes(N, m.nr, sizeof(double));
  double *gs = scratch + slot * (int64_t)xslot_doubles(N);
  const WarpBuf<double> b = carve_warp_buf<double>(base, N, m.nr, gs);
  for (int64_t i = slot; i < n; i += (int64_t)gridDim.x * (blockDim.x / XL)) {
    XV yy, ff;
#pragma unroll
    for (int r = 0; r < XWR; ++r) {
      const int g = lane + XL * r;
      yy.v[r] = g < N ? y[(int64_t)g * n + i] : 0.0;
    }
    warp_chem<XL, double>(m, b, P[i], yy, ff, true);
#pragma unroll
    for (int r = 0; r < XWR; ++r) {
      const int g = lane + XL * r;
      if (g < N) f[(int64_t)g * n + i] = ff.v[r];
    }
    for (int e = lane; e < N * N; e += XL) J[(int64_t)e * n + i] = b.J[(e / N) * b.ld + e % N];
    XG::sync();
    warp_chem<XL, double>(m, b, P[i], yy, ff, false);
#pragma unroll
    for (int r = 0; r < XWR; ++r) {
      const int g = lane + XL * r;
      if (g < N) f2[(int64_t)g * n + i] = ff.v[r];
    }
    XG::sync();
  }
}

}  // namespace

struct kin_exprb {
  int device = 0;
  MechLayout L;
  double *d_tab = nullptr;
  int *d_itab = nullptr;
  unsigned long long *d_totals = nullptr;
  double *d_scratch = nullptr;
  int64_t slots = 0;
  cudaStream_t last_stream = nullptr;
};

extern "C" void kin_exprb_destroy(kin_exprb *x) {
  if (!x) return;
  cudaFree(x->d_tab);
  cudaFree(x->d_itab);
  cudaFree(x->d_totals);
  cudaFree(x->d_scratch);
  delete x;
}

extern "C" int kin_exprb_create(const kin_mech_desc *desc, kin_exprb **out) {
  if (!desc || !out) return KIN_ERR_INVALID_ARG;
  *out = nullptr;
  MechLayout L;
  std::vector<double> dt;
  std::vector<int> it;
  const int rc = build_tables(desc, L, dt, it);
  if (rc) return rc;
  if (xS(L.ns) > XG::CAP) return KIN_ERR_UNSUPPORTED;  // augmented matrix on one warp
  int dev = 0, sms = 0;
  KIN_CUDA_TRY(cudaGetDevice(&dev));
  KIN_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  kin_exprb *x = new kin_exprb();
  x->device = dev;
  x->L = L;
  x->slots = (int64_t)sms * 16;  // one per resident warp (128 registers: at most 16 per SM)
  const size_t sbytes = (size_t)x->slots * xslot_doubles(L.ns) * sizeof(double);
  if (cudaMalloc(&x->d_tab, sizeof(double) * L.nd) != cudaSuccess ||
      cudaMalloc(&x->d_itab, sizeof(int) * L.ni) != cudaSuccess ||
      cudaMalloc(&x->d_totals, sizeof(unsigned long long) * 16) != cudaSuccess ||
      cudaMalloc(&x->d_scratch, sbytes) != cudaSuccess) {
    (void)cudaGetLastError();
    kin_exprb_destroy(x);
    return KIN_ERR_NOMEM;
  }
  if (cudaMemcpy(x->d_tab, dt.data(), sizeof(double) * L.nd, cudaMemcpyHostToDevice) !=
          cudaSuccess ||
      cudaMemcpy(x->d_itab, it.data(), sizeof(int) * L.ni, cudaMemcpyHostToDevice) !=
          cudaSuccess ||
      cudaMemset(x->d_totals, 0, sizeof(unsigned long long) * 16) != cudaSuccess) {
    (void)cudaGetLastError();
    kin_exprb_destroy(x);
    return KIN_ERR_CUDA;
  }
  *out = x;
  return KIN_OK;
}

extern "C" int kin_integrate_exprb(kin_exprb *x, double *Y, double *T, const double *P,
                                   int64_t n, double dt, double rtol, double atol, double kappa,
                                   const double *h0, int32_t max_steps, int32_t *status,
                                   int32_t *counters, void *stream) {
  if (!x || n < 0) return KIN_ERR_INVALID_ARG;
  if (n > 0 && (!Y || !T || !P)) return KIN_ERR_INVALID_ARG;
  if (!(dt > 0.0) || !(rtol > 0.0) || !(atol > 0.0) || !std::isfinite(dt) || !(kappa >= 0.0) ||
      !std::isfinite(kappa) || max_steps < 1)
    return KIN_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  x->last_stream = st;
  KIN_CUDA_TRY(cudaMemsetAsync(x->d_totals, 0, sizeof(unsigned long long) * 16, st));
  if (n == 0) return KIN_OK;
  int dev = 0, sms = 0;
  KIN_CUDA_TRY(cudaGetDevice(&dev));
  if (dev != x->device) return KIN_ERR_INVALID_ARG;
  KIN_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  XArgs a;
  a.L = x->L;
  a.tab = x->d_tab;
  a.itab = x->d_itab;
  a.Y = Y;
  a.T = T;
  a.P = P;
  a.status = status;
  a.counters = counters;
  a.totals = x->d_totals;
  a.p.rtol = rtol;
  a.p.atol = atol;
  a.p.dt = dt;
  a.p.kappa = kappa;
  a.p.max_steps = max_steps;
  a.p.n = n;
  a.p.h0 = h0;
  a.scratch = x->d_scratch;
  a.slots = x->slots;
  const size_t budget = 227 * 1024, per = warp_buf_bytes(x->L.ns, x->L.nr, sizeof(double));
  auto kern = k_integrate_exprb;
  int warps = 0, per_sm = 0;
  for (int wp = 8; wp >= 1; wp >>= 1) {
    const size_t smw = (size_t)wp * per;
    if (smw > budget) continue;
    KIN_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smw));
    int nb = 0;
    KIN_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, 32 * wp, smw));
    if (nb * wp > per_sm * warps) {
      warps = wp;
      per_sm = nb;
    }
  }
  if (warps < 1 || per_sm < 1) return KIN_ERR_UNSUPPORTED;
  const size_t sm = (size_t)warps * per;
  KIN_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
  int64_t grid = (int64_t)sms * per_sm;
  const int64_t need = (n + warps - 1) / warps;
  if (grid > need) grid = need;
  if (grid * warps > x->slots) grid = x->slots / warps;  // one workspace slot per warp
  if (grid < 1) return KIN_ERR_UNSUPPORTED;
  kern<<<(unsigned)grid, 32 * warps, sm, st>>>(a);
  KIN_CUDA_TRY(cudaGetLastError());
  return KIN_OK;
}

extern "C" int kin_exprb_get_stats(kin_exprb *x, int64_t *out) {
  if (!x || !out) return KIN_ERR_INVALID_ARG;
  unsigned long long t[16];
  KIN_CUDA_TRY(cudaStreamSynchronize(x->last_stream));
  KIN_CUDA_TRY(cudaMemcpy(t, x->d_totals, sizeof t, cudaMemcpyDeviceToHost));
  for (int i = 0; i < 9; ++i) out[i] = (int64_t)t[i];
  return out[7] > 0 ? KIN_ERR_STATE_FAILED : KIN_OK;
}

extern "C" int kin_exprb_phi(kin_exprb *x, const double *H, int32_t m, int32_t p, double tau,
                             double *out, void *stream) {
  if (!x || !H || !out || m < 1 || p < 1 || m > x->L.ns || p > XKP || !std::isfinite(tau))
    return KIN_ERR_INVALID_ARG;
  k_exprb_phi<<<1, XL, 0, (cudaStream_t)stream>>>(H, m, p, tau, out, x->d_scratch, x->L.ns);
  KIN_CUDA_TRY(cudaGetLastError());
  return KIN_OK;
}

extern "C" int kin_exprb_chem(kin_exprb *x, const double *y, const double *P, int64_t n,
                              double *f, double *f_rates, double *J, void *stream) {
  if (!x || n < 0 || (n > 0 && (!y || !P || !f || !f_rates || !J))) return KIN_ERR_INVALID_ARG;
  if (n == 0) return KIN_OK;
  const size_t sm = warp_buf_bytes(x->L.ns, x->L.nr, sizeof(double));
  KIN_CUDA_TRY(cudaFuncSetAttribute(k_exprb_chem, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)sm));
  const int64_t grid = n < x->slots ? n : x->slots;
  k_exprb_chem<<<(unsigned)grid, XL, sm, (cudaStream_t)stream>>>(
      x->L, x->d_tab, x->d_itab, y, P, n, f, f_rates, J, x->d_scratch, x->slots);
  KIN_CUDA_TRY(cudaGetLastError());
  return KIN_OK;
}
