// Device-side chemistry and dense linear algebra for the Radau kernels.
//
// Chemistry (Sec. 2.1 of Curtis, Niemeyer & Sung: the constant-pressure,
// mass-fraction-based reactor with pyJac-style source terms and analytical
// Jacobian): NASA-7 thermo, reversible Arrhenius / third-body / Troe rates
// with reverse rates from equilibrium constants, dY/dt and dT/dt, and the
// Jacobian df/dy.  State y = [T, Y_0 .. Y_{ns-2}]; the last species is inert.
//
// Linear algebra (Sec. 2.1: the GPU Radau needs custom LU and solves): LU
// with partial pivoting (first row of largest |a|, or |Re|+|Im| for complex)
// and forward/back substitution, templated on the storage/arithmetic type so
// the Newton matrices can be factorised in FP32 or FP64.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace kin {

constexpr double RU = 8314.46261815324;  // J/(kmol K)
constexpr double PATM = 101325.0;        // Pa
constexpr double LN10 = 2.302585092994045684;

// ---------------------------------------------------------------------------
// Mechanism tables.  Built on the host (kin_api), staged into shared memory
// by each CTA; every lane of a warp reads the same entry at the same time in
// the one-state-per-thread layout, so the reads are broadcasts.
// ---------------------------------------------------------------------------
struct MechLayout {
  int ns, nr, neff;
  int nd, ni;  // table sizes in doubles / ints
  // double-table offsets
  int dW, dinvW, dTmid, dcp, dh, ds, dlnA, db, dTh, dtroe, deff;
  // int-table offsets
  int islot, imeta, ieff0, itroe, ieffsp;
};

// per-species coefficient blocks (two ranges each):
//   cp/R = c0 + T(c1 + T(c2 + T(c3 + T c4)))                 (5)
//   h/RT = c0 + T(c1 + T(c2 + T(c3 + T c4))) + c5 / T        (6)
//   s/R  = c0 lnT + T(c1 + T(c2 + T(c3 + T c4))) + c5        (6)
constexpr int NCP = 5, NH = 6, NS = 6;
// Troe block per falloff reaction: k0 lnA, k0 b, k0 Theta, a, 1/T***, 1/T*, T**
constexpr int NTROE = 7;

// reaction meta word: bits 0-1 type, 2-3 #reactants, 4-5 #products,
// 6-7 unused, 8-15 #efficiency entries, 16-31 troe index
__device__ __forceinline__ int meta_type(int w) { return w & 3; }
__device__ __forceinline__ int meta_nreac(int w) { return (w >> 2) & 3; }
__device__ __forceinline__ int meta_nprod(int w) { return (w >> 4) & 3; }
__device__ __forceinline__ int meta_neff(int w) { return (w >> 8) & 255; }
__device__ __forceinline__ int meta_troe(int w) { return w >> 16; }

struct MechView {
  int ns, nr;
  const double *W, *invW, *Tmid, *cp, *h, *s, *lnA, *b, *Th, *troe, *eff;
  const int *slot, *meta, *eff0, *effsp;
};

__device__ __forceinline__ MechView make_view(const MechLayout &L, const double *d, const int *i) {
  MechView v;
  v.ns = L.ns;
  v.nr = L.nr;
  v.W = d + L.dW;
  v.invW = d + L.dinvW;
  v.Tmid = d + L.dTmid;
  v.cp = d + L.dcp;
  v.h = d + L.dh;
  v.s = d + L.ds;
  v.lnA = d + L.dlnA;
  v.b = d + L.db;
  v.Th = d + L.dTh;
  v.troe = d + L.dtroe;
  v.eff = d + L.deff;
  v.slot = i + L.islot;
  v.meta = i + L.imeta;
  v.eff0 = i + L.ieff0;
  v.effsp = i + L.ieffsp;
  return v;
}

// Copy the tables from global memory into this CTA's shared memory.
__device__ __forceinline__ MechView stage_tables(const MechLayout &L, const double *gd,
                                                 const int *gi, double *smem) {
  int *si = reinterpret_cast<int *>(smem + L.nd);
  for (int k = threadIdx.x; k < L.nd; k += blockDim.x) smem[k] = gd[k];
  for (int k = threadIdx.x; k < L.ni; k += blockDim.x) si[k] = gi[k];
  __syncthreads();
  return make_view(L, smem, si);
}

// ---------------------------------------------------------------------------
// Thermodynamics (NASA-7)
// ---------------------------------------------------------------------------
__device__ __forceinline__ int range_of(const MechView &m, int k, double T) {
  return T < m.Tmid[k] ? 0 : 1;
}

__device__ __forceinline__ double poly_cp(const double *c, double T) {
  return c[0] + T * (c[1] + T * (c[2] + T * (c[3] + T * c[4])));
}
__device__ __forceinline__ double poly_h(const double *c, double T, double invT) {
  return c[0] + T * (c[1] + T * (c[2] + T * (c[3] + T * c[4]))) + c[5] * invT;
}
__device__ __forceinline__ double poly_s(const double *c, double T, double logT) {
  return c[0] * logT + T * (c[1] + T * (c[2] + T * (c[3] + T * c[4]))) + c[5];
}
// d(cp/R)/dT from the cp coefficients
__device__ __forceinline__ double poly_dcp(const double *c, double T) {
  return c[1] + T * (2.0 * c[2] + T * (3.0 * c[3] + T * 4.0 * c[4]));
}

// ---------------------------------------------------------------------------
// Troe falloff factor Pfac = Pr/(1+Pr) F, Pr = k0 [M] / k_inf, with its
// logarithmic derivatives in T (at fixed [M]) and in [M].
// ---------------------------------------------------------------------------
struct TroeOut {
  double P, dlnP_dT, dlnP_dM;
};

template <bool DERIV>
__device__ __forceinline__ TroeOut troe_factor(const double *tp, double T, double logT,
                                               double invT, double kinf, double dlnkinf,
                                               double M) {
  TroeOut o;
  double k0 = exp(tp[0] + tp[1] * logT - tp[2] * invT);
  double a = tp[3];
  double e3 = exp(-T * tp[4]), e1 = exp(-T * tp[5]), e2 = exp(-tp[6] * invT);
  double Fc = (1.0 - a) * e3 + a * e1 + e2;
  double lFc = log10(Fc);
  double Pr = k0 * M / kinf;
  double L = log10(Pr);
  double c = -0.4 - 0.67 * lFc, nn = 0.75 - 1.27 * lFc;
  const double d = 0.14;
  double u = L + c, v = nn - d * u;
  double X = u / v;
  double den = 1.0 + X * X;
  double lF = lFc / den;
  o.P = Pr / (1.0 + Pr) * exp(lF * LN10);
  o.dlnP_dT = 0.0;
  o.dlnP_dM = 0.0;
  if (DERIV) {
    double dFc = -(1.0 - a) * tp[4] * e3 - a * tp[5] * e1 + tp[6] * invT * invT * e2;
    double dX_dL = nn / (v * v);
    double dv = -1.27 + d * 0.67;
    double dX_dlFc = (-0.67 * v - u * dv) / (v * v);
    double dlF_dL = -lFc * 2.0 * X * dX_dL / (den * den);
    double dlF_dlFc = 1.0 / den - lFc * 2.0 * X * dX_dlFc / (den * den);
    double dlnk0 = tp[1] * invT + tp[2] * invT * invT;
    double dL_dT = (dlnk0 - dlnkinf) / LN10;
    double dlnP_dL = LN10 / (1.0 + Pr) + LN10 * dlF_dL;
    o.dlnP_dT = dlnP_dL * dL_dT + dlF_dlFc * dFc / Fc;
    o.dlnP_dM = dlnP_dL / (M * LN10);
  }
  return o;
}

// ---------------------------------------------------------------------------
// Right-hand side f(y).  Scratch arrays (MAXN each): C, g, hs, wd.
// Returns 0, or KIN_STATE_NONFINITE (4) if any output is not finite.
// ---------------------------------------------------------------------------
template <int MAXN>
struct ChemScratch {
  double C[MAXN], g[MAXN], hs[MAXN], cpk[MAXN], wd[MAXN];
};

template <int MAXN>
__device__ __noinline__ int rhs(const MechView &m, double P, const double *y, double *f,
                   ChemScratch<MAXN> &w) {
  const int ns = m.ns, in = ns - 1;
  const double T = y[0];
  double sumY = 0.0, S = 0.0;
  for (int k = 0; k < in; ++k) {
    double Yk = y[1 + k];
    sumY += Yk;
    S += Yk * m.invW[k];
  }
  const double Yin = 1.0 - sumY;
  S += Yin * m.invW[in];
  const double rho = P / (RU * T * S);
  const double logT = log(T), invT = 1.0 / T;
  double cpm = 0.0;
  for (int k = 0; k < ns; ++k) {
    double Yk = (k < in) ? y[1 + k] : Yin;
    w.C[k] = rho * Yk * m.invW[k];
    int r = range_of(m, k, T);
    double cp = poly_cp(m.cp + (2 * k + r) * NCP, T);
    double h = poly_h(m.h + (2 * k + r) * NH, T, invT);
    double s = poly_s(m.s + (2 * k + r) * NS, T, logT);
    w.g[k] = s - h;
    w.hs[k] = h;
    cpm += Yk * cp * m.invW[k];
    w.wd[k] = 0.0;
  }
  const double Ctot = rho * S;
  const double lnPf = log(PATM / RU) - logT;
  for (int i = 0; i < m.nr; ++i) {
    const int meta = m.meta[i];
    const int *sl = m.slot + 6 * i;
    double kf = exp(m.lnA[i] + m.b[i] * logT - m.Th[i] * invT);
    int nre = meta_nreac(meta), npr = meta_nprod(meta);
    double lnKc = (npr - nre) * lnPf, fwd = 1.0, rev = 1.0;
    for (int s = 0; s < nre; ++s) {
      lnKc -= w.g[sl[s]];
      fwd *= w.C[sl[s]];
    }
    for (int s = 0; s < npr; ++s) {
      lnKc += w.g[sl[3 + s]];
      rev *= w.C[sl[3 + s]];
    }
    double kr = kf * exp(-lnKc);
    double q = kf * fwd - kr * rev;
    int type = meta_type(meta);
    if (type != 0) {
      double M = Ctot;
      int e0 = m.eff0[i], ne = meta_neff(meta);
      for (int e = 0; e < ne; ++e) M += m.eff[e0 + e] * w.C[m.effsp[e0 + e]];
      if (type == 1) {
        q *= M;
      } else {
        TroeOut t = troe_factor<false>(m.troe + NTROE * meta_troe(meta), T, logT, invT, kf,
                                       0.0, M);
        q *= t.P;
      }
    }
    for (int s = 0; s < nre; ++s) w.wd[sl[s]] -= q;
    for (int s = 0; s < npr; ++s) w.wd[sl[3 + s]] += q;
  }
  double Hw = 0.0;
  for (int k = 0; k < in; ++k) Hw += w.hs[k] * w.wd[k];
  // f_T = -sum_k H_k wdot_k / (rho cp),  H_k = (h/RT) Ru T, cp = Ru cpm
  f[0] = -(Hw * T) / (rho * cpm);
  bool ok = isfinite(f[0]);
  for (int k = 0; k < in; ++k) {
    f[1 + k] = m.W[k] * w.wd[k] / rho;
    ok &= isfinite(f[1 + k]);
  }
  return ok ? 0 : 4;
}

// ---------------------------------------------------------------------------
// Analytical Jacobian J (row-major N x N, N = ns), assembled from the sparse
// reaction structure:
//   dq/dY_j = (rho/W_j) D_j - (rho/W_in) D_in - (m_j/S) sigma',
//   D_k = dq/dC_k without the uniform [M] part (that part multiplies
//   d(sum C)/dY_j = 0 at fixed T, P), m_j = 1/W_j - 1/W_in,
//   dq/dT = dq/dT|_C - sigma/T with sigma = sum_k dq/dC_k C_k.
// Rows: dY_k/dt = W_k wdot_k/rho and dT/dt = -sum H_k wdot_k/(rho cp) by
// the product and quotient rules (rho, cp and H_k depend on y).
// ---------------------------------------------------------------------------
template <int MAXN>
struct JacScratch {
  double A[MAXN], B[MAXN], Tc[MAXN], dcp[MAXN], mj[MAXN];
};

template <int MAXN>
__device__ __noinline__ int jac_analytic(const MechView &m, double P, const double *y, double *J,
                            ChemScratch<MAXN> &w, JacScratch<MAXN> &x) {
  const int ns = m.ns, in = ns - 1, N = ns;
  const double T = y[0];
  double sumY = 0.0, S = 0.0;
  for (int k = 0; k < in; ++k) {
    sumY += y[1 + k];
    S += y[1 + k] * m.invW[k];
  }
  const double Yin = 1.0 - sumY;
  S += Yin * m.invW[in];
  const double rho = P / (RU * T * S);
  const double logT = log(T), invT = 1.0 / T;
  double cpm = 0.0, dcpm = 0.0;
  for (int k = 0; k < ns; ++k) {
    double Yk = (k < in) ? y[1 + k] : Yin;
    w.C[k] = rho * Yk * m.invW[k];
    int r = range_of(m, k, T);
    const double *cc = m.cp + (2 * k + r) * NCP;
    double cp = poly_cp(cc, T);
    double h = poly_h(m.h + (2 * k + r) * NH, T, invT);
    double s = poly_s(m.s + (2 * k + r) * NS, T, logT);
    w.g[k] = s - h;
    w.hs[k] = h;
    w.cpk[k] = cp;
    x.dcp[k] = poly_dcp(cc, T);
    cpm += Yk * cp * m.invW[k];
    dcpm += Yk * x.dcp[k] * m.invW[k];
    w.wd[k] = 0.0;
    x.A[k] = 0.0;
    x.B[k] = 0.0;
    x.Tc[k] = 0.0;
  }
  for (int q = 0; q < N * N; ++q) J[q] = 0.0;
  for (int j = 0; j < in; ++j) x.mj[j] = m.invW[j] - m.invW[in];
  const double Ctot = rho * S;
  const double lnPf = log(PATM / RU) - logT;
  for (int i = 0; i < m.nr; ++i) {
    const int meta = m.meta[i];
    const int *sl = m.slot + 6 * i;
    const int nre = meta_nreac(meta), npr = meta_nprod(meta), type = meta_type(meta);
    double kf = exp(m.lnA[i] + m.b[i] * logT - m.Th[i] * invT);
    double dlnkf = m.b[i] * invT + m.Th[i] * invT * invT;
    double lnKc = (npr - nre) * lnPf, dH = 0.0, fwd = 1.0, rev = 1.0;
    for (int s = 0; s < nre; ++s) {
      lnKc -= w.g[sl[s]];
      dH -= w.hs[sl[s]];
      fwd *= w.C[sl[s]];
    }
    for (int s = 0; s < npr; ++s) {
      lnKc += w.g[sl[3 + s]];
      dH += w.hs[sl[3 + s]];
      rev *= w.C[sl[3 + s]];
    }
    double kr = kf * exp(-lnKc);
    // d ln Kc / dT = sum nu (h/RT) / T - (sum nu) / T
    double dlnkr = dlnkf - (dH - (npr - nre)) * invT;
    double phi = 1.0, dphi_dT = 0.0, dphi_dM = 0.0, M = Ctot;
    const int e0 = m.eff0[i], ne = meta_neff(meta);
    if (type != 0) {
      for (int e = 0; e < ne; ++e) M += m.eff[e0 + e] * w.C[m.effsp[e0 + e]];
      if (type == 1) {
        phi = M;
        dphi_dM = 1.0;
      } else {
        TroeOut t = troe_factor<true>(m.troe + NTROE * meta_troe(meta), T, logT, invT, kf,
                                      dlnkf, M);
        phi = t.P;
        dphi_dT = t.P * t.dlnP_dT;
        dphi_dM = t.P * t.dlnP_dM;
      }
    }
    const double Rn = kf * fwd - kr * rev;
    const double q = phi * Rn;
    const double u = Rn * dphi_dM;
    const double sig_p = phi * (nre * kf * fwd - npr * kr * rev) + u * (M - Ctot);
    const double dqdT = phi * (kf * dlnkf * fwd - kr * dlnkr * rev) + Rn * dphi_dT -
                        (sig_p + u * Ctot) * invT;
    // row updates: nu = -1 per reactant slot, +1 per product slot
    for (int rs = 0; rs < nre + npr; ++rs) {
      const int row = (rs < nre) ? sl[rs] : sl[3 + rs - nre];
      const double nu = (rs < nre) ? -1.0 : 1.0;
      w.wd[row] += nu * q;
      x.B[row] += nu * sig_p;
      x.Tc[row] += nu * dqdT;
      double *Jr = J + (1 + row) * N;
      // mass-action columns
      for (int cs = 0; cs < nre + npr; ++cs) {
        const int col = (cs < nre) ? sl[cs] : sl[3 + cs - nre];
        double p = 1.0;
        if (cs < nre) {
          for (int t = 0; t < nre; ++t)
            if (t != cs) p *= w.C[sl[t]];
          p *= phi * kf;
        } else {
          for (int t = 0; t < npr; ++t)
            if (t != cs - nre) p *= w.C[sl[3 + t]];
          p *= -phi * kr;
        }
        if (col != in)
          Jr[1 + col] += nu * rho * m.invW[col] * p;
        else
          x.A[row] += nu * p;
      }
      // efficiency columns
      for (int e = 0; e < ne; ++e) {
        const int col = m.effsp[e0 + e];
        const double p = u * m.eff[e0 + e];
        if (col != in)
          Jr[1 + col] += nu * rho * m.invW[col] * p;
        else
          x.A[row] += nu * p;
      }
    }
  }
  // rank-one and inert terms, then the temperature column of dwdot/dy
  const double rWin = rho * m.invW[in];
  for (int k = 0; k < in; ++k) {
    double *Jr = J + (1 + k) * N;
    Jr[0] = x.Tc[k];
    for (int j = 0; j < in; ++j) Jr[1 + j] -= rWin * x.A[k] + x.mj[j] / S * x.B[k];
  }
  // T row from the dwdot/dy rows (before they are scaled)
  double Hw = 0.0, CPw = 0.0;
  for (int k = 0; k < in; ++k) {
    Hw += w.hs[k] * w.wd[k];
    CPw += w.cpk[k] * w.wd[k];
  }
  Hw *= RU * T;   // sum H_k wdot_k, J/(m^3 s)
  CPw *= RU;      // sum Cp_k wdot_k
  const double rcp = rho * cpm * RU;
  const double cpin = w.cpk[in] * m.invW[in];
  for (int c = 0; c < N; ++c) {
    double dHw = (c == 0) ? CPw : 0.0;
    for (int k = 0; k < in; ++k) dHw += w.hs[k] * RU * T * J[(1 + k) * N + c];
    double drho, dcp;
    if (c == 0) {
      drho = -rho * invT;
      dcp = dcpm * RU;
    } else {
      drho = -rho * x.mj[c - 1] / S;
      dcp = (w.cpk[c - 1] * m.invW[c - 1] - cpin) * RU;
    }
    const double drcp = cpm * RU * drho + rho * dcp;
    J[c] = -dHw / rcp + Hw / (rcp * rcp) * drcp;
  }
  bool ok = true;
  for (int k = 0; k < in; ++k) {
    double *Jr = J + (1 + k) * N;
    const double a = m.W[k] / rho, bb = m.W[k] * w.wd[k] / (rho * rho);
    Jr[0] = a * Jr[0] - bb * (-rho * invT);
    for (int j = 0; j < in; ++j) Jr[1 + j] = a * Jr[1 + j] - bb * (-rho * x.mj[j] / S);
  }
  for (int q = 0; q < N * N; ++q) ok &= isfinite(J[q]);
  return ok ? 0 : 4;
}

// ---------------------------------------------------------------------------
// Dense LU with partial pivoting (row-major, leading dimension n).
// Returns 0 or k+1 when column k has no nonzero pivot.
// ---------------------------------------------------------------------------
template <typename LT>
__device__ __noinline__ int lu_real(int n, LT *a, int *ip) {
  for (int k = 0; k < n; ++k) {
    int p = k;
    LT amax = fabs(a[k * n + k]);
    for (int i = k + 1; i < n; ++i) {
      LT v = fabs(a[i * n + k]);
      if (v > amax) {
        amax = v;
        p = i;
      }
    }
    ip[k] = p;
    if (amax == LT(0)) return k + 1;
    if (p != k)
      for (int j = 0; j < n; ++j) {
        LT t = a[k * n + j];
        a[k * n + j] = a[p * n + j];
        a[p * n + j] = t;
      }
    const LT inv = LT(1) / a[k * n + k];
    for (int i = k + 1; i < n; ++i) {
      LT l = a[i * n + k] * inv;
      a[i * n + k] = l;
      if (l != LT(0))
        for (int j = k + 1; j < n; ++j) a[i * n + j] -= l * a[k * n + j];
    }
  }
  return 0;
}

template <typename LT, typename VT>
__device__ __noinline__ void lu_solve_real(int n, const LT *lu, const int *ip, VT *b) {
  for (int k = 0; k < n; ++k) {
    int p = ip[k];
    if (p != k) {
      VT t = b[k];
      b[k] = b[p];
      b[p] = t;
    }
  }
  for (int i = 1; i < n; ++i) {
    LT s = LT(b[i]);
    for (int j = 0; j < i; ++j) s -= lu[i * n + j] * LT(b[j]);
    b[i] = VT(s);
  }
  for (int i = n - 1; i >= 0; --i) {
    LT s = LT(b[i]);
    for (int j = i + 1; j < n; ++j) s -= lu[i * n + j] * LT(b[j]);
    b[i] = VT(s / lu[i * n + i]);
  }
}

// complex (a + ib) / (c + id), Smith's scaling
template <typename LT>
__device__ __forceinline__ void cdiv(LT a, LT b, LT c, LT d, LT &re, LT &im) {
  if (fabs(c) >= fabs(d)) {
    LT r = d / c, den = c + d * r;
    re = (a + b * r) / den;
    im = (b - a * r) / den;
  } else {
    LT r = c / d, den = c * r + d;
    re = (a * r + b) / den;
    im = (b * r - a) / den;
  }
}

template <typename LT>
__device__ __noinline__ int lu_cplx(int n, LT *ar, LT *ai, int *ip) {
  for (int k = 0; k < n; ++k) {
    int p = k;
    LT amax = fabs(ar[k * n + k]) + fabs(ai[k * n + k]);
    for (int i = k + 1; i < n; ++i) {
      LT v = fabs(ar[i * n + k]) + fabs(ai[i * n + k]);
      if (v > amax) {
        amax = v;
        p = i;
      }
    }
    ip[k] = p;
    if (amax == LT(0)) return k + 1;
    if (p != k)
      for (int j = 0; j < n; ++j) {
        LT t = ar[k * n + j];
        ar[k * n + j] = ar[p * n + j];
        ar[p * n + j] = t;
        t = ai[k * n + j];
        ai[k * n + j] = ai[p * n + j];
        ai[p * n + j] = t;
      }
    const LT pr = ar[k * n + k], pi = ai[k * n + k];
    for (int i = k + 1; i < n; ++i) {
      LT lr, li;
      cdiv(ar[i * n + k], ai[i * n + k], pr, pi, lr, li);
      ar[i * n + k] = lr;
      ai[i * n + k] = li;
      if (lr != LT(0) || li != LT(0))
        for (int j = k + 1; j < n; ++j) {
          LT ur = ar[k * n + j], ui = ai[k * n + j];
          ar[i * n + j] -= lr * ur - li * ui;
          ai[i * n + j] -= lr * ui + li * ur;
        }
    }
  }
  return 0;
}

template <typename LT, typename VT>
__device__ __noinline__ void lu_solve_cplx(int n, const LT *lr, const LT *li, const int *ip, VT *br,
                              VT *bi) {
  for (int k = 0; k < n; ++k) {
    int p = ip[k];
    if (p != k) {
      VT t = br[k];
      br[k] = br[p];
      br[p] = t;
      t = bi[k];
      bi[k] = bi[p];
      bi[p] = t;
    }
  }
  for (int i = 1; i < n; ++i) {
    LT sr = LT(br[i]), si = LT(bi[i]);
    for (int j = 0; j < i; ++j) {
      LT xr = LT(br[j]), xi = LT(bi[j]);
      sr -= lr[i * n + j] * xr - li[i * n + j] * xi;
      si -= lr[i * n + j] * xi + li[i * n + j] * xr;
    }
    br[i] = VT(sr);
    bi[i] = VT(si);
  }
  for (int i = n - 1; i >= 0; --i) {
    LT sr = LT(br[i]), si = LT(bi[i]);
    for (int j = i + 1; j < n; ++j) {
      LT xr = LT(br[j]), xi = LT(bi[j]);
      sr -= lr[i * n + j] * xr - li[i * n + j] * xi;
      si -= lr[i * n + j] * xi + li[i * n + j] * xr;
    }
    LT qr, qi;
    cdiv(sr, si, lr[i * n + i], li[i * n + i], qr, qi);
    br[i] = VT(qr);
    bi[i] = VT(qi);
  }
}

}  // namespace kin
