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
  int ntroe, nfall;  // device order: Troe reactions [0, ntroe), third-body [ntroe, nfall)
  int nd, ni;  // table sizes in doubles / ints
  // double-table offsets
  int dW, dinvW, dTmid, dcp, dh, dg, dlnA, db, dTh, dtroe, deff, dexp, dnu, dcsrnu;
  // int-table offsets
  int islot, imeta, ieff0, itroe, ieffsp;
  int icsr0, icsr;  // species -> (reaction, net nu) lists: offsets [ns+1], entries
};

// per-species coefficient blocks (two ranges each):
//   cp/R = c0 + T(c1 + T(c2 + T(c3 + T c4)))                 (5)
//   h/RT = c0 + T(c1 + T(c2 + T(c3 + T c4))) + c5 / T        (6)
//   g    = s/R - h/RT
//        = c0 lnT + T(c1 + T(c2 + T(c3 + T c4))) + c5 + c6 / T (7)
constexpr int NCP = 5, NH = 6, NG = 7;
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
  int ns, nr, ntroe, nfall;
  const double *W, *invW, *Tmid, *cp, *h, *gb, *lnA, *b, *Th, *troe, *eff, *etab;
  const double *dnu;      // per reaction: sum of product minus reactant coefficients
  const double *csrnu;    // per species -> reaction entry: the net coefficient nu
  const int *slot, *meta, *eff0, *effsp;
  const int *csr0, *csr;  // entry = reaction << 4 | (nu + 8)
};

__device__ __forceinline__ MechView make_view(const MechLayout &L, const double *d, const int *i) {
  MechView v;
  v.ns = L.ns;
  v.nr = L.nr;
  v.ntroe = L.ntroe;
  v.nfall = L.nfall;
  v.W = d + L.dW;
  v.invW = d + L.dinvW;
  v.Tmid = d + L.dTmid;
  v.cp = d + L.dcp;
  v.h = d + L.dh;
  v.gb = d + L.dg;
  v.lnA = d + L.dlnA;
  v.b = d + L.db;
  v.Th = d + L.dTh;
  v.troe = d + L.dtroe;
  v.eff = d + L.deff;
  v.etab = d + L.dexp;
  v.dnu = d + L.dnu;
  v.csrnu = d + L.dcsrnu;
  v.slot = i + L.islot;
  v.meta = i + L.imeta;
  v.eff0 = i + L.ieff0;
  v.effsp = i + L.ieffsp;
  v.csr0 = i + L.icsr0;
  v.csr = i + L.icsr;
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
__device__ __forceinline__ double poly_g(const double *c, double T, double logT, double invT) {
  return c[0] * logT + T * (c[1] + T * (c[2] + T * (c[3] + T * c[4]))) + c[5] + c[6] * invT;
}
// d(cp/R)/dT from the cp coefficients
__device__ __forceinline__ double poly_dcp(const double *c, double T) {
  return c[1] + T * (2.0 * c[2] + T * (3.0 * c[3] + T * 4.0 * c[4]));
}

// ---------------------------------------------------------------------------
// Exponential for the rate expressions: Tang's table-driven method
// (ACM TOMS 15, 1989).  exp(x) = 2^m 2^(j/256) exp(r) with N = round(256 x /
// ln 2), j = N mod 256, m = N div 256, r = x - N ln2/256 (|r| <= ln2/512,
// computed with ln2/256 split into a 29-bit head, so N*head is exact, and a
// tail); exp(r) = 1 + r + r^2/2 + r^3/6 + r^4/24 (truncation below 4e-17).
// The 256 values 2^(j/256) are rounded doubles computed by the host.  Valid
// for |x| < 700 (the result stays a normal number), checked on the high word
// with integer arithmetic; outside that range the library exp() is used.
// ---------------------------------------------------------------------------
constexpr int EXP_TAB = 256;

__device__ __forceinline__ double kexp(double x, const double *tab) {
  if ((__double2hiint(x) & 0x7fffffff) >= 0x4085E000) return exp(x);  // |x| >= 700, NaN
  const double inv = 0x1.71547652b82fep+8;    // 256 / ln 2
  const double hi = 0x1.62e42ff000000p-9;     // ln2/256, 29 significant bits
  const double lo = -0x1.718432a1b0e26p-43;   // ln2/256 - hi
  const double shifter = 0x1.8p52;            // 1.5 * 2^52: rounds to an integer
  double kd = fma(x, inv, shifter);
  const int N = (int)(unsigned)__double2loint(kd);
  kd -= shifter;
  double r = fma(-kd, hi, x);
  r = fma(-kd, lo, r);
  double q = fma(r, 1.0 / 24.0, 1.0 / 6.0);
  q = fma(q, r, 0.5);
  q = fma(q, r, 1.0);
  const double p = q * r;                     // exp(r) - 1
  const double tj = tab[N & (EXP_TAB - 1)];
  const double v = fma(tj, p, tj);
  const long long m = (long long)(N >> 8);     // floor division (arithmetic shift)
  return __longlong_as_double(__double_as_longlong(v) + (m << 52));
}

// ---------------------------------------------------------------------------
// Troe falloff factor Pfac = Pr/(1+Pr) F, Pr = k0 [M] / k_inf, with its
// logarithmic derivatives in T (at fixed [M]) and in [M].  lnkinf is the
// high-pressure rate's Arrhenius exponent (ln k_inf), so ln Pr is formed from
// the two exponents and ln [M] without dividing the rate constants.
// ---------------------------------------------------------------------------
struct TroeOut {
  double P, dlnP_dT, dlnP_dM;
};

template <bool DERIV>
__device__ __forceinline__ TroeOut troe_factor(const double *tp, double T, double logT,
                                               double invT, double lnkinf, double dlnkinf,
                                               double M, const double *etab) {
  TroeOut o;
  double a = tp[3];
  double e3 = kexp(-T * tp[4], etab), e1 = kexp(-T * tp[5], etab), e2 = kexp(-tp[6] * invT, etab);
  double Fc = (1.0 - a) * e3 + a * e1 + e2;
  double lFc = log10(Fc);
  const double lnPr = (tp[0] + tp[1] * logT - tp[2] * invT) - lnkinf + log(M);
  const double Pr = kexp(lnPr, etab);
  const double L = lnPr * (1.0 / LN10);  // log10 Pr
  double c = -0.4 - 0.67 * lFc, nn = 0.75 - 1.27 * lFc;
  const double d = 0.14;
  double u = L + c, v = nn - d * u;
  // log10 F = lFc / (1 + (u/v)^2) = lFc v^2 / (v^2 + u^2): one division
  const double v2 = v * v;
  o.P = Pr / (1.0 + Pr) * kexp(lFc * v2 / (v2 + u * u) * LN10, etab);
  o.dlnP_dT = 0.0;
  o.dlnP_dM = 0.0;
  if (DERIV) {
    double X = u / v;
    double den = 1.0 + X * X;
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
// Source terms and (optionally) the analytical Jacobian at one point.
//
// f(y): thermo per species, then per reaction kf = exp(lnA + b lnT - Theta/T),
// Kc from the Gibbs energies, kr = kf exp(-ln Kc), q = phi (kf prod C' -
// kr prod C''), wdot scattered to the species, dY/dt = W wdot/rho and
// dT/dt = -sum H wdot / (rho cp).  Rates are always FP64.
//
// J = df/dy (row-major N x N in the matrix type JT) reuses the same rates and
// is assembled from the sparse reaction structure:
//   dq/dY_j = (rho/W_j) D_j - (rho/W_in) D_in - (m_j/S) sigma',
//   D_k = dq/dC_k without the uniform [M] part (that part multiplies
//   d(sum C)/dY_j = 0 at fixed T, P), m_j = 1/W_j - 1/W_in,
//   dq/dT = dq/dT|_C - sigma/T, sigma = sum_k dq/dC_k C_k,
// then dY_k/dt = W_k wdot_k/rho and dT/dt = -sum H_k wdot_k/(rho cp) by the
// product and quotient rules.  Per-reaction scalars are formed in FP64 and
// the assembly arithmetic runs in JT (FP32 when the Newton matrices are FP32).
// Returns 0, or 4 (KIN_STATE_NONFINITE) for a non-finite f or J.
// ---------------------------------------------------------------------------
template <int MAXN>
struct ChemScratch {
  double C[MAXN], g[MAXN], hs[MAXN], cpk[MAXN], wd[MAXN];
};

// One thread's vector in the block's shared memory, element k at p[k * stride]:
// the threads of a block are interleaved, so a warp's accesses to the same k
// are consecutive doubles (no bank conflicts).
struct SmemVec {
  double *p;
  int stride;
  __device__ __forceinline__ double &operator[](int k) const { return p[k * stride]; }
};

// The same scratch with the arrays the reaction loop gathers from and scatters
// to (C, g, wdot) in shared memory, the others in the thread's own memory.
template <int MAXN>
struct ChemScratchS {
  SmemVec C, g, wd;
  double hs[MAXN], cpk[MAXN];
  // three vectors of ns doubles per thread of the block, at base
  __device__ __forceinline__ void bind(double *base, int ns) {
    const int nt = blockDim.x, t = threadIdx.x;
    C = SmemVec{base + t, nt};
    g = SmemVec{base + ns * nt + t, nt};
    wd = SmemVec{base + 2 * ns * nt + t, nt};
  }
  __host__ __device__ static size_t bytes(int ns, int nt) { return 3 * sizeof(double) * ns * nt; }
};

template <int MAXN, typename JT>
struct JacScratch {
  JT A[MAXN], B[MAXN], Tc[MAXN], mj[MAXN], Cj[MAXN], rW[MAXN];
  double dcp[MAXN];
};

// Unroll factor of the per-species and per-reaction loops of chem_eval: more
// independent FP64 chains in flight per thread (a build-time tuning knob).
#ifndef KIN_RHS_UNROLL
#define KIN_RHS_UNROLL 1
#endif
constexpr int RHS_UNROLL = KIN_RHS_UNROLL;

template <int MAXN, typename JT, typename CS>
__device__ __noinline__ int chem_eval(const MechView &m, double P, const double *y,
                                      double *f, JT *J, bool wantJ, CS &w,
                                      JacScratch<MAXN, JT> &x) {
  const int ns = m.ns, in = ns - 1, N = ns;
  const double T = y[0];
  double sumY = 0.0, S = 0.0;
  for (int k = 0; k < in; ++k) {
    const double Yk = y[1 + k];
    sumY += Yk;
    S += Yk * m.invW[k];
  }
  const double Yin = 1.0 - sumY;
  S += Yin * m.invW[in];
  const double rho = P / (RU * T * S);
  const double logT = log(T), invT = 1.0 / T;
  double cpm = 0.0, dcpm = 0.0;
#pragma unroll RHS_UNROLL
  for (int k = 0; k < ns; ++k) {
    const double Yk = (k < in) ? y[1 + k] : Yin;
    const double YW = Yk * m.invW[k];
    w.C[k] = rho * YW;
    // the range test on the bit patterns (both are positive): integer pipe
    const int r = (__double_as_longlong(T) < __double_as_longlong(m.Tmid[k])) ? 0 : 1;
    const double *cc = m.cp + (2 * k + r) * NCP;
    const double cp = poly_cp(cc, T);
    const double h = poly_h(m.h + (2 * k + r) * NH, T, invT);
    w.g[k] = poly_g(m.gb + (2 * k + r) * NG, T, logT, invT);
    w.hs[k] = h;
    cpm = fma(YW, cp, cpm);
    w.wd[k] = 0.0;
    if (wantJ) {
      w.cpk[k] = cp;  // per-species cp only for the Jacobian's temperature terms
      x.dcp[k] = poly_dcp(cc, T);
      dcpm = fma(YW, x.dcp[k], dcpm);
      x.A[k] = JT(0);
      x.B[k] = JT(0);
      x.Tc[k] = JT(0);
      x.Cj[k] = JT(w.C[k]);
      x.rW[k] = JT(rho * m.invW[k]);
    }
  }
  if (wantJ) {
    for (int q = 0; q < N * N; ++q) J[q] = JT(0);
    for (int j = 0; j < in; ++j) x.mj[j] = JT(m.invW[j] - m.invW[in]);
  }
  const double Ctot = rho * S;
  const double lnPf = 2.5003366899611787 - logT;  // ln(Patm / Ru) - ln T
#pragma unroll RHS_UNROLL
  for (int i = 0; i < m.nr; ++i) {
    const int meta = m.meta[i];
    const int *sl = m.slot + 6 * i;
    const int nre = meta_nreac(meta), npr = meta_nprod(meta), type = meta_type(meta);
    const double lnkf = m.lnA[i] + m.b[i] * logT - m.Th[i] * invT;
    const double kf = kexp(lnkf, m.etab);
    // every reaction has a reactant and a product (checked when the mechanism
    // is created): the first of each seeds the Gibbs sum and the products
    double fwd = w.C[sl[0]], rev = w.C[sl[3]];
    double lnKc = fma(m.dnu[i], lnPf, w.g[sl[3]] - w.g[sl[0]]);
    for (int s = 1; s < nre; ++s) {
      lnKc -= w.g[sl[s]];
      fwd *= w.C[sl[s]];
    }
    for (int s = 1; s < npr; ++s) {
      lnKc += w.g[sl[3 + s]];
      rev *= w.C[sl[3 + s]];
    }
    const double iKc = kexp(-lnKc, m.etab);  // 1 / Kc, so kr = kf / Kc
    double phi = 1.0, dphi_dT = 0.0, dphi_dM = 0.0, M = Ctot;
    const int e0 = m.eff0[i], ne = meta_neff(meta);
    // d ln kf / dT, needed only for the Jacobian
    const double dlnkf = wantJ ? m.b[i] * invT + m.Th[i] * invT * invT : 0.0;
    if (type != 0) {
      for (int e = 0; e < ne; ++e) M += m.eff[e0 + e] * w.C[m.effsp[e0 + e]];
      if (type == 1) {
        phi = M;
        dphi_dM = 1.0;
      } else {
        // the derivatives only when the Jacobian is assembled
        const double *tp = m.troe + NTROE * meta_troe(meta);
        TroeOut t = wantJ ? troe_factor<true>(tp, T, logT, invT, lnkf, dlnkf, M, m.etab)
                          : troe_factor<false>(tp, T, logT, invT, lnkf, dlnkf, M, m.etab);
        phi = t.P;
        dphi_dT = t.P * t.dlnP_dT;
        dphi_dM = t.P * t.dlnP_dM;
      }
    }
    const double Rn = kf * fma(-iKc, rev, fwd);  // kf prod C' - kr prod C''
    const double q = (type != 0) ? phi * Rn : Rn;
    for (int s = 0; s < nre; ++s) w.wd[sl[s]] -= q;
    for (int s = 0; s < npr; ++s) w.wd[sl[3 + s]] += q;
    if (wantJ) {
      const double kr = kf * iKc;
      // d ln Kc / dT = sum nu (h/RT) / T - (sum nu) / T
      double dH = 0.0;
      for (int s = 0; s < nre; ++s) dH -= w.hs[sl[s]];
      for (int s = 0; s < npr; ++s) dH += w.hs[sl[3 + s]];
      const double dlnkr = dlnkf - (dH - m.dnu[i]) * invT;
      const double u = Rn * dphi_dM;
      const double sig_p = phi * (nre * kf * fwd - npr * kr * rev) + u * (M - Ctot);
      const double dqdT = phi * (kf * dlnkf * fwd - kr * dlnkr * rev) + Rn * dphi_dT -
                          (sig_p + u * Ctot) * invT;
      const JT pkf = JT(phi * kf), pkr = JT(-phi * kr), uJ = JT(u);
      const JT sJ = JT(sig_p), tJ = JT(dqdT);
      for (int rs = 0; rs < nre + npr; ++rs) {
        const int row = (rs < nre) ? sl[rs] : sl[3 + rs - nre];
        const JT nu = (rs < nre) ? JT(-1) : JT(1);
        x.B[row] += nu * sJ;
        x.Tc[row] += nu * tJ;
        JT *Jr = J + (1 + row) * N;
        for (int cs = 0; cs < nre + npr; ++cs) {
          const int col = (cs < nre) ? sl[cs] : sl[3 + cs - nre];
          JT p = (cs < nre) ? pkf : pkr;
          if (cs < nre) {
            for (int t = 0; t < nre; ++t)
              if (t != cs) p *= x.Cj[sl[t]];
          } else {
            for (int t = 0; t < npr; ++t)
              if (t != cs - nre) p *= x.Cj[sl[3 + t]];
          }
          if (col != in)
            Jr[1 + col] += nu * x.rW[col] * p;
          else
            x.A[row] += nu * p;
        }
        for (int e = 0; e < ne; ++e) {
          const int col = m.effsp[e0 + e];
          const JT p = uJ * JT(m.eff[e0 + e]);
          if (col != in)
            Jr[1 + col] += nu * x.rW[col] * p;
          else
            x.A[row] += nu * p;
        }
      }
    }
  }
  double Hw = 0.0;
  for (int k = 0; k < in; ++k) Hw += w.hs[k] * w.wd[k];
  // f_T = -sum_k H_k wdot_k / (rho cp),  H_k = (h/RT) Ru T, cp = Ru cpm
  f[0] = -(Hw * T) / (rho * cpm);
  // finiteness on the exponent bits (integer pipe): all ones = inf or NaN
  int nonfinite = (__double2hiint(f[0]) & 0x7ff00000) == 0x7ff00000;
  const double irho = 1.0 / rho;
  for (int k = 0; k < in; ++k) {
    f[1 + k] = m.W[k] * w.wd[k] * irho;
    nonfinite |= (__double2hiint(f[1 + k]) & 0x7ff00000) == 0x7ff00000;
  }
  if (!wantJ) return nonfinite ? 4 : 0;
  bool ok = !nonfinite;
  double CPw = 0.0;
  for (int k = 0; k < in; ++k) CPw += w.cpk[k] * w.wd[k];
  // rank-one and inert terms, then the temperature column of dwdot/dy
  const double iSd = 1.0 / S;
  const JT rWin = x.rW[in], iS = JT(iSd);
  for (int k = 0; k < in; ++k) {
    JT *Jr = J + (1 + k) * N;
    Jr[0] = x.Tc[k];
    const JT a = rWin * x.A[k], b = iS * x.B[k];
    for (int j = 0; j < in; ++j) Jr[1 + j] -= a + x.mj[j] * b;
  }
  // T row from the dwdot/dy rows (before they are scaled); h/RT in the
  // matrix type once per species (the Cj scratch is free by now)
  for (int k = 0; k < in; ++k) x.Cj[k] = JT(w.hs[k]);
  const double HwJ = Hw * RU * T;      // sum H_k wdot_k
  const double CPwJ = CPw * RU;        // sum Cp_k wdot_k
  const double rcp = rho * cpm * RU;
  const double cpin = w.cpk[in] * m.invW[in];
  const JT hfac = JT(RU * T / rcp);    // dHw/dy enters as -RU T sum h_k J_kc / rcp
  const JT g2 = JT(HwJ / (rcp * rcp));
  const double rhoS = rho * iSd;
  for (int c = 0; c < N; ++c) {
    JT dh = JT(0);
    for (int k = 0; k < in; ++k) dh += x.Cj[k] * J[(1 + k) * N + c];
    double drcp;
    if (c == 0) {
      drcp = cpm * RU * (-rho * invT) + rho * dcpm * RU;
    } else {
      drcp = cpm * RU * (-rhoS * (m.invW[c - 1] - m.invW[in])) +
             rho * (w.cpk[c - 1] * m.invW[c - 1] - cpin) * RU;
    }
    const JT extra = (c == 0) ? JT(-CPwJ / rcp) : JT(0);
    J[c] = -hfac * dh + extra + g2 * JT(drcp);
  }
  for (int k = 0; k < in; ++k) {
    JT *Jr = J + (1 + k) * N;
    const JT a = JT(m.W[k] * irho), bb = JT(m.W[k] * w.wd[k] * irho * irho);
    Jr[0] = a * Jr[0] + bb * JT(rho * invT);
    const JT bS = bb * JT(rhoS);
    for (int j = 0; j < in; ++j) Jr[1 + j] = a * Jr[1 + j] + bS * x.mj[j];
  }
  // in the matrix type itself: no widening conversion per entry
  for (int q = 0; q < N * N; ++q) ok &= isfinite(J[q]);
  return ok ? 0 : 4;
}

// f only (the Jacobian scratch is not touched when wantJ is false)
template <int MAXN, typename JT, typename CS>
__device__ __forceinline__ int rhs(const MechView &m, double P, const double *y, double *f,
                                   CS &w, JacScratch<MAXN, JT> &x) {
  return chem_eval<MAXN, JT>(m, P, y, f, (JT *)nullptr, false, w, x);
}

// ---------------------------------------------------------------------------
// Dense LU with partial pivoting (row-major, leading dimension n).  The loops
// stay rolled (#pragma unroll 1) to keep the instruction footprint small.
// Returns 0 or k+1 when column k has no nonzero pivot.
// ---------------------------------------------------------------------------
template <typename LT>
__device__ __noinline__ int lu_real(int n, LT *a, int *ip) {
  #pragma unroll 1
  for (int k = 0; k < n; ++k) {
    int p = k;
    LT amax = fabs(a[k * n + k]);
    #pragma unroll 1
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
      #pragma unroll 1
      for (int j = 0; j < n; ++j) {
        LT t = a[k * n + j];
        a[k * n + j] = a[p * n + j];
        a[p * n + j] = t;
      }
    const LT inv = LT(1) / a[k * n + k];
    #pragma unroll 1
    for (int i = k + 1; i < n; ++i) {
      LT l = a[i * n + k] * inv;
      a[i * n + k] = l;
      if (l != LT(0))
        #pragma unroll 1
        for (int j = k + 1; j < n; ++j) a[i * n + j] -= l * a[k * n + j];
    }
  }
  return 0;
}

// Solve LU x = b in place.  The right-hand side is rounded to the matrix
// type once, the substitution runs in LT, and the result is widened back.
template <int MAXN, typename LT, typename VT>
__device__ __noinline__ void lu_solve_real(int n, const LT *lu, const int *ip, VT *b) {
  LT v[MAXN];
  #pragma unroll 1
  for (int k = 0; k < n; ++k) v[k] = LT(b[k]);
  #pragma unroll 1
  for (int k = 0; k < n; ++k) {
    const int p = ip[k];
    if (p != k) {
      const LT t = v[k];
      v[k] = v[p];
      v[p] = t;
    }
  }
  #pragma unroll 1
  for (int i = 1; i < n; ++i) {
    LT s = v[i];
    #pragma unroll 1
    for (int j = 0; j < i; ++j) s -= lu[i * n + j] * v[j];
    v[i] = s;
  }
  #pragma unroll 1
  for (int i = n - 1; i >= 0; --i) {
    LT s = v[i];
    #pragma unroll 1
    for (int j = i + 1; j < n; ++j) s -= lu[i * n + j] * v[j];
    v[i] = s / lu[i * n + i];
  }
  #pragma unroll 1
  for (int k = 0; k < n; ++k) b[k] = VT(v[k]);
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

// Complex matrices of the thread layouts keep (re, im) interleaved, so an
// entry is one 8-byte (FP32) or 16-byte (FP64) access.
template <typename LT>
struct CplxOf;
template <>
struct CplxOf<float> {
  using type = float2;
};
template <>
struct CplxOf<double> {
  using type = double2;
};
template <typename LT>
using cplx_t = typename CplxOf<LT>::type;

template <typename LT>
__device__ __noinline__ int lu_cplx(int n, cplx_t<LT> *a, int *ip) {
  #pragma unroll 1
  for (int k = 0; k < n; ++k) {
    int p = k;
    LT amax = fabs(a[k * n + k].x) + fabs(a[k * n + k].y);
    #pragma unroll 1
    for (int i = k + 1; i < n; ++i) {
      const cplx_t<LT> e = a[i * n + k];
      LT v = fabs(e.x) + fabs(e.y);
      if (v > amax) {
        amax = v;
        p = i;
      }
    }
    ip[k] = p;
    if (amax == LT(0)) return k + 1;
    if (p != k)
      #pragma unroll 1
      for (int j = 0; j < n; ++j) {
        const cplx_t<LT> t = a[k * n + j];
        a[k * n + j] = a[p * n + j];
        a[p * n + j] = t;
      }
    const cplx_t<LT> pk = a[k * n + k];
    #pragma unroll 1
    for (int i = k + 1; i < n; ++i) {
      LT lr, li;
      cdiv(a[i * n + k].x, a[i * n + k].y, pk.x, pk.y, lr, li);
      a[i * n + k].x = lr;
      a[i * n + k].y = li;
      if (lr != LT(0) || li != LT(0))
        #pragma unroll 1
        for (int j = k + 1; j < n; ++j) {
          const cplx_t<LT> u = a[k * n + j];
          cplx_t<LT> e = a[i * n + j];
          e.x -= lr * u.x - li * u.y;
          e.y -= lr * u.y + li * u.x;
          a[i * n + j] = e;
        }
    }
  }
  return 0;
}

template <int MAXN, typename LT, typename VT>
__device__ __noinline__ void lu_solve_cplx(int n, const cplx_t<LT> *l, const int *ip, VT *br,
                                           VT *bi) {
  cplx_t<LT> v[MAXN];
  #pragma unroll 1
  for (int k = 0; k < n; ++k) {
    v[k].x = LT(br[k]);
    v[k].y = LT(bi[k]);
  }
  #pragma unroll 1
  for (int k = 0; k < n; ++k) {
    const int p = ip[k];
    if (p != k) {
      const cplx_t<LT> t = v[k];
      v[k] = v[p];
      v[p] = t;
    }
  }
  #pragma unroll 1
  for (int i = 1; i < n; ++i) {
    LT sr = v[i].x, si = v[i].y;
    #pragma unroll 1
    for (int j = 0; j < i; ++j) {
      const cplx_t<LT> x = v[j], m = l[i * n + j];
      sr -= m.x * x.x - m.y * x.y;
      si -= m.x * x.y + m.y * x.x;
    }
    v[i].x = sr;
    v[i].y = si;
  }
  #pragma unroll 1
  for (int i = n - 1; i >= 0; --i) {
    LT sr = v[i].x, si = v[i].y;
    #pragma unroll 1
    for (int j = i + 1; j < n; ++j) {
      const cplx_t<LT> x = v[j], m = l[i * n + j];
      sr -= m.x * x.x - m.y * x.y;
      si -= m.x * x.y + m.y * x.x;
    }
    LT qr, qi;
    cdiv(sr, si, l[i * n + i].x, l[i * n + i].y, qr, qi);
    v[i].x = qr;
    v[i].y = qi;
  }
  #pragma unroll 1
  for (int k = 0; k < n; ++k) {
    br[k] = VT(v[k].x);
    bi[k] = VT(v[k].y);
  }
}

}  // namespace kin
