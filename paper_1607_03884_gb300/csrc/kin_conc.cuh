// Radau IIA on the concentration-based reactor, one state per group of L
// lanes, with a sparse LU of the Newton matrices: the reformulation the
// paper proposes for large models (Sec. 3.3, "memory traffic"; Sec. 4),
// where a Jacobian in species concentrations is sparse and admits sparse
// factorisation.
//
// State (per unit mass of mixture, constant pressure): T, the volume V and
// the moles n_k of every species but the last, the inert bath gas, whose
// moles close P V = n Ru T.  With C_k = n_k / V and Ctot = P / (Ru T):
//   dn_k/dt = V wdot_k,   dT/dt = -sum_k H_k wdot_k / sum_k C_k Cp_k,
//   dV/dt = V (sum_k wdot_k / Ctot + (dT/dt) / T).
// Two species are coupled in the Jacobian only through a reaction both take
// part in, or a collision efficiency that differs from the bath gas's (which
// must be the default, 1); the T and V rows and columns are full.
//
// The group's vectors hold the variables in elimination order: the host
// (kin_conc.cu) orders the species by minimum degree and puts T and V last,
// so the LU needs no pivoting and fills only the symbolic pattern it lists:
// per pivot k the rows below it in column k of L and the columns right of it
// in row k of U.  Minimum degree leaves a trailing block that is full (from
// pivot k0 on); there the update runs dense, without the lists' indirection.
// The matrices are stored dense (N x (N+1), as in the mass-fraction layout);
// entries outside the pattern stay zero, so the back substitution and the
// forward one past k0 run over whole columns.
// The step driver (warp_init_sys / warp_step_sys) is the mass-fraction
// layout's, with ConcSys as its system.  The moles' absolute tolerance is
// atol / W_k, so that an error in n_k weighs as the mass-fraction error
// W_k dn_k does in the mass-fraction form (T and V take atol).
#pragma once
#include "kin_warp.cuh"

namespace kin {

struct ConcView {
  int N;           // ns + 1 unknowns
  int k0;          // pivots k0 .. N-1 form a full trailing block
  int posT, posV;  // elements of T and V
  const int *var;  // [N] element -> variable: 0 T, 1 V, 2 + k the moles of species k
  const int *posn; // [ns - 1] species k -> element
  const int *lp, *li;  // L by columns: rows li[lp[k] .. lp[k+1]) below pivot k
  const int *up, *uj;  // U by rows: columns uj[up[k] .. up[k+1]) right of pivot k
  const int *cp, *ci;  // U by columns: rows ci[cp[k] .. cp[k+1]) above pivot k
  const double *aw;    // [N] factor on atol per element: 1 for T and V, 1 / W_k for n_k
};

// ---------------------------------------------------------------------------
// Source terms (and the analytical Jacobian, in element order) of the
// concentration-based form.  Rates as warp_chem; returns 0 or 4 (non-finite).
// ---------------------------------------------------------------------------
template <int L, typename LT>
__device__ __noinline__ int conc_chem(const MechView &m, const ConcView &cv, const WarpBuf<LT> &b,
                                      double P, const WVecT<Grp<L>::WR> &y,
                                      WVecT<Grp<L>::WR> &f, bool wantJ) {
  using G = Grp<L>;
  constexpr int WR = G::WR;
  const int lane = G::lane();
  const int ns = m.ns, in = ns - 1, N = cv.N, ld = b.ld;
  const double T = elem<L>(y, cv.posT), V = elem<L>(y, cv.posV);
  const double iV = 1.0 / V, invT = 1.0 / T, logT = log(T);
  const double Ctot = P / (RU * T);
  double sC = 0.0;
#pragma unroll
  for (int r = 0; r < WR; ++r) {
    const int g = lane + L * r;
    if (g < N) {
      const int v = cv.var[g];
      if (v >= 2) {
        const double c = y.v[r] * iV;
        b.C[v - 2] = c;
        sC += c;
      }
    }
  }
  sC = G::sum(sC);  // sum of the active species' concentrations
  if (lane == 0) b.C[in] = Ctot - sC;
  G::sync();
  double cpl = 0.0, dcpl = 0.0;
#pragma unroll
  for (int r = 0; r < WR; ++r) {
    const int k = lane + L * r;
    if (k < ns) {
      const int rg = range_of(m, k, T);
      const double *cc = m.cp + (2 * k + rg) * NCP;
      const double cp = poly_cp(cc, T);
      b.g[k] = poly_g(m.gb + (2 * k + rg) * NG, T, logT, invT);
      b.hs[k] = poly_h(m.h + (2 * k + rg) * NH, T, invT);
      b.cpk[k] = cp;
      cpl += b.C[k] * cp;
      if (wantJ) {
        dcpl += b.C[k] * poly_dcp(cc, T);
        b.B[k] = 0.0;
        b.Tc[k] = 0.0;
      }
    }
  }
  const double Cs = G::sum(cpl);  // sum_k C_k cp_k / R
  const double dCsT = wantJ ? G::sum(dcpl) : 0.0;
  if (wantJ)
    for (int e = lane; e < N * ld; e += L) b.Jd[e] = 0.0;
  G::sync();
  const double lnPf = 2.5003366899611787 - logT;  // ln(Patm / Ru) - ln T
  if (!wantJ) {  // Troe, third-body and elementary reactions in rounds of their own
    for (int i0 = 0; i0 < m.ntroe; i0 += L)
      if (i0 + lane < m.ntroe)
        b.q[i0 + lane] = falloff_rate(m, b.C, b.g, i0 + lane, T, logT, invT, lnPf, Ctot);
    for (int i0 = m.ntroe; i0 < m.nfall; i0 += L)
      if (i0 + lane < m.nfall)
        b.q[i0 + lane] = falloff_rate(m, b.C, b.g, i0 + lane, T, logT, invT, lnPf, Ctot);
    for (int i0 = m.nfall; i0 < m.nr; i0 += L)
      if (i0 + lane < m.nr) b.q[i0 + lane] = elem_rate(m, b.C, b.g, i0 + lane, logT, invT, lnPf);
  } else {
    for (int i0 = 0; i0 < m.nr; i0 += L) {
      const int i = i0 + lane;
      if (i >= m.nr) continue;
      const int meta = m.meta[i];
      const int *sl = m.slot + 6 * i;
      const int nre = meta_nreac(meta), npr = meta_nprod(meta), type = meta_type(meta);
      const double lnkf = m.lnA[i] + m.b[i] * logT - m.Th[i] * invT;
      const double kf = kexp(lnkf, m.etab);
      double lnKc = m.dnu[i] * lnPf, dH = 0.0, fwd = 1.0, rev = 1.0;
      for (int s = 0; s < nre; ++s) {
        lnKc -= b.g[sl[s]];
        dH -= b.hs[sl[s]];
        fwd *= b.C[sl[s]];
      }
      for (int s = 0; s < npr; ++s) {
        lnKc += b.g[sl[3 + s]];
        dH += b.hs[sl[3 + s]];
        rev *= b.C[sl[3 + s]];
      }
      const double kr = kf * kexp(-lnKc, m.etab);
      double phi = 1.0, dphi_dT = 0.0, dphi_dM = 0.0, M = Ctot;
      const int e0 = m.eff0[i], ne = meta_neff(meta);
      const double dlnkf = m.b[i] * invT + m.Th[i] * invT * invT;
      if (type != 0) {
        for (int e = 0; e < ne; ++e) M += m.eff[e0 + e] * b.C[m.effsp[e0 + e]];
        if (type == 1) {
          phi = M;
          dphi_dM = 1.0;
        } else {
          const TroeOut t = troe_factor<true>(m.troe + NTROE * meta_troe(meta), T, logT, invT,
                                              lnkf, dlnkf, M, m.etab);
          phi = t.P;
          dphi_dT = t.P * t.dlnP_dT;
          dphi_dM = t.P * t.dlnP_dM;
        }
      }
      const double Rn = kf * fwd - kr * rev;
      b.q[i] = phi * Rn;
      // partials of q: d/dn_l = (mass action + u eff'_l) / V; d/dV = -sig / V
      // (sig = sum_l C_l dq/dC_l + u (M - Ctot)); d/dT at fixed n, V, where
      // only Ctot (and with it M and the bath gas) moves
      const double dlnkr = dlnkf - (dH - m.dnu[i]) * invT;
      const double u = Rn * dphi_dM;
      const double sig = phi * (nre * kf * fwd - npr * kr * rev) + u * (M - Ctot);
      const double dqdT = phi * (kf * dlnkf * fwd - kr * dlnkr * rev) + Rn * dphi_dT -
                          u * Ctot * invT;
      const double pkf = phi * kf, pkr = -phi * kr;
      for (int rs = 0; rs < nre + npr; ++rs) {
        const int row = (rs < nre) ? sl[rs] : sl[3 + rs - nre];
        const double nu = (rs < nre) ? -1.0 : 1.0;
        atomicAdd(&b.B[row], nu * sig);
        atomicAdd(&b.Tc[row], nu * dqdT);
        double *Jr = b.Jd + cv.posn[row] * ld;
        for (int cs = 0; cs < nre + npr; ++cs) {
          const int col = (cs < nre) ? sl[cs] : sl[3 + cs - nre];
          double p = (cs < nre) ? pkf : pkr;
          if (cs < nre) {
            for (int t = 0; t < nre; ++t)
              if (t != cs) p *= b.C[sl[t]];
          } else {
            for (int t = 0; t < npr; ++t)
              if (t != cs - nre) p *= b.C[sl[3 + t]];
          }
          atomicAdd(&Jr[cv.posn[col]], nu * p);
        }
        for (int e = 0; e < ne; ++e)
          atomicAdd(&Jr[cv.posn[m.effsp[e0 + e]]], nu * u * m.eff[e0 + e]);
      }
    }
  }
  G::sync();
  // production rates gathered per species (deterministic), mixture sums
  double hw = 0.0, ww = 0.0;
#pragma unroll
  for (int r = 0; r < WR; ++r) {
    const int k = lane + L * r;
    if (k < in) {
      double w = 0.0;
      for (int e = m.csr0[k]; e < m.csr0[k + 1]; ++e) w += m.csrnu[e] * b.q[m.csr[e] >> 4];
      b.wd[k] = w;
      hw += b.hs[k] * w;
      ww += w;
    }
  }
  const double Hs = G::sum(hw), Ws = G::sum(ww);
  const double fT = -T * Hs / Cs;
  const double fV = V * (Ws / Ctot + fT * invT);
  G::sync();
  bool ok = isfinite(fT) && isfinite(fV);
#pragma unroll
  for (int r = 0; r < WR; ++r) {
    const int g = lane + L * r;
    if (g < N) {
      const int v = cv.var[g];
      const double val = (v == 0) ? fT : (v == 1) ? fV : V * b.wd[v - 2];
      f.v[r] = val;
      ok &= isfinite(val);
    }
  }
  if (!wantJ) return G::all(ok) ? 0 : 4;
  // species rows: the T and V columns; sums the T and V rows need
  double sHB = 0.0, sHT = 0.0, sCW = 0.0, sB = 0.0, sTc = 0.0, sCC = 0.0;
#pragma unroll
  for (int r = 0; r < WR; ++r) {
    const int k = lane + L * r;
    if (k < in) {
      double *Jr = b.Jd + cv.posn[k] * ld;
      Jr[cv.posT] = V * b.Tc[k];
      Jr[cv.posV] = b.wd[k] - b.B[k];
      sHB += b.hs[k] * b.B[k];
      sHT += b.hs[k] * b.Tc[k];
      sCW += b.cpk[k] * b.wd[k];
      sB += b.B[k];
      sTc += b.Tc[k];
      sCC += b.cpk[k] * b.C[k];
    }
  }
  sHB = G::sum(sHB);
  sHT = G::sum(sHT);
  sCW = G::sum(sCW);
  sB = G::sum(sB);
  sTc = G::sum(sTc);
  sCC = G::sum(sCC);
  G::sync();
  // T row: f_T = -(T Hs) / Cs, so dT-row = -(d(T Hs) + fT dCs) / Cs; the V
  // row from it: f_V = V (Ws / Ctot + f_T / T)
  const double cpin = b.cpk[in];
  double rowT[WR], rowV[WR];
#pragma unroll
  for (int r = 0; r < WR; ++r) {
    const int c = lane + L * r;
    rowT[r] = rowV[r] = 0.0;
    if (c < N) {
      const int v = cv.var[c];
      double dTH, dCs, dWs;  // d(T Hs), dCs, d(sum wdot) * V along phi_c
      if (v >= 2) {
        double sh = 0.0, sw = 0.0;
        for (int k = 0; k < in; ++k) {
          const double jk = b.Jd[cv.posn[k] * ld + c];
          sh += b.hs[k] * jk;
          sw += jk;
        }
        dTH = T * iV * sh;
        dCs = (b.cpk[v - 2] - cpin) * iV;
        dWs = sw;
      } else if (v == 1) {
        dTH = -T * iV * sHB;
        dCs = (cpin * sC - sCC) * iV;
        dWs = -sB;
      } else {
        dTH = sCW + T * sHT;
        dCs = dCsT - cpin * Ctot * invT;
        dWs = V * sTc;
      }
      const double jt = -(dTH + fT * dCs) / Cs;
      double jv = dWs / Ctot + V * jt * invT;
      if (v == 1) jv += Ws / Ctot + fT * invT;
      if (v == 0) jv += V * (Ws / (Ctot * T) - fT * invT * invT);
      rowT[r] = jt;
      rowV[r] = jv;
    }
  }
  G::sync();
#pragma unroll
  for (int r = 0; r < WR; ++r) {
    const int c = lane + L * r;
    if (c < N) {
      b.Jd[cv.posT * ld + c] = rowT[r];
      b.Jd[cv.posV * ld + c] = rowV[r];
    }
  }
  G::sync();
  bool okJ = true;
  for (int e = lane; e < N * N; e += L) {
    const int q = (e / N) * ld + e % N;
    const double v = b.Jd[q];
    okJ &= isfinite(v);
    b.J[q] = LT(v);  // one rounding per entry (none in FP64)
  }
  G::sync();
  return G::all(ok && okJ) ? 0 : 4;
}

// ---------------------------------------------------------------------------
// Sparse LU without pivoting over the symbolic pattern, and the solves.
// A pivot that is zero (or not finite) reports the matrix singular, as the
// dense factorisation does when no pivot is left.
// ---------------------------------------------------------------------------
template <int L, typename LT>
__device__ __noinline__ int sparse_lu_real(const ConcView &cv, int ld, LT *a) {
  using G = Grp<L>;
  const int N = cv.N, lane = G::lane();
  for (int k = 0; k < N; ++k) {
    const LT piv = a[k * ld + k];
    if (!(fabs(piv) > LT(0))) return k + 1;
    const LT inv = LT(1) / piv;
    if (k < cv.k0) {  // sparse head: the pattern's rows and columns
      const int l0 = cv.lp[k], l1 = cv.lp[k + 1];
      for (int e = l0 + lane; e < l1; e += L) a[cv.li[e] * ld + k] *= inv;
      G::sync();
      for (int e = cv.up[k] + lane; e < cv.up[k + 1]; e += L) {
        const int j = cv.uj[e];
        const LT u = a[k * ld + j];
        if (u != LT(0))
          for (int q = l0; q < l1; ++q) {
            const int i = cv.li[q];
            a[i * ld + j] -= a[i * ld + k] * u;
          }
      }
    } else {  // full trailing block: the dense update, lanes over columns
      for (int i = k + 1 + lane; i < N; i += L) a[i * ld + k] *= inv;
      G::sync();
      for (int j = k + 1 + lane; j < N; j += L) {
        const LT u = a[k * ld + j];
        if (u != LT(0))
          for (int i = k + 1; i < N; ++i) a[i * ld + j] -= a[i * ld + k] * u;
      }
    }
    G::sync();
  }
  return 0;
}

template <int L, typename LT>
__device__ __noinline__ int sparse_lu_cplx(const ConcView &cv, int ld, LT *ar, LT *ai) {
  using G = Grp<L>;
  const int N = cv.N, lane = G::lane();
  for (int k = 0; k < N; ++k) {
    const LT pr = ar[k * ld + k], pi = ai[k * ld + k];
    if (!(fabs(pr) + fabs(pi) > LT(0))) return k + 1;
    const bool head = k < cv.k0;
    const int l0 = cv.lp[k], l1 = cv.lp[k + 1];
    const int ib = head ? l0 : k + 1, ie = head ? l1 : N;  // multiplier rows
    for (int e = ib + lane; e < ie; e += L) {
      const int i = head ? cv.li[e] : e;
      LT lr, li;
      cdiv(ar[i * ld + k], ai[i * ld + k], pr, pi, lr, li);
      ar[i * ld + k] = lr;
      ai[i * ld + k] = li;
    }
    G::sync();
    const int jb = head ? cv.up[k] : k + 1, je = head ? cv.up[k + 1] : N;
    for (int e = jb + lane; e < je; e += L) {
      const int j = head ? cv.uj[e] : e;
      const LT ur = ar[k * ld + j], ui = ai[k * ld + j];
      if (ur != LT(0) || ui != LT(0)) {
        if (head) {
          for (int q = l0; q < l1; ++q) {
            const int i = cv.li[q];
            const LT lr = ar[i * ld + k], li = ai[i * ld + k];
            ar[i * ld + j] -= lr * ur - li * ui;
            ai[i * ld + j] -= lr * ui + li * ur;
          }
        } else {
          for (int i = k + 1; i < N; ++i) {
            const LT lr = ar[i * ld + k], li = ai[i * ld + k];
            ar[i * ld + j] -= lr * ur - li * ui;
            ai[i * ld + j] -= lr * ui + li * ur;
          }
        }
      }
    }
    G::sync();
  }
  return 0;
}

// Solve LU x = rhs over the pattern: rhs/result in x (registers, FP64), the
// substitution in LT through the group's vector v.
template <int L, typename LT>
__device__ __noinline__ void sparse_solve_real(const ConcView &cv, int ld, const LT *lu, LT *v,
                                               WVecT<Grp<L>::WR> &x) {
  using G = Grp<L>;
  constexpr int WR = G::WR;
  const int N = cv.N, lane = G::lane();
#pragma unroll
  for (int r = 0; r < WR; ++r) {
    const int g = lane + L * r;
    if (g < N) v[g] = LT(x.v[r]);
  }
  G::sync();
  for (int j = 0; j < N; ++j) {  // forward, unit lower triangle
    const LT xj = v[j];
    if (j < cv.k0) {
      for (int e = cv.lp[j] + lane; e < cv.lp[j + 1]; e += L) {
        const int i = cv.li[e];
        v[i] -= lu[i * ld + j] * xj;
      }
    } else {
#pragma unroll
      for (int r = 0; r < WR; ++r) {
        const int i = lane + L * r;
        if (i > j && i < N) v[i] -= lu[i * ld + j] * xj;
      }
    }
    G::sync();
  }
  for (int i = N - 1; i >= 0; --i) {  // backward (entries outside the pattern are zero)
    const LT xi = v[i] / lu[i * ld + i];
    G::sync();
    if (lane == (i & (L - 1))) v[i] = xi;
#pragma unroll
    for (int r = 0; r < WR; ++r) {
      const int i2 = lane + L * r;
      if (i2 < i) v[i2] -= lu[i2 * ld + i] * xi;
    }
    G::sync();
  }
#pragma unroll
  for (int r = 0; r < WR; ++r) {
    const int g = lane + L * r;
    if (g < N) x.v[r] = double(v[g]);
  }
  G::sync();
}

template <int L, typename LT>
__device__ __noinline__ void sparse_solve_cplx(const ConcView &cv, int ld, const LT *lr,
                                               const LT *li, LT *vr, LT *vi,
                                               WVecT<Grp<L>::WR> &xr, WVecT<Grp<L>::WR> &xi) {
  using G = Grp<L>;
  constexpr int WR = G::WR;
  const int N = cv.N, lane = G::lane();
#pragma unroll
  for (int r = 0; r < WR; ++r) {
    const int g = lane + L * r;
    if (g < N) {
      vr[g] = LT(xr.v[r]);
      vi[g] = LT(xi.v[r]);
    }
  }
  G::sync();
  for (int j = 0; j < N; ++j) {
    const LT xr_ = vr[j], xi_ = vi[j];
    if (j < cv.k0) {
      for (int e = cv.lp[j] + lane; e < cv.lp[j + 1]; e += L) {
        const int i = cv.li[e];
        const LT a = lr[i * ld + j], c = li[i * ld + j];
        vr[i] -= a * xr_ - c * xi_;
        vi[i] -= a * xi_ + c * xr_;
      }
    } else {
#pragma unroll
      for (int r = 0; r < WR; ++r) {
        const int i = lane + L * r;
        if (i > j && i < N) {
          const LT a = lr[i * ld + j], c = li[i * ld + j];
          vr[i] -= a * xr_ - c * xi_;
          vi[i] -= a * xi_ + c * xr_;
        }
      }
    }
    G::sync();
  }
  for (int i = N - 1; i >= 0; --i) {
    LT qr, qi;
    cdiv(vr[i], vi[i], lr[i * ld + i], li[i * ld + i], qr, qi);
    G::sync();
    if (lane == (i & (L - 1))) {
      vr[i] = qr;
      vi[i] = qi;
    }
#pragma unroll
    for (int r = 0; r < WR; ++r) {
      const int i2 = lane + L * r;
      if (i2 < i) {
        const LT a = lr[i2 * ld + i], c = li[i2 * ld + i];
        vr[i2] -= a * qr - c * qi;
        vi[i2] -= a * qi + c * qr;
      }
    }
    G::sync();
  }
#pragma unroll
  for (int r = 0; r < WR; ++r) {
    const int g = lane + L * r;
    if (g < N) {
      xr.v[r] = double(vr[g]);
      xi.v[r] = double(vi[g]);
    }
  }
  G::sync();
}

// E1 = gamma/h - J and E2 = (alpha + i beta)/h - J from the stored J, then
// their sparse factorisations
template <int L, typename LT>
__device__ int conc_factor(const ConcView &cv, const WarpBuf<LT> &b, double h) {
  const double fac1 = RC.gam / h, alphn = RC.alp / h, betan = RC.bet / h;
  const int lane = Grp<L>::lane(), ld = b.ld, N = cv.N;
  for (int e = lane; e < N * N; e += L) {
    const int i = e / N, j = e % N;
    const LT Jv = b.J[i * ld + j];
    b.E1[i * ld + j] = (i == j) ? LT(fac1) - Jv : -Jv;
    b.E2r[i * ld + j] = (i == j) ? LT(alphn) - Jv : -Jv;
    b.E2i[i * ld + j] = (i == j) ? LT(betan) : LT(0);
  }
  Grp<L>::sync();
  const int s1 = sparse_lu_real<L, LT>(cv, ld, b.E1);
  if (s1) return s1;
  return sparse_lu_cplx<L, LT>(cv, ld, b.E2r, b.E2i);
}

template <int L, typename LT>
struct ConcSys {
  using WV = WVecT<Grp<L>::WR>;
  const MechView *m;
  const ConcView *cv;
  __device__ __forceinline__ int n() const { return cv->N; }
  __device__ __forceinline__ double atol_w(int g) const { return g < cv->N ? cv->aw[g] : 1.0; }
  __device__ __forceinline__ int chem(const WarpBuf<LT> &b, double P, const WV &y, WV &f,
                                      bool wantJ) const {
    return conc_chem<L, LT>(*m, *cv, b, P, y, f, wantJ);
  }
  __device__ __forceinline__ int factor(const WarpBuf<LT> &b, double h) const {
    return conc_factor<L, LT>(*cv, b, h);
  }
  __device__ __forceinline__ void solve_real(const WarpBuf<LT> &b, WV &x) const {
    sparse_solve_real<L, LT>(*cv, b.ld, b.E1, b.v1, x);
  }
  __device__ __forceinline__ void solve_cplx(const WarpBuf<LT> &b, WV &xr, WV &xi) const {
    sparse_solve_cplx<L, LT>(*cv, b.ld, b.E2r, b.E2i, b.v1, b.v2, xr, xi);
  }
};

}  // namespace kin
