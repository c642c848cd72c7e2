/*
 * Oracle chemistry: thermodynamics, source terms and Jacobians of the
 * constant-pressure reactor.  TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * The paper takes its source terms and its analytical constant-pressure,
 * mass-fraction-based Jacobian from pyJac (Sec. 2.1) and does not print the
 * equations; what follows is the textbook formulation written out directly:
 *
 *   NASA-7:  cp/R = a1 + a2 T + a3 T^2 + a4 T^3 + a5 T^4
 *            h/RT = a1 + a2 T/2 + a3 T^2/3 + a4 T^3/4 + a5 T^4/5 + a6/T
 *            s/R  = a1 ln T + a2 T + a3 T^2/2 + a4 T^3/3 + a5 T^4/4 + a7
 *   mixture: 1/Wbar = sum Y_k/W_k,  rho = P Wbar / (Ru T),  C_k = rho Y_k / W_k
 *   rates:   k = A T^b exp(-Theta/T);  Kc = Kp (Patm/(Ru T))^(sum nu);
 *            ln Kp = sum_k nu_k (s_k/R - h_k/RT);  kr = kf / Kc;
 *            q = Phi (kf prod C^nu' - kr prod C^nu'') with Phi = 1,
 *            [M] = sum eff_k C_k (third body) or the Troe falloff factor
 *            Pr/(1+Pr) F (Pr = k0 [M]/k_inf, Troe/Gilbert F).
 *   ODE:     dY_k/dt = W_k wdot_k / rho,   dT/dt = -sum_k H_k wdot_k / (rho cp)
 *            with H_k = (h_k/RT) Ru T the molar enthalpy, cp = sum Y_k cp_k/W_k.
 *
 * The analytical Jacobian is assembled by the chain rule through the
 * concentrations: dq/dC (dense, nr x ns) times dC/dy (ns x N), plus the
 * explicit temperature dependences of k_f, K_c, the falloff factor, rho,
 * the enthalpies and cp.  It is deliberately the slow dense product so that
 * each factor can be checked by eye.
 */
#include <float.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include "oracle.h"

static const double *nasa_set(const orc_mech *m, int k, double T) {
  const double *p = m->nasa + 17 * (size_t)k;
  return (T < p[1]) ? p + 3 : p + 10;
}

/* NASA-7 cp/R, h/RT, s/R per species (Sec. 2.1: thermo behind the reverse rates). */
void orc_thermo(const orc_mech *m, double T, double *cp_R, double *h_RT, double *s_R) {
  for (int k = 0; k < m->ns; ++k) {
    const double *a = nasa_set(m, k, T);
    double T2 = T * T, T3 = T2 * T, T4 = T3 * T;
    cp_R[k] = a[0] + a[1] * T + a[2] * T2 + a[3] * T3 + a[4] * T4;
    h_RT[k] = a[0] + a[1] * T / 2.0 + a[2] * T2 / 3.0 + a[3] * T3 / 4.0 + a[4] * T4 / 5.0 + a[5] / T;
    s_R[k] = a[0] * log(T) + a[1] * T + a[2] * T2 / 2.0 + a[3] * T3 / 3.0 + a[4] * T4 / 4.0 + a[6];
  }
}

/* d(cp/R)/dT per species */
static void thermo_dcp(const orc_mech *m, double T, double *dcp_R) {
  for (int k = 0; k < m->ns; ++k) {
    const double *a = nasa_set(m, k, T);
    dcp_R[k] = a[1] + 2.0 * a[2] * T + 3.0 * a[3] * T * T + 4.0 * a[4] * T * T * T;
  }
}

static double arrhenius(const double *p, double T) {
  return p[0] * pow(T, p[1]) * exp(-p[2] / T);
}

static double dln_arrhenius_dT(const double *p, double T) {
  return p[1] / T + p[2] / (T * T);
}

/* net stoichiometric coefficient of species k in reaction i */
static int nu_of(const orc_mech *m, int i, int k) {
  int nu = 0;
  for (int s = 0; s < 3; ++s) {
    if (m->prod[3 * i + s] == k) nu += 1;
    if (m->reac[3 * i + s] == k) nu -= 1;
  }
  return nu;
}

static int slots_used(const int32_t *sl) {
  int c = 0;
  for (int s = 0; s < 3; ++s) c += (sl[s] >= 0);
  return c;
}

/* product over the filled slots of C (mass-action term) */
static double mass_action(const int32_t *sl, const double *C) {
  double p = 1.0;
  for (int s = 0; s < 3; ++s)
    if (sl[s] >= 0) p *= C[sl[s]];
  return p;
}

/* d(mass_action)/dC_k = sum over the slots holding k of the product of the other slots */
static double mass_action_dC(const int32_t *sl, const double *C, int k) {
  double d = 0.0;
  for (int s = 0; s < 3; ++s) {
    if (sl[s] != k) continue;
    double p = 1.0;
    for (int t = 0; t < 3; ++t)
      if (t != s && sl[t] >= 0) p *= C[sl[t]];
    d += p;
  }
  return d;
}

/* Troe falloff factor Pfac = Pr/(1+Pr) F and its logarithmic derivatives.
 * Textbook Troe/Gilbert form with log = log10:
 *   Fcent = (1-a) exp(-T/T3) + a exp(-T/T1) + exp(-T2/T)   (T3, T1, T2 = T***, T*, T**)
 *   c = -0.4 - 0.67 log Fcent,  n = 0.75 - 1.27 log Fcent,  d = 0.14
 *   log F = log Fcent / (1 + ((log Pr + c)/(n - d (log Pr + c)))^2)        */
typedef struct {
  double Pfac, dlnP_dT, dlnP_dM;
} troe_out;

static troe_out troe(const double *fall, const double *arrh_inf, double T, double M) {
  troe_out o;
  const double ln10 = log(10.0);
  double k0 = arrhenius(fall, T), kinf = arrhenius(arrh_inf, T);
  double a = fall[3], T3 = fall[4], T1 = fall[5], T2 = fall[6];
  double e3 = exp(-T / T3), e1 = exp(-T / T1), e2 = exp(-T2 / T);
  double Fc = (1.0 - a) * e3 + a * e1 + e2;
  double dFc_dT = -(1.0 - a) / T3 * e3 - a / T1 * e1 + T2 / (T * T) * e2;
  double lFc = log10(Fc);
  double Pr = k0 * M / kinf;
  double L = log10(Pr);
  double c = -0.4 - 0.67 * lFc, nn = 0.75 - 1.27 * lFc, d = 0.14;
  double u = L + c, v = nn - d * u, X = u / v;
  double den = 1.0 + X * X;
  double lF = lFc / den;
  o.Pfac = Pr / (1.0 + Pr) * pow(10.0, lF);
  double dX_dL = nn / (v * v);
  double du = -0.67, dv = -1.27 - d * du;
  double dX_dlFc = (du * v - u * dv) / (v * v);
  double dlF_dL = -lFc * 2.0 * X * dX_dL / (den * den);
  double dlF_dlFc = 1.0 / den - lFc * 2.0 * X * dX_dlFc / (den * den);
  double dlFc_dT = dFc_dT / (Fc * ln10);
  double dL_dT = (dln_arrhenius_dT(fall, T) - dln_arrhenius_dT(arrh_inf, T)) / ln10;
  double dL_dM = 1.0 / (M * ln10);
  double dlnP_dL = ln10 / (1.0 + Pr) + ln10 * dlF_dL;
  o.dlnP_dT = dlnP_dL * dL_dT + ln10 * dlF_dlFc * dlFc_dT;
  o.dlnP_dM = dlnP_dL * dL_dM;
  return o;
}

static double third_body(const orc_mech *m, int i, const double *C) {
  double M = 0.0;
  for (int k = 0; k < m->ns; ++k) M += m->eff[(size_t)i * m->ns + k] * C[k];
  return M;
}

/* Per-reaction quantities at (T, C): everything the source term and the
 * Jacobian need. */
typedef struct {
  double kf, kr, phi, fwd, rev;
  double dlnkf_dT, dlnkr_dT, dphi_dT, dphi_dM;
} rxn_terms;

static rxn_terms reaction(const orc_mech *m, int i, double T, const double *C,
                          const double *h_RT, const double *s_R) {
  rxn_terms r;
  const int32_t *re = m->reac + 3 * i, *pr = m->prod + 3 * i;
  const double *ar = m->arrh + 3 * i;
  r.kf = arrhenius(ar, T);
  r.dlnkf_dT = dln_arrhenius_dT(ar, T);
  /* equilibrium constant from the thermo (reverse rate) */
  double dg = 0.0, dh = 0.0;
  int dnu = slots_used(pr) - slots_used(re);
  for (int k = 0; k < m->ns; ++k) {
    int nu = nu_of(m, i, k);
    if (nu == 0) continue;
    dg += nu * (s_R[k] - h_RT[k]);
    dh += nu * h_RT[k];
  }
  double lnKc = dg + dnu * log(ORC_PATM / (ORC_RU * T));
  r.kr = r.kf / exp(lnKc);
  /* d ln Kc/dT = sum nu (h/RT)/T - (sum nu)/T   (van 't Hoff) */
  r.dlnkr_dT = r.dlnkf_dT - (dh / T - dnu / T);
  r.fwd = mass_action(re, C);
  r.rev = mass_action(pr, C);
  r.phi = 1.0;
  r.dphi_dT = 0.0;
  r.dphi_dM = 0.0;
  if (m->rtype[i] == 1) {
    r.phi = third_body(m, i, C);
    r.dphi_dM = 1.0;
  } else if (m->rtype[i] == 2) {
    double M = third_body(m, i, C);
    troe_out t = troe(m->fall + 7 * i, ar, T, M);
    r.phi = t.Pfac;
    r.dphi_dT = t.Pfac * t.dlnP_dT;
    r.dphi_dM = t.Pfac * t.dlnP_dM;
  }
  return r;
}

/* effective forward / reverse rate constants (phi included) at (T, C) */
void orc_rate_constants(const orc_mech *m, double T, const double *C, double *kf_eff,
                        double *kr_eff) {
  int ns = m->ns;
  double *cp = malloc(sizeof(double) * 3 * ns), *h = cp + ns, *s = h + ns;
  orc_thermo(m, T, cp, h, s);
  for (int i = 0; i < m->nr; ++i) {
    rxn_terms r = reaction(m, i, T, C, h, s);
    kf_eff[i] = r.phi * r.kf;
    kr_eff[i] = r.phi * r.kr;
  }
  free(cp);
}

/* molar production rates wdot [ns] (kmol/m^3/s) from T, P and full Y */
void orc_wdot(const orc_mech *m, double T, double P, const double *Yfull, double *wdot) {
  int ns = m->ns;
  double *C = malloc(sizeof(double) * 4 * ns), *cp = C + ns, *h = cp + ns, *s = h + ns;
  double S = 0.0;
  for (int k = 0; k < ns; ++k) S += Yfull[k] / m->W[k];
  double rho = P / (ORC_RU * T * S);
  for (int k = 0; k < ns; ++k) C[k] = rho * Yfull[k] / m->W[k];
  orc_thermo(m, T, cp, h, s);
  for (int k = 0; k < ns; ++k) wdot[k] = 0.0;
  for (int i = 0; i < m->nr; ++i) {
    rxn_terms r = reaction(m, i, T, C, h, s);
    double q = r.phi * (r.kf * r.fwd - r.kr * r.rev);
    for (int k = 0; k < ns; ++k) wdot[k] += nu_of(m, i, k) * q;
  }
  free(C);
}

/* Unpack y = [T, Y_0..Y_{ns-2}] into the full mass-fraction vector. */
static void full_Y(const orc_mech *m, const double *y, double *Y) {
  double sum = 0.0;
  for (int k = 0; k < m->ns - 1; ++k) {
    Y[k] = y[1 + k];
    sum += Y[k];
  }
  Y[m->ns - 1] = 1.0 - sum;
}

/* Right-hand side f(y) of the constant-pressure reactor (Sec. 2.1). */
int orc_rhs(const orc_mech *m, double P, const double *y, double *f) {
  int ns = m->ns;
  double T = y[0];
  double *Y = malloc(sizeof(double) * 5 * ns), *wdot = Y + ns, *cp = wdot + ns, *h = cp + ns,
         *s = h + ns;
  full_Y(m, y, Y);
  orc_wdot(m, T, P, Y, wdot);
  orc_thermo(m, T, cp, h, s);
  double S = 0.0, cpm = 0.0, Hw = 0.0;
  for (int k = 0; k < ns; ++k) {
    S += Y[k] / m->W[k];
    cpm += Y[k] * cp[k] * ORC_RU / m->W[k];
    Hw += h[k] * ORC_RU * T * wdot[k];
  }
  double rho = P / (ORC_RU * T * S);
  f[0] = -Hw / (rho * cpm);
  for (int k = 0; k < ns - 1; ++k) f[1 + k] = m->W[k] * wdot[k] / rho;
  int ok = 1;
  for (int k = 0; k < ns; ++k) ok &= isfinite(f[k]);
  free(Y);
  return ok ? 0 : ORC_NONFINITE;
}

/* Analytical Jacobian J[i*N + j] = d f_i / d y_j (row-major), the
 * constant-pressure mass-fraction form (Sec. 2.1, Sec. 3.4). */
int orc_jac(const orc_mech *m, double P, const double *y, double *J) {
  int ns = m->ns, nr = m->nr, N = ns, in = ns - 1;
  double T = y[0];
  double *Y = calloc((size_t)ns * 8, sizeof(double));
  double *C = Y + ns, *cp = C + ns, *h = cp + ns, *s = h + ns, *dcp = s + ns, *wdot = dcp + ns,
         *mj = wdot + ns;
  double *dqdC = calloc((size_t)nr * ns, sizeof(double));  /* d q_i / d C_k at fixed T */
  double *dqdT = calloc((size_t)nr, sizeof(double));       /* d q_i / d T at fixed C */
  double *dCdy = calloc((size_t)ns * N, sizeof(double));    /* d C_k / d y_j */
  double *dqdy = calloc((size_t)nr * N, sizeof(double));
  double *dwdy = calloc((size_t)ns * N, sizeof(double));
  full_Y(m, y, Y);
  double S = 0.0;
  for (int k = 0; k < ns; ++k) S += Y[k] / m->W[k];
  double rho = P / (ORC_RU * T * S);
  for (int k = 0; k < ns; ++k) C[k] = rho * Y[k] / m->W[k];
  orc_thermo(m, T, cp, h, s);
  thermo_dcp(m, T, dcp);
  for (int k = 0; k < ns; ++k) wdot[k] = 0.0;

  for (int i = 0; i < nr; ++i) {
    rxn_terms r = reaction(m, i, T, C, h, s);
    const int32_t *re = m->reac + 3 * i, *pr = m->prod + 3 * i;
    double Rnet = r.kf * r.fwd - r.kr * r.rev;
    double q = r.phi * Rnet;
    for (int k = 0; k < ns; ++k) wdot[k] += nu_of(m, i, k) * q;
    for (int k = 0; k < ns; ++k) {
      double d = r.phi * (r.kf * mass_action_dC(re, C, k) - r.kr * mass_action_dC(pr, C, k));
      if (m->rtype[i] != 0) d += Rnet * r.dphi_dM * m->eff[(size_t)i * ns + k];
      dqdC[(size_t)i * ns + k] = d;
    }
    dqdT[i] = r.phi * (r.kf * r.dlnkf_dT * r.fwd - r.kr * r.dlnkr_dT * r.rev) + Rnet * r.dphi_dT;
  }
  /* dC/dy: column 0 is T, column 1+j is Y_j (j < ns-1, the inert absorbs -1) */
  for (int j = 0; j < ns - 1; ++j) mj[j] = 1.0 / m->W[j] - 1.0 / m->W[in];
  for (int k = 0; k < ns; ++k) {
    dCdy[(size_t)k * N + 0] = -C[k] / T;
    for (int j = 0; j < ns - 1; ++j) {
      double d = -C[k] * mj[j] / S;
      if (k == j) d += rho / m->W[k];
      if (k == in) d -= rho / m->W[k];
      dCdy[(size_t)k * N + 1 + j] = d;
    }
  }
  for (int i = 0; i < nr; ++i)
    for (int j = 0; j < N; ++j) {
      double d = (j == 0) ? dqdT[i] : 0.0;
      for (int k = 0; k < ns; ++k) d += dqdC[(size_t)i * ns + k] * dCdy[(size_t)k * N + j];
      dqdy[(size_t)i * N + j] = d;
    }
  for (int k = 0; k < ns; ++k)
    for (int j = 0; j < N; ++j) {
      double d = 0.0;
      for (int i = 0; i < nr; ++i) d += nu_of(m, i, k) * dqdy[(size_t)i * N + j];
      dwdy[(size_t)k * N + j] = d;
    }
  /* mixture quantities and their derivatives */
  double cpm = 0.0, dcpm_dT = 0.0, Hw = 0.0, dHw_dT = 0.0;
  for (int k = 0; k < ns; ++k) {
    cpm += Y[k] * cp[k] * ORC_RU / m->W[k];
    dcpm_dT += Y[k] * dcp[k] * ORC_RU / m->W[k];
    Hw += h[k] * ORC_RU * T * wdot[k];
    dHw_dT += cp[k] * ORC_RU * wdot[k];
  }
  double rcp = rho * cpm;
  for (int j = 0; j < N; ++j) {
    double drho, dcpm, dHw = (j == 0) ? dHw_dT : 0.0;
    if (j == 0) {
      drho = -rho / T;
      dcpm = dcpm_dT;
    } else {
      drho = -rho * mj[j - 1] / S;
      dcpm = cp[j - 1] * ORC_RU / m->W[j - 1] - cp[in] * ORC_RU / m->W[in];
    }
    for (int k = 0; k < ns; ++k) dHw += h[k] * ORC_RU * T * dwdy[(size_t)k * N + j];
    double drcp = cpm * drho + rho * dcpm;
    J[(size_t)0 * N + j] = -dHw / rcp + Hw / (rcp * rcp) * drcp;
    for (int k = 0; k < ns - 1; ++k)
      J[(size_t)(1 + k) * N + j] =
          m->W[k] / rho * dwdy[(size_t)k * N + j] - m->W[k] * wdot[k] / (rho * rho) * drho;
  }
  int ok = 1;
  for (size_t q = 0; q < (size_t)N * N; ++q) ok &= isfinite(J[q]);
  free(Y);
  free(dqdC);
  free(dqdT);
  free(dCdy);
  free(dqdy);
  free(dwdy);
  return ok ? 0 : ORC_NONFINITE;
}

/* The chemistry's difference-quotient Jacobian: the generic one-sided rule
 * of orc_fd_jacobian (radau.c, "based on that of CVODE", Sec. 2.1) applied to
 * orc_rhs at fixed pressure. */
typedef struct {
  const orc_mech *m;
  double P;
} fd_ctx;

static int fd_rhs(void *c, double t, const double *y, double *f) {
  (void)t;
  const fd_ctx *k = (const fd_ctx *)c;
  return orc_rhs(k->m, k->P, y, f);
}

int orc_jac_fd(const orc_mech *m, double P, const double *y, const double *f0, double h,
               const double *scal, double *J) {
  fd_ctx c = {m, P};
  return orc_fd_jacobian(m->ns, fd_rhs, &c, 0.0, y, f0, h, scal, J);
}

/* ------------------------------------------------------------------------
 * Concentration-based form: the reformulation the paper proposes for a
 * sparse Jacobian and a sparse LU (Sec. 3.3 and Sec. 4, after Schwer et al.
 * and the planned sparse pyJac).  The state is extensive, per unit mass of
 * mixture: phi = [T, V, n_0 .. n_{ns-2}] with V the volume (m^3) and n_k the
 * moles (kmol) of every species but the last, the inert bath gas, whose
 * moles close the ideal-gas law at the fixed pressure:
 *   C_k = n_k / V (k < in),   Ctot = P / (Ru T),   C_in = Ctot - sum_{k<in} C_k
 *   dn_k/dt = V wdot_k                                  (k < in)
 *   dT/dt   = -sum_k H_k wdot_k / sum_k C_k Cp_k        (the same energy equation)
 *   dV/dt   = V (sum_k wdot_k / Ctot + (dT/dt) / T)     (d/dt of P V = n Ru T)
 * with H_k = Ru T (h/RT)_k and Cp_k = Ru (cp/R)_k.  The Jacobian goes through
 * the concentrations as orc_jac does: dq/dC (nr x ns) times dC/dphi
 * (ns x (ns+1)), plus the explicit temperature dependences.  A species pair
 * is coupled only through a reaction that both take part in, or a collision
 * efficiency that differs from the bath gas's; rows and columns of T and V
 * are full.
 * ---------------------------------------------------------------------- */

/* C[ns] of the state phi; returns Ctot */
static double conc_of(const orc_mech *m, double P, const double *phi, double *C) {
  int in = m->ns - 1;
  double T = phi[0], V = phi[1], Ctot = P / (ORC_RU * T), s = 0.0;
  for (int k = 0; k < in; ++k) {
    C[k] = phi[2 + k] / V;
    s += C[k];
  }
  C[in] = Ctot - s;
  return Ctot;
}

/* molar production rates from (T, C) */
static void wdot_of_C(const orc_mech *m, double T, const double *C, const double *h_RT,
                      const double *s_R, double *wdot) {
  for (int k = 0; k < m->ns; ++k) wdot[k] = 0.0;
  for (int i = 0; i < m->nr; ++i) {
    rxn_terms r = reaction(m, i, T, C, h_RT, s_R);
    double q = r.phi * (r.kf * r.fwd - r.kr * r.rev);
    for (int k = 0; k < m->ns; ++k) wdot[k] += nu_of(m, i, k) * q;
  }
}

int orc_rhs_conc(const orc_mech *m, double P, const double *phi, double *f) {
  int ns = m->ns, in = ns - 1;
  double T = phi[0], V = phi[1];
  double *C = malloc(sizeof(double) * 5 * ns), *wdot = C + ns, *cp = wdot + ns, *h = cp + ns,
         *s = h + ns;
  double Ctot = conc_of(m, P, phi, C);
  orc_thermo(m, T, cp, h, s);
  wdot_of_C(m, T, C, h, s, wdot);
  double Hs = 0.0, Cs = 0.0, Ws = 0.0;
  for (int k = 0; k < ns; ++k) {
    Hs += h[k] * wdot[k];
    Cs += C[k] * cp[k];
    Ws += wdot[k];
  }
  double fT = -T * Hs / Cs;
  f[0] = fT;
  f[1] = V * (Ws / Ctot + fT / T);
  for (int k = 0; k < in; ++k) f[2 + k] = V * wdot[k];
  int ok = 1;
  for (int k = 0; k < ns + 1; ++k) ok &= isfinite(f[k]);
  free(C);
  return ok ? 0 : ORC_NONFINITE;
}

/* J[i*(ns+1) + j] = d f_i / d phi_j of the concentration-based form */
int orc_jac_conc(const orc_mech *m, double P, const double *phi, double *J) {
  int ns = m->ns, nr = m->nr, in = ns - 1, N = ns + 1;
  double T = phi[0], V = phi[1];
  double *C = calloc((size_t)ns * 6, sizeof(double));
  double *cp = C + ns, *h = cp + ns, *s = h + ns, *dcp = s + ns, *wdot = dcp + ns;
  double *dqdC = calloc((size_t)nr * ns, sizeof(double));
  double *dqdT = calloc((size_t)nr, sizeof(double));
  double *dCdp = calloc((size_t)ns * N, sizeof(double));   /* d C_k / d phi_j */
  double *dqdp = calloc((size_t)nr * N, sizeof(double));
  double *dwdp = calloc((size_t)ns * N, sizeof(double));
  double Ctot = conc_of(m, P, phi, C);
  orc_thermo(m, T, cp, h, s);
  thermo_dcp(m, T, dcp);
  for (int k = 0; k < ns; ++k) wdot[k] = 0.0;
  for (int i = 0; i < nr; ++i) {
    rxn_terms r = reaction(m, i, T, C, h, s);
    const int32_t *re = m->reac + 3 * i, *pr = m->prod + 3 * i;
    double Rnet = r.kf * r.fwd - r.kr * r.rev;
    double q = r.phi * Rnet;
    for (int k = 0; k < ns; ++k) wdot[k] += nu_of(m, i, k) * q;
    for (int k = 0; k < ns; ++k) {
      double d = r.phi * (r.kf * mass_action_dC(re, C, k) - r.kr * mass_action_dC(pr, C, k));
      if (m->rtype[i] != 0) d += Rnet * r.dphi_dM * m->eff[(size_t)i * ns + k];
      dqdC[(size_t)i * ns + k] = d;
    }
    dqdT[i] = r.phi * (r.kf * r.dlnkf_dT * r.fwd - r.kr * r.dlnkr_dT * r.rev) + Rnet * r.dphi_dT;
  }
  /* dC/dphi: column 0 is T, column 1 is V, column 2+l is n_l */
  double Sact = 0.0;
  for (int k = 0; k < in; ++k) Sact += C[k];
  for (int k = 0; k < in; ++k) {
    dCdp[(size_t)k * N + 1] = -C[k] / V;
    dCdp[(size_t)k * N + 2 + k] = 1.0 / V;
  }
  dCdp[(size_t)in * N + 0] = -Ctot / T;
  dCdp[(size_t)in * N + 1] = Sact / V;
  for (int l = 0; l < in; ++l) dCdp[(size_t)in * N + 2 + l] = -1.0 / V;
  for (int i = 0; i < nr; ++i)
    for (int j = 0; j < N; ++j) {
      double d = (j == 0) ? dqdT[i] : 0.0;
      for (int k = 0; k < ns; ++k) d += dqdC[(size_t)i * ns + k] * dCdp[(size_t)k * N + j];
      dqdp[(size_t)i * N + j] = d;
    }
  for (int k = 0; k < ns; ++k)
    for (int j = 0; j < N; ++j) {
      double d = 0.0;
      for (int i = 0; i < nr; ++i) d += nu_of(m, i, k) * dqdp[(size_t)i * N + j];
      dwdp[(size_t)k * N + j] = d;
    }
  /* mixture sums and their derivatives */
  double Hs = 0.0, Cs = 0.0, Ws = 0.0;
  for (int k = 0; k < ns; ++k) {
    Hs += h[k] * wdot[k];
    Cs += C[k] * cp[k];
    Ws += wdot[k];
  }
  double fT = -T * Hs / Cs;
  for (int j = 0; j < N; ++j) {
    double a = 0.0, c = 0.0;
    for (int k = 0; k < ns; ++k) {
      a += T * h[k] * dwdp[(size_t)k * N + j];
      c += cp[k] * dCdp[(size_t)k * N + j];
    }
    if (j == 0)
      for (int k = 0; k < ns; ++k) {
        a += cp[k] * wdot[k];   /* d(T h_k)/dT = cp_k (h in units of RT) */
        c += C[k] * dcp[k];
      }
    /* T row: f_T = -(T Hs) / Cs; a = d(T Hs)/dphi_j, c = dCs/dphi_j */
    J[(size_t)0 * N + j] = -a / Cs + (T * Hs) * c / (Cs * Cs);
  }
  for (int j = 0; j < N; ++j) {
    double dW = 0.0;
    for (int k = 0; k < ns; ++k) dW += dwdp[(size_t)k * N + j];
    double JT = J[(size_t)0 * N + j];
    /* V row: f_V = V (Ws / Ctot + fT / T), Ctot = P / (Ru T) */
    double inner = dW / Ctot + JT / T;
    if (j == 0) inner += Ws / (Ctot * T) - fT / (T * T);
    double dV = V * inner;
    if (j == 1) dV += Ws / Ctot + fT / T;
    J[(size_t)1 * N + j] = dV;
    /* species rows: f_k = V wdot_k */
    for (int k = 0; k < in; ++k) {
      double d = V * dwdp[(size_t)k * N + j];
      if (j == 1) d += wdot[k];
      J[(size_t)(2 + k) * N + j] = d;
    }
  }
  int ok = 1;
  for (size_t q = 0; q < (size_t)N * N; ++q) ok &= isfinite(J[q]);
  free(C);
  free(dqdC);
  free(dqdT);
  free(dCdp);
  free(dqdp);
  free(dwdp);
  return ok ? 0 : ORC_NONFINITE;
}
