// libkin: kernels and the C ABI declared in include/kin.h.
//
// One global step of n independent constant-pressure reactor states with
// Radau IIA (Sec. 2.1 of Curtis, Niemeyer & Sung).  Two launch layouts:
//   PLAIN  one thread per state, grid covers n (the paper's organisation);
//   QUEUE  a persistent grid sized from the occupancy calculator; each lane
//          attempts one step per loop trip and pops the next state index from
//          an atomic counter when its state is finished, so finished lanes
//          never wait for the slowest lane of their warp (Sec. 3.3).
// Mechanism tables are staged into shared memory per CTA.
#include <cuda_runtime.h>

#include <cmath>
#include <algorithm>
#include <complex>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <vector>

#include "../../include/kin.h"
#include "kin_internal.h"
#include "kin_kernels.cuh"

using namespace kin;

// One tuned launch configuration (kin_autotune) and the key it answers.
struct TuneEntry {
  int lu_fp32, jac_fd, dt_decade, n_log2;
  int layout, block, refill, lanes;
};

struct kin_mech {
  int device;
  std::mutex tune_mu;
  std::vector<TuneEntry> tuned;            // at most kMaxTuned entries
  MechLayout L;
  double *d_tab = nullptr;
  int *d_itab = nullptr;
  unsigned long long *d_totals = nullptr;  // [0..6] sums, [7] failed, [8] max steps, [9] queue,
                                           // [10] order entries out of range
  void *d_order_ws = nullptr;              // kin_order_states workspace
  void *d_gscratch = nullptr;              // WARP layout: per-group Jacobian slots
  int64_t gslots = 0;
  cudaStream_t last_stream = nullptr;
  // host-call buffers
  double *h_Y = nullptr, *h_T = nullptr, *h_P = nullptr;
  int32_t *h_status = nullptr, *h_cnt = nullptr;
  double *h_key = nullptr;    // host entry: ordering key and permutation
  int32_t *h_order = nullptr;
  int64_t h_cap = 0;
};

// ---------------------------------------------------------------------------
// Radau constants from closed forms (Hairer & Wanner IV.5 / IV.8)
// ---------------------------------------------------------------------------
static void inv3(const double *m, double *r) {
  double d = m[0] * (m[4] * m[8] - m[5] * m[7]) - m[1] * (m[3] * m[8] - m[5] * m[6]) +
             m[2] * (m[3] * m[7] - m[4] * m[6]);
  r[0] = (m[4] * m[8] - m[5] * m[7]) / d;
  r[1] = (m[2] * m[7] - m[1] * m[8]) / d;
  r[2] = (m[1] * m[5] - m[2] * m[4]) / d;
  r[3] = (m[5] * m[6] - m[3] * m[8]) / d;
  r[4] = (m[0] * m[8] - m[2] * m[6]) / d;
  r[5] = (m[2] * m[3] - m[0] * m[5]) / d;
  r[6] = (m[3] * m[7] - m[4] * m[6]) / d;
  r[7] = (m[1] * m[6] - m[0] * m[7]) / d;
  r[8] = (m[0] * m[4] - m[1] * m[3]) / d;
}

static RadauConst radau_constants_host() {
  RadauConst rc;
  const double s6 = std::sqrt(6.0);
  rc.c1 = (4.0 - s6) / 10.0;
  rc.c2 = (4.0 + s6) / 10.0;
  // eigenvalues of A: real u1 and al +- i be (cube-root closed forms)
  const double c9 = std::cbrt(9.0), c81 = std::cbrt(81.0);
  const double u1 = (6.0 + c81 - c9) / 30.0;
  const double al = (12.0 - c81 + c9) / 60.0;
  const double be = (c81 + c9) * std::sqrt(3.0) / 60.0;
  const double cno = al * al + be * be;
  rc.gam = 1.0 / u1;  // eigenvalues of A^-1
  rc.alp = al / cno;
  rc.bet = be / cno;
  // A from its closed-form entries, M = A^-1
  const double A[9] = {(88.0 - 7.0 * s6) / 360.0,   (296.0 - 169.0 * s6) / 1800.0,
                       (-2.0 + 3.0 * s6) / 225.0,   (296.0 + 169.0 * s6) / 1800.0,
                       (88.0 + 7.0 * s6) / 360.0,   (-2.0 - 3.0 * s6) / 225.0,
                       (16.0 - s6) / 36.0,          (16.0 + s6) / 36.0,
                       1.0 / 9.0};
  double M[9];
  inv3(A, M);
  // eigenvector for gam with last entry 1: 2x2 system from the first two rows
  double v[3];
  {
    const double a = M[0] - rc.gam, b = M[1], c = M[3], d = M[4] - rc.gam;
    const double r0 = -M[2], r1 = -M[5], det = a * d - b * c;
    v[0] = (r0 * d - b * r1) / det;
    v[1] = (a * r1 - c * r0) / det;
    v[2] = 1.0;
    const double nv = std::sqrt(v[0] * v[0] + v[1] * v[1] + 1.0);
    for (double &q : v) q /= nv;
  }
  // eigenvector for alp + i bet with last entry 1
  std::complex<double> w0, w1;
  {
    const std::complex<double> lam(rc.alp, rc.bet);
    const std::complex<double> a = M[0] - lam, b = M[1], c = M[3], d = M[4] - lam;
    const std::complex<double> r0 = -M[2], r1 = -M[5], det = a * d - b * c;
    w0 = (r0 * d - b * r1) / det;
    w1 = (a * r1 - c * r0) / det;
  }
  // columns: v, Re w, -Im w  (w = T2 - i T3)
  const double T[9] = {v[0], w0.real(), -w0.imag(), v[1], w1.real(), -w1.imag(),
                       v[2], 1.0,       0.0};
  std::memcpy(rc.T, T, sizeof T);
  inv3(rc.T, rc.TI);
  rc.d[0] = -(13.0 + 7.0 * s6) / 3.0;
  rc.d[1] = (-13.0 + 7.0 * s6) / 3.0;
  rc.d[2] = -1.0 / 3.0;
  rc.ic1 = 1.0 / rc.c1;
  rc.ic2 = 1.0 / rc.c2;
  rc.ic1m1 = 1.0 / (rc.c1 - 1.0);
  rc.ic2m1 = 1.0 / (rc.c2 - 1.0);
  rc.ic1mc2 = 1.0 / (rc.c1 - rc.c2);
  return rc;
}

static std::mutex g_const_mu;
static bool g_const_done[64];

int kin::ensure_constants(int dev) {
  std::lock_guard<std::mutex> lk(g_const_mu);
  if (dev < 0 || dev >= 64) return KIN_ERR_CUDA;
  if (g_const_done[dev]) return KIN_OK;
  RadauConst rc = radau_constants_host();
  int r;
  if ((r = kin_consts_16d(rc)) || (r = kin_consts_16f(rc)) || (r = kin_consts_64d(rc)) ||
      (r = kin_consts_64f(rc)) || (r = kin_consts_grpd(rc)) || (r = kin_consts_grpf(rc)))
    return r;
  g_const_done[dev] = true;
  return KIN_OK;
}

template <int MAXN>
__global__ void k_rhs(MechLayout L, const double *tab, const int *itab, const double *y,
                      const double *P, int64_t n, double *f) {
  extern __shared__ double smem[];
  const MechView m = stage_tables(L, tab, itab, smem);
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int N = m.ns;
  double yy[MAXN], ff[MAXN];
  ChemScratch<MAXN> cs;
  JacScratch<MAXN, double> js;
  for (int k = 0; k < N; ++k) yy[k] = y[(int64_t)k * n + i];
  rhs<MAXN, double>(m, P[i], yy, ff, cs, js);
  for (int k = 0; k < N; ++k) f[(int64_t)k * n + i] = ff[k];
}

template <int MAXN>
__global__ void k_jac(MechLayout L, const double *tab, const int *itab, const double *y,
                      const double *P, int64_t n, int fd, double h, const double *scal,
                      double *Jout) {
  extern __shared__ double smem[];
  const MechView m = stage_tables(L, tab, itab, smem);
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int N = m.ns;
  double yy[MAXN], f0[MAXN], sc[MAXN], u[MAXN], fu[MAXN];
  double J[MAXN * MAXN];
  ChemScratch<MAXN> cs;
  JacScratch<MAXN, double> js;
  for (int k = 0; k < N; ++k) yy[k] = y[(int64_t)k * n + i];
  if (!fd) {
    chem_eval<MAXN, double>(m, P[i], yy, f0, J, true, cs, js);
  } else {
    for (int k = 0; k < N; ++k) sc[k] = scal[(int64_t)k * n + i];
    rhs<MAXN, double>(m, P[i], yy, f0, cs, js);
    double mininc = 0.0;
    for (int j = 0; j < N; ++j) {
      const double inc = fd_increment(N, yy, f0, sc, h, j, mininc, j == 0);
      for (int k = 0; k < N; ++k) u[k] = yy[k];
      u[j] = yy[j] + inc;
      rhs<MAXN, double>(m, P[i], u, fu, cs, js);
      for (int k = 0; k < N; ++k) J[k * N + j] = (fu[k] - f0[k]) / inc;
    }
  }
  for (int q = 0; q < N * N; ++q) Jout[(int64_t)q * n + i] = J[q];
}

__global__ void k_exp(const double *tab, const double *x, double *y, int64_t n) {
  __shared__ double t[EXP_TAB];
  for (int j = threadIdx.x; j < EXP_TAB; j += blockDim.x) t[j] = tab[j];
  __syncthreads();
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] = kexp(x[i], t);
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
extern "C" int kin_options_default(kin_options *o) {
  if (!o) return KIN_ERR_INVALID_ARG;
  std::memset(o, 0, sizeof *o);
  o->layout = KIN_LAYOUT_AUTO;
  o->lu_fp32 = 0;
  o->jac_fd = 0;
  o->max_steps = 100000;
  o->nit = 7;
  o->block = 0;
  o->grid_per_sm = 0;
  o->transform_tol = 1;
  o->queue_refill = 0;
  o->stop_after = 0;
  o->order = nullptr;
  o->lanes = 0;
  o->h_fixed = 0.0;
  o->order_by = 0;
  return KIN_OK;
}

extern "C" const char *kin_status_string(int s) {
  switch (s) {
    case KIN_OK: return "ok";
    case KIN_ERR_INVALID_ARG: return "invalid argument";
    case KIN_ERR_CUDA: return "CUDA error";
    case KIN_ERR_NOMEM: return "out of device memory";
    case KIN_ERR_MECH: return "invalid mechanism description";
    case KIN_ERR_STATE_FAILED: return "one or more states failed";
    case KIN_ERR_UNSUPPORTED: return "unsupported configuration";
    default: return "unknown status";
  }
}

extern "C" int kin_radau_constants(double *out, int32_t len) {
  if (!out || len < 27) return KIN_ERR_INVALID_ARG;
  RadauConst rc = radau_constants_host();
  out[0] = rc.c1;
  out[1] = rc.c2;
  out[2] = 1.0;
  out[3] = rc.gam;
  out[4] = rc.alp;
  out[5] = rc.bet;
  for (int i = 0; i < 9; ++i) out[6 + i] = rc.T[i];
  for (int i = 0; i < 9; ++i) out[15 + i] = rc.TI[i];
  for (int i = 0; i < 3; ++i) out[24 + i] = rc.d[i];
  return KIN_OK;
}

// Validate a mechanism description and build its device tables on the host.
int kin::build_tables(const kin_mech_desc *d, MechLayout &L, std::vector<double> &dt,
                      std::vector<int> &it) {
  if (!d) return KIN_ERR_INVALID_ARG;
  const int ns = d->ns, nr = d->nr;
  if (ns < 2 || ns > KIN_MAX_SPECIES || nr < 1) return KIN_ERR_INVALID_ARG;
  if (!d->W || !d->nasa || !d->reac || !d->prod || !d->arrh || !d->rtype || !d->eff || !d->fall)
    return KIN_ERR_INVALID_ARG;
  const int in = ns - 1;
  for (int k = 0; k < ns; ++k) {
    if (!(d->W[k] > 0.0)) return KIN_ERR_MECH;
    const double *p = d->nasa + 17 * k;
    if (!(p[0] > 0.0 && p[1] > 0.0 && p[2] > 0.0)) return KIN_ERR_MECH;
  }
  int neff = 0, ntroe = 0;
  for (int i = 0; i < nr; ++i) {
    int nre = 0, npr = 0;
    for (int s = 0; s < 3; ++s) {
      const int r = d->reac[3 * i + s], p = d->prod[3 * i + s];
      if (r < -1 || r >= ns || p < -1 || p >= ns) return KIN_ERR_MECH;
      if (r == in || p == in) return KIN_ERR_MECH;
      nre += (r >= 0);
      npr += (p >= 0);
    }
    if (nre == 0 || npr == 0) return KIN_ERR_MECH;
    const int t = d->rtype[i];
    if (t < 0 || t > 2) return KIN_ERR_MECH;
    if (t != 0) {
      for (int k = 0; k < ns; ++k)
        if (d->eff[(size_t)i * ns + k] != 1.0) ++neff;
    }
    if (t == 2) ++ntroe;
    if (!(d->arrh[3 * i] > 0.0)) return KIN_ERR_MECH;
    if (t == 2 && !(d->fall[7 * i] > 0.0 && d->fall[7 * i + 4] > 0.0 && d->fall[7 * i + 5] > 0.0))
      return KIN_ERR_MECH;
  }
  L = MechLayout{};
  L.ns = ns;
  L.nr = nr;
  L.neff = neff;
  L.ntroe = ntroe;
  L.nfall = 0;
  for (int i = 0; i < nr; ++i) L.nfall += d->rtype[i] != 0;
  int o = 0;
  L.dW = o; o += ns;
  L.dinvW = o; o += ns;
  L.dTmid = o; o += ns;
  L.dcp = o; o += 2 * ns * NCP;
  L.dh = o; o += 2 * ns * NH;
  L.dg = o; o += 2 * ns * NG;
  L.dlnA = o; o += nr;
  L.db = o; o += nr;
  L.dTh = o; o += nr;
  L.dtroe = o; o += NTROE * (ntroe > 0 ? ntroe : 1);
  L.deff = o; o += (neff > 0 ? neff : 1);
  L.dexp = o; o += EXP_TAB;
  L.dnu = o; o += nr;
  int q = 0;
  L.islot = q; q += 6 * nr;
  L.imeta = q; q += nr;
  L.ieff0 = q; q += nr;
  L.itroe = q;
  L.ieffsp = q; q += (neff > 0 ? neff : 1);
  // Device order of the reactions: Troe falloff first, then third-body, then
  // elementary, each by reactant and product count (stable).  Kernels that
  // spread reactions over lanes then meet the falloff branches in the first
  // rounds only and run the slot loops with equal trip counts; results
  // depend on the order only through summation rounding.
  std::vector<int> perm(nr);
  for (int i = 0; i < nr; ++i) perm[i] = i;
  auto rkey = [&](int i) {
    int nre = 0, npr = 0;
    for (int s2 = 0; s2 < 3; ++s2) {
      nre += d->reac[3 * i + s2] >= 0;
      npr += d->prod[3 * i + s2] >= 0;
    }
    const int t = d->rtype[i], cls = t == 2 ? 0 : t == 1 ? 1 : 2;
    return cls * 16 + nre * 4 + npr;
  };
  std::stable_sort(perm.begin(), perm.end(), [&](int a, int b) { return rkey(a) < rkey(b); });
  // species-major list of (reaction, net coefficient) for gathered production rates
  std::vector<std::vector<int>> sp_list(ns);
  for (int i = 0; i < nr; ++i) {
    const int src = perm[i];
    for (int k = 0; k < ns; ++k) {
      int nu = 0;
      for (int s2 = 0; s2 < 3; ++s2)
        nu += (d->prod[3 * src + s2] == k) - (d->reac[3 * src + s2] == k);
      if (nu != 0) sp_list[k].push_back((i << 4) | (nu + 8));
    }
  }
  int ncsr = 0;
  for (int k = 0; k < ns; ++k) ncsr += (int)sp_list[k].size();
  L.icsr0 = q; q += ns + 1;
  L.icsr = q; q += (ncsr > 0 ? ncsr : 1);
  L.ni = q;
  L.dcsrnu = o; o += (ncsr > 0 ? ncsr : 1);
  L.nd = o;
  dt.assign(L.nd, 0.0);
  it.assign(L.ni, 0);
  for (int k = 0; k < ns; ++k) {
    dt[L.dW + k] = d->W[k];
    dt[L.dinvW + k] = 1.0 / d->W[k];
    const double *p = d->nasa + 17 * k;
    dt[L.dTmid + k] = p[1];
    for (int r = 0; r < 2; ++r) {
      const double *a = p + 3 + 7 * r;
      double *cp = &dt[L.dcp + (2 * k + r) * NCP];
      double *h = &dt[L.dh + (2 * k + r) * NH];
      double *g = &dt[L.dg + (2 * k + r) * NG];
      for (int j = 0; j < 5; ++j) cp[j] = a[j];
      h[0] = a[0]; h[1] = a[1] / 2.0; h[2] = a[2] / 3.0; h[3] = a[3] / 4.0; h[4] = a[4] / 5.0;
      h[5] = a[5];
      // g = s/R - h/RT: a0 (ln T - 1) + a1 T/2 + a2 T^2/6 + a3 T^3/12 + a4 T^4/20 + a6 - a5/T
      g[0] = a[0]; g[1] = a[1] / 2.0; g[2] = a[2] / 6.0; g[3] = a[3] / 12.0;
      g[4] = a[4] / 20.0; g[5] = a[6] - a[0]; g[6] = -a[5];
    }
  }
  // 2^(j/256), rounded to double, for the table-driven exponential
  for (int j = 0; j < EXP_TAB; ++j) dt[L.dexp + j] = (double)exp2l((long double)j / EXP_TAB);
  int e = 0, tr = 0;
  for (int i = 0; i < nr; ++i) {
    const int src = perm[i];  // description index of device reaction i
    dt[L.dlnA + i] = std::log(d->arrh[3 * src]);
    dt[L.db + i] = d->arrh[3 * src + 1];
    dt[L.dTh + i] = d->arrh[3 * src + 2];
    int nre = 0, npr = 0;
    for (int s = 0; s < 3; ++s) {
      if (d->reac[3 * src + s] >= 0) it[L.islot + 6 * i + nre++] = d->reac[3 * src + s];
      if (d->prod[3 * src + s] >= 0) it[L.islot + 6 * i + 3 + npr++] = d->prod[3 * src + s];
    }
    const int t = d->rtype[src];
    int ne = 0;
    it[L.ieff0 + i] = e;
    if (t != 0) {
      for (int k = 0; k < ns; ++k) {
        const double ef = d->eff[(size_t)src * ns + k];
        if (ef != 1.0) {
          dt[L.deff + e] = ef - 1.0;
          it[L.ieffsp + e] = k;
          ++e;
          ++ne;
        }
      }
    }
    if (ne > 255) return KIN_ERR_MECH;
    int troe_idx = 0;
    if (t == 2) {
      const double *f = d->fall + 7 * src;
      double *tp = &dt[L.dtroe + NTROE * tr];
      tp[0] = std::log(f[0]);
      tp[1] = f[1];
      tp[2] = f[2];
      tp[3] = f[3];
      tp[4] = 1.0 / f[4];
      tp[5] = 1.0 / f[5];
      tp[6] = f[6];
      troe_idx = tr++;
    }
    it[L.imeta + i] = t | (nre << 2) | (npr << 4) | (ne << 8) | (troe_idx << 16);
    dt[L.dnu + i] = (double)(npr - nre);
  }
  {
    int c = 0;
    for (int k = 0; k < ns; ++k) {
      it[L.icsr0 + k] = c;
      for (int code : sp_list[k]) {
        dt[L.dcsrnu + c] = (double)((code & 15) - 8);
        it[L.icsr + c++] = code;
      }
    }
    it[L.icsr0 + ns] = c;
  }
  if (smem_bytes(L) > 200 * 1024) return KIN_ERR_UNSUPPORTED;
  return KIN_OK;
}

extern "C" int kin_mech_create(const kin_mech_desc *d, kin_mech **out) {
  if (!d || !out) return KIN_ERR_INVALID_ARG;
  *out = nullptr;
  MechLayout L;
  std::vector<double> dt;
  std::vector<int> it;
  int brc = build_tables(d, L, dt, it);
  if (brc) return brc;
  int dev = 0;
  KIN_CUDA_TRY(cudaGetDevice(&dev));
  int rc = ensure_constants(dev);
  if (rc) return rc;
  int sms = 0;
  KIN_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  kin_mech *m = new kin_mech();
  m->device = dev;
  m->L = L;
  // WARP layout: one Jacobian slot (with the complex matrix when that lives
  // in global memory) per resident group: up to 64 groups of 4-16 lanes per
  // SM for ns <= 15, 16 whole warps per SM beyond
  m->gslots = (int64_t)sms * (L.ns <= 15 ? 64 : 16);
  const size_t gbytes =
      (size_t)m->gslots * warp_slot_mats(sizeof(double)) * L.ns * (L.ns + 1) * sizeof(double);
  if (cudaMalloc(&m->d_tab, sizeof(double) * L.nd) != cudaSuccess ||
      cudaMalloc(&m->d_itab, sizeof(int) * L.ni) != cudaSuccess ||
      cudaMalloc(&m->d_totals, sizeof(unsigned long long) * 16) != cudaSuccess ||
      cudaMalloc(&m->d_order_ws, order_workspace_bytes()) != cudaSuccess ||
      cudaMalloc(&m->d_gscratch, gbytes) != cudaSuccess) {
    (void)cudaGetLastError();
    kin_destroy(m);
    return KIN_ERR_NOMEM;
  }
  if (cudaMemcpy(m->d_tab, dt.data(), sizeof(double) * L.nd, cudaMemcpyHostToDevice) !=
          cudaSuccess ||
      cudaMemcpy(m->d_itab, it.data(), sizeof(int) * L.ni, cudaMemcpyHostToDevice) !=
          cudaSuccess ||
      cudaMemset(m->d_totals, 0, sizeof(unsigned long long) * 16) != cudaSuccess) {
    (void)cudaGetLastError();
    kin_destroy(m);
    return KIN_ERR_CUDA;
  }
  *out = m;
  return KIN_OK;
}

extern "C" void kin_destroy(kin_mech *m) {
  if (!m) return;
  cudaFree(m->d_tab);
  cudaFree(m->d_itab);
  cudaFree(m->d_totals);
  cudaFree(m->d_order_ws);
  cudaFree(m->d_gscratch);
  cudaFree(m->h_Y);
  cudaFree(m->h_T);
  cudaFree(m->h_P);
  cudaFree(m->h_status);
  cudaFree(m->h_key);
  cudaFree(m->h_order);
  cudaFree(m->h_cnt);
  delete m;
}

int kin::launch_dispatch(const KernelArgs &a, const kin_options &o, cudaStream_t st,
                         int sms) {
  if (o.layout == KIN_LAYOUT_WARP && o.lanes != 0 && o.lanes != 32)
    return o.lu_fp32 ? kin_launch_grpf(a, o, st, sms) : kin_launch_grpd(a, o, st, sms);
  if (a.L.ns <= SMALL_MAXN && o.layout != KIN_LAYOUT_WARP)
    return o.lu_fp32 ? kin_launch_16f(a, o, st, sms) : kin_launch_16d(a, o, st, sms);
  return o.lu_fp32 ? kin_launch_64f(a, o, st, sms) : kin_launch_64d(a, o, st, sms);
}

static constexpr size_t kMaxTuned = 64;

static int dt_decade(double dt) { return (int)std::floor(std::log10(dt)); }
static int n_log2(int64_t n) {
  int b = 0;
  while (b < 62 && ((int64_t)1 << (b + 1)) <= n) ++b;
  return b;
}

// KIN_LAYOUT_AUTO: the tuning cache's entry for (precision, Jacobian, dt
// decade) nearest in log2 n, else the size rule (PLAIN up to 16 species,
// WARP beyond; PLAIN at a fixed step, where WARP is not available).
static void resolve_auto(kin_mech *m, int64_t n, double dt, kin_options &o) {
  if (o.layout != KIN_LAYOUT_AUTO) return;
  const int dd = dt_decade(dt), nb = n_log2(n > 0 ? n : 1);
  const TuneEntry *best = nullptr;
  {
    std::lock_guard<std::mutex> lk(m->tune_mu);
    for (const TuneEntry &e : m->tuned) {
      if (e.lu_fp32 != (o.lu_fp32 != 0) || e.jac_fd != (o.jac_fd != 0) || e.dt_decade != dd)
        continue;
      if (!best || std::abs(e.n_log2 - nb) < std::abs(best->n_log2 - nb)) best = &e;
    }
    if (best && !(o.h_fixed > 0.0 && best->layout == KIN_LAYOUT_WARP)) {
      o.layout = best->layout;
      o.block = best->block;
      o.queue_refill = best->refill;
      o.lanes = best->lanes;
      return;
    }
  }
  if (m->L.ns <= SMALL_MAXN || o.h_fixed > 0.0) {
    o.layout = KIN_LAYOUT_PLAIN;
    o.block = 64;
    o.lanes = 0;
  } else {
    o.layout = KIN_LAYOUT_WARP;
    o.block = 0;
    o.lanes = 32;
  }
}

static void remember_tuning(kin_mech *m, int64_t n, double dt, const kin_options &best) {
  TuneEntry e{best.lu_fp32 != 0, best.jac_fd != 0, dt_decade(dt), n_log2(n),
              best.layout, best.block, best.queue_refill, best.lanes};
  std::lock_guard<std::mutex> lk(m->tune_mu);
  for (TuneEntry &x : m->tuned)
    if (x.lu_fp32 == e.lu_fp32 && x.jac_fd == e.jac_fd && x.dt_decade == e.dt_decade &&
        x.n_log2 == e.n_log2) {
      x = e;
      return;
    }
  if (m->tuned.size() >= kMaxTuned) m->tuned.erase(m->tuned.begin());
  m->tuned.push_back(e);
}

extern "C" int kin_resolve_options(kin_mech *m, int64_t n, double dt, const kin_options *opt,
                                   kin_options *out) {
  if (!m || !out || n < 0 || !(dt > 0.0) || !std::isfinite(dt)) return KIN_ERR_INVALID_ARG;
  kin_options o;
  if (opt) {
    o = *opt;
  } else {
    kin_options_default(&o);
  }
  resolve_auto(m, n, dt, o);
  *out = o;
  return KIN_OK;
}

static int check_common(kin_mech *m, const void *Y, const void *T, const void *P, int64_t n,
                        double dt, double rtol, double atol) {
  if (!m || n < 0) return KIN_ERR_INVALID_ARG;
  if (n > 0 && (!Y || !T || !P)) return KIN_ERR_INVALID_ARG;
  if (!(dt > 0.0) || !(rtol > 0.0) || !(atol > 0.0) || !std::isfinite(dt))
    return KIN_ERR_INVALID_ARG;
  return KIN_OK;
}

extern "C" int kin_integrate_ex(kin_mech *m, double *Y, double *T, const double *P, int64_t n,
                                double dt, double rtol, double atol, const kin_options *opt,
                                int32_t *status, int32_t *counters, void *stream) {
  int rc = check_common(m, Y, T, P, n, dt, rtol, atol);
  if (rc) return rc;
  kin_options o;
  if (opt) {
    o = *opt;
  } else {
    kin_options_default(&o);
  }
  if (o.layout != KIN_LAYOUT_PLAIN && o.layout != KIN_LAYOUT_QUEUE && o.layout != KIN_LAYOUT_WARP &&
      o.layout != KIN_LAYOUT_AUTO)
    return KIN_ERR_INVALID_ARG;
  if (o.nit < 1 || o.nit > 50 || o.max_steps < 1) return KIN_ERR_INVALID_ARG;
  if (o.queue_refill < 0 || o.queue_refill > 32 || o.stop_after < 0) return KIN_ERR_INVALID_ARG;
  if (o.order && n > INT32_MAX) return KIN_ERR_INVALID_ARG;
  if (o.order_by != 0) return KIN_ERR_INVALID_ARG;  // host entry only (kin_order_states here)
  if (o.lanes != 0 && o.lanes != 4 && o.lanes != 8 && o.lanes != 16 && o.lanes != 32)
    return KIN_ERR_INVALID_ARG;
  if (!(o.h_fixed >= 0.0) || !std::isfinite(o.h_fixed)) return KIN_ERR_INVALID_ARG;
  if (o.block != 0 && (o.block < 32 || o.block > 64 || o.block % 32)) return KIN_ERR_INVALID_ARG;
  resolve_auto(m, n, dt, o);
  if (o.h_fixed > 0.0 && o.layout == KIN_LAYOUT_WARP) return KIN_ERR_UNSUPPORTED;
  cudaStream_t st = (cudaStream_t)stream;
  m->last_stream = st;
  KIN_CUDA_TRY(cudaMemsetAsync(m->d_totals, 0, sizeof(unsigned long long) * 16, st));
  if (n == 0) return KIN_OK;
  KernelArgs a;
  a.L = m->L;
  a.tab = m->d_tab;
  a.itab = m->d_itab;
  a.Y = Y;
  a.T = T;
  a.P = P;
  a.status = status;
  a.counters = counters;
  a.totals = m->d_totals;
  double r = rtol, at = atol;
  if (o.transform_tol) {
    const double quot = atol / rtol;
    r = 0.1 * std::pow(rtol, 2.0 / 3.0);
    at = r * quot;
  }
  a.rp.rtol = r;
  a.rp.atol = at;
  a.rp.fnewt = std::fmax(10.0 * UROUND / r, std::fmin(0.03, std::sqrt(r)));
  a.rp.dt = dt;
  a.rp.nit = o.nit;
  a.rp.max_steps = o.max_steps;
  a.rp.n = n;
  a.rp.h0 = o.h0;
  a.rp.z0 = o.z0;
  a.rp.h_first = o.h_first;
  a.rp.z_first = o.z_first;
  a.rp.stop_after = o.stop_after;
  a.rp.hfixed = o.h_fixed;
  a.refill_min = o.queue_refill > 0 ? o.queue_refill : 1;
  a.order = o.order;
  a.gscratch = m->d_gscratch;
  a.gslots = m->gslots;
  int dev = 0, sms = 0;
  KIN_CUDA_TRY(cudaGetDevice(&dev));
  if (dev != m->device) return KIN_ERR_INVALID_ARG;
  KIN_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  return launch_dispatch(a, o, st, sms);
}

extern "C" int kin_integrate(kin_mech *m, double *Y, double *T, const double *P, int64_t n,
                             double dt, double rtol, double atol, void *stream) {
  return kin_integrate_ex(m, Y, T, P, n, dt, rtol, atol, nullptr, nullptr, nullptr, stream);
}

template <typename X>
static int grow(X **p, int64_t count) {
  cudaFree(*p);
  *p = nullptr;
  KIN_CUDA_TRY(cudaMalloc(p, sizeof(X) * (size_t)count));
  return KIN_OK;
}

extern "C" int kin_integrate_host(kin_mech *m, double *Y, double *T, const double *P, int64_t n,
                                  double dt, double rtol, double atol, const kin_options *opt,
                                  int32_t *status, int32_t *counters, void *stream) {
  int rc = check_common(m, Y, T, P, n, dt, rtol, atol);
  if (rc) return rc;
  if (opt && (opt->h0 || opt->z0 || opt->h_first || opt->z_first || opt->order))
    return KIN_ERR_INVALID_ARG;
  if (opt && opt->order_by != 0 && opt->order_by != 1) return KIN_ERR_INVALID_ARG;
  if (opt && opt->order_by && n > INT32_MAX) return KIN_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  const int ns = m->L.ns;
  if (n > m->h_cap) {
    if ((rc = grow(&m->h_Y, n * ns)) || (rc = grow(&m->h_T, n)) || (rc = grow(&m->h_P, n)) ||
        (rc = grow(&m->h_status, n)) || (rc = grow(&m->h_cnt, n * KIN_NCOUNTERS)) ||
        (rc = grow(&m->h_key, n)) || (rc = grow(&m->h_order, n))) {
      m->h_cap = 0;
      return rc;
    }
    m->h_cap = n;
  }
  kin_options o;
  if (opt) {
    o = *opt;
  } else {
    kin_options_default(&o);
  }
  const bool order = o.order_by == 1;
  o.order_by = 0;  // handled here; the device entry takes the explicit order
  if (n == 0) return kin_integrate_ex(m, m->h_Y, m->h_T, m->h_P, 0, dt, rtol, atol, &o, nullptr,
                                      nullptr, stream);
  KIN_CUDA_TRY(cudaMemcpyAsync(m->h_Y, Y, sizeof(double) * n * ns, cudaMemcpyHostToDevice, st));
  KIN_CUDA_TRY(cudaMemcpyAsync(m->h_T, T, sizeof(double) * n, cudaMemcpyHostToDevice, st));
  KIN_CUDA_TRY(cudaMemcpyAsync(m->h_P, P, sizeof(double) * n, cudaMemcpyHostToDevice, st));
  if (order) {  // stiffness ordering into the entry's own buffers
    rc = kin_order_states(m, m->h_Y, m->h_T, m->h_P, n, rtol, atol, KIN_KEY_STEP_HEURISTIC,
                          m->h_key, m->h_order, stream);
    if (rc) return rc;
    o.order = m->h_order;
  }
  rc = kin_integrate_ex(m, m->h_Y, m->h_T, m->h_P, n, dt, rtol, atol, &o,
                        status ? m->h_status : nullptr, counters ? m->h_cnt : nullptr, stream);
  if (rc) return rc;
  KIN_CUDA_TRY(cudaMemcpyAsync(Y, m->h_Y, sizeof(double) * n * ns, cudaMemcpyDeviceToHost, st));
  KIN_CUDA_TRY(cudaMemcpyAsync(T, m->h_T, sizeof(double) * n, cudaMemcpyDeviceToHost, st));
  if (status)
    KIN_CUDA_TRY(cudaMemcpyAsync(status, m->h_status, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, st));
  if (counters)
    KIN_CUDA_TRY(cudaMemcpyAsync(counters, m->h_cnt, sizeof(int32_t) * n * KIN_NCOUNTERS,
                                 cudaMemcpyDeviceToHost, st));
  KIN_CUDA_TRY(cudaStreamSynchronize(st));
  return KIN_OK;
}

extern "C" int kin_get_stats(kin_mech *m, int64_t *out) {
  if (!m || !out) return KIN_ERR_INVALID_ARG;
  unsigned long long t[16];
  KIN_CUDA_TRY(cudaStreamSynchronize(m->last_stream));
  KIN_CUDA_TRY(cudaMemcpy(t, m->d_totals, sizeof t, cudaMemcpyDeviceToHost));
  for (int i = 0; i < 9; ++i) out[i] = (int64_t)t[i];
  if (t[10] > 0) return KIN_ERR_INVALID_ARG;  // order entries outside [0, n) were skipped
  return out[7] > 0 ? KIN_ERR_STATE_FAILED : KIN_OK;
}

extern "C" int kin_order_states(kin_mech *m, const double *Y, const double *T, const double *P,
                                int64_t n, double rtol, double atol, int32_t key_mode,
                                double *key, int32_t *order, void *stream) {
  if (!m || n < 0 || n > INT32_MAX) return KIN_ERR_INVALID_ARG;
  if (key_mode != KIN_KEY_GIVEN && key_mode != KIN_KEY_STEP_HEURISTIC &&
      key_mode != KIN_KEY_GIVEN_LOG)
    return KIN_ERR_INVALID_ARG;
  if (n == 0) return KIN_OK;
  if (!key || !order) return KIN_ERR_INVALID_ARG;
  const bool compute = key_mode == KIN_KEY_STEP_HEURISTIC;
  if (compute) {
    if (!Y || !T || !P || !(rtol > 0.0) || !(atol > 0.0)) return KIN_ERR_INVALID_ARG;
  }
  int dev = 0, sms = 0;
  KIN_CUDA_TRY(cudaGetDevice(&dev));
  if (dev != m->device) return KIN_ERR_INVALID_ARG;
  KIN_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  // the integrator's default tolerance transform (Hairer-Wanner)
  const double r = 0.1 * std::pow(rtol, 2.0 / 3.0), at = compute ? r * (atol / rtol) : 0.0;
  return launch_order(m->L, m->d_tab, m->d_itab, Y, T, P, n, r, at, compute,
                      key_mode == KIN_KEY_GIVEN_LOG, key, order, m->d_order_ws,
                      (cudaStream_t)stream, sms);
}

extern "C" int kin_rhs(kin_mech *m, const double *y, const double *P, int64_t n, double *f,
                       void *stream) {
  if (!m || n < 0 || (n > 0 && (!y || !P || !f))) return KIN_ERR_INVALID_ARG;
  if (n == 0) return KIN_OK;
  cudaStream_t st = (cudaStream_t)stream;
  const size_t sm = smem_bytes(m->L);
  const int block = 64;
  const unsigned grid = (unsigned)((n + block - 1) / block);
  if (m->L.ns <= 16) {
    KIN_CUDA_TRY(cudaFuncSetAttribute(k_rhs<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    k_rhs<16><<<grid, block, sm, st>>>(m->L, m->d_tab, m->d_itab, y, P, n, f);
  } else {
    KIN_CUDA_TRY(cudaFuncSetAttribute(k_rhs<64>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    k_rhs<64><<<grid, block, sm, st>>>(m->L, m->d_tab, m->d_itab, y, P, n, f);
  }
  KIN_CUDA_TRY(cudaGetLastError());
  return KIN_OK;
}

extern "C" int kin_jacobian(kin_mech *m, const double *y, const double *P, int64_t n, int32_t fd,
                            double h, const double *scal, double *J, void *stream) {
  if (!m || n < 0 || (n > 0 && (!y || !P || !J)) || (fd && !scal)) return KIN_ERR_INVALID_ARG;
  if (n == 0) return KIN_OK;
  cudaStream_t st = (cudaStream_t)stream;
  const size_t sm = smem_bytes(m->L);
  const int block = 64;
  const unsigned grid = (unsigned)((n + block - 1) / block);
  if (m->L.ns <= 16) {
    KIN_CUDA_TRY(cudaFuncSetAttribute(k_jac<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    k_jac<16><<<grid, block, sm, st>>>(m->L, m->d_tab, m->d_itab, y, P, n, fd, h, scal, J);
  } else {
    KIN_CUDA_TRY(cudaFuncSetAttribute(k_jac<64>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    k_jac<64><<<grid, block, sm, st>>>(m->L, m->d_tab, m->d_itab, y, P, n, fd, h, scal, J);
  }
  KIN_CUDA_TRY(cudaGetLastError());
  return KIN_OK;
}

extern "C" int kin_exp(kin_mech *m, const double *x, double *y, int64_t n, void *stream) {
  if (!m || n < 0 || (n > 0 && (!x || !y))) return KIN_ERR_INVALID_ARG;
  if (n == 0) return KIN_OK;
  const int block = 256;
  k_exp<<<(unsigned)((n + block - 1) / block), block, 0, (cudaStream_t)stream>>>(
      m->d_tab + m->L.dexp, x, y, n);
  KIN_CUDA_TRY(cudaGetLastError());
  return KIN_OK;
}

extern "C" int kin_autotune(kin_mech *m, const double *Y, const double *T, const double *P,
                            int64_t n, double dt, double rtol, double atol, const kin_options *base,
                            kin_options *best, double *seconds, int32_t max_candidates,
                            void *stream) {
  int rc = check_common(m, Y, T, P, n, dt, rtol, atol);
  if (rc) return rc;
  if (!best || n < 1 || max_candidates < 1) return KIN_ERR_INVALID_ARG;
  kin_options b;
  if (base) {
    b = *base;
  } else {
    kin_options_default(&b);
  }
  if (b.h0 || b.z0 || b.h_first || b.z_first) return KIN_ERR_INVALID_ARG;
  struct Cand {
    int layout, block, refill, lanes;
  };
  // thread layouts only while the per-thread matrices stay on chip (N <= 16);
  // beyond that a state per warp is the one layout that fits
  const Cand small[] = {{KIN_LAYOUT_PLAIN, 64, 0, 0}, {KIN_LAYOUT_PLAIN, 32, 0, 0},
                        {KIN_LAYOUT_QUEUE, 64, 1, 0}, {KIN_LAYOUT_QUEUE, 64, 4, 0},
                        {KIN_LAYOUT_QUEUE, 64, 8, 0}, {KIN_LAYOUT_QUEUE, 64, 16, 0},
                        {KIN_LAYOUT_QUEUE, 64, 32, 0}, {KIN_LAYOUT_QUEUE, 32, 1, 0},
                        {KIN_LAYOUT_WARP, 0, 0, 32}, {KIN_LAYOUT_WARP, 0, 0, 16},
                        {KIN_LAYOUT_WARP, 0, 0, 8}, {KIN_LAYOUT_WARP, 0, 0, 4}};
  const Cand large[] = {{KIN_LAYOUT_WARP, 0, 0, 32}};
  const bool is_small = m->L.ns <= 16;
  const Cand *cands = is_small ? small : large;
  const int ncand = !is_small ? 1 : (m->L.ns <= 15 ? 12 : 9);
  const int nc = ncand < max_candidates ? ncand : max_candidates;
  if (nc == 1) {
    *best = b;
    best->layout = cands[0].layout;
    best->block = cands[0].block;
    best->queue_refill = cands[0].refill;
    best->lanes = cands[0].lanes;
    remember_tuning(m, n, dt, *best);
    return KIN_OK;
  }
  cudaStream_t st = (cudaStream_t)stream;
  const int ns = m->L.ns;
  double *y = nullptr, *t = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int best_i = -1;
  float best_ms = 0.0f;
  auto cleanup = [&]() {
    cudaFree(y);
    cudaFree(t);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
  };
  if (cudaMalloc(&y, sizeof(double) * n * ns) != cudaSuccess ||
      cudaMalloc(&t, sizeof(double) * n) != cudaSuccess ||
      cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    (void)cudaGetLastError();
    cleanup();
    return KIN_ERR_NOMEM;
  }
  // the first candidate runs twice: the first launch also pays one-time costs
  float prev_group_ms = -1.0f;  // the last WARP candidate's time
  for (int run = -1; run < nc; ++run) {
    const Cand &c = cands[run < 0 ? 0 : run];
    // smaller lane groups only pay when the larger one came close: stop
    // timing them once a WARP candidate ran over twice the best time
    if (run >= 0 && c.layout == KIN_LAYOUT_WARP && prev_group_ms > 2.0f * best_ms) {
      if (seconds) seconds[run] = -1.0;
      continue;
    }
    kin_options o = b;
    o.layout = c.layout;
    o.block = c.block;
    o.queue_refill = c.refill;
    o.lanes = c.lanes;
    if (cudaMemcpyAsync(y, Y, sizeof(double) * n * ns, cudaMemcpyDeviceToDevice, st) !=
            cudaSuccess ||
        cudaMemcpyAsync(t, T, sizeof(double) * n, cudaMemcpyDeviceToDevice, st) != cudaSuccess ||
        cudaEventRecord(e0, st) != cudaSuccess) {
      (void)cudaGetLastError();
      cleanup();
      return KIN_ERR_CUDA;
    }
    rc = kin_integrate_ex(m, y, t, P, n, dt, rtol, atol, &o, nullptr, nullptr, stream);
    float ms = 0.0f;
    if (rc || cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
        cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
      (void)cudaGetLastError();
      cleanup();
      return rc ? rc : KIN_ERR_CUDA;
    }
    if (run < 0) continue;
    if (c.layout == KIN_LAYOUT_WARP) prev_group_ms = ms;
    if (seconds) seconds[run] = ms * 1e-3;
    if (best_i < 0 || ms < best_ms) {
      best_i = run;
      best_ms = ms;
    }
  }
  cleanup();
  *best = b;
  best->layout = cands[best_i].layout;
  best->block = cands[best_i].block;
  best->queue_refill = cands[best_i].refill;
  best->lanes = cands[best_i].lanes;
  remember_tuning(m, n, dt, *best);
  return KIN_OK;
}
