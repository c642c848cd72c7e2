// Concentration-based reactor with a sparse LU (kin_conc_* of the C ABI):
// the host's symbolic analysis, the state-per-group kernel and its launch.
// The reformulation is the one the paper proposes for large models (Sec. 3.3,
// Sec. 4); kin_conc.cuh has the device side and the equations.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

#include "../../include/kin.h"
#include "kin_conc.cuh"
#include "kin_internal.h"

using namespace kin;

namespace {

// Structure of the Newton matrices of the concentration-based form and its
// elimination: phi = [T, V, n_0 .. n_{ns-2}]; element g of the group's
// vectors holds phi[var[g]].
struct ConcStructure {
  int N = 0;
  int k0 = 0;                 // pivots k0 .. N-1 form a full trailing block
  std::vector<int> var;       // [N] element -> phi index
  std::vector<uint8_t> pat;   // [N*N] filled L + U pattern in element order
  std::vector<int> lp, li, up, uj, cp, ci;
  int64_t nnz_J = 0, nnz_LU = 0;
};

// The pattern of J in phi order: full T and V rows and columns, the
// diagonal, and species pairs that share a reaction or where one is a
// collider with a non-default efficiency in a reaction of the other.
int conc_pattern(const kin_mech_desc *d, std::vector<uint8_t> &A) {
  if (!d || !d->reac || !d->prod || !d->rtype || !d->eff) return KIN_ERR_INVALID_ARG;
  const int ns = d->ns, nr = d->nr, in = ns - 1, N = ns + 1;
  if (ns < 2 || ns > KIN_MAX_SPECIES || nr < 1) return KIN_ERR_INVALID_ARG;
  A.assign((size_t)N * N, 0);
  for (int i = 0; i < N; ++i) {
    A[(size_t)i * N + i] = 1;
    A[(size_t)0 * N + i] = A[(size_t)1 * N + i] = 1;
    A[(size_t)i * N + 0] = A[(size_t)i * N + 1] = 1;
  }
  for (int i = 0; i < nr; ++i) {
    int sp[6], np = 0;
    for (int s = 0; s < 3; ++s) {
      const int r = d->reac[3 * i + s], p = d->prod[3 * i + s];
      if (r < -1 || r >= ns || p < -1 || p >= ns || r == in || p == in) return KIN_ERR_MECH;
      if (r >= 0) sp[np++] = r;
      if (p >= 0) sp[np++] = p;
    }
    std::vector<int> cols(sp, sp + np);
    if (d->rtype[i] != 0) {
      // the bath gas's concentration follows from the others: its efficiency
      // must be the default for the coupling to stay sparse
      if (d->eff[(size_t)i * ns + in] != 1.0) return KIN_ERR_UNSUPPORTED;
      for (int k = 0; k < in; ++k)
        if (d->eff[(size_t)i * ns + k] != 1.0) cols.push_back(k);
    }
    for (int a = 0; a < np; ++a)
      for (int c : cols) A[(size_t)(2 + sp[a]) * N + 2 + c] = 1;
  }
  return KIN_OK;
}

int conc_analyse(const kin_mech_desc *d, ConcStructure &S) {
  std::vector<uint8_t> A;
  int rc = conc_pattern(d, A);
  if (rc) return rc;
  const int ns = d->ns, N = ns + 1, m = ns - 1;
  S = ConcStructure{};
  S.N = N;
  for (uint8_t x : A) S.nnz_J += x;
  // minimum degree on the species block's symmetric structure (T and V
  // touch every species and go last); ties to the lowest index
  std::vector<uint64_t> adj(m, 0);
  for (int a = 0; a < m; ++a)
    for (int c = 0; c < m; ++c)
      if (a != c && (A[(size_t)(2 + a) * N + 2 + c] || A[(size_t)(2 + c) * N + 2 + a]))
        adj[a] |= 1ull << c;
  uint64_t alive = (m == 64) ? ~0ull : ((1ull << m) - 1ull);
  for (int step = 0; step < m; ++step) {
    int best = -1, bd = 1 << 30;
    for (int a = 0; a < m; ++a) {
      if (!((alive >> a) & 1ull)) continue;
      const int deg = __builtin_popcountll(adj[a] & alive);
      if (deg < bd) {
        bd = deg;
        best = a;
      }
    }
    const uint64_t nb = adj[best] & alive & ~(1ull << best);
    for (int c = 0; c < m; ++c)
      if ((nb >> c) & 1ull) adj[c] |= nb & ~(1ull << c);
    alive &= ~(1ull << best);
    S.var.push_back(2 + best);
  }
  S.var.push_back(0);
  S.var.push_back(1);
  // filled pattern in element order (no pivoting: the fill of Gaussian
  // elimination in this order)
  std::vector<uint8_t> &P = S.pat;
  P.assign((size_t)N * N, 0);
  for (int g = 0; g < N; ++g)
    for (int h = 0; h < N; ++h) P[(size_t)g * N + h] = A[(size_t)S.var[g] * N + S.var[h]];
  for (int k = 0; k < N; ++k)
    for (int i = k + 1; i < N; ++i) {
      if (!P[(size_t)i * N + k]) continue;
      for (int j = k + 1; j < N; ++j)
        if (P[(size_t)k * N + j]) P[(size_t)i * N + j] = 1;
    }
  for (uint8_t x : P) S.nnz_LU += x;
  S.lp.assign(1, 0);
  S.up.assign(1, 0);
  S.cp.assign(1, 0);
  for (int k = 0; k < N; ++k) {
    for (int i = k + 1; i < N; ++i)
      if (P[(size_t)i * N + k]) S.li.push_back(i);
    for (int j = k + 1; j < N; ++j)
      if (P[(size_t)k * N + j]) S.uj.push_back(j);
    for (int i = 0; i < k; ++i)
      if (P[(size_t)i * N + k]) S.ci.push_back(i);
    S.lp.push_back((int)S.li.size());
    S.up.push_back((int)S.uj.size());
    S.cp.push_back((int)S.ci.size());
  }
  S.k0 = N;
  for (int k = N - 1; k >= 0; --k) {
    const int l = S.lp[k + 1] - S.lp[k], u = S.up[k + 1] - S.up[k];
    if (l != N - 1 - k || u != N - 1 - k) break;
    S.k0 = k;
  }
  return KIN_OK;
}

// Operations of one real factorisation and one real solve over the pattern:
// per pivot a division and |L_k| multiplications, 2 |L_k| |U_k| for the
// update; per solve 2 per off-diagonal entry of L and U and N divisions.
void conc_counts(const ConcStructure &S, int64_t *out) {
  int64_t lu = 0, sol = S.N;
  for (int k = 0; k < S.N; ++k) {
    const int64_t l = S.lp[k + 1] - S.lp[k], u = S.up[k + 1] - S.up[k];
    lu += 1 + l + 2 * l * u;
    sol += 2 * l + 2 * (S.cp[k + 1] - S.cp[k]);
  }
  out[0] = S.nnz_J;
  out[1] = S.nnz_LU;
  out[2] = lu;
  out[3] = sol;
}

// offsets into the device int table: var | posn | lp | li | up | uj | cp | ci
struct ConcArgs {
  KernelArgs a;
  int N, k0, posT, posV;
  const int *ctab;
  const double *aw;
  int o_posn, o_lp, o_li, o_up, o_uj, o_cp, o_ci;
};

template <int L, typename LT>
__global__ void __launch_bounds__(256) k_integrate_conc(ConcArgs ca) {
  using G = Grp<L>;
  constexpr int WR = G::WR;
  extern __shared__ double smem[];
  const KernelArgs &a = ca.a;
  const MechView m = make_view(a.L, a.tab, a.itab);
  ConcView cv;
  cv.N = ca.N;
  cv.k0 = ca.k0;
  cv.posT = ca.posT;
  cv.posV = ca.posV;
  cv.var = ca.ctab;
  cv.posn = ca.ctab + ca.o_posn;
  cv.lp = ca.ctab + ca.o_lp;
  cv.li = ca.ctab + ca.o_li;
  cv.up = ca.ctab + ca.o_up;
  cv.uj = ca.ctab + ca.o_uj;
  cv.cp = ca.ctab + ca.o_cp;
  cv.ci = ca.ctab + ca.o_ci;
  cv.aw = ca.aw;
  const int N = cv.N, ns = m.ns, in = ns - 1, lane = G::lane(), grp = (int)(threadIdx.x / L);
  const int64_t n = a.rp.n;
  char *base = reinterpret_cast<char *>(smem) + (size_t)grp * warp_buf_bytes(N, m.nr, sizeof(LT));
  const int64_t slot = (int64_t)blockIdx.x * (blockDim.x / L) + grp;  // < gslots (launch)
  LT *Jg = reinterpret_cast<LT *>(a.gscratch) +
           slot * (int64_t)warp_slot_mats(sizeof(LT)) * N * (N + 1);
  const WarpBuf<LT> b = carve_warp_buf<LT>(base, N, m.nr, Jg);
  const ConcSys<L, LT> sys{&m, &cv};
  unsigned long long *queue = a.totals + 9;
  WStateT<WR> w;
  StepState s;
  for (;;) {
    unsigned long long t = 0;
    if (lane == 0) t = atomicAdd(queue, 1ull);
    t = G::bcast(t, 0);
    if (t >= (unsigned long long)n) break;
    int64_t idx = 0;
    if (lane == 0) idx = state_of(a, (int64_t)t);
    idx = G::bcast(idx, 0);
    if (idx < 0) continue;
    const double P = a.P[idx], T0 = a.T[idx];
    // phi per unit mass: n_k = Y_k / W_k, V = Ru T sum_k (Y_k / W_k) / P
    double sS = 0.0;
#pragma unroll
    for (int r = 0; r < WR; ++r) {
      const int k = lane + L * r;
      if (k < ns) sS += a.Y[(int64_t)k * n + idx] * m.invW[k];
    }
    sS = G::sum(sS);
#pragma unroll
    for (int r = 0; r < WR; ++r) {
      const int g = lane + L * r;
      const int v = g < N ? cv.var[g] : -1;
      w.y.v[r] = (v == 0)   ? T0
                 : (v == 1) ? RU * T0 * sS / P
                 : (v >= 2) ? a.Y[(int64_t)(v - 2) * n + idx] * m.invW[v - 2]
                            : 0.0;
    }
    // every attempt ends the loop or counts a step; max_steps bounds it
    bool done = warp_init_sys<L, LT, false>(sys, b, P, w, s, a.rp, idx);
    while (!done) done = warp_step_sys<L, LT, false>(sys, b, P, w, s, a.rp, idx);
    // back to mass fractions: the bath gas's moles close P V = n Ru T; Y_k is
    // W_k n_k over the mixture's mass
    const double T1 = elem<L>(w.y, cv.posT), V1 = elem<L>(w.y, cv.posV);
    double sn = 0.0, sm = 0.0;
#pragma unroll
    for (int r = 0; r < WR; ++r) {
      const int g = lane + L * r;
      const int v = g < N ? cv.var[g] : -1;
      if (v >= 2) {
        sn += w.y.v[r];
        sm += m.W[v - 2] * w.y.v[r];
      }
    }
    sn = G::sum(sn);
    sm = G::sum(sm);
    const double nin = P * V1 / (RU * T1) - sn;
    const double imass = 1.0 / (sm + m.W[in] * nin);
#pragma unroll
    for (int r = 0; r < WR; ++r) {
      const int g = lane + L * r;
      const int v = g < N ? cv.var[g] : -1;
      if (v >= 2) a.Y[(int64_t)(v - 2) * n + idx] = m.W[v - 2] * w.y.v[r] * imass;
    }
    if (lane == 0) {
      a.T[idx] = T1;
      a.Y[(int64_t)in * n + idx] = m.W[in] * nin * imass;
      if (a.status) a.status[idx] = s.status;
      if (a.counters) {
        const int32_t c[8] = {s.nstep, s.naccpt, s.nrejct, s.nfcn, s.njac, s.ndec, s.nsol,
                              s.status};
        for (int q = 0; q < 8; ++q) a.counters[(int64_t)q * n + idx] = c[q];
      }
      const unsigned long long c7[7] = {
          (unsigned long long)s.nstep, (unsigned long long)s.naccpt, (unsigned long long)s.nrejct,
          (unsigned long long)s.nfcn,  (unsigned long long)s.njac,   (unsigned long long)s.ndec,
          (unsigned long long)s.nsol};
      for (int q = 0; q < 7; ++q) atomicAdd(a.totals + q, c7[q]);
      if (s.status) atomicAdd(a.totals + 7, 1ull);
      atomicMax(a.totals + 8, (unsigned long long)s.nstep);
    }
    G::sync();
  }
}

template <int L, typename LT>
int launch_conc(const ConcArgs &ca, cudaStream_t st, int sms) {
  using G = Grp<L>;
  const KernelArgs &a = ca.a;
  if (ca.N > G::CAP) return KIN_ERR_UNSUPPORTED;
  if (!a.gscratch || a.gslots < 1) return KIN_ERR_UNSUPPORTED;
  const size_t budget = 227 * 1024, per_grp = warp_buf_bytes(ca.N, a.L.nr, sizeof(LT));
  auto kern = k_integrate_conc<L, LT>;
  // the block size (1 to 8 warps) that keeps the most warps resident per SM
  int warps = 0, per_sm = 0;
  for (int wp = 8; wp >= 1; wp >>= 1) {
    const size_t smw = (size_t)wp * (32 / L) * per_grp;
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
  const size_t sm = (size_t)warps * (32 / L) * per_grp;
  KIN_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
  int64_t grid = (int64_t)sms * per_sm;
  const int64_t per_block = (int64_t)warps * (32 / L);
  const int64_t need = (a.rp.n + per_block - 1) / per_block;
  if (grid > need) grid = need;
  if (grid * per_block > a.gslots) grid = a.gslots / per_block;  // one J slot per group
  if (grid < 1) return KIN_ERR_UNSUPPORTED;
  kern<<<(unsigned)grid, 32 * warps, sm, st>>>(ca);
  KIN_CUDA_TRY(cudaGetLastError());
  return KIN_OK;
}

}  // namespace

struct kin_conc {
  int device = 0;
  MechLayout L;
  ConcStructure S;
  double *d_tab = nullptr;
  int *d_itab = nullptr;
  int *d_ctab = nullptr;
  double *d_aw = nullptr;  // [N] factor on atol per element
  int o_posn = 0, o_lp = 0, o_li = 0, o_up = 0, o_uj = 0, o_cp = 0, o_ci = 0;
  unsigned long long *d_totals = nullptr;
  void *d_gscratch = nullptr;
  int64_t gslots = 0;
  cudaStream_t last_stream = nullptr;
};

extern "C" int kin_conc_analyse(const kin_mech_desc *desc, int32_t *var, uint8_t *pattern,
                                int64_t *counts) {
  if (!desc) return KIN_ERR_INVALID_ARG;
  ConcStructure S;
  const int rc = conc_analyse(desc, S);
  if (rc) return rc;
  if (var)
    for (int g = 0; g < S.N; ++g) var[g] = S.var[g];
  if (pattern) std::memcpy(pattern, S.pat.data(), S.pat.size());
  if (counts) conc_counts(S, counts);
  return KIN_OK;
}

extern "C" void kin_conc_destroy(kin_conc *c) {
  if (!c) return;
  cudaFree(c->d_tab);
  cudaFree(c->d_itab);
  cudaFree(c->d_ctab);
  cudaFree(c->d_aw);
  cudaFree(c->d_totals);
  cudaFree(c->d_gscratch);
  delete c;
}

extern "C" int kin_conc_create(const kin_mech_desc *desc, kin_conc **out) {
  if (!desc || !out) return KIN_ERR_INVALID_ARG;
  *out = nullptr;
  MechLayout L;
  std::vector<double> dt;
  std::vector<int> it;
  int rc = build_tables(desc, L, dt, it);
  if (rc) return rc;
  ConcStructure S;
  rc = conc_analyse(desc, S);
  if (rc) return rc;
  if (S.N > Grp<32>::CAP) return KIN_ERR_UNSUPPORTED;
  // the Radau constants of this translation unit's kernels, from the same
  // closed forms as every other kernel's
  double k[27];
  rc = kin_radau_constants(k, 27);
  if (rc) return rc;
  RadauConst rk{};
  rk.c1 = k[0];
  rk.c2 = k[1];
  rk.gam = k[3];
  rk.alp = k[4];
  rk.bet = k[5];
  for (int i = 0; i < 9; ++i) rk.T[i] = k[6 + i];
  for (int i = 0; i < 9; ++i) rk.TI[i] = k[15 + i];
  for (int i = 0; i < 3; ++i) rk.d[i] = k[24 + i];
  rk.ic1 = 1.0 / rk.c1;
  rk.ic2 = 1.0 / rk.c2;
  rk.ic1m1 = 1.0 / (rk.c1 - 1.0);
  rk.ic2m1 = 1.0 / (rk.c2 - 1.0);
  rk.ic1mc2 = 1.0 / (rk.c1 - rk.c2);
  KIN_CUDA_TRY(cudaMemcpyToSymbol(RC, &rk, sizeof rk));
  // device int table: var | posn | lp | li | up | uj | cp | ci
  const int N = S.N, ns = desc->ns;
  std::vector<int> ct(S.var.begin(), S.var.end());
  kin_conc *c = new kin_conc();
  c->o_posn = (int)ct.size();
  ct.resize(ct.size() + (ns - 1));
  for (int g = 0; g < N; ++g)
    if (S.var[g] >= 2) ct[c->o_posn + S.var[g] - 2] = g;
  auto append = [&](const std::vector<int> &v) {
    const int o = (int)ct.size();
    ct.insert(ct.end(), v.begin(), v.end());
    if (v.empty()) ct.push_back(0);
    return o;
  };
  c->o_lp = append(S.lp);
  c->o_li = append(S.li);
  c->o_up = append(S.up);
  c->o_uj = append(S.uj);
  c->o_cp = append(S.cp);
  c->o_ci = append(S.ci);
  c->L = L;
  c->S = S;
  // the moles' absolute tolerance is atol / W_k (T and V: atol)
  std::vector<double> aw(N, 1.0);
  for (int g = 0; g < N; ++g)
    if (S.var[g] >= 2) aw[g] = 1.0 / desc->W[S.var[g] - 2];
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    (void)cudaGetLastError();
    delete c;
    return KIN_ERR_CUDA;
  }
  c->device = dev;
  // one Jacobian slot (with the complex matrix when that is global) per
  // resident warp: at most 16 whole-warp groups per SM
  c->gslots = (int64_t)sms * 16;
  const size_t gbytes =
      (size_t)c->gslots * warp_slot_mats(sizeof(double)) * N * (N + 1) * sizeof(double);
  if (cudaMalloc(&c->d_tab, sizeof(double) * L.nd) != cudaSuccess ||
      cudaMalloc(&c->d_itab, sizeof(int) * L.ni) != cudaSuccess ||
      cudaMalloc(&c->d_ctab, sizeof(int) * ct.size()) != cudaSuccess ||
      cudaMalloc(&c->d_aw, sizeof(double) * N) != cudaSuccess ||
      cudaMalloc(&c->d_totals, sizeof(unsigned long long) * 16) != cudaSuccess ||
      cudaMalloc(&c->d_gscratch, gbytes) != cudaSuccess) {
    (void)cudaGetLastError();
    kin_conc_destroy(c);
    return KIN_ERR_NOMEM;
  }
  if (cudaMemcpy(c->d_tab, dt.data(), sizeof(double) * L.nd, cudaMemcpyHostToDevice) !=
          cudaSuccess ||
      cudaMemcpy(c->d_itab, it.data(), sizeof(int) * L.ni, cudaMemcpyHostToDevice) !=
          cudaSuccess ||
      cudaMemcpy(c->d_ctab, ct.data(), sizeof(int) * ct.size(), cudaMemcpyHostToDevice) !=
          cudaSuccess ||
      cudaMemcpy(c->d_aw, aw.data(), sizeof(double) * N, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemset(c->d_totals, 0, sizeof(unsigned long long) * 16) != cudaSuccess) {
    (void)cudaGetLastError();
    kin_conc_destroy(c);
    return KIN_ERR_CUDA;
  }
  *out = c;
  return KIN_OK;
}

extern "C" int kin_integrate_conc(kin_conc *c, double *Y, double *T, const double *P, int64_t n,
                                  double dt, double rtol, double atol, const kin_options *opt,
                                  int32_t *status, int32_t *counters, void *stream) {
  if (!c || n < 0) return KIN_ERR_INVALID_ARG;
  if (n > 0 && (!Y || !T || !P)) return KIN_ERR_INVALID_ARG;
  if (!(dt > 0.0) || !(rtol > 0.0) || !(atol > 0.0) || !std::isfinite(dt))
    return KIN_ERR_INVALID_ARG;
  kin_options o;
  if (opt) {
    o = *opt;
  } else {
    kin_options_default(&o);
  }
  if (o.layout != KIN_LAYOUT_WARP && o.layout != KIN_LAYOUT_AUTO) return KIN_ERR_UNSUPPORTED;
  if (o.lanes != 0 && o.lanes != 32) return KIN_ERR_UNSUPPORTED;
  if (o.jac_fd || o.h_fixed != 0.0 || o.z0 || o.z_first) return KIN_ERR_UNSUPPORTED;
  if (o.nit < 1 || o.nit > 50 || o.max_steps < 1 || o.stop_after < 0) return KIN_ERR_INVALID_ARG;
  if (o.order && n > INT32_MAX) return KIN_ERR_INVALID_ARG;
  if (o.order_by != 0) return KIN_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  c->last_stream = st;
  KIN_CUDA_TRY(cudaMemsetAsync(c->d_totals, 0, sizeof(unsigned long long) * 16, st));
  if (n == 0) return KIN_OK;
  int dev = 0, sms = 0;
  KIN_CUDA_TRY(cudaGetDevice(&dev));
  if (dev != c->device) return KIN_ERR_INVALID_ARG;
  KIN_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  ConcArgs ca;
  KernelArgs &a = ca.a;
  a.L = c->L;
  a.tab = c->d_tab;
  a.itab = c->d_itab;
  a.Y = Y;
  a.T = T;
  a.P = P;
  a.status = status;
  a.counters = counters;
  a.totals = c->d_totals;
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
  a.rp.z0 = nullptr;
  a.rp.h_first = o.h_first;
  a.rp.z_first = nullptr;
  a.rp.stop_after = o.stop_after;
  a.rp.hfixed = 0.0;
  a.refill_min = 1;
  a.order = o.order;
  a.gscratch = c->d_gscratch;
  a.gslots = c->gslots;
  ca.N = c->S.N;
  ca.k0 = c->S.k0;
  ca.posT = ca.posV = -1;
  for (int g = 0; g < ca.N; ++g) {
    if (c->S.var[g] == 0) ca.posT = g;
    if (c->S.var[g] == 1) ca.posV = g;
  }
  ca.ctab = c->d_ctab;
  ca.aw = c->d_aw;
  ca.o_posn = c->o_posn;
  ca.o_lp = c->o_lp;
  ca.o_li = c->o_li;
  ca.o_up = c->o_up;
  ca.o_uj = c->o_uj;
  ca.o_cp = c->o_cp;
  ca.o_ci = c->o_ci;
  return o.lu_fp32 ? launch_conc<32, float>(ca, st, sms) : launch_conc<32, double>(ca, st, sms);
}

extern "C" int kin_conc_get_stats(kin_conc *c, int64_t *out) {
  if (!c || !out) return KIN_ERR_INVALID_ARG;
  unsigned long long t[16];
  KIN_CUDA_TRY(cudaStreamSynchronize(c->last_stream));
  KIN_CUDA_TRY(cudaMemcpy(t, c->d_totals, sizeof t, cudaMemcpyDeviceToHost));
  for (int i = 0; i < 9; ++i) out[i] = (int64_t)t[i];
  if (t[10] > 0) return KIN_ERR_INVALID_ARG;
  return out[7] > 0 ? KIN_ERR_STATE_FAILED : KIN_OK;
}
