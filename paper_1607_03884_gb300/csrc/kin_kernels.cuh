// Integration kernels (PLAIN and QUEUE layouts) and their launch helper,
// instantiated per (species capacity, matrix precision) in the kin_tu_*.cu
// translation units so that the library compiles in parallel.
#pragma once
#include <cuda_runtime.h>

#include "../../include/kin.h"
#include "kin_radau.cuh"
#include "kin_warp.cuh"

namespace kin {

#define KIN_CUDA_TRY(expr)                                                    \
  do {                                                                        \
    cudaError_t e_ = (expr);                                                  \
    if (e_ != cudaSuccess) {                                                  \
      (void)cudaGetLastError();                                               \
      return e_ == cudaErrorMemoryAllocation ? KIN_ERR_NOMEM : KIN_ERR_CUDA; \
    }                                                                         \
  } while (0)

__host__ __device__ inline size_t smem_bytes(const MechLayout &L) {
  return sizeof(double) * (size_t)L.nd + sizeof(int) * (size_t)L.ni;
}

// Species capacity of the small-mechanism thread kernels: the per-thread
// workspace is sized for it (a smaller one spills less).
#ifndef KIN_SMALL_MAXN
#define KIN_SMALL_MAXN 16
#endif
constexpr int SMALL_MAXN = KIN_SMALL_MAXN;

struct KernelArgs {
  MechLayout L;
  const double *tab;
  const int *itab;
  double *Y, *T;
  const double *P;
  int32_t *status, *counters;
  unsigned long long *totals;
  RadauParams rp;
  int refill_min;        // QUEUE: idle lanes of a warp that trigger a refill
  const int32_t *order;  // slot -> state permutation or null (identity)
  void *gscratch;        // WARP: per-group Jacobian slots (N x (N+1) doubles each)
  int64_t gslots;        // number of slots in gscratch
};

// The state a slot carries: order[slot] when an order is given, else the
// slot itself.  Entries outside [0, n) are skipped (-1) and counted in
// totals[10], so a bad permutation cannot reach memory out of bounds.
__device__ __forceinline__ int64_t state_of(const KernelArgs &a, int64_t slot) {
  if (!a.order) return slot;
  const int32_t s = a.order[slot];
  if (s < 0 || (int64_t)s >= a.rp.n) {
    atomicAdd(a.totals + 10, 1ull);
    return -1;
  }
  return (int64_t)s;
}

template <int MAXN, typename LT>
__device__ void load_state(Work<MAXN, LT> &w, const KernelArgs &a, int N, int64_t i) {
  const int64_t n = a.rp.n;
  w.y[0] = a.T[i];
  for (int k = 0; k < N - 1; ++k) w.y[1 + k] = a.Y[(int64_t)k * n + i];
}

template <int MAXN, typename LT>
__device__ void store_state(const Work<MAXN, LT> &w, const StepState &s, const KernelArgs &a,
                            int N, int64_t i) {
  const int64_t n = a.rp.n;
  a.T[i] = w.y[0];
  double sum = 0.0;
  for (int k = 0; k < N - 1; ++k) {
    a.Y[(int64_t)k * n + i] = w.y[1 + k];
    sum += w.y[1 + k];
  }
  a.Y[(int64_t)(N - 1) * n + i] = 1.0 - sum;
  if (a.status) a.status[i] = s.status;
  if (a.counters) {
    const int32_t c[8] = {s.nstep, s.naccpt, s.nrejct, s.nfcn, s.njac, s.ndec, s.nsol, s.status};
    for (int q = 0; q < 8; ++q) a.counters[(int64_t)q * n + i] = c[q];
  }
  const unsigned long long c7[7] = {(unsigned long long)s.nstep, (unsigned long long)s.naccpt,
                                    (unsigned long long)s.nrejct, (unsigned long long)s.nfcn,
                                    (unsigned long long)s.njac, (unsigned long long)s.ndec,
                                    (unsigned long long)s.nsol};
  for (int q = 0; q < 7; ++q) atomicAdd(a.totals + q, c7[q]);
  if (s.status) atomicAdd(a.totals + 7, 1ull);
  atomicMax(a.totals + 8, (unsigned long long)s.nstep);
}

// Tuning of the thread layouts (measured on 2^18 H2 states; the per-thread
// workspace spills, so latency hiding matters more than spill volume):
//   * 64 threads per block and at least KIN_THREAD_MIN_BLOCKS resident blocks
//     per SM, which caps a thread's registers (20: 48 registers, 40 warps per
//     SM; 0 leaves the allocator free: 168 registers, 12 warps);
//   * the mechanism tables read through L1 rather than staged in shared
//     memory per block (-DKIN_THREAD_TABLES_SMEM stages them), with the
//     unified L1/shared memory split towards L1 (KIN_THREAD_CARVEOUT, percent
//     given to shared memory; -1 = driver default).
// Together: 144k -> 178k states/s (FP32 matrices) and 106k -> 131k (FP64).
#ifndef KIN_THREAD_MIN_BLOCKS
#define KIN_THREAD_MIN_BLOCKS 20
#endif
#if KIN_THREAD_MIN_BLOCKS > 0
#define KIN_THREAD_BOUNDS __launch_bounds__(64, KIN_THREAD_MIN_BLOCKS)
#else
#define KIN_THREAD_BOUNDS __launch_bounds__(64)
#endif
#ifndef KIN_THREAD_CARVEOUT
#define KIN_THREAD_CARVEOUT 0
#endif
#ifdef KIN_THREAD_TABLES_SMEM
#define KIN_THREAD_VIEW(a, smem) stage_tables((a).L, (a).tab, (a).itab, smem)
#else
#define KIN_THREAD_VIEW(a, smem) make_view((a).L, (a).tab, (a).itab)
#endif

// Dynamic shared memory of a thread-layout block: the staged tables (if any),
// then the right-hand side's shared scratch (if any), 8-byte aligned.
__host__ __device__ inline size_t thread_tables_bytes(const MechLayout &L) {
#ifdef KIN_THREAD_TABLES_SMEM
  return (smem_bytes(L) + 7) / 8 * 8;
#else
  (void)L;
  return 0;
#endif
}
template <int MAXN>
__host__ __device__ inline size_t thread_smem_bytes(const MechLayout &L, int block) {
#ifdef KIN_THREAD_SCRATCH_SMEM
  return thread_tables_bytes(L) + ChemScratchS<MAXN>::bytes(L.ns, block);
#else
  (void)block;
  return thread_tables_bytes(L);
#endif
}
template <int MAXN, typename LT>
__device__ __forceinline__ void bind_scratch(Work<MAXN, LT> &w, const KernelArgs &a, double *smem) {
#ifdef KIN_THREAD_SCRATCH_SMEM
  w.cs.bind(smem + thread_tables_bytes(a.L) / 8, a.L.ns);
#else
  (void)w;
  (void)a;
  (void)smem;
#endif
}

template <int MAXN, typename LT, bool FDJ>
__global__ void KIN_THREAD_BOUNDS k_integrate_plain(KernelArgs a) {
  extern __shared__ double smem[];
  const MechView m = KIN_THREAD_VIEW(a, smem);
  const int64_t slot = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (slot >= a.rp.n) return;
  const int64_t i = state_of(a, slot);
  if (i < 0) return;
  Work<MAXN, LT> w;
  bind_scratch(w, a, smem);
  StepState s;
  const int N = m.ns;
  load_state(w, a, N, i);
  integrate_plain<MAXN, LT, FDJ>(m, a.P[i], w, s, a.rp, i);
  store_state(w, s, a, N, i);
}

template <int MAXN, typename LT, bool FDJ>
__global__ void KIN_THREAD_BOUNDS k_integrate_queue(KernelArgs a) {
  extern __shared__ double smem[];
  const MechView m = KIN_THREAD_VIEW(a, smem);
  const int N = m.ns;
  const int64_t n = a.rp.n;
  const unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  unsigned long long *queue = a.totals + 9;
  Work<MAXN, LT> w;
  bind_scratch(w, a, smem);
  StepState s;
  int64_t idx = -1;
  double P = 0.0;
  bool exhausted = false;  // warp-uniform: the queue has no more states
  // One step attempt per trip for every lane that holds a state.  Idle lanes
  // wait until refill_min of the warp's lanes are idle, then take that many
  // states with one atomic, so refilled lanes start their integrations
  // together.  Every state ends after at most max_steps attempts, so the
  // warp's loop is bounded.
  for (;;) {
    const unsigned idle = __ballot_sync(FULL, idx < 0);
    if (exhausted && idle == FULL) break;
    const int nidle = __popc(idle);
    if (!exhausted && nidle >= a.refill_min) {
      const int leader = __ffs(idle) - 1;
      unsigned long long base = 0;
      if (lane == leader) base = atomicAdd(queue, (unsigned long long)nidle);
      base = __shfl_sync(FULL, base, leader);
      if (base + (unsigned long long)nidle >= (unsigned long long)n) exhausted = true;
      if (idx < 0) {
        const unsigned long long t = base + __popc(idle & ((1u << lane) - 1u));
        if (t < (unsigned long long)n) idx = state_of(a, (int64_t)t);
        if (idx >= 0) {
          P = a.P[idx];
          load_state(w, a, N, idx);
          if (radau_init<MAXN, LT, FDJ>(m, P, w, s, a.rp, idx)) {
            store_state(w, s, a, N, idx);
            idx = -1;
          }
        }
      }
    }
    if (idx >= 0 && radau_step<MAXN, LT, FDJ>(m, P, w, s, a.rp, idx)) {
      store_state(w, s, a, N, idx);
      idx = -1;
    }
  }
}

// WARP layout: one state per group of L lanes; groups pop states from the
// atomic queue.
// Register cap of the WARP kernels (0: the compiler's choice under the
// 256-thread bound): a build-time tuning knob.
#ifndef KIN_WARP_MAXNREG
#define KIN_WARP_MAXNREG 0
#endif
#if KIN_WARP_MAXNREG > 0
#define KIN_WARP_BOUNDS __maxnreg__(KIN_WARP_MAXNREG)
#else
#define KIN_WARP_BOUNDS __launch_bounds__(256)
#endif

template <int L, typename LT, bool FDJ>
__global__ void KIN_WARP_BOUNDS k_integrate_lanes(KernelArgs a) {
  using G = Grp<L>;
  constexpr int WR = G::WR;
  extern __shared__ double smem[];
  // the mechanism tables are read through L1 from global memory: shared
  // memory holds only the groups' matrices and vectors
  const MechView m = make_view(a.L, a.tab, a.itab);
  const int N = m.ns, lane = G::lane(), grp = (int)(threadIdx.x / L);
  const int64_t n = a.rp.n;
  char *base = reinterpret_cast<char *>(smem) + (size_t)grp * warp_buf_bytes(N, m.nr, sizeof(LT));
  const int64_t slot = (int64_t)blockIdx.x * (blockDim.x / L) + grp;  // < gslots (launch)
  LT *Jg = reinterpret_cast<LT *>(a.gscratch) +
           slot * (int64_t)warp_slot_mats(sizeof(LT)) * N * (N + 1);
  const WarpBuf<LT> b = carve_warp_buf<LT>(base, N, m.nr, Jg);
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
    const double P = a.P[idx];
#pragma unroll
    for (int r = 0; r < WR; ++r) {
      const int g = lane + L * r;
      w.y.v[r] = (g == 0) ? a.T[idx] : (g < N ? a.Y[(int64_t)(g - 1) * n + idx] : 0.0);
    }
    // every attempt ends the loop or counts a step; max_steps bounds it
    bool done = warp_init<L, LT, FDJ>(m, b, P, w, s, a.rp, idx);
    while (!done) done = warp_step<L, LT, FDJ>(m, b, P, w, s, a.rp, idx);
    double sum = 0.0;
#pragma unroll
    for (int r = 0; r < WR; ++r) {
      const int g = lane + L * r;
      if (g == 0) a.T[idx] = w.y.v[r];
      if (g >= 1 && g < N) {
        a.Y[(int64_t)(g - 1) * n + idx] = w.y.v[r];
        sum += w.y.v[r];
      }
    }
    sum = G::sum(sum);
    if (lane == 0) {
      a.Y[(int64_t)(N - 1) * n + idx] = 1.0 - sum;
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

// Shared memory of one block of `warps` warps for L lanes per state.
__host__ __device__ inline size_t lanes_smem_bytes(const MechLayout &L_, int lanes, size_t lt,
                                                   int warps) {
  return (size_t)warps * (32 / lanes) * warp_buf_bytes(L_.ns, L_.nr, lt);
}

template <int L, typename LT, bool FDJ>
int launch_lanes(const KernelArgs &a, cudaStream_t st, int sms) {
  using G = Grp<L>;
  if (a.L.ns >= G::CAP) return KIN_ERR_UNSUPPORTED;
  if (!a.gscratch || a.gslots < 1) return KIN_ERR_UNSUPPORTED;
  const size_t budget = 227 * 1024;
  auto kern = k_integrate_lanes<L, LT, FDJ>;
  // the block size (1 to 8 warps) that keeps the most warps resident per SM
  int warps = 0, per_sm = 0;
  for (int w = 8; w >= 1; w >>= 1) {
    const size_t smw = lanes_smem_bytes(a.L, L, sizeof(LT), w);
    if (smw > budget) continue;
    KIN_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smw));
    int b = 0;
    KIN_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kern, 32 * w, smw));
    if (b * w > per_sm * warps) {
      warps = w;
      per_sm = b;
    }
  }
  if (warps < 1 || per_sm < 1) return KIN_ERR_UNSUPPORTED;
  const size_t sm = lanes_smem_bytes(a.L, L, sizeof(LT), warps);
  KIN_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
  int64_t grid = (int64_t)sms * per_sm;
  const int64_t per_block = (int64_t)warps * (32 / L);
  const int64_t need = (a.rp.n + per_block - 1) / per_block;
  if (grid > need) grid = need;
  if (grid * per_block > a.gslots) grid = a.gslots / per_block;  // one J slot per group
  if (grid < 1) return KIN_ERR_UNSUPPORTED;
  kern<<<(unsigned)grid, 32 * warps, sm, st>>>(a);
  KIN_CUDA_TRY(cudaGetLastError());
  return KIN_OK;
}

template <int MAXN, typename LT, bool FDJ>
int launch_t(const KernelArgs &a, const kin_options &o, cudaStream_t st, int sms) {
  if (o.layout == KIN_LAYOUT_WARP) {
    if constexpr (MAXN == 64) {
      if (a.L.ns > 63) return KIN_ERR_UNSUPPORTED;
      return launch_lanes<32, LT, FDJ>(a, st, sms);
    } else {
      return KIN_ERR_UNSUPPORTED;
    }
  }
  const int block = o.block > 0 ? o.block : 64;
  if (block > 64 || block % 32) return KIN_ERR_INVALID_ARG;
  const size_t sm = thread_smem_bytes<MAXN>(a.L, block);
  const int carve = KIN_THREAD_CARVEOUT;  // percent of the unified L1 given to shared memory
  if (o.layout == KIN_LAYOUT_PLAIN) {
    auto kern = k_integrate_plain<MAXN, LT, FDJ>;
    KIN_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    KIN_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, carve));
    const int64_t grid = (a.rp.n + block - 1) / block;
    kern<<<(unsigned)grid, block, sm, st>>>(a);
  } else {
    auto kern = k_integrate_queue<MAXN, LT, FDJ>;
    KIN_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    KIN_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, carve));
    int per_sm = o.grid_per_sm;
    if (per_sm <= 0) {
      KIN_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, block, sm));
      if (per_sm < 1) per_sm = 1;
    }
    int64_t grid = (int64_t)sms * per_sm;
    const int64_t need = (a.rp.n + block - 1) / block;
    if (grid > need) grid = need;
    kern<<<(unsigned)grid, block, sm, st>>>(a);
  }
  KIN_CUDA_TRY(cudaGetLastError());
  return KIN_OK;
}


// Per-TU entry points: launch for one (MAXN, LT) pair and upload this TU's
// copy of the Radau constants.
#define KIN_DEFINE_TU(NAME, MAXN, LT)                                                   \
  int kin_launch_##NAME(const KernelArgs &a, const kin_options &o, cudaStream_t st,    \
                        int sms) {                                                     \
    return o.jac_fd ? launch_t<MAXN, LT, true>(a, o, st, sms)                          \
                    : launch_t<MAXN, LT, false>(a, o, st, sms);                        \
  }                                                                                    \
  int kin_consts_##NAME(const RadauConst &rc) {                                        \
    KIN_CUDA_TRY(cudaMemcpyToSymbol(RC, &rc, sizeof rc));                              \
    return KIN_OK;                                                                     \
  }

#define KIN_DECLARE_TU(NAME)                                                            \
  int kin_launch_##NAME(const KernelArgs &a, const kin_options &o, cudaStream_t st,    \
                        int sms);                                                      \
  int kin_consts_##NAME(const RadauConst &rc);

// Groups of 4, 8 or 16 lanes per state (at most 15 species) for one matrix
// precision, in their own translation units.
#define KIN_DEFINE_GROUP_TU(NAME, LT)                                                   \
  int kin_launch_##NAME(const KernelArgs &a, const kin_options &o, cudaStream_t st,    \
                        int sms) {                                                     \
    const bool fd = o.jac_fd != 0;                                                     \
    switch (o.lanes) {                                                                 \
      case 4: return fd ? launch_lanes<4, LT, true>(a, st, sms)                        \
                        : launch_lanes<4, LT, false>(a, st, sms);                      \
      case 8: return fd ? launch_lanes<8, LT, true>(a, st, sms)                        \
                        : launch_lanes<8, LT, false>(a, st, sms);                      \
      case 16: return fd ? launch_lanes<16, LT, true>(a, st, sms)                      \
                         : launch_lanes<16, LT, false>(a, st, sms);                    \
      default: return KIN_ERR_INVALID_ARG;                                             \
    }                                                                                  \
  }                                                                                    \
  int kin_consts_##NAME(const RadauConst &rc) {                                        \
    KIN_CUDA_TRY(cudaMemcpyToSymbol(RC, &rc, sizeof rc));                              \
    return KIN_OK;                                                                     \
  }

KIN_DECLARE_TU(16d)
KIN_DECLARE_TU(16f)
KIN_DECLARE_TU(64d)
KIN_DECLARE_TU(64f)
KIN_DECLARE_TU(grpd)
KIN_DECLARE_TU(grpf)

}  // namespace kin
