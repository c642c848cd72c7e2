// Stiffness-ordered batching: a permutation of the states that puts states of
// similar stiffness next to each other, stiffest first.
//
// The paper names thread divergence from differing internal step counts as
// the main limiter of the per-thread integrator (Sec. 3.3, Sec. 4.2) and
// suggests grouping similar states.  The key is the natural logarithm of a
// first-step size: either the Hairer-Wanner starting-step heuristic
// (0.01 d0/d1 with d0 = ||y||, d1 = ||f(y)|| in the weighted RMS norm, one
// right-hand side per state) or a key the caller supplies (the predictor's
// h0, taken by its logarithm).  The permutation is a counting sort of the key into 4096
// equal-width bins between its minimum and maximum: min/max, histogram,
// exclusive scan, scatter.  The order inside a bin is not specified; the
// integration of a state does not depend on the slot that carries it.
#include "kin_internal.h"

namespace kin {

constexpr int ORDER_BINS = 4096;

// order-preserving map of finite doubles onto unsigned 64-bit integers
__device__ __forceinline__ unsigned long long key_bits(double k) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(k);
  return (u >> 63) ? ~u : (u | 0x8000000000000000ull);
}

__device__ __forceinline__ double bits_key(unsigned long long u) {
  const unsigned long long v = (u >> 63) ? (u & 0x7fffffffffffffffull) : ~u;
  return __longlong_as_double((long long)v);
}

template <int MAXN>
__global__ void k_order_key(MechLayout L, const double *tab, const int *itab, const double *Y,
                            const double *T, const double *P, int64_t n, double rtol,
                            double atol, double *key) {
  extern __shared__ double smem[];
  const MechView m = stage_tables(L, tab, itab, smem);
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int N = m.ns;
  double y[MAXN], f[MAXN];
  ChemScratch<MAXN> cs;
  JacScratch<MAXN, double> js;
  y[0] = T[i];
  for (int k = 0; k < N - 1; ++k) y[1 + k] = Y[(int64_t)k * n + i];
  const int bad = rhs<MAXN, double>(m, P[i], y, f, cs, js);
  double s0 = 0.0, s1 = 0.0;
  for (int k = 0; k < N; ++k) {
    const double sc = atol + rtol * fabs(y[k]);
    const double a = y[k] / sc, b = f[k] / sc;
    s0 += a * a;
    s1 += b * b;
  }
  const double d0 = sqrt(s0 / N), d1 = sqrt(s1 / N);
  const double h0 = (d0 < 1e-5 || d1 < 1e-5) ? 1e-6 : 0.01 * d0 / d1;
  key[i] = bad ? -INFINITY : log(h0);  // a state whose rates fail goes first
}

// ws: [0] min bits, [1] max bits (u64) of the finite keys, then ORDER_BINS
// u32 counts (cursors after the scan)
__global__ void k_order_init(unsigned long long *ws) {
  if (threadIdx.x == 0) {
    ws[0] = ~0ull;
    ws[1] = 0ull;
  }
  unsigned int *cnt = reinterpret_cast<unsigned int *>(ws + 2);
  for (int b = threadIdx.x; b < ORDER_BINS; b += blockDim.x) cnt[b] = 0u;
}

// the sort key of state i: the key itself, or its natural logarithm
__device__ __forceinline__ double key_at(const double *key, int64_t i, bool logk) {
  return logk ? log(key[i]) : key[i];  // log: 0 -> -inf (first), negative -> NaN (last)
}

__global__ void k_order_minmax(const double *key, bool logk, int64_t n, unsigned long long *ws) {
  unsigned long long lo = ~0ull, hi = 0ull;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double k = key_at(key, i, logk);
    if (!isfinite(k)) continue;
    const unsigned long long u = key_bits(k);
    lo = u < lo ? u : lo;
    hi = u > hi ? u : hi;
  }
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long a = __shfl_xor_sync(0xffffffffu, lo, o);
    const unsigned long long b = __shfl_xor_sync(0xffffffffu, hi, o);
    lo = a < lo ? a : lo;
    hi = b > hi ? b : hi;
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMin(ws, lo);
    atomicMax(ws + 1, hi);
  }
}

// -inf first; +inf and NaN last; finite keys in equal-width bins over [lo, hi]
__device__ __forceinline__ int order_bin(double k, double lo, double span) {
  if (k == -INFINITY) return 0;
  if (!isfinite(k)) return ORDER_BINS - 1;
  if (!(span > 0.0) || !isfinite(span)) return 0;  // one distinct finite key
  const double x = (k - lo) / span * ORDER_BINS;
  int b = x >= 0.0 ? (int)x : 0;
  return b < ORDER_BINS ? b : ORDER_BINS - 1;
}

__global__ void k_order_hist(const double *key, bool logk, int64_t n, unsigned long long *ws) {
  __shared__ unsigned int h[ORDER_BINS];
  for (int b = threadIdx.x; b < ORDER_BINS; b += blockDim.x) h[b] = 0u;
  __syncthreads();
  const double lo = bits_key(ws[0]), hi = bits_key(ws[1]);
  const double span = hi - lo;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    atomicAdd(&h[order_bin(key_at(key, i, logk), lo, span)], 1u);
  __syncthreads();
  unsigned int *cnt = reinterpret_cast<unsigned int *>(ws + 2);
  for (int b = threadIdx.x; b < ORDER_BINS; b += blockDim.x)
    if (h[b]) atomicAdd(&cnt[b], h[b]);
}

// exclusive scan of the bin counts in place (one block of 1024 threads)
__global__ void k_order_scan(unsigned long long *ws) {
  constexpr int PER = ORDER_BINS / 1024;
  __shared__ unsigned int part[1024];
  unsigned int *cnt = reinterpret_cast<unsigned int *>(ws + 2);
  const int t = threadIdx.x;
  unsigned int v[PER], s = 0u;
  for (int j = 0; j < PER; ++j) {
    v[j] = cnt[t * PER + j];
    s += v[j];
  }
  part[t] = s;
  __syncthreads();
  for (int o = 1; o < 1024; o <<= 1) {  // Hillis-Steele inclusive scan
    const unsigned int a = t >= o ? part[t - o] : 0u;
    __syncthreads();
    part[t] += a;
    __syncthreads();
  }
  unsigned int run = part[t] - s;
  for (int j = 0; j < PER; ++j) {
    cnt[t * PER + j] = run;
    run += v[j];
  }
}

__global__ void k_order_scatter(const double *key, bool logk, int64_t n,
                                unsigned long long *ws, int32_t *order) {
  const double lo = bits_key(ws[0]), hi = bits_key(ws[1]);
  const double span = hi - lo;
  unsigned int *cur = reinterpret_cast<unsigned int *>(ws + 2);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const unsigned int pos = atomicAdd(&cur[order_bin(key_at(key, i, logk), lo, span)], 1u);
    order[pos] = (int32_t)i;
  }
}

size_t order_workspace_bytes() {
  return 2 * sizeof(unsigned long long) + ORDER_BINS * sizeof(unsigned int);
}

int launch_order(const MechLayout &L, const double *tab, const int *itab, const double *Y,
                 const double *T, const double *P, int64_t n, double rtol, double atol,
                 bool compute_key, bool log_key, double *key, int32_t *order, void *ws_v,
                 cudaStream_t st, int sms) {
  unsigned long long *ws = static_cast<unsigned long long *>(ws_v);
  k_order_init<<<1, 1024, 0, st>>>(ws);
  if (compute_key) {
    const size_t sm = smem_bytes(L);
    const int block = 64;
    const unsigned grid = (unsigned)((n + block - 1) / block);
    if (L.ns <= 16) {
      KIN_CUDA_TRY(cudaFuncSetAttribute(k_order_key<16>,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
      k_order_key<16><<<grid, block, sm, st>>>(L, tab, itab, Y, T, P, n, rtol, atol, key);
    } else {
      KIN_CUDA_TRY(cudaFuncSetAttribute(k_order_key<64>,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
      k_order_key<64><<<grid, block, sm, st>>>(L, tab, itab, Y, T, P, n, rtol, atol, key);
    }
    KIN_CUDA_TRY(cudaGetLastError());
  }
  const int64_t want = (n + 255) / 256;
  const unsigned grid = (unsigned)(want < 4 * (int64_t)sms ? (want > 0 ? want : 1) : 4 * sms);
  const bool lg = log_key && !compute_key;
  k_order_minmax<<<grid, 256, 0, st>>>(key, lg, n, ws);
  k_order_hist<<<grid, 256, 0, st>>>(key, lg, n, ws);
  k_order_scan<<<1, 1024, 0, st>>>(ws);
  k_order_scatter<<<grid, 256, 0, st>>>(key, lg, n, ws, order);
  KIN_CUDA_TRY(cudaGetLastError());
  return KIN_OK;
}

}  // namespace kin
