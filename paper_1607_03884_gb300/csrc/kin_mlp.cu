// The step/guess predictor: a small MLP trained on trajectories the
// integrator itself generates, mapping a reactor state to the first internal
// step size and the Newton starting stages of the first step.  Radau keeps
// its error test and step control, so the network can only save rejected
// steps and Newton iterations (it changes no accepted result beyond the
// integrator's tolerance).
//
// Network: x (din) -> 3 x [Linear(width) -> SiLU] -> Linear(dout).
// Two arithmetic modes:
//   BF16  tensor cores (mma.sync m16n8k16, BF16 operands, FP32 accumulate);
//         activations are rounded to BF16 between layers, master weights and
//         the optimiser stay FP32;
//   FP32  CUDA-core FMA everywhere (a check mode for gradient tests).
// Training: MSE loss, backprop, Adam with bias correction.
// Features for the integrator: log T, log P, log dt, log10(max(Y_k, 1e-12))
// (all species), standardised with caller-given moments; outputs: log h0 and
// the 3 N stage increments, de-standardised.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <random>
#include <vector>

#include "kin_internal.h"

using namespace kin;

namespace {

constexpr int LAYERS = 4;

__device__ __forceinline__ float silu(float a) { return a / (1.0f + __expf(-a)); }
__device__ __forceinline__ float silu_grad(float a) {
  const float s = 1.0f / (1.0f + __expf(-a));
  return s * (1.0f + a * (1.0f - s));
}

// ---------------------------------------------------------------------------
// GEMM, generic strides: C[m][n] (+)= sum_k A(m,k) B(k,n) with
// A(m,k) = A[m*sam + k*sak], B(k,n) = B[k*sbk + n*sbn]; out of range = 0.
// BF16 tensor-core version: a warp computes a 16 x 32 tile (four n8 MMAs per
// k16 step); a block stacks four warps in m (64 x 32).
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned short bf_at(const __nv_bfloat16 *p, int64_t i, bool ok) {
  return ok ? __bfloat16_as_ushort(p[i]) : (unsigned short)0;
}

__global__ void k_gemm_bf16(int M, int N, int K, const __nv_bfloat16 *A, int64_t sam, int64_t sak,
                            const __nv_bfloat16 *B, int64_t sbk, int64_t sbn, float *C,
                            int64_t ldc, int accumulate) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int g = lane >> 2, t = lane & 3;
  const int m0 = blockIdx.x * 64 + warp * 16;
  const int n0 = blockIdx.y * 32;
  float acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.0f;
  const int r0 = m0 + g, r1 = m0 + g + 8;
  for (int k0 = 0; k0 < K; k0 += 16) {
    const int ka = k0 + 2 * t, kb = k0 + 2 * t + 8;
    unsigned a[4];
    {
      const bool ok00 = r0 < M && ka < K, ok01 = r0 < M && ka + 1 < K;
      const bool ok10 = r1 < M && ka < K, ok11 = r1 < M && ka + 1 < K;
      const bool ok02 = r0 < M && kb < K, ok03 = r0 < M && kb + 1 < K;
      const bool ok12 = r1 < M && kb < K, ok13 = r1 < M && kb + 1 < K;
      a[0] = bf_at(A, r0 * sam + ka * sak, ok00) | ((unsigned)bf_at(A, r0 * sam + (ka + 1) * sak, ok01) << 16);
      a[1] = bf_at(A, r1 * sam + ka * sak, ok10) | ((unsigned)bf_at(A, r1 * sam + (ka + 1) * sak, ok11) << 16);
      a[2] = bf_at(A, r0 * sam + kb * sak, ok02) | ((unsigned)bf_at(A, r0 * sam + (kb + 1) * sak, ok03) << 16);
      a[3] = bf_at(A, r1 * sam + kb * sak, ok12) | ((unsigned)bf_at(A, r1 * sam + (kb + 1) * sak, ok13) << 16);
    }
#pragma unroll
    for (int nt = 0; nt < 4; ++nt) {
      const int c = n0 + nt * 8 + g;
      const bool okc = c < N;
      unsigned b0 = bf_at(B, ka * sbk + c * sbn, okc && ka < K) |
                    ((unsigned)bf_at(B, (ka + 1) * sbk + c * sbn, okc && ka + 1 < K) << 16);
      unsigned b1 = bf_at(B, kb * sbk + c * sbn, okc && kb < K) |
                    ((unsigned)bf_at(B, (kb + 1) * sbk + c * sbn, okc && kb + 1 < K) << 16);
      asm volatile(
          "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
          "{%8,%9}, {%0,%1,%2,%3};\n"
          : "+f"(acc[nt][0]), "+f"(acc[nt][1]), "+f"(acc[nt][2]), "+f"(acc[nt][3])
          : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
    }
  }
#pragma unroll
  for (int nt = 0; nt < 4; ++nt) {
    const int c = n0 + nt * 8 + 2 * t;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int r = h ? r1 : r0;
      if (r >= M) continue;
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        if (c + q >= N) continue;
        float v = acc[nt][2 * h + q];
        float *dst = C + (int64_t)r * ldc + c + q;
        *dst = accumulate ? *dst + v : v;
      }
    }
  }
}

// FP32 CUDA-core version (check mode): one output per thread.
__global__ void k_gemm_f32(int M, int N, int K, const float *A, int64_t sam, int64_t sak,
                           const float *B, int64_t sbk, int64_t sbn, float *C, int64_t ldc,
                           int accumulate) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (int64_t)M * N) return;
  const int m = (int)(idx / N), n = (int)(idx % N);
  float s = 0.0f;
  for (int k = 0; k < K; ++k) s = fmaf(A[m * sam + k * sak], B[k * sbk + n * sbn], s);
  float *dst = C + (int64_t)m * ldc + n;
  *dst = accumulate ? *dst + s : s;
}

// ---------------------------------------------------------------------------
// Elementwise kernels
// ---------------------------------------------------------------------------
// a = C + b (stored), h = silu(a) (or a for the last layer) as f32 and bf16
__global__ void k_bias_act(int64_t M, int N, const float *C, const float *b, float *a, float *hf,
                           __nv_bfloat16 *hb, int act) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= M * N) return;
  const float v = C[i] + b[i % N];
  if (a) a[i] = v;
  const float h = act ? silu(v) : v;
  if (hf) hf[i] = h;
  if (hb) hb[i] = __float2bfloat16(h);
}

// gather rows of a [R][d] set: dst[r] = src[rows[r]]; an index outside
// [0, R) gives a zero row
__global__ void k_gather_rows(int64_t M, int d, const float *src, int64_t R,
                              const int32_t *rows, float *dst) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= M * d) return;
  const int64_t r = i / d;
  const int c = (int)(i % d);
  const int32_t s = rows[r];
  dst[i] = (s >= 0 && (int64_t)s < R) ? src[(int64_t)s * d + c] : 0.0f;
}

// pad/convert an input block [M][din] f32 -> [M][ld] (f32 and bf16), zero pad
__global__ void k_pack_input(int64_t M, int din, int ld, const float *X, float *xf,
                             __nv_bfloat16 *xb) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= M * ld) return;
  const int64_t r = i / ld;
  const int c = (int)(i % ld);
  const float v = c < din ? X[r * din + c] : 0.0f;
  if (xf) xf[i] = v;
  if (xb) xb[i] = __float2bfloat16(v);
}

// loss gradient g = 2 (y - t) / (M dout) on the first dout columns, loss sum
__global__ void k_mse_grad(int64_t M, int dout, int ld, const float *y, const float *tgt, float *g,
                           __nv_bfloat16 *gb, float *loss) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  float l = 0.0f;
  if (i < M * ld) {
    const int64_t r = i / ld;
    const int c = (int)(i % ld);
    float v = 0.0f;
    if (c < dout) {
      const float d = y[i] - tgt[r * dout + c];
      v = 2.0f * d / (float)(M * dout);
      l = d * d / (float)(M * dout);
    }
    g[i] = v;
    if (gb) gb[i] = __float2bfloat16(v);
  }
  if (loss) {
    for (int o = 16; o > 0; o >>= 1) l += __shfl_down_sync(0xffffffffu, l, o);
    if ((threadIdx.x & 31) == 0 && l != 0.0f) atomicAdd(loss, l);
  }
}

// g = dH * silu'(a)
__global__ void k_silu_back(int64_t n, const float *dH, const float *a, float *g,
                            __nv_bfloat16 *gb) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float v = dH[i] * silu_grad(a[i]);
  g[i] = v;
  if (gb) gb[i] = __float2bfloat16(v);
}

// column sums: out[c] = sum_r g[r][c]
__global__ void k_colsum(int64_t M, int N, const float *g, float *out) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= N) return;
  float s = 0.0f;
  for (int64_t r = 0; r < M; ++r) s += g[r * N + c];
  out[c] = s;
}

// Adam with bias correction on the masked parameters
__global__ void k_adam(int64_t n, float *p, const float *grad, float *m, float *v,
                       const unsigned char *mask, float lr, float b1, float b2, float eps,
                       float c1, float c2) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n || !mask[i]) return;
  const float gi = grad[i];
  const float mi = b1 * m[i] + (1.0f - b1) * gi;
  const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

__global__ void k_to_bf16(int64_t n, const float *x, __nv_bfloat16 *y) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] = __float2bfloat16(x[i]);
}

// column mean and standard deviation of X [M][d] (two-pass, FP64 sums)
__global__ void k_moments(int64_t M, int d, const float *X, float *mean, float *stdv) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= d) return;
  double s = 0.0;
  for (int64_t r = 0; r < M; ++r) s += X[r * d + c];
  const double mu = s / (double)M;
  double q = 0.0;
  for (int64_t r = 0; r < M; ++r) {
    const double e = X[r * d + c] - mu;
    q += e * e;
  }
  mean[c] = (float)mu;
  stdv[c] = (float)fmax(sqrt(q / (double)M), 1e-12);
}

// features of the integrator's states: [log T, log P, log dt, log10 Y_k], standardised
__global__ void k_features(int64_t n, int ns, const double *Y, const double *T, const double *P,
                           double dt, const float *mean, const float *stdv, float *X) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int din = 3 + ns;
  float *x = X + i * din;
  x[0] = (float)log(T[i]);
  x[1] = (float)log(P[i]);
  x[2] = (float)log(dt);
  for (int k = 0; k < ns; ++k) x[3 + k] = (float)log10(fmax(Y[(int64_t)k * n + i], 1e-12));
  if (mean)
    for (int c = 0; c < din; ++c) x[c] = (x[c] - mean[c]) / stdv[c];
}

// network outputs -> h0 (clipped to [1e-14, dt]) and stage guesses [3N][n]
__global__ void k_unpack_prediction(int64_t n, int dout, int ld, const float *y, const float *mean,
                                    const float *stdv, double dt, double *h0, double *z0) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float *r = y + i * ld;
  if (h0) {
    double lh = (double)r[0] * stdv[0] + mean[0];
    double h = exp(lh);
    h0[i] = fmin(fmax(h, 1e-14), dt);
  }
  if (z0)
    for (int c = 1; c < dout; ++c) z0[(int64_t)(c - 1) * n + i] = (double)r[c] * stdv[c] + mean[c];
}

// training targets: [log h, z_1..z_3N] from the integrator's first-step outputs
__global__ void k_targets(int64_t n, int nz, const double *h, const double *z, float *tgt) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float *t = tgt + i * (1 + nz);
  t[0] = (float)log(h[i]);
  for (int c = 0; c < nz; ++c) t[1 + c] = (float)z[(int64_t)c * n + i];
}

__global__ void k_standardise(int64_t M, int d, float *X, const float *mean, const float *stdv) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= M * d) return;
  const int c = (int)(i % d);
  X[i] = (X[i] - mean[c]) / stdv[c];
}

inline unsigned blocks(int64_t n, int b = 256) { return (unsigned)((n + b - 1) / b); }

}  // namespace

struct kin_mlp {
  int din, dinp, width, dout, doutp, precision;
  int K[LAYERS], N[LAYERS];
  int64_t woff[LAYERS], boff[LAYERS], np;
  float *p = nullptr, *grad = nullptr, *m = nullptr, *v = nullptr;
  unsigned char *mask = nullptr;
  __nv_bfloat16 *wb = nullptr;  // bf16 copy of the weight blocks (same offsets)
  int64_t step = 0;
  // activations (capacity rows)
  int64_t cap = 0;
  float *xf = nullptr, *a[LAYERS] = {}, *hf[LAYERS] = {}, *C = nullptr, *g = nullptr,
        *dH = nullptr, *y = nullptr, *loss = nullptr;
  float *xg = nullptr, *tg = nullptr;  // gathered minibatch rows (train_step_rows)
  __nv_bfloat16 *xb = nullptr, *hb[LAYERS] = {}, *gb = nullptr;
};

static int mlp_reserve(kin_mlp *n, int64_t rows) {
  if (rows <= n->cap) return KIN_OK;
  cudaFree(n->xg);
  cudaFree(n->tg);
  n->xg = n->tg = nullptr;
  cudaFree(n->xf);
  cudaFree(n->xb);
  cudaFree(n->C);
  cudaFree(n->g);
  cudaFree(n->dH);
  cudaFree(n->gb);
  for (int l = 0; l < LAYERS; ++l) {
    cudaFree(n->a[l]);
    cudaFree(n->hf[l]);
    cudaFree(n->hb[l]);
  }
  n->cap = 0;
  const int64_t wmax = n->width > n->doutp ? n->width : n->doutp;
  KIN_CUDA_TRY(cudaMalloc(&n->xg, sizeof(float) * rows * n->din));
  KIN_CUDA_TRY(cudaMalloc(&n->tg, sizeof(float) * rows * n->dout));
  KIN_CUDA_TRY(cudaMalloc(&n->xf, sizeof(float) * rows * n->dinp));
  KIN_CUDA_TRY(cudaMalloc(&n->xb, sizeof(__nv_bfloat16) * rows * n->dinp));
  KIN_CUDA_TRY(cudaMalloc(&n->C, sizeof(float) * rows * wmax));
  KIN_CUDA_TRY(cudaMalloc(&n->g, sizeof(float) * rows * wmax));
  KIN_CUDA_TRY(cudaMalloc(&n->dH, sizeof(float) * rows * wmax));
  KIN_CUDA_TRY(cudaMalloc(&n->gb, sizeof(__nv_bfloat16) * rows * wmax));
  for (int l = 0; l < LAYERS; ++l) {
    KIN_CUDA_TRY(cudaMalloc(&n->a[l], sizeof(float) * rows * n->N[l]));
    KIN_CUDA_TRY(cudaMalloc(&n->hf[l], sizeof(float) * rows * n->N[l]));
    KIN_CUDA_TRY(cudaMalloc(&n->hb[l], sizeof(__nv_bfloat16) * rows * n->N[l]));
  }
  n->y = n->hf[LAYERS - 1];
  n->cap = rows;
  return KIN_OK;
}

static void gemm(const kin_mlp *n, cudaStream_t st, int M, int N, int K, bool bf, const void *A,
                 int64_t sam, int64_t sak, const void *B, int64_t sbk, int64_t sbn, float *C,
                 int64_t ldc, int acc) {
  if (bf) {
    dim3 grid((M + 63) / 64, (N + 31) / 32);
    k_gemm_bf16<<<grid, 128, 0, st>>>(M, N, K, (const __nv_bfloat16 *)A, sam, sak,
                                      (const __nv_bfloat16 *)B, sbk, sbn, C, ldc, acc);
  } else {
    k_gemm_f32<<<blocks((int64_t)M * N), 256, 0, st>>>(M, N, K, (const float *)A, sam, sak,
                                                       (const float *)B, sbk, sbn, C, ldc, acc);
  }
}

// forward pass over M rows already packed in xf/xb; leaves y = hf[L-1]
static int mlp_forward_packed(kin_mlp *n, int64_t M, cudaStream_t st) {
  const bool bf = n->precision == 0;
  for (int l = 0; l < LAYERS; ++l) {
    const void *in = bf ? (l ? (const void *)n->hb[l - 1] : (const void *)n->xb)
                        : (l ? (const void *)n->hf[l - 1] : (const void *)n->xf);
    const void *W = bf ? (const void *)(n->wb + n->woff[l]) : (const void *)(n->p + n->woff[l]);
    gemm(n, st, (int)M, n->N[l], n->K[l], bf, in, n->K[l], 1, W, n->N[l], 1, n->C, n->N[l], 0);
    const int act = l < LAYERS - 1;
    k_bias_act<<<blocks(M * n->N[l]), 256, 0, st>>>(M, n->N[l], n->C, n->p + n->boff[l], n->a[l],
                                                    n->hf[l], bf ? n->hb[l] : nullptr, act);
  }
  KIN_CUDA_TRY(cudaGetLastError());
  return KIN_OK;
}

// backward pass (after mlp_forward_packed and k_mse_grad into g/gb): grad
static int mlp_backward(kin_mlp *n, int64_t M, cudaStream_t st) {
  const bool bf = n->precision == 0;
  for (int l = LAYERS - 1; l >= 0; --l) {
    const int K = n->K[l], N = n->N[l];
    const void *hin = bf ? (l ? (const void *)n->hb[l - 1] : (const void *)n->xb)
                         : (l ? (const void *)n->hf[l - 1] : (const void *)n->xf);
    const void *gv = bf ? (const void *)n->gb : (const void *)n->g;
    // dW[i][o] = sum_b h[b][i] g[b][o]
    gemm(n, st, K, N, (int)M, bf, hin, 1, K, gv, N, 1, n->grad + n->woff[l], N, 0);
    k_colsum<<<blocks(N, 128), 128, 0, st>>>(M, N, n->g, n->grad + n->boff[l]);
    if (l == 0) break;
    // dH[b][i] = sum_o g[b][o] W[i][o]
    const void *W = bf ? (const void *)(n->wb + n->woff[l]) : (const void *)(n->p + n->woff[l]);
    gemm(n, st, (int)M, K, N, bf, gv, N, 1, W, 1, N, n->dH, K, 0);
    k_silu_back<<<blocks(M * K), 256, 0, st>>>(M * K, n->dH, n->a[l - 1], n->g,
                                               bf ? n->gb : nullptr);
  }
  KIN_CUDA_TRY(cudaGetLastError());
  return KIN_OK;
}

static int mlp_pack(kin_mlp *n, const float *X, int64_t M, cudaStream_t st) {
  int rc = mlp_reserve(n, M);
  if (rc) return rc;
  k_pack_input<<<blocks(M * n->dinp), 256, 0, st>>>(M, n->din, n->dinp, X, n->xf,
                                                    n->precision == 0 ? n->xb : nullptr);
  KIN_CUDA_TRY(cudaGetLastError());
  return KIN_OK;
}

static int mlp_refresh_bf16(kin_mlp *n, cudaStream_t st) {
  k_to_bf16<<<blocks(n->np), 256, 0, st>>>(n->np, n->p, n->wb);
  KIN_CUDA_TRY(cudaGetLastError());
  return KIN_OK;
}

extern "C" int kin_mlp_create(int32_t din, int32_t width, int32_t dout, int32_t precision,
                              uint64_t seed, kin_mlp **out) {
  if (!out || din < 1 || width < 8 || dout < 1 || din > 4096 || width > 4096 || dout > 4096 ||
      (precision != 0 && precision != 1))
    return KIN_ERR_INVALID_ARG;
  *out = nullptr;
  kin_mlp *n = new kin_mlp();
  n->din = din;
  n->dinp = (din + 15) / 16 * 16;
  n->width = width;
  n->dout = dout;
  n->doutp = (dout + 7) / 8 * 8;
  n->precision = precision;
  int64_t off = 0;
  for (int l = 0; l < LAYERS; ++l) {
    n->K[l] = l == 0 ? n->dinp : width;
    n->N[l] = l == LAYERS - 1 ? n->doutp : width;
    n->woff[l] = off;
    off += (int64_t)n->K[l] * n->N[l];
    n->boff[l] = off;
    off += n->N[l];
  }
  n->np = off;
  // He-style uniform initialisation, zero biases; padding stays zero
  std::vector<float> p(off, 0.0f);
  std::vector<unsigned char> mask(off, 0);
  std::mt19937_64 rng(seed);
  for (int l = 0; l < LAYERS; ++l) {
    const int kin_ = l == 0 ? din : width, nout = l == LAYERS - 1 ? dout : width;
    const float lim = std::sqrt(6.0f / (float)kin_);
    std::uniform_real_distribution<float> U(-lim, lim);
    for (int i = 0; i < kin_; ++i)
      for (int o = 0; o < nout; ++o) {
        p[n->woff[l] + (int64_t)i * n->N[l] + o] = U(rng);
        mask[n->woff[l] + (int64_t)i * n->N[l] + o] = 1;
      }
    for (int o = 0; o < nout; ++o) mask[n->boff[l] + o] = 1;
  }
  if (cudaMalloc(&n->p, sizeof(float) * off) != cudaSuccess ||
      cudaMalloc(&n->grad, sizeof(float) * off) != cudaSuccess ||
      cudaMalloc(&n->m, sizeof(float) * off) != cudaSuccess ||
      cudaMalloc(&n->v, sizeof(float) * off) != cudaSuccess ||
      cudaMalloc(&n->mask, off) != cudaSuccess ||
      cudaMalloc(&n->wb, sizeof(__nv_bfloat16) * off) != cudaSuccess ||
      cudaMalloc(&n->loss, sizeof(float)) != cudaSuccess) {
    (void)cudaGetLastError();
    kin_mlp_destroy(n);
    return KIN_ERR_NOMEM;
  }
  if (cudaMemcpy(n->p, p.data(), sizeof(float) * off, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(n->mask, mask.data(), off, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemset(n->m, 0, sizeof(float) * off) != cudaSuccess ||
      cudaMemset(n->v, 0, sizeof(float) * off) != cudaSuccess ||
      cudaMemset(n->grad, 0, sizeof(float) * off) != cudaSuccess ||
      mlp_refresh_bf16(n, nullptr) != KIN_OK || cudaDeviceSynchronize() != cudaSuccess) {
    (void)cudaGetLastError();
    kin_mlp_destroy(n);
    return KIN_ERR_CUDA;
  }
  *out = n;
  return KIN_OK;
}

extern "C" void kin_mlp_destroy(kin_mlp *n) {
  if (!n) return;
  cudaFree(n->p);
  cudaFree(n->grad);
  cudaFree(n->m);
  cudaFree(n->v);
  cudaFree(n->mask);
  cudaFree(n->wb);
  cudaFree(n->loss);
  cudaFree(n->xg);
  cudaFree(n->tg);
  cudaFree(n->xf);
  cudaFree(n->xb);
  cudaFree(n->C);
  cudaFree(n->g);
  cudaFree(n->dH);
  cudaFree(n->gb);
  for (int l = 0; l < LAYERS; ++l) {
    cudaFree(n->a[l]);
    cudaFree(n->hf[l]);
    cudaFree(n->hb[l]);
  }
  delete n;
}

// parameter exchange in the unpadded layout W0 [din][w], b0, W1, b1, W2, b2, W3 [w][dout], b3
extern "C" int64_t kin_mlp_num_params(const kin_mlp *n) {
  if (!n) return -1;
  return (int64_t)n->din * n->width + n->width + 2 * ((int64_t)n->width * n->width + n->width) +
         (int64_t)n->width * n->dout + n->dout;
}

static int mlp_copy_params(kin_mlp *n, float *host, const float *dev_src, bool to_host) {
  std::vector<float> full(n->np);
  if (to_host) {
    KIN_CUDA_TRY(cudaMemcpy(full.data(), dev_src, sizeof(float) * n->np, cudaMemcpyDeviceToHost));
  } else {
    KIN_CUDA_TRY(cudaMemcpy(full.data(), n->p, sizeof(float) * n->np, cudaMemcpyDeviceToHost));
  }
  int64_t q = 0;
  for (int l = 0; l < LAYERS; ++l) {
    const int kin_ = l == 0 ? n->din : n->width, nout = l == LAYERS - 1 ? n->dout : n->width;
    for (int i = 0; i < kin_; ++i)
      for (int o = 0; o < nout; ++o) {
        float &f = full[n->woff[l] + (int64_t)i * n->N[l] + o];
        if (to_host) host[q++] = f; else f = host[q++];
      }
    for (int o = 0; o < nout; ++o) {
      float &f = full[n->boff[l] + o];
      if (to_host) host[q++] = f; else f = host[q++];
    }
  }
  if (!to_host) {
    KIN_CUDA_TRY(cudaMemcpy(n->p, full.data(), sizeof(float) * n->np, cudaMemcpyHostToDevice));
    int rc = mlp_refresh_bf16(n, nullptr);
    if (rc) return rc;
    KIN_CUDA_TRY(cudaDeviceSynchronize());
  }
  return KIN_OK;
}

extern "C" int kin_mlp_get_params(kin_mlp *n, float *host, int64_t len) {
  if (!n || !host || len != kin_mlp_num_params(n)) return KIN_ERR_INVALID_ARG;
  return mlp_copy_params(n, host, n->p, true);
}

extern "C" int kin_mlp_set_params(kin_mlp *n, const float *host, int64_t len) {
  if (!n || !host || len != kin_mlp_num_params(n)) return KIN_ERR_INVALID_ARG;
  n->step = 0;
  KIN_CUDA_TRY(cudaMemset(n->m, 0, sizeof(float) * n->np));
  KIN_CUDA_TRY(cudaMemset(n->v, 0, sizeof(float) * n->np));
  return mlp_copy_params(n, const_cast<float *>(host), nullptr, false);
}

extern "C" int kin_mlp_forward(kin_mlp *n, const float *X, float *Y, int64_t M, void *stream) {
  if (!n || M < 0 || (M > 0 && (!X || !Y))) return KIN_ERR_INVALID_ARG;
  if (M == 0) return KIN_OK;
  cudaStream_t st = (cudaStream_t)stream;
  int rc = mlp_pack(n, X, M, st);
  if (rc || (rc = mlp_forward_packed(n, M, st))) return rc;
  KIN_CUDA_TRY(cudaMemcpy2DAsync(Y, sizeof(float) * n->dout, n->y, sizeof(float) * n->doutp,
                                 sizeof(float) * n->dout, M, cudaMemcpyDeviceToDevice, st));
  return KIN_OK;
}

// gradients (unpadded layout, dev [num_params]) of the MSE loss on (X, T)
extern "C" int kin_mlp_grad(kin_mlp *n, const float *X, const float *T, int64_t M, float *grad_out,
                            float *loss_out, void *stream) {
  if (!n || M < 1 || !X || !T) return KIN_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  int rc = mlp_pack(n, X, M, st);
  if (rc || (rc = mlp_forward_packed(n, M, st))) return rc;
  KIN_CUDA_TRY(cudaMemsetAsync(n->loss, 0, sizeof(float), st));
  k_mse_grad<<<blocks(M * n->doutp), 256, 0, st>>>(M, n->dout, n->doutp, n->y, T, n->g,
                                                   n->precision == 0 ? n->gb : nullptr, n->loss);
  if ((rc = mlp_backward(n, M, st))) return rc;
  if (loss_out)
    KIN_CUDA_TRY(cudaMemcpyAsync(loss_out, n->loss, sizeof(float), cudaMemcpyDeviceToDevice, st));
  if (grad_out) {
    // gather the unpadded layout on the host side of the stream
    KIN_CUDA_TRY(cudaStreamSynchronize(st));
    std::vector<float> full(n->np), packed(kin_mlp_num_params(n));
    KIN_CUDA_TRY(cudaMemcpy(full.data(), n->grad, sizeof(float) * n->np, cudaMemcpyDeviceToHost));
    int64_t q = 0;
    for (int l = 0; l < LAYERS; ++l) {
      const int kin_ = l == 0 ? n->din : n->width, nout = l == LAYERS - 1 ? n->dout : n->width;
      for (int i = 0; i < kin_; ++i)
        for (int o = 0; o < nout; ++o) packed[q++] = full[n->woff[l] + (int64_t)i * n->N[l] + o];
      for (int o = 0; o < nout; ++o) packed[q++] = full[n->boff[l] + o];
    }
    KIN_CUDA_TRY(cudaMemcpy(grad_out, packed.data(), sizeof(float) * q, cudaMemcpyHostToDevice));
  }
  return KIN_OK;
}

// one Adam step on a minibatch (X dev [M][din], T dev [M][dout]); loss_out dev scalar or NULL
extern "C" int kin_mlp_train_step(kin_mlp *n, const float *X, const float *T, int64_t M, float lr,
                                  float *loss_out, void *stream) {
  if (!n || M < 1 || !X || !T || !(lr > 0.0f)) return KIN_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  int rc = mlp_pack(n, X, M, st);
  if (rc || (rc = mlp_forward_packed(n, M, st))) return rc;
  KIN_CUDA_TRY(cudaMemsetAsync(n->loss, 0, sizeof(float), st));
  k_mse_grad<<<blocks(M * n->doutp), 256, 0, st>>>(M, n->dout, n->doutp, n->y, T, n->g,
                                                   n->precision == 0 ? n->gb : nullptr, n->loss);
  if ((rc = mlp_backward(n, M, st))) return rc;
  n->step++;
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.0f - std::pow(b1, (float)n->step), c2 = 1.0f - std::pow(b2, (float)n->step);
  k_adam<<<blocks(n->np), 256, 0, st>>>(n->np, n->p, n->grad, n->m, n->v, n->mask, lr, b1, b2,
                                        1e-8f, c1, c2);
  if ((rc = mlp_refresh_bf16(n, st))) return rc;
  if (loss_out)
    KIN_CUDA_TRY(cudaMemcpyAsync(loss_out, n->loss, sizeof(float), cudaMemcpyDeviceToDevice, st));
  return KIN_OK;
}

extern "C" int kin_mlp_train_step_rows(kin_mlp *n, const float *X, const float *T, int64_t R,
                                       const int32_t *rows, int64_t M, float lr, float *loss_out,
                                       void *stream) {
  if (!n || M < 1 || R < 1 || !X || !T || !rows || !(lr > 0.0f)) return KIN_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  int rc = mlp_reserve(n, M);
  if (rc) return rc;
  k_gather_rows<<<blocks(M * n->din), 256, 0, st>>>(M, n->din, X, R, rows, n->xg);
  k_gather_rows<<<blocks(M * n->dout), 256, 0, st>>>(M, n->dout, T, R, rows, n->tg);
  KIN_CUDA_TRY(cudaGetLastError());
  return kin_mlp_train_step(n, n->xg, n->tg, M, lr, loss_out, stream);
}

extern "C" int kin_moments(const float *X, int64_t M, int32_t d, float *mean, float *stdv,
                           void *stream) {
  if (!X || M < 1 || d < 1 || !mean || !stdv) return KIN_ERR_INVALID_ARG;
  k_moments<<<blocks(d, 64), 64, 0, (cudaStream_t)stream>>>(M, d, X, mean, stdv);
  KIN_CUDA_TRY(cudaGetLastError());
  return KIN_OK;
}

extern "C" int kin_mlp_features(int32_t ns, const double *Y, const double *T, const double *P,
                                int64_t n, double dt, const float *mean, const float *stdv,
                                float *X, void *stream) {
  if (ns < 2 || n < 0 || (n > 0 && (!Y || !T || !P || !X)) || !(dt > 0.0) ||
      ((mean == nullptr) != (stdv == nullptr)))
    return KIN_ERR_INVALID_ARG;
  if (n == 0) return KIN_OK;
  k_features<<<blocks(n), 256, 0, (cudaStream_t)stream>>>(n, ns, Y, T, P, dt, mean, stdv, X);
  KIN_CUDA_TRY(cudaGetLastError());
  return KIN_OK;
}

extern "C" int kin_mlp_targets(int32_t nz, const double *h, const double *z, int64_t n,
                               const float *mean, const float *stdv, float *tgt, void *stream) {
  if (nz < 1 || n < 1 || !h || !z || !tgt || ((mean == nullptr) != (stdv == nullptr)))
    return KIN_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  k_targets<<<blocks(n), 256, 0, st>>>(n, nz, h, z, tgt);
  if (mean) k_standardise<<<blocks(n * (1 + nz)), 256, 0, st>>>(n, 1 + nz, tgt, mean, stdv);
  KIN_CUDA_TRY(cudaGetLastError());
  return KIN_OK;
}

extern "C" int kin_mlp_predict(kin_mlp *net, int32_t ns, const double *Y, const double *T,
                               const double *P, int64_t n, double dt, const float *in_mean,
                               const float *in_std, const float *out_mean, const float *out_std,
                               double *h0, double *z0, void *stream) {
  if (!net || n < 0 || !in_mean || !in_std || !out_mean || !out_std || net->din != 3 + ns ||
      net->din > (net->width > net->doutp ? net->width : net->doutp) ||
      net->dout != 1 + 3 * ns || (!h0 && !z0))
    return KIN_ERR_INVALID_ARG;
  if (n == 0) return KIN_OK;
  cudaStream_t st = (cudaStream_t)stream;
  int rc = mlp_reserve(net, n);
  if (rc) return rc;
  // features straight into the f32 input block (din <= dinp), then pack in place
  k_features<<<blocks(n), 256, 0, st>>>(n, ns, Y, T, P, dt, in_mean, in_std, net->dH);
  if ((rc = mlp_pack(net, net->dH, n, st)) || (rc = mlp_forward_packed(net, n, st))) return rc;
  k_unpack_prediction<<<blocks(n), 256, 0, st>>>(n, net->dout, net->doutp, net->y, out_mean,
                                                 out_std, dt, h0, z0);
  KIN_CUDA_TRY(cudaGetLastError());
  return KIN_OK;
}
