// The step/guess predictor: a small MLP trained on trajectories the
// integrator itself generates, mapping a reactor state to the first internal
// step size and the Newton starting stages of the first step.  Radau keeps
// its error test and step control, so the network can only save rejected
// steps and Newton iterations (it changes no accepted result beyond the
// integrator's tolerance).
//
// Network: x (din) -> 3 x [Linear(width) -> SiLU] -> Linear(dout).
// Two arithmetic modes:
//   BF16  5th-generation tensor cores (tcgen05.mma, BF16 operands, FP32
//         accumulators in tensor memory);
//         activations are rounded to BF16 between layers, master weights and
//         the optimiser stay FP32;
//   FP32  CUDA-core FMA everywhere (a check mode for gradient tests).
// Training: MSE loss, backprop, Adam with bias correction.
// Features for the integrator: log T, log P, log dt, log10(max(Y_k, 1e-12))
// (all species), standardised with caller-given moments; outputs: log h0 and
// the 3 N stage increments, de-standardised.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
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
//
// BF16 version on the 5th-generation tensor cores (tcgen05): a CTA of four
// warps owns a 128 x 128 tile of C.  Per 64-wide slice of K, the warps copy
// A (128 x 64) and B (as its transpose, 128 x 64, K contiguous) into shared
// memory in the canonical no-swizzle K-major layout (8-row x 16-byte core
// matrices, 128 B each: core (g, c) of rows 8g.. and K columns 8c.. at
// (8 g + c) * 128 bytes), one thread issues four m128n128k16 MMAs into the
// tile's FP32 accumulator in tensor memory (TMEM, 128 columns), and their
// completion is signalled on an mbarrier before the slice is overwritten.
// The epilogue reads the accumulator back with tcgen05.ld (warp w owns TMEM
// lanes 32w..32w+31, the tile's rows) and writes or adds C.  Every wait is
// bounded: on expiry the kernel sets *err, waits (bounded) for its MMAs and
// loads, frees its TMEM and returns.
// A K-contiguous operand with 16-byte rows (the forward pass and the input
// gradients) is loaded by the tensor memory accelerator instead: one thread
// issues eight cp.async.bulk.tensor boxes of 8 K x 128 rows per slice, each
// landing as 16 core matrices in a row (core (g, c) at c * 2048 + g * 128
// bytes), completion counted in bytes on a second mbarrier; the TMA fills
// rows and K past the matrix with zeros.
// ---------------------------------------------------------------------------
constexpr int TC_BM = 128, TC_BN = 128, TC_BK = 64;
constexpr int TC_THREADS = 128;
constexpr uint32_t TC_TMEM_COLS = 128;
// 16 KB per operand slice; the dynamic allocation is padded so that at most
// four CTAs share an SM (4 x 128 of its 512 TMEM columns)
constexpr size_t TC_SMEM = 2 * TC_BM * TC_BK * sizeof(__nv_bfloat16) + 20 * 1024;
constexpr long long TC_SPIN_LIMIT = 1ll << 26;

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// shared-memory matrix descriptor, no swizzle: start address, leading byte
// offset (next core matrix along K), stride byte offset (next 8 rows), the
// fixed version bits 46-48 = 0b001
__device__ __forceinline__ uint64_t tc_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// instruction descriptor of kind::f16: FP32 accumulator (bits 4-5 = 1), BF16
// A and B (bits 7-9, 10-12 = 1), both K-major, N >> 3 at bits 17-22, M >> 4 at
// bits 24-28
__host__ __device__ constexpr uint32_t tc_idesc(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ bool tc_wait(uint32_t mbar, uint32_t phase) {
  for (long long it = 0; it < TC_SPIN_LIMIT; ++it) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(mbar), "r"(phase)
        : "memory");
    if (done) return true;
  }
  return false;
}

// byte offset of element (r, k) of a 128 x 64 K-major slice
__device__ __forceinline__ int tc_off(int r, int k) {
  return (((r >> 3) * (TC_BK / 8) + (k >> 3)) << 7) + ((r & 7) << 4) + ((k & 7) << 1);
}

// 16-byte copy of a core-matrix row (8 consecutive K) when the operand is
// K-contiguous and the row lies inside the matrix, else element by element
__device__ __forceinline__ void tc_stage_row(unsigned char *dst, const __nv_bfloat16 *src_row,
                                             int64_t sk, bool vec, bool row_ok, int gk, int ke) {
  if (vec && row_ok && gk + 8 <= ke) {
    *reinterpret_cast<uint4 *>(dst) = *reinterpret_cast<const uint4 *>(src_row + gk);
    return;
  }
  __nv_bfloat16 *d = reinterpret_cast<__nv_bfloat16 *>(dst);
#pragma unroll
  for (int e = 0; e < 8; ++e)
    d[e] = (row_ok && gk + e < ke) ? src_row[(int64_t)(gk + e) * sk] : __float2bfloat16(0.0f);
}

// Split K: CTA z sums K in [z kchunk, min(K, (z + 1) kchunk)) and writes its
// partial tile to C + z cz (the caller reduces the partials).
// tma: bit 0 loads A, bit 1 loads B through the tensor maps (rows x K, K
// innermost, boxes of 8 x 128); the split-K chunks are multiples of the slice
__global__ void __launch_bounds__(TC_THREADS) k_gemm_tc(int M, int N, int K,
                                                       const __nv_bfloat16 *A, int64_t sam,
                                                       int64_t sak, const __nv_bfloat16 *B,
                                                       int64_t sbk, int64_t sbn, float *C,
                                                       int64_t ldc, int accumulate, int *err,
                                                       int kchunk, int64_t cz,
                                                       const __grid_constant__ CUtensorMap tmA,
                                                       const __grid_constant__ CUtensorMap tmB,
                                                       int tma) {
  extern __shared__ __align__(1024) unsigned char tc_smem[];
  __shared__ __align__(8) unsigned long long mbar, mfull;
  __shared__ uint32_t tmem_base;
  unsigned char *sA = tc_smem, *sB = tc_smem + TC_BM * TC_BK * 2;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m0 = blockIdx.x * TC_BM, n0 = blockIdx.y * TC_BN;
  const uint32_t mb = smem_u32(&mbar), mf = smem_u32(&mfull);
  const bool ta = (tma & 1) != 0, tb = (tma & 2) != 0;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&tmem_base)),
                 "r"(TC_TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mb) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mf) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base;
  const int kb = blockIdx.z * kchunk, ke = min(K, kb + kchunk);
  C += (int64_t)blockIdx.z * cz;
  // K-contiguous operands are staged 16 bytes (a core-matrix row) at a time
  const bool a_k1 = sak == 1, b_k1 = sbk == 1;
  const bool a_vec = a_k1 && sam % 8 == 0 && (reinterpret_cast<uintptr_t>(A) & 15) == 0;
  const bool b_vec = b_k1 && sbn % 8 == 0 && (reinterpret_cast<uintptr_t>(B) & 15) == 0;
  const bool a_kfast = sak <= sam, b_kfast = sbk <= sbn;
  uint32_t phase = 0, fphase = 0;
  bool ok = true, tma_pending = false;
  const int nk = (ke - kb + TC_BK - 1) / TC_BK;
  for (int kt = 0; kt < nk && ok; ++kt) {
    const int k0 = kb + kt * TC_BK;
    if ((ta || tb) && tid == 0) {  // x = k0 + 8 j: a multiple of 8 elements (16 bytes)
      const uint32_t bytes = (ta ? TC_BM * TC_BK * 2u : 0u) + (tb ? TC_BN * TC_BK * 2u : 0u);
      asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mf), "r"(bytes)
                   : "memory");
#pragma unroll
      for (int j = 0; j < TC_BK / 8; ++j) {
        if (ta)
          asm volatile(
              "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
              " [%0], [%1, {%2, %3}], [%4];" ::"r"(smem_u32(sA) + (uint32_t)(j * TC_BM * 16)),
              "l"(reinterpret_cast<uint64_t>(&tmA)), "r"(k0 + 8 * j), "r"(m0), "r"(mf)
              : "memory");
        if (tb)
          asm volatile(
              "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
              " [%0], [%1, {%2, %3}], [%4];" ::"r"(smem_u32(sB) + (uint32_t)(j * TC_BN * 16)),
              "l"(reinterpret_cast<uint64_t>(&tmB)), "r"(k0 + 8 * j), "r"(n0), "r"(mf)
              : "memory");
      }
    }
    tma_pending = ta || tb;
    // stage the other slices (zero outside the matrices and the K range)
    if (ta) {
    } else if (a_k1) {
      for (int e = tid; e < TC_BM * (TC_BK / 8); e += TC_THREADS) {
        const int r = e >> 3, kc = (e & 7) * 8, gm = m0 + r;
        tc_stage_row(sA + tc_off(r, kc), A + (int64_t)(gm < M ? gm : 0) * sam, 1, a_vec,
                     gm < M, k0 + kc, ke);
      }
    } else {
      for (int e = tid; e < TC_BM * TC_BK; e += TC_THREADS) {
        const int r = a_kfast ? e / TC_BK : e % TC_BM, k = a_kfast ? e % TC_BK : e / TC_BM;
        const int gm = m0 + r, gk = k0 + k;
        const __nv_bfloat16 v = (gm < M && gk < ke) ? A[(int64_t)gm * sam + (int64_t)gk * sak]
                                                    : __float2bfloat16(0.0f);
        *reinterpret_cast<__nv_bfloat16 *>(sA + tc_off(r, k)) = v;
      }
    }
    if (tb) {
    } else if (b_k1) {
      for (int e = tid; e < TC_BN * (TC_BK / 8); e += TC_THREADS) {
        const int c = e >> 3, kc = (e & 7) * 8, gn = n0 + c;
        tc_stage_row(sB + tc_off(c, kc), B + (int64_t)(gn < N ? gn : 0) * sbn, 1, b_vec,
                     gn < N, k0 + kc, ke);
      }
    } else {
      for (int e = tid; e < TC_BN * TC_BK; e += TC_THREADS) {
        const int c = b_kfast ? e / TC_BK : e % TC_BN, k = b_kfast ? e % TC_BK : e / TC_BN;
        const int gn = n0 + c, gk = k0 + k;
        const __nv_bfloat16 v = (gn < N && gk < ke) ? B[(int64_t)gk * sbk + (int64_t)gn * sbn]
                                                    : __float2bfloat16(0.0f);
        *reinterpret_cast<__nv_bfloat16 *>(sB + tc_off(c, k)) = v;
      }
    }
    // make the generic-proxy writes visible to the tensor core (async proxy)
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (ta || tb) {  // the TMA boxes have landed
      ok = __syncthreads_and(tc_wait(mf, fphase)) != 0;
      fphase ^= 1u;
      tma_pending = !ok;
      if (!ok) break;
    }
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t idesc = tc_idesc(TC_BM, TC_BN);
#pragma unroll
      for (int s = 0; s < TC_BK / 16; ++s) {
        // k16 step s covers K cores 2s and 2s + 1
        // K cores 128 B apart, 8-row groups 1024 B (threads' layout); or K
        // cores 2048 B apart, row groups 128 B (the TMA boxes)
        const uint64_t da = ta ? tc_desc(smem_u32(sA) + 4096u * s, 2048u, 128u)
                               : tc_desc(smem_u32(sA) + 256u * s, 128u, (TC_BK / 8) * 128u);
        const uint64_t db = tb ? tc_desc(smem_u32(sB) + 4096u * s, 2048u, 128u)
                               : tc_desc(smem_u32(sB) + 256u * s, 128u, (TC_BK / 8) * 128u);
        const uint32_t acc = (kt > 0 || s > 0) ? 1u : 0u;
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
            "l"(da), "l"(db), "r"(idesc), "r"(acc)
            : "memory");
      }
      asm volatile(
          "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mb)
          : "memory");
    }
    // the slice may be overwritten once its MMAs have completed; every
    // thread leaves the loop on the same trip
    ok = tc_wait(mb, phase);
    phase ^= 1u;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    ok = __syncthreads_and(ok) != 0;
  }
  if (ok) {
    const int row = m0 + warp * 32 + lane;
    for (int c0 = 0; c0 < TC_BN; c0 += 16) {
      uint32_t v[16];
      const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
          "%14,%15}, [%16];\n"
          : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
            "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]),
            "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
          : "r"(taddr)
          : "memory");
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      if (row < M) {
        float *dst = C + (int64_t)row * ldc + n0 + c0;
#pragma unroll
        for (int j = 0; j < 16; ++j)
          if (n0 + c0 + j < N) {
            const float x = __uint_as_float(v[j]);
            dst[j] = accumulate ? dst[j] + x : x;
          }
      }
    }
  } else {
    if (tid == 0) atomicOr(err, 1);
    if (tma_pending) (void)tc_wait(mf, fphase);  // boxes still landing
    else (void)tc_wait(mb, phase ^ 1u);          // the last commit, if it is still pending
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(TC_TMEM_COLS)
                 : "memory");
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

// y [N][K] = bf16(x [K][N])^T: a weight block with K contiguous, so the
// forward GEMMs stage their B operand 16 bytes at a time
__global__ void k_to_bf16_t(int K, int N, const float *x, __nv_bfloat16 *y) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (int64_t)K * N) return;
  const int k = (int)(i / N), n = (int)(i % N);
  y[(int64_t)n * K + k] = __float2bfloat16(x[i]);
}

// C[m][n] (+)= sum over the S partial tiles ws[s][m][n] (split-K GEMMs; a
// fixed summation order, so results do not depend on scheduling)
__global__ void k_splitk_reduce(int M, int N, int S, const float *ws, float *C, int64_t ldc,
                                int accumulate) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (int64_t)M * N) return;
  const int m = (int)(i / N), n = (int)(i % N);
  float v = 0.0f;
  for (int q = 0; q < S; ++q) v += ws[(int64_t)q * M * N + i];
  float *dst = C + (int64_t)m * ldc + n;
  *dst = accumulate ? *dst + v : v;
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
  __nv_bfloat16 *wbt = nullptr; // the same blocks transposed ([N][K] at the same offsets)
  float *ws = nullptr;          // split-K partial tiles
  int64_t ws_floats = 0;
  int64_t step = 0;
  // activations (capacity rows)
  int64_t cap = 0;
  float *xf = nullptr, *a[LAYERS] = {}, *hf[LAYERS] = {}, *C = nullptr, *g = nullptr,
        *dH = nullptr, *y = nullptr, *loss = nullptr;
  float *xg = nullptr, *tg = nullptr;  // gathered minibatch rows (train_step_rows)
  int *err = nullptr;                  // set by a tensor-core GEMM whose wait expired
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

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link
// against the driver library); null when unavailable
static PFN_cuTensorMapEncodeTiled_v12000 tmap_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = [] {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      p = nullptr;
    (void)cudaGetLastError();
    return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }();
  return fn;
}

// tensor map of a rows x cols BF16 matrix with row stride ld (elements),
// boxes of 8 columns x 128 rows, zero fill outside; false when the layout
// does not allow the TMA (16-byte base and rows)
static bool make_tmap(CUtensorMap *m, const void *base, int64_t rows, int64_t cols, int64_t ld) {
  std::memset(m, 0, sizeof *m);
  auto enc = tmap_encoder();
  if (!enc || (reinterpret_cast<uintptr_t>(base) & 15) || (ld * 2) % 16 || ld < cols ||
      rows < 1 || cols < 1)
    return false;
  const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
  const cuuint32_t box[2] = {8, 128}, es[2] = {1, 1};
  return enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(base), dims, strides, box,
             es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
             CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
         CUDA_SUCCESS;
}

// TMA operand loads (1) or the threads' copies only (0): a build-time knob
#ifndef KIN_MLP_TMA
#define KIN_MLP_TMA 1
#endif

static void gemm(const kin_mlp *n, cudaStream_t st, int M, int N, int K, bool bf, const void *A,
                 int64_t sam, int64_t sak, const void *B, int64_t sbk, int64_t sbn, float *C,
                 int64_t ldc, int acc) {
  if (bf) {
    CUtensorMap tmA, tmB;
    int tma = 0;
    if (KIN_MLP_TMA && sak == 1 && make_tmap(&tmA, A, M, K, sam)) tma |= 1;
    if (KIN_MLP_TMA && sbk == 1 && make_tmap(&tmB, B, N, K, sbn)) tma |= 2;
    if (!(tma & 1)) std::memset(&tmA, 0, sizeof tmA);
    if (!(tma & 2)) std::memset(&tmB, 0, sizeof tmB);
    dim3 grid((M + TC_BM - 1) / TC_BM, (N + TC_BN - 1) / TC_BN, 1);
    // few output tiles and a long K (the weight gradients: K = batch rows):
    // split K over up to 2 x 152 CTAs, partial tiles reduced in fixed order
    const int64_t tiles = (int64_t)grid.x * grid.y, kt = (K + TC_BK - 1) / TC_BK;
    int S = 1;
    if (tiles < 2 * 152 && kt >= 8) {
      S = (int)std::min<int64_t>(kt / 4, (2 * 152 + tiles - 1) / tiles);
      while (S > 1 && (int64_t)S * M * N > n->ws_floats) --S;
    }
    if (S > 1) {
      const int kchunk = (int)((kt + S - 1) / S) * TC_BK;
      S = (K + kchunk - 1) / kchunk;  // every split holds at least one K slice
      grid.z = S;
      k_gemm_tc<<<grid, TC_THREADS, TC_SMEM, st>>>(M, N, K, (const __nv_bfloat16 *)A, sam, sak,
                                                   (const __nv_bfloat16 *)B, sbk, sbn, n->ws, N,
                                                   0, n->err, kchunk, (int64_t)M * N, tmA, tmB,
                                                   tma);
      k_splitk_reduce<<<blocks((int64_t)M * N), 256, 0, st>>>(M, N, S, n->ws, C, ldc, acc);
    } else {
      k_gemm_tc<<<grid, TC_THREADS, TC_SMEM, st>>>(M, N, K, (const __nv_bfloat16 *)A, sam, sak,
                                                   (const __nv_bfloat16 *)B, sbk, sbn, C, ldc,
                                                   acc, n->err, (int)kt * TC_BK, 0, tmA, tmB,
                                                   tma);
    }
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
    if (bf)  // B(k, n) = W[k][n] from the transposed copy (K contiguous)
      gemm(n, st, (int)M, n->N[l], n->K[l], bf, in, n->K[l], 1, n->wbt + n->woff[l], 1,
           n->K[l], n->C, n->N[l], 0);
    else
      gemm(n, st, (int)M, n->N[l], n->K[l], bf, in, n->K[l], 1, n->p + n->woff[l], n->N[l], 1,
           n->C, n->N[l], 0);
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
  for (int l = 0; l < LAYERS; ++l)
    k_to_bf16_t<<<blocks((int64_t)n->K[l] * n->N[l]), 256, 0, st>>>(
        n->K[l], n->N[l], n->p + n->woff[l], n->wbt + n->woff[l]);
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
  {  // split-K workspace: up to 64 partial tiles of the largest weight block, 64 MB at most
    int64_t big = 0;
    for (int l = 0; l < LAYERS; ++l) big = std::max<int64_t>(big, (int64_t)n->K[l] * n->N[l]);
    n->ws_floats = std::max<int64_t>(big, std::min<int64_t>(64 * big, 16ll << 20));
  }
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
      cudaMalloc(&n->wbt, sizeof(__nv_bfloat16) * off) != cudaSuccess ||
      cudaMalloc(&n->ws, sizeof(float) * n->ws_floats) != cudaSuccess ||
      cudaMalloc(&n->loss, sizeof(float)) != cudaSuccess ||
      cudaMalloc(&n->err, sizeof(int)) != cudaSuccess) {
    (void)cudaGetLastError();
    kin_mlp_destroy(n);
    return KIN_ERR_NOMEM;
  }
  if (cudaMemcpy(n->p, p.data(), sizeof(float) * off, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(n->mask, mask.data(), off, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemset(n->m, 0, sizeof(float) * off) != cudaSuccess ||
      cudaMemset(n->v, 0, sizeof(float) * off) != cudaSuccess ||
      cudaMemset(n->grad, 0, sizeof(float) * off) != cudaSuccess ||
      cudaMemset(n->err, 0, sizeof(int)) != cudaSuccess ||
      cudaFuncSetAttribute(k_gemm_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)TC_SMEM) != cudaSuccess ||
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
  cudaFree(n->wbt);
  cudaFree(n->ws);
  cudaFree(n->loss);
  cudaFree(n->err);
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
    int e = 0;
    KIN_CUDA_TRY(cudaMemcpy(&e, n->err, sizeof e, cudaMemcpyDeviceToHost));
    if (e) return KIN_ERR_CUDA;  // a tensor-core wait expired
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
