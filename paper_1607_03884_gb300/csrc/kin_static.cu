// kin_integrate_static: the one entry point of libkin that allocates nothing.
// (The CUDA driver may still reserve local memory for a kernel's per-thread
// frame at its first launch on a device; see include/kin.h.)
//
// Some callers cannot call cudaMalloc: code running inside a host framework
// whose allocator owns (and has reserved) all device memory, plugins that are
// not allowed to allocate, or real-time loops that must not allocate once
// started.  For them this entry point keeps everything the integration
// kernel needs beyond the caller's inputs and outputs -- the mechanism tables
// and the work-queue / statistics counters -- in one file-scope device array
// of fixed size, instead of the cudaMalloc'd workspace of a kin_mech.
//
// The array (KIN_STATIC_SCRATCH_BYTES) is part of the library image: every
// GPU that loads libkin holds it until the process exits.  All calls share
// it and it keeps the last call's contents; each call rewrites the tables and
// clears the counters before its launch, so two calls whose GPU work overlaps
// (on different streams) race on it and must not be issued.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>
#include <vector>

#include "kin_internal.h"

using namespace kin;

namespace {

constexpr size_t kTableBytes = 64 * 1024;   // mechanism tables (doubles, then ints)
constexpr size_t kCounterBytes = 256;       // totals and the queue counter (16 x u64)
static_assert(kTableBytes + kCounterBytes == KIN_STATIC_SCRATCH_BYTES, "scratch size");

// In host code this name is only a host-side stand-in for the device array;
// the device address comes from cudaGetSymbolAddress (kept per device below).
static __device__ __align__(256) unsigned char g_scratch[KIN_STATIC_SCRATCH_BYTES];

std::mutex g_mu;
unsigned char *g_addr[64];  // device address of g_scratch per device (set-up done when non-null)

int scratch_address(int dev, unsigned char **out) {
  std::lock_guard<std::mutex> lk(g_mu);
  if (dev < 0 || dev >= 64) return KIN_ERR_CUDA;
  if (!g_addr[dev]) {
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess || !p) {
      (void)cudaGetLastError();
      return KIN_ERR_CUDA;
    }
    g_addr[dev] = static_cast<unsigned char *>(p);
  }
  *out = g_addr[dev];
  return KIN_OK;
}

}  // namespace

extern "C" int kin_integrate_static(const kin_mech_desc *desc, double *Y, double *T,
                                    const double *P, int64_t n, double dt, double rtol,
                                    double atol, int32_t *status, void *stream) {
  if (!desc || n < 0 || (n > 0 && (!Y || !T || !P))) return KIN_ERR_INVALID_ARG;
  if (!(dt > 0.0) || !(rtol > 0.0) || !(atol > 0.0) || !std::isfinite(dt))
    return KIN_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  // The tables are uploaded from host vectors this call frees: a graph
  // captured from it would replay copies from freed memory.  Refuse capture
  // before any CUDA work is issued.
  {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) {
      (void)cudaGetLastError();
      return KIN_ERR_UNSUPPORTED;
    }
    if (cs != cudaStreamCaptureStatusNone) return KIN_ERR_UNSUPPORTED;
  }
  MechLayout L;
  std::vector<double> dtab;
  std::vector<int> itab;
  int rc = build_tables(desc, L, dtab, itab);
  if (rc) return rc;
  const size_t dbytes = sizeof(double) * (size_t)L.nd, ibytes = sizeof(int) * (size_t)L.ni;
  if (dbytes + ibytes > kTableBytes) return KIN_ERR_UNSUPPORTED;  // beyond the static array
  int dev = 0, sms = 0;
  KIN_CUDA_TRY(cudaGetDevice(&dev));
  if ((rc = ensure_constants(dev))) return rc;
  unsigned char *base = nullptr;
  if ((rc = scratch_address(dev, &base))) return rc;
  KIN_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  double *tab = reinterpret_cast<double *>(base);
  int *itb = reinterpret_cast<int *>(base + dbytes);
  unsigned long long *totals = reinterpret_cast<unsigned long long *>(base + kTableBytes);
  KIN_CUDA_TRY(cudaMemcpyAsync(tab, dtab.data(), dbytes, cudaMemcpyHostToDevice, st));
  KIN_CUDA_TRY(cudaMemcpyAsync(itb, itab.data(), ibytes, cudaMemcpyHostToDevice, st));
  KIN_CUDA_TRY(cudaMemsetAsync(totals, 0, kCounterBytes, st));
  if (n == 0) return KIN_OK;
  kin_options o;
  kin_options_default(&o);
  // the default options without a tuning cache or a per-mechanism
  // workspace: one state per thread (the WARP layout needs Jacobian slots)
  o.layout = KIN_LAYOUT_PLAIN;
  o.block = 64;
  KernelArgs a;
  a.L = L;
  a.tab = tab;
  a.itab = itb;
  a.Y = Y;
  a.T = T;
  a.P = P;
  a.status = status;
  a.counters = nullptr;
  a.totals = totals;
  const double quot = atol / rtol;
  const double r = 0.1 * std::pow(rtol, 2.0 / 3.0);
  a.rp.rtol = r;
  a.rp.atol = r * quot;
  a.rp.fnewt = std::fmax(10.0 * UROUND / r, std::fmin(0.03, std::sqrt(r)));
  a.rp.dt = dt;
  a.rp.nit = o.nit;
  a.rp.max_steps = o.max_steps;
  a.rp.n = n;
  a.rp.h0 = nullptr;
  a.rp.z0 = nullptr;
  a.rp.h_first = nullptr;
  a.rp.z_first = nullptr;
  a.rp.stop_after = 0;
  a.rp.hfixed = 0.0;
  a.refill_min = 1;
  a.order = nullptr;
  a.gscratch = nullptr;  // the thread layout needs no group slots
  a.gslots = 0;
  return launch_dispatch(a, o, st, sms);
}
