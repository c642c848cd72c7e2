// Host-side helpers shared by the C-ABI translation units of libkin.
#pragma once
#include <cuda_runtime.h>

#include <vector>

#include "../../include/kin.h"
#include "kin_kernels.cuh"

namespace kin {
// Validate a mechanism description and build its device tables on the host.
int build_tables(const kin_mech_desc *d, MechLayout &L, std::vector<double> &dt,
                 std::vector<int> &it);
// Upload the Radau constants to every kernel translation unit, once per device.
int ensure_constants(int dev);
// Launch the integration kernel that matches the options and species count.
int launch_dispatch(const KernelArgs &a, const kin_options &o, cudaStream_t st, int sms);
// Stiffness ordering (kin_order.cu): device workspace size and launcher.
size_t order_workspace_bytes();
int launch_order(const MechLayout &L, const double *tab, const int *itab, const double *Y,
                 const double *T, const double *P, int64_t n, double rtol, double atol,
                 bool compute_key, bool log_key, double *key, int32_t *order, void *ws,
                 cudaStream_t st, int sms);
}  // namespace kin
