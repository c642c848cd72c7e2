// Radau kernels for up to SMALL_MAXN (16) species with double Newton matrices.
#include "kin_kernels.cuh"

namespace kin {
KIN_DEFINE_TU(16d, SMALL_MAXN, double)
}  // namespace kin
