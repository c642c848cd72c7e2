// Radau kernels for up to SMALL_MAXN (16) species with float Newton matrices.
#include "kin_kernels.cuh"

namespace kin {
KIN_DEFINE_TU(16f, SMALL_MAXN, float)
}  // namespace kin
