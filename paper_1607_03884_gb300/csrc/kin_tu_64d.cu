// Radau kernels for up to 64 species with double Newton matrices.
#include "kin_kernels.cuh"

namespace kin {
KIN_DEFINE_TU(64d, 64, double)
}  // namespace kin
