// Radau kernels for up to 64 species with float Newton matrices.
#include "kin_kernels.cuh"

namespace kin {
KIN_DEFINE_TU(64f, 64, float)
}  // namespace kin
