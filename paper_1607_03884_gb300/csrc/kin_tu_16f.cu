// Radau kernels for up to 16 species with float Newton matrices.
#include "kin_kernels.cuh"

namespace kin {
KIN_DEFINE_TU(16f, 16, float)
}  // namespace kin
