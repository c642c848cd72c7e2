// Radau kernels for up to 16 species with double Newton matrices.
#include "kin_kernels.cuh"

namespace kin {
KIN_DEFINE_TU(16d, 16, double)
}  // namespace kin
