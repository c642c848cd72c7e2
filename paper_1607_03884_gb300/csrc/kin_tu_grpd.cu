// Group kernels (4, 8 or 16 lanes per state, up to 15 species) with double
// Newton matrices.
#include "kin_kernels.cuh"

namespace kin {
KIN_DEFINE_GROUP_TU(grpd, double)
}  // namespace kin
