// Kernel instantiations for points of dimension 36.
#include "esom_fused.cuh"

namespace esom {
ESOM_DEFINE_D(36)
}  // namespace esom
