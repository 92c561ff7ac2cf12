// Kernel instantiations for points of dimension 24.
#include "esom_fused.cuh"

namespace esom {
ESOM_DEFINE_D(24)
}  // namespace esom
