// Kernel instantiations for points of dimension 64.
#include "esom_fused.cuh"

namespace esom {
ESOM_DEFINE_D(64)
}  // namespace esom
