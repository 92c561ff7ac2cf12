// Kernel instantiations for points of dimension 12.
#include "esom_fused.cuh"

namespace esom {
ESOM_DEFINE_D(12)
}  // namespace esom
