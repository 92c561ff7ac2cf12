// Kernel instantiations for points of dimension 8.
#include "esom_fused.cuh"

namespace esom {
ESOM_DEFINE_D(8)
}  // namespace esom
