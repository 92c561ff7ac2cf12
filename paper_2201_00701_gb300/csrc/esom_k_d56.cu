// Kernel instantiations for points of dimension 56.
#include "esom_fused.cuh"

namespace esom {
ESOM_DEFINE_D(56)
}  // namespace esom
