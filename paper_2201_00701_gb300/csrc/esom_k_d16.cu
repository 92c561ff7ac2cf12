// Kernel instantiations for points of dimension 16.
#include "esom_fused.cuh"

namespace esom {
ESOM_DEFINE_D(16)
}  // namespace esom
