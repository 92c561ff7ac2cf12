// Kernel instantiations for points of dimension 32.
#include "esom_fused.cuh"

namespace esom {
ESOM_DEFINE_D(32)
}  // namespace esom
