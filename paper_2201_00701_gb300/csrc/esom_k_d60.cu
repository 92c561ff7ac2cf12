// Kernel instantiations for points of dimension 60.
#include "esom_fused.cuh"

namespace esom {
ESOM_DEFINE_D(60)
}  // namespace esom
