// Kernel instantiations for points of dimension 4.
#include "esom_fused.cuh"

namespace esom {
ESOM_DEFINE_D(4)
}  // namespace esom
