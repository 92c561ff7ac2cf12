// Kernel instantiations for points of dimension 20.
#include "esom_fused.cuh"

namespace esom {
ESOM_DEFINE_D(20)
}  // namespace esom
