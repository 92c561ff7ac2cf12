// Kernel instantiations for points of dimension 40.
#include "esom_fused.cuh"

namespace esom {
ESOM_DEFINE_D(40)
}  // namespace esom
