// Kernel instantiations for points of dimension 44.
#include "esom_fused.cuh"

namespace esom {
ESOM_DEFINE_D(44)
}  // namespace esom
