// Kernel instantiations for points of dimension 28.
#include "esom_fused.cuh"

namespace esom {
ESOM_DEFINE_D(28)
}  // namespace esom
