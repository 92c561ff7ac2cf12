// Kernel instantiations for points of dimension 48.
#include "esom_fused.cuh"

namespace esom {
ESOM_DEFINE_D(48)
}  // namespace esom
