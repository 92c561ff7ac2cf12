// Kernel instantiations for points of dimension 52.
#include "esom_fused.cuh"

namespace esom {
ESOM_DEFINE_D(52)
}  // namespace esom
