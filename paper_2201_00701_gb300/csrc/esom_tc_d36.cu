// Tensor-core screened kernel instantiations for points of dimension 36.
#include "esom_tc.cuh"

namespace esom {
ESOM_DEFINE_TC_D(36)
}  // namespace esom
