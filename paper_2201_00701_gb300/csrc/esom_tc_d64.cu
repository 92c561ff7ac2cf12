// Tensor-core screened kernel instantiations for points of dimension 64.
#include "esom_tc.cuh"

namespace esom {
ESOM_DEFINE_TC_D(64)
}  // namespace esom
