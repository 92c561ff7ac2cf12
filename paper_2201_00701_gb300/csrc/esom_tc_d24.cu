// Tensor-core screened kernel instantiations for points of dimension 24.
#include "esom_tc.cuh"

namespace esom {
ESOM_DEFINE_TC_D(24)
}  // namespace esom
