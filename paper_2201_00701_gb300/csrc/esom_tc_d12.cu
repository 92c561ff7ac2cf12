// Tensor-core screened kernel instantiations for points of dimension 12.
#include "esom_tc.cuh"

namespace esom {
ESOM_DEFINE_TC_D(12)
}  // namespace esom
