// Tensor-core screened kernel instantiations for points of dimension 8.
#include "esom_tc.cuh"

namespace esom {
ESOM_DEFINE_TC_D(8)
}  // namespace esom
