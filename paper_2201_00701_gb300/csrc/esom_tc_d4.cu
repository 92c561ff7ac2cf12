// Tensor-core screened kernel instantiations for points of dimension 4.
#include "esom_tc.cuh"

namespace esom {
ESOM_DEFINE_TC_D(4)
}  // namespace esom
