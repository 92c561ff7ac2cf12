// Tensor-core screened kernel instantiations for points of dimension 56.
#include "esom_tc.cuh"

namespace esom {
ESOM_DEFINE_TC_D(56)
}  // namespace esom
