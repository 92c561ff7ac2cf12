// Tensor-core screened kernel instantiations for points of dimension 16.
#include "esom_tc.cuh"

namespace esom {
ESOM_DEFINE_TC_D(16)
}  // namespace esom
