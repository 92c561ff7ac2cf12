// Tensor-core screened kernel instantiations for points of dimension 32.
#include "esom_tc.cuh"

namespace esom {
ESOM_DEFINE_TC_D(32)
}  // namespace esom
