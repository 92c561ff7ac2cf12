// Tensor-core screened kernel instantiations for points of dimension 60.
#include "esom_tc.cuh"

namespace esom {
ESOM_DEFINE_TC_D(60)
}  // namespace esom
