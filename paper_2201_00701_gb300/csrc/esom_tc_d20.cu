// Tensor-core screened kernel instantiations for points of dimension 20.
#include "esom_tc.cuh"

namespace esom {
ESOM_DEFINE_TC_D(20)
}  // namespace esom
