// Tensor-core screened kernel instantiations for points of dimension 40.
#include "esom_tc.cuh"

namespace esom {
ESOM_DEFINE_TC_D(40)
}  // namespace esom
