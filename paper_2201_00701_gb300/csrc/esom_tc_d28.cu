// Tensor-core screened kernel instantiations for points of dimension 28.
#include "esom_tc.cuh"

namespace esom {
ESOM_DEFINE_TC_D(28)
}  // namespace esom
