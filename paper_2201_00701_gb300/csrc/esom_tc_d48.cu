// Tensor-core screened kernel instantiations for points of dimension 48.
#include "esom_tc.cuh"

namespace esom {
ESOM_DEFINE_TC_D(48)
}  // namespace esom
