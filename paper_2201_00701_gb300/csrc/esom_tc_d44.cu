// Tensor-core screened kernel instantiations for points of dimension 44.
#include "esom_tc.cuh"

namespace esom {
ESOM_DEFINE_TC_D(44)
}  // namespace esom
