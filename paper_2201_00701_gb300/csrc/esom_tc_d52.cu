// Tensor-core screened kernel instantiations for points of dimension 52.
#include "esom_tc.cuh"

namespace esom {
ESOM_DEFINE_TC_D(52)
}  // namespace esom
