// Internal interface to the paper-variant ablation kernels
// (esom_variants.cuh, esom_variants_*.cu).  Not part of the ABI.
#pragma once

#include "esom_kernels.h"

namespace esom {

// Base and Bitonic k-NN (the library's neighbours, bit for bit) and the
// Registers projection from given neighbours.  Grids are sized from a.n; the
// k-NN variants write a.idx / a.dist2, the projection reads them and writes
// a.out.
struct VariantOps {
    cudaError_t (*knn_base)(const FusedArgs &a, cudaStream_t stream);
    cudaError_t (*knn_bitonic)(const FusedArgs &a, cudaStream_t stream);
    cudaError_t (*project_registers)(const FusedArgs &a, cudaStream_t stream);
};
const VariantOps *variant_ops(int D);

}  // namespace esom
