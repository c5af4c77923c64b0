// Symmetric-tile tensor-core product: RBF kernel, bfloat16 halves.
#include "mv_tcs_inst.cuh"

namespace lgp {
namespace tcs {
template cudaError_t dispatch_kind<kFmtBF16, LGP_RBF>(int, int, dim3, const CUtensorMap &, const CUtensorMap &,
                                               const CUtensorMap &, const TcsArgs &, cudaStream_t);
}  // namespace tcs
}  // namespace lgp
