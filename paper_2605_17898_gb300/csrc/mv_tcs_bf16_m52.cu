// Symmetric-tile tensor-core product: Matern-5/2 kernel, bfloat16 halves.
#include "mv_tcs_inst.cuh"

namespace lgp {
namespace tcs {
template cudaError_t dispatch_kind<kFmtBF16, LGP_MATERN52>(int, int, dim3, const CUtensorMap &, const CUtensorMap &,
                                               const CUtensorMap &, const TcsArgs &, cudaStream_t);
}  // namespace tcs
}  // namespace lgp
