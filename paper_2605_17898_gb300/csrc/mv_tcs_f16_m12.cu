// Symmetric-tile tensor-core product: Matern-1/2 kernel, scaled float16 halves.
#include "mv_tcs_inst.cuh"

namespace lgp {
namespace tcs {
template cudaError_t dispatch_kind<kFmtF16, LGP_MATERN12>(int, int, dim3, const CUtensorMap &, const CUtensorMap &,
                                               const CUtensorMap &, const TcsArgs &, cudaStream_t);
}  // namespace tcs
}  // namespace lgp
