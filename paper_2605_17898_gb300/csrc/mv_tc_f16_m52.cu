// Row split tensor-core product: Matern-5/2 kernel, scaled float16 halves.
#include "mv_tc_inst.cuh"

namespace lgp {
namespace tc {
template cudaError_t dispatch_kind<kFmtF16, LGP_MATERN52>(int, int, dim3, const CUtensorMap &, const CUtensorMap &, const TcArgs &,
                                               cudaStream_t);
}  // namespace tc
}  // namespace lgp
