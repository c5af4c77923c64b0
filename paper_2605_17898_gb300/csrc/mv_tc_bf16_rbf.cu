// Row split tensor-core product: RBF kernel, bfloat16 halves.
#include "mv_tc_inst.cuh"

namespace lgp {
namespace tc {
template cudaError_t dispatch_kind<kFmtBF16, LGP_RBF>(int, int, dim3, const CUtensorMap &, const CUtensorMap &, const TcArgs &,
                                               cudaStream_t);
}  // namespace tc
}  // namespace lgp
