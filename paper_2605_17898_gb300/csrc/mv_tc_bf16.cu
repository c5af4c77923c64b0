// Split tensor-core product, bfloat16 halves.
#include "mv_tc_inst.cuh"

namespace lgp {
namespace tc {
cudaError_t dispatch_bf16(int kind, int D, int T, dim3 grid, const CUtensorMap &mx, const CUtensorMap &mv,
                          const TcArgs &a, cudaStream_t st) {
    return dispatch_fmt<kFmtBF16>(kind, D, T, grid, mx, mv, a, st);
}
}  // namespace tc
}  // namespace lgp
