// Symmetric split tensor-core product, bfloat16 halves.
#include "mv_tcs_inst.cuh"

namespace lgp {
namespace tcs {
cudaError_t dispatch_bf16(int kind, int D, int T, dim3 grid, const CUtensorMap &mx, const CUtensorMap &mv,
                         const CUtensorMap &mo, const TcsArgs &a, cudaStream_t st) {
    return dispatch_fmt<kFmtBF16>(kind, D, T, grid, mx, mv, mo, a, st);
}
}  // namespace tcs
}  // namespace lgp
