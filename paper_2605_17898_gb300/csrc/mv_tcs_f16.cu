// Symmetric split tensor-core product, scaled float16 halves.
#include "mv_tcs_inst.cuh"

namespace lgp {
namespace tcs {
cudaError_t dispatch_f16(int kind, int D, int T, dim3 grid, const CUtensorMap &mx, const CUtensorMap &mv,
                         const CUtensorMap &mo, const TcsArgs &a, cudaStream_t st) {
    return dispatch_fmt<kFmtF16>(kind, D, T, grid, mx, mv, mo, a, st);
}
}  // namespace tcs
}  // namespace lgp
