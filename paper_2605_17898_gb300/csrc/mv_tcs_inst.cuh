// Instantiation of the symmetric split tensor-core product for one 16-bit format (included once
// per format).
#pragma once

#include "mv_tcs.cuh"

namespace lgp {
namespace tcs {

template <int KIND, int D, int T, int FMT>
cudaError_t launch_tcs_inst(dim3 grid, const CUtensorMap &mx, const CUtensorMap &mv, const CUtensorMap &mo,
                            const TcsArgs &a,
                            cudaStream_t st) {
    constexpr int DP = D <= 4 ? 4 : 8;
    constexpr int bytes = TcsLayout<T, DP>::kBytes;
    static bool configured = false;
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(mv_tcs_kernel<KIND, D, T, FMT>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
        if (e != cudaSuccess) return e;
        configured = true;
    }
    mv_tcs_kernel<KIND, D, T, FMT><<<grid, kThreads, bytes, st>>>(mx, mv, mo, a);
    return cudaGetLastError();
}

template <int KIND, int T, int FMT>
cudaError_t dispatch_d(int D, dim3 grid, const CUtensorMap &mx, const CUtensorMap &mv, const CUtensorMap &mo,
                            const TcsArgs &a,
                       cudaStream_t st) {
    switch (D) {
        case 1: return launch_tcs_inst<KIND, 1, T, FMT>(grid, mx, mv, mo, a, st);
        case 2: return launch_tcs_inst<KIND, 2, T, FMT>(grid, mx, mv, mo, a, st);
        case 3: return launch_tcs_inst<KIND, 3, T, FMT>(grid, mx, mv, mo, a, st);
        case 4: return launch_tcs_inst<KIND, 4, T, FMT>(grid, mx, mv, mo, a, st);
        case 5: return launch_tcs_inst<KIND, 5, T, FMT>(grid, mx, mv, mo, a, st);
        case 6: return launch_tcs_inst<KIND, 6, T, FMT>(grid, mx, mv, mo, a, st);
        case 7: return launch_tcs_inst<KIND, 7, T, FMT>(grid, mx, mv, mo, a, st);
        case 8: return launch_tcs_inst<KIND, 8, T, FMT>(grid, mx, mv, mo, a, st);
    }
    return cudaErrorInvalidValue;
}

template <int FMT>
cudaError_t dispatch_fmt(int kind, int D, int T, dim3 grid, const CUtensorMap &mx, const CUtensorMap &mv,
                         const CUtensorMap &mo, const TcsArgs &a, cudaStream_t st) {
    if (kind == LGP_RBF)
        return T == 16 ? dispatch_d<LGP_RBF, 16, FMT>(D, grid, mx, mv, mo, a, st)
                       : dispatch_d<LGP_RBF, 32, FMT>(D, grid, mx, mv, mo, a, st);
    return T == 16 ? dispatch_d<LGP_MATERN52, 16, FMT>(D, grid, mx, mv, mo, a, st)
                   : dispatch_d<LGP_MATERN52, 32, FMT>(D, grid, mx, mv, mo, a, st);
}

cudaError_t dispatch_bf16(int kind, int D, int T, dim3 grid, const CUtensorMap &mx, const CUtensorMap &mv,
                          const CUtensorMap &mo, const TcsArgs &a, cudaStream_t st);
cudaError_t dispatch_f16(int kind, int D, int T, dim3 grid, const CUtensorMap &mx, const CUtensorMap &mv,
                         const CUtensorMap &mo, const TcsArgs &a, cudaStream_t st);

}  // namespace tcs
}  // namespace lgp
