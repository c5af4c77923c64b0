// Instantiation of the symmetric split tensor-core product for one 16-bit format (included once
// per format).
#pragma once

#include "mv_tcs.cuh"

namespace lgp {
namespace tcs {

template <int KIND, int D, int T, int FMT, bool DOT = false, bool BANDED = false>
cudaError_t launch_tcs_inst(dim3 grid, const CUtensorMap &mx, const CUtensorMap &mv, const CUtensorMap &mo,
                            const TcsArgs &a,
                            cudaStream_t st) {
    constexpr int DP = D <= 4 ? 4 : 8;
    constexpr int bytes = DOT ? TcdLayout<T, DP>::kBytes : TcsLayout<T, DP>::kBytes;
    static bool configured = false;
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(mv_tcs_kernel<KIND, D, T, FMT, DOT, BANDED>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
        if (e != cudaSuccess) return e;
        configured = true;
    }
    mv_tcs_kernel<KIND, D, T, FMT, DOT, BANDED><<<grid, DOT ? kDotThreads : kThreads, bytes, st>>>(mx, mv, mo, a);
    return cudaGetLastError();
}

// The dot-form instance: the banded tile order when the band is narrower than the triangle
// (TcsArgs::band < nb), else the single-band one.
template <int KIND, int DP, int T, int FMT>
cudaError_t launch_tcs_dot(dim3 grid, const CUtensorMap &mx, const CUtensorMap &mv, const CUtensorMap &mo,
                           const TcsArgs &a, cudaStream_t st) {
    return a.band < a.nb ? launch_tcs_inst<KIND, DP, T, FMT, true, true>(grid, mx, mv, mo, a, st)
                         : launch_tcs_inst<KIND, DP, T, FMT, true, false>(grid, mx, mv, mo, a, st);
}

// Dot-form instances exist for RBF, Matern-5/2 and Matern-3/2 at the padded widths 4 and 8, each with
// and without the banded tile order. The difference form walks the single-band order at every size.
template <int KIND>
constexpr bool has_dot_form() { return KIND == LGP_RBF || KIND == LGP_MATERN52 || KIND == LGP_MATERN32; }

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

// One (format, kind) pair: every D and T. Instantiated in its own translation unit
// (mv_tcs_<fmt>_<kind>.cu) so that the instantiations compile in parallel.
template <int FMT, int KIND>
cudaError_t dispatch_kind(int D, int T, dim3 grid, const CUtensorMap &mx, const CUtensorMap &mv, const CUtensorMap &mo,
                          const TcsArgs &a, cudaStream_t st) {
    if (a.dot) {
        if constexpr (has_dot_form<KIND>()) {
            if (D < 1 || D > 8) return cudaErrorInvalidValue;
            if (D <= 4)
                return T == 16 ? launch_tcs_dot<KIND, 4, 16, FMT>(grid, mx, mv, mo, a, st)
                               : launch_tcs_dot<KIND, 4, 32, FMT>(grid, mx, mv, mo, a, st);
            return T == 16 ? launch_tcs_dot<KIND, 8, 16, FMT>(grid, mx, mv, mo, a, st)
                           : launch_tcs_dot<KIND, 8, 32, FMT>(grid, mx, mv, mo, a, st);
        }
        return cudaErrorInvalidValue;
    }
    return T == 16 ? dispatch_d<KIND, 16, FMT>(D, grid, mx, mv, mo, a, st)
                   : dispatch_d<KIND, 32, FMT>(D, grid, mx, mv, mo, a, st);
}

#define LGP_TCS_KIND_DECL(FMT, KIND)                                                                                \
    extern template cudaError_t dispatch_kind<FMT, KIND>(int, int, dim3, const CUtensorMap &, const CUtensorMap &,  \
                                                         const CUtensorMap &, const TcsArgs &, cudaStream_t);
LGP_TCS_KIND_DECL(kFmtBF16, LGP_RBF)
LGP_TCS_KIND_DECL(kFmtBF16, LGP_MATERN52)
LGP_TCS_KIND_DECL(kFmtBF16, LGP_MATERN12)
LGP_TCS_KIND_DECL(kFmtBF16, LGP_MATERN32)
LGP_TCS_KIND_DECL(kFmtF16, LGP_RBF)
LGP_TCS_KIND_DECL(kFmtF16, LGP_MATERN52)
LGP_TCS_KIND_DECL(kFmtF16, LGP_MATERN12)
LGP_TCS_KIND_DECL(kFmtF16, LGP_MATERN32)
#undef LGP_TCS_KIND_DECL

template <int FMT>
cudaError_t dispatch_fmt(int kind, int D, int T, dim3 grid, const CUtensorMap &mx, const CUtensorMap &mv,
                         const CUtensorMap &mo, const TcsArgs &a, cudaStream_t st) {
    switch (kind) {
        case LGP_RBF: return dispatch_kind<FMT, LGP_RBF>(D, T, grid, mx, mv, mo, a, st);
        case LGP_MATERN52: return dispatch_kind<FMT, LGP_MATERN52>(D, T, grid, mx, mv, mo, a, st);
        case LGP_MATERN12: return dispatch_kind<FMT, LGP_MATERN12>(D, T, grid, mx, mv, mo, a, st);
        case LGP_MATERN32: return dispatch_kind<FMT, LGP_MATERN32>(D, T, grid, mx, mv, mo, a, st);
    }
    return cudaErrorInvalidValue;
}

inline cudaError_t dispatch_bf16(int kind, int D, int T, dim3 grid, const CUtensorMap &mx, const CUtensorMap &mv,
                                 const CUtensorMap &mo, const TcsArgs &a, cudaStream_t st) {
    return dispatch_fmt<kFmtBF16>(kind, D, T, grid, mx, mv, mo, a, st);
}
inline cudaError_t dispatch_f16(int kind, int D, int T, dim3 grid, const CUtensorMap &mx, const CUtensorMap &mv,
                                const CUtensorMap &mo, const TcsArgs &a, cudaStream_t st) {
    return dispatch_fmt<kFmtF16>(kind, D, T, grid, mx, mv, mo, a, st);
}

}  // namespace tcs
}  // namespace lgp
