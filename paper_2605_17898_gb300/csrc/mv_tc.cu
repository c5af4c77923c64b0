// Tensor-core (tcgen05) split-BF16 product: placeholder until the kernel lands.
#include "lgp_internal.cuh"

namespace lgp {

bool tc_supported(int t) { (void)t; return false; }
int64_t tc_vsplit_bytes(int64_t Np, int t) { return 2 * Np * t * 2; }
int64_t mv_tc_partial_floats(int64_t Np, int t, int num_sms) { (void)Np; (void)t; (void)num_sms; return 0; }
cudaError_t launch_mv_tc(const KernelParams &, const float *, int64_t, int64_t, const float *, int64_t, float *,
                         int64_t, int, void *, float *, int64_t, const int *, int *, long long, int, cudaStream_t) {
    return cudaErrorNotSupported;
}

}  // namespace lgp
