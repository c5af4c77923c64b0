// FP32 SIMT product kernels instantiated for the Matern-3/2 kernel.
#include "mv_simt.cuh"

LGP_DEFINE_SIMT_DISPATCH(LGP_MATERN32, m32)
