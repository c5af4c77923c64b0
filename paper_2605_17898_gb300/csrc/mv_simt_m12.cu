// FP32 SIMT product kernels instantiated for the Matern-1/2 kernel.
#include "mv_simt.cuh"

LGP_DEFINE_SIMT_DISPATCH(LGP_MATERN12, m12)
