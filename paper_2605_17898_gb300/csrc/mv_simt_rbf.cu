// FP32 SIMT product kernels instantiated for the RBF kernel.
#include "mv_simt.cuh"

LGP_DEFINE_SIMT_DISPATCH(LGP_RBF, rbf)
