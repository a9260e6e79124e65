// Kernel instantiations for one storage precision (LBM_MIX_FP16).
#include "lbm_kernels.cuh"

LBM_DEFINE_PREC(f16, LBM_MIX_FP16)
