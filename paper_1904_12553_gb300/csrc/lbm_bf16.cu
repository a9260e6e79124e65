// Kernel instantiations for one storage precision (LBM_MIX_BF16).
#include "lbm_kernels.cuh"

LBM_DEFINE_PREC(bf16, LBM_MIX_BF16)
