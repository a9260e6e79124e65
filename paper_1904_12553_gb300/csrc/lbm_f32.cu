// Kernel instantiations for one storage precision (LBM_FP32).
#include "lbm_kernels.cuh"

LBM_DEFINE_PREC(f32, LBM_FP32)
