// Kernel instantiations for one storage precision (LBM_FP64).
#include "lbm_kernels.cuh"

LBM_DEFINE_PREC(f64, LBM_FP64)
