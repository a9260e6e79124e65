// Self-test of the failure path of the bounded device waits. The pipelined
// kernels wait on mbarriers for their TMA copies with a bounded wait; when it
// gives up, the CTA sets the handle's device error word and the next
// lbm_nphase_moments / lbm_nphase_diagnostics call reports LBM_ETIMEOUT.
// Here one warp waits, with the same bounded wait, on an mbarrier that
// nothing arrives at, so the host side of that path can be tested on a GPU
// without a fault or a hang.
#include <cuda_runtime.h>

#include "lbm_kernels.cuh"
#include "lbm_nphase.h"

namespace lbm {
__global__ void stall_probe_kernel(int *err) {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  const bool ok = mbar_wait(&bar, 0);  // no arrival: gives up at the bound
  if (!ok && threadIdx.x == 0) atomicExch(err, 1);
}
}  // namespace lbm

extern "C" lbm_status lbm_nphase_selftest_wait_timeout(lbm_nphase_t *h) {
  if (!h) return LBM_EINVAL;
  lbm::stall_probe_kernel<<<1, 32, 0, h->stream>>>(h->g.err);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    h->cuda_err = (int)e;
    return LBM_ECUDA;
  }
  return LBM_OK;
}
