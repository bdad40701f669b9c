// The FP64 instantiation of the persistent BLR-QR scheduler kernel: every
// step of the factorization in double precision.
#include "blr_tasks.cuh"

int blr_run_factor_fp64(const SchedParams& P, int ctas, cudaStream_t st) {
  int rc = blr_cuda_check(cudaFuncSetAttribute(k_factor<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               BLR_SMEM_BYTES), "smem attribute");
  if (rc) return rc;
  k_factor<double><<<ctas, BLR_NT, BLR_SMEM_BYTES, st>>>(P);
  return blr_cuda_check(cudaGetLastError(), "launch k_factor<double>");
}
