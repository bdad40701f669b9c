// The FP64 instantiation of the persistent BLR-QR scheduler kernel: every
// step of the factorization in double precision.
#include "blr_tasks.cuh"

int blr_run_factor_fp64(const SchedParams& P, int ctas, cudaStream_t st) {
  // set once per device (a launch may be under stream capture, where the
  // attribute call is not a stream operation)
  static bool done[64] = {};
  int dev = 0;
  int rc = blr_cuda_check(cudaGetDevice(&dev), "cudaGetDevice");
  if (rc) return rc;
  if (dev < 0 || dev >= 64 || !done[dev]) {
    rc = blr_cuda_check(cudaFuncSetAttribute(k_factor<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             BLR_SMEM_BYTES), "smem attribute");
    if (rc) return rc;
    if (dev >= 0 && dev < 64) done[dev] = true;
  }
  k_factor<double><<<ctas, BLR_NT, BLR_SMEM_BYTES, st>>>(P);
  return blr_cuda_check(cudaGetLastError(), "launch k_factor<double>");
}
