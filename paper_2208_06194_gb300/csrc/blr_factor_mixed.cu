// The mixed-precision instantiation of the persistent BLR-QR scheduler
// kernel: Householder panels, norms, tau and T in FP64; trailing compact-WY
// updates and the rounded additions in FP32.
#include "blr_tasks.cuh"

int blr_run_factor_mixed(const SchedParams& P, int ctas, cudaStream_t st) {
  // set once per device (a launch may be under stream capture, where the
  // attribute call is not a stream operation)
  static bool done[64] = {};
  int dev = 0;
  int rc = blr_cuda_check(cudaGetDevice(&dev), "cudaGetDevice");
  if (rc) return rc;
  if (dev < 0 || dev >= 64 || !done[dev]) {
    rc = blr_cuda_check(cudaFuncSetAttribute(k_factor<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             BLR_SMEM_BYTES), "smem attribute");
    if (rc) return rc;
    if (dev >= 0 && dev < 64) done[dev] = true;
  }
  k_factor<float><<<ctas, BLR_NT, BLR_SMEM_BYTES, st>>>(P);
  return blr_cuda_check(cudaGetLastError(), "launch k_factor<float>");
}
