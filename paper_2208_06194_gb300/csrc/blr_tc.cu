// Stand-alone launch of the tensor-core GEMM building block (blr_tc.cuh):
// D = A B for FP64 device matrices with 3xTF32 products and FP32
// accumulation in TMEM.  It checks, in isolation, the primitive that the
// mixed-precision trapezoidal updates run on.
#include "blr_tc.cuh"

namespace {

constexpr int kTcN = 256;   // columns of D per CTA
constexpr size_t kTcStageFloats = 2 * (2 * (size_t)TC_M * TC_KC + 2 * (size_t)kTcN * TC_KC);
constexpr size_t kTcSmemBytes = kTcStageFloats * sizeof(float) + 1024;

__global__ void __launch_bounds__(BLR_NT, 1)
    k_tc_gemm(const double* A, long long lda, const double* B, long long ldb, double* D, long long ldd, int m,
              int n, int k, int* status, unsigned long long limit_ns) {
  extern __shared__ __align__(1024) float tc_smem[];
  __shared__ uint64_t bars[2];
  __shared__ uint32_t phase[2];
  __shared__ uint32_t tmem_base;
  __shared__ int unsafe;
  if (threadIdx.x < 32) tmem_alloc(&tmem_base, 512);   // main and cross-term accumulators
  if (threadIdx.x == 0) {
    mbar_init(&bars[0], 1);
    mbar_init(&bars[1], 1);
    phase[0] = phase[1] = 0;
    unsafe = 0;
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  TcCtx t;
  t.tmem = tmem_base;
  t.bar = bars;
  t.phase = phase;
  t.buf = tc_smem;
  t.bcap = kTcN;
  t.status = status;
  t.limit_ns = limit_ns;
  t.unsafe = &unsafe;
  const int mb = blockIdx.x, nb = blockIdx.y;
  const int m0 = mb * TC_M, n0 = nb * kTcN;
  const int mrow = min(TC_M, m - m0);
  const int ncol = min(kTcN, n - n0);
  const int ncol16 = (ncol + 15) & ~15;
  // A(r, kk) = A[(m0 + r) + kk * lda]; B^T(nn, kk) = B[kk + (n0 + nn) * ldb]
  const bool ok = tc_gemm_tile(t, 0, A + m0, 1, lda, mrow, B + (long long)n0 * ldb, ldb, 1, ncol, ncol16, k);
  if (ok) {
    tc_epilogue(t, 0, ncol16, [&](int r, int c, float v) {
      if (r < mrow && c < ncol) D[(m0 + r) + (long long)(n0 + c) * ldd] = (double)v;
    });
  }
  tc_fence_before();
  __syncthreads();
  if (threadIdx.x < 32 && !unsafe) tmem_dealloc(tmem_base, 512);
}

}  // namespace

extern "C" int blr_tc_gemm_selftest(const double* a_dev, int lda, const double* b_dev, int ldb, double* d_dev,
                                    int ldd, int m, int n, int k, void* stream) {
  if (!a_dev || !b_dev || !d_dev || m <= 0 || n <= 0 || k <= 0 || lda < m || ldb < k || ldd < m) {
    blr_set_error("blr_tc_gemm_selftest: bad arguments");
    return BLR_ERR_INVALID;
  }
  cudaStream_t st = (cudaStream_t)stream;
  int* status = nullptr;
  int rc = blr_cuda_check(cudaMalloc(&status, sizeof(int)), "status");
  if (rc) return rc;
  do {
    if ((rc = blr_cuda_check(cudaMemsetAsync(status, 0, sizeof(int), st), "memset"))) break;
    if ((rc = blr_cuda_check(cudaFuncSetAttribute(k_tc_gemm, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                  (int)kTcSmemBytes), "smem attribute")))
      break;
    dim3 grid((m + TC_M - 1) / TC_M, (n + kTcN - 1) / kTcN);
    k_tc_gemm<<<grid, BLR_NT, kTcSmemBytes, st>>>(a_dev, lda, b_dev, ldb, d_dev, ldd, m, n, k, status,
                                                  2000000000ull);
    if ((rc = blr_cuda_check(cudaGetLastError(), "launch k_tc_gemm"))) break;
    int s = 0;
    if ((rc = blr_cuda_check(cudaMemcpyAsync(&s, status, sizeof(int), cudaMemcpyDeviceToHost, st), "status"))) break;
    if ((rc = blr_cuda_check(cudaStreamSynchronize(st), "k_tc_gemm"))) break;
    if (s & ST_TIMEOUT) {
      blr_set_error("blr_tc_gemm_selftest: tensor-core completion wait timed out");
      rc = BLR_ERR_TIMEOUT;
    }
  } while (0);
  cudaFree(status);
  return rc;
}
