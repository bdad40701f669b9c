// BLR compression on the device (Section 3.1): diagonal tiles dense (weak
// admissibility), every other tile either its best rank-r approximation
// (one-sided Jacobi SVD, fixed rank) or a truncated column-pivoted
// Householder QR stopped at ||R22||_F <= tol ||A_ij||_F (the truncated
// rank-revealing QR used for compression in Section 5), which gives U with
// orthonormal columns.  A tile needing rank > the dense threshold stays
// dense (Section 3.1 fallback).
#include <cstdio>
#include "blr_device.cuh"

namespace {

struct CompressParams {
  int m, n, b, p, q, cap, dense_rank, fixed_rank;
  double tol;
  const double* a;
  long long lda;
  const double* x;
  const double* y;
  int dim, kernel;
  const double* scale;
  double* tiles;
  int* rank;
  double* scratch;
  size_t slab;
  int* status;
  const unsigned char* inadmissible;   // p*q flags (j*p + i), or NULL: weak admissibility
};

__device__ __forceinline__ double kernel_entry(const CompressParams& P, int gi, int gj) {
  double r2 = 0.0;
  for (int d = 0; d < P.dim; d++) {
    double diff = P.x[d + (size_t)gi * P.dim] - P.y[d + (size_t)gj * P.dim];
    r2 += diff * diff;
  }
  const double r = sqrt(r2);
  double v = (P.kernel == BLR_KERNEL_YUKAWA3D) ? exp(-r) / (r + 1e-3) : 1.0 / (r + 1e-3);
  if (P.scale) v *= P.scale[gj];
  return v;
}

__global__ void __launch_bounds__(BLR_NT, 1) k_compress(CompressParams P) {
  extern __shared__ double smem[];
  Ctx c;
  c.s = sm_carve(smem);
  c.status = P.status;
  c.fma = 0.0;
  const int b = P.b;
  double* W = P.scratch + (size_t)blockIdx.x * P.slab;   // b x b working tile
  double* A0 = W + (size_t)b * b;                        // original tile
  double* E = A0 + (size_t)b * b;                        // b x b (U build)
  double* tau = E + (size_t)b * b;                       // b
  for (int t = blockIdx.x; t < P.p * P.q; t += gridDim.x) {
    const int i = t % P.p, j = t / P.p;
    double* dest = P.tiles + (size_t)t * b * b;
    __syncthreads();
    for (int e = threadIdx.x; e < b * b; e += BLR_NT) {
      int r = e % b, cc = e / b;
      int gi = i * b + r, gj = j * b + cc;
      double v = P.a ? P.a[gi + (size_t)gj * P.lda] : kernel_entry(P, gi, gj);
      W[e] = v;
      A0[e] = v;
    }
    __syncthreads();
    if (i == j || (P.inadmissible && P.inadmissible[t])) {
      copy_mat(dest, b, A0, b, b, b);
      if (threadIdx.x == 0) P.rank[t] = -1;
      continue;
    }
    if (P.fixed_rank > 0) {
      double* sig = c.s.vec;
      int* order = c.s.ivec;
      jacobi_svd(W, b, b, sig, order, c);
      // keep min(fixed_rank, #nonzero sigma) columns so that U stays orthonormal
      __shared__ int rsh;
      if (threadIdx.x == 0) {
        int r = 0;
        while (r < P.fixed_rank && sig[order[r]] > 0.0) r++;
        rsh = r;
      }
      __syncthreads();
      const int r = rsh;
      for (int e = threadIdx.x; e < b * r; e += BLR_NT) {
        int a = e % b, l = e / b;
        int col = order[l];
        dest[a + (size_t)l * b] = W[a + (size_t)col * b] / sig[col];
      }
      __syncthreads();
      // V = A^T U
      gemm(b, r, b, 1.0, A0, b, true, dest, b, false, 0.0, dest + (size_t)b * P.cap, b, c);
      if (threadIdx.x == 0) P.rank[t] = r;
      continue;
    }
    // truncated pivoted QR
    double part = 0.0;
    for (int e = threadIdx.x; e < b * b; e += BLR_NT) part += A0[e] * A0[e];
    const double nrm2 = block_sum(part, c.s.red);
    const double tol2 = P.tol * P.tol * nrm2;
    int* perm = c.s.ivec;
    __shared__ int over_sh;
    const int r = qrcp(W, b, b, b, tol2, P.dense_rank, perm, tau, &over_sh, c);
    if (over_sh) {
      copy_mat(dest, b, A0, b, b, b);
      __syncthreads();
      if (threadIdx.x == 0) P.rank[t] = -1;
      continue;
    }
    // U = Q [I_r; 0]
    zero_mat(E, b, b, r);
    __syncthreads();
    for (int l = threadIdx.x; l < r; l += BLR_NT) E[l + (size_t)l * b] = 1.0;
    __syncthreads();
    apply_q_unblocked(W, b, b, r, tau, E, b, r, false, c);
    copy_mat(dest, b, E, b, b, r);
    // V = P R_r^T: V(perm[cc], l) = R(l, cc) for cc >= l
    double* V = dest + (size_t)b * P.cap;
    for (int e = threadIdx.x; e < b * r; e += BLR_NT) {
      int cc = e % b, l = e / b;
      V[perm[cc] + (size_t)l * b] = (cc >= l) ? W[l + (size_t)cc * b] : 0.0;
    }
    __syncthreads();
    if (threadIdx.x == 0) P.rank[t] = r;
  }
}

}  // namespace

int blr_compress_impl(const double* a_dev, int lda, const double* x_dev, const double* y_dev, int dim,
                      int kernel_id, const double* scale_dev, int m, int n, const blr_opts* o,
                      blr_matrix* out, cudaStream_t st, const unsigned char* inadmissible_dev) {
  CompressParams P{};
  P.inadmissible = inadmissible_dev;
  P.m = m; P.n = n; P.b = out->b; P.p = out->p; P.q = out->q; P.cap = out->cap;
  P.dense_rank = (o->dense_rank > 0 && o->dense_rank <= out->cap) ? o->dense_rank : out->cap;
  P.fixed_rank = o->fixed_rank;
  P.tol = o->tol;
  P.a = a_dev; P.lda = lda;
  P.x = x_dev; P.y = y_dev; P.dim = dim; P.kernel = kernel_id; P.scale = scale_dev;
  P.tiles = out->tiles; P.rank = out->rank;
  const int ntiles = P.p * P.q;
  int ctas = 2 * blr_num_sms();
  if (ctas > ntiles) ctas = ntiles;
  P.slab = (size_t)3 * P.b * P.b + P.b + 64;
  int rc = BLR_OK;
  int* status = nullptr;
  if ((rc = blr_cuda_check(cudaMalloc(&P.scratch, sizeof(double) * P.slab * ctas), "compress scratch"))) return rc;
  if ((rc = blr_cuda_check(cudaMalloc(&status, sizeof(int)), "compress status"))) { cudaFree(P.scratch); return rc; }
  P.status = status;
  do {
    if ((rc = blr_cuda_check(cudaMemsetAsync(status, 0, sizeof(int), st), "memset"))) break;
    if ((rc = blr_cuda_check(cudaMemsetAsync(out->tiles, 0, sizeof(double) * (size_t)ntiles * P.b * P.b, st), "memset tiles"))) break;
    if ((rc = blr_cuda_check(cudaFuncSetAttribute(k_compress, cudaFuncAttributeMaxDynamicSharedMemorySize, BLR_SMEM_BYTES), "smem attribute"))) break;
    k_compress<<<ctas, BLR_NT, BLR_SMEM_BYTES, st>>>(P);
    if ((rc = blr_cuda_check(cudaGetLastError(), "launch k_compress"))) break;
    if ((rc = blr_cuda_check(cudaStreamSynchronize(st), "k_compress"))) break;
    int s = 0;
    cudaMemcpy(&s, status, sizeof(int), cudaMemcpyDeviceToHost);
    if (s & ST_NUMERIC) { blr_set_error("compression met a non-finite value"); rc = BLR_ERR_NUMERIC; }
  } while (0);
  cudaFree(P.scratch);
  cudaFree(status);
  return rc;
}
