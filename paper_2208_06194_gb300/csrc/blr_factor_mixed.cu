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

// ---------------------------------------------------------------------------
// blr_tc_update_bench: the dense prepared trapezoidal update (the body that
// carries most of the mixed path's work) timed on its own.  Every CTA of a
// persistent grid repeats the update on its own b x b tiles Ct, Cb with one
// shared slot of prepared operands; the values are synthetic (bounded), so
// the timing is that of the data movement and the products, not of a
// factorization.
// ---------------------------------------------------------------------------
namespace {

__global__ void k_bench_fill(double* d, size_t n, float* f, size_t nf) {
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n + nf; e += (size_t)gridDim.x * blockDim.x) {
    unsigned x = (unsigned)(e * 2654435761u) ^ 0x9e3779b9u;
    x ^= x >> 15;
    x *= 0x2c1b3c6du;
    x ^= x >> 12;
    const float v = (float)(x & 0xffff) / 65536.0f - 0.5f;
    if (e < n) d[e] = v;
    else f[e - n] = v * 0.01f;
  }
}

template <int V>
__global__ void __launch_bounds__(BLR_NT, 1)
    k_tc_update_bench(SchedParams P, double* ct_all, double* cb_all, const float* slot, int reps,
                      unsigned long long* ns_out) {
  extern __shared__ double smem[];
  Ctx c;
  c.s = sm_carve(smem);
  c.status = P.status;
  c.fma = 0.0;
  __shared__ uint64_t tc_bars[2];
  __shared__ uint32_t tc_phase[2];
  __shared__ uint32_t tc_tmem;
  __shared__ uint64_t tq_full[2], tq_empty[2];
  __shared__ uint32_t tq_ph[4];
  __shared__ int tc_unsafe;
  if (threadIdx.x < 32) tmem_alloc(&tc_tmem, 512);
  if (threadIdx.x == 0) {
    mbar_init(&tc_bars[0], 1);
    mbar_init(&tc_bars[1], 1);
    tc_phase[0] = tc_phase[1] = 0;
    for (int s2 = 0; s2 < 2; s2++) {
      mbar_init(&tq_full[s2], 1);
      mbar_init(&tq_empty[s2], 1);
    }
    for (int s2 = 0; s2 < 4; s2++) tq_ph[s2] = 0;
    tc_unsafe = 0;
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  TcCtx tcx;
  tcx.tmem = tc_tmem;
  tcx.bar = tc_bars;
  tcx.phase = tc_phase;
  tcx.buf = reinterpret_cast<float*>(smem);
  tcx.bcap = 256;
  tcx.status = P.status;
  tcx.limit_ns = (unsigned long long)P.watchdog_ns;
  tcx.unsafe = &tc_unsafe;
  TcBulk tq{tq_full, tq_empty, tq_ph};
  TaskEnv env{&P, P.scratch + (size_t)blockIdx.x * P.slab, 0, false, &tcx, &tq, nullptr, -1, nullptr, 0};
  const size_t bb = (size_t)P.b * P.b;
  double* Ct = ct_all + blockIdx.x * bb;
  double* Cb = cb_all + blockIdx.x * bb;
  __syncthreads();
  const unsigned long long t0 = gtimer();
  for (int r = 0; r < reps; r++) {
    env.used = 0;
    tc_apply_prepared<V>(env, slot, Ct, Cb, c);
  }
  __syncthreads();
  if (threadIdx.x == 0) ns_out[blockIdx.x] = gtimer() - t0;
  tc_fence_before();
  __syncthreads();
  if (threadIdx.x < 32 && !tc_unsafe) tmem_dealloc(tc_tmem, 512);
}

template <int V>
int launch_update_bench(const SchedParams& P, int ctas, double* ct, double* cb, const float* slot, int reps,
                        unsigned long long* ns, cudaStream_t st) {
  int rc = blr_cuda_check(cudaFuncSetAttribute(k_tc_update_bench<V>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               BLR_SMEM_BYTES), "smem attribute");
  if (rc) return rc;
  k_tc_update_bench<V><<<ctas, BLR_NT, BLR_SMEM_BYTES, st>>>(P, ct, cb, slot, reps, ns);
  return blr_cuda_check(cudaGetLastError(), "launch k_tc_update_bench");
}

}  // namespace

extern "C" int blr_tc_update_bench(int b, int ctas, int reps, int variant, double* ms_per_update,
                                   double* aggregate_tflops) {
  if (b < 128 || b > BLR_BMAX || b % 128 != 0 || ctas < 1 || reps < 1 || !ms_per_update) {
    blr_set_error("blr_tc_update_bench: b must be a multiple of 128 in [128, %d], ctas and reps >= 1", BLR_BMAX);
    return BLR_ERR_INVALID;
  }
  static const int kVariants[] = {0, 1, 2, 3, 4, 6, 9, 11, 15, 17, 19};
  bool known = false;
  for (int v : kVariants) known = known || v == variant;
  if (!known) {
    blr_set_error("blr_tc_update_bench: variant %d not built (0, 1, 2, 3, 4, 6, 9, 11, 15, 17, 19)", variant);
    return BLR_ERR_INVALID;
  }
  const int Rp = b;
  const size_t bb = (size_t)b * b, slot_floats = (size_t)6 * Rp * b, slab = (size_t)4 * bb;
  double *ct = nullptr, *cb = nullptr, *scratch = nullptr;
  float* slot = nullptr;
  int* status = nullptr;
  unsigned long long* ns = nullptr;
  unsigned long long* phase = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int rc = BLR_OK;
  do {
    if ((rc = blr_cuda_check(cudaMalloc(&ct, sizeof(double) * bb * ctas * 2), "bench tiles"))) break;
    cb = ct + bb * ctas;
    if ((rc = blr_cuda_check(cudaMalloc(&scratch, sizeof(double) * slab * ctas), "bench scratch"))) break;
    if ((rc = blr_cuda_check(cudaMalloc(&slot, sizeof(float) * slot_floats), "bench slot"))) break;
    if ((rc = blr_cuda_check(cudaMalloc(&status, sizeof(int)), "bench status"))) break;
    if ((rc = blr_cuda_check(cudaMalloc(&ns, sizeof(unsigned long long) * ctas), "bench timers"))) break;
    if ((rc = blr_cuda_check(cudaMemset(status, 0, sizeof(int)), "memset"))) break;
    k_bench_fill<<<4 * blr_num_sms(), 256>>>(ct, bb * ctas * 2, slot, slot_floats);
    if ((rc = blr_cuda_check(cudaDeviceSynchronize(), "bench fill"))) break;
    SchedParams P{};
#ifdef BLR_PHASE_TIMING
    if ((rc = blr_cuda_check(cudaMalloc(&P.phase, 32 * sizeof(unsigned long long)), "phase counters"))) break;
    cudaMemset(P.phase, 0, 32 * sizeof(unsigned long long));
    phase = P.phase;
#endif
    P.b = b;
    P.cap = b / 2;
    P.prep_rp = Rp;
    P.status = status;
    P.watchdog_ns = 2000000000ll;
    P.scratch = scratch;
    P.slab = slab;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0);
    switch (variant) {
      case 0: rc = launch_update_bench<0>(P, ctas, ct, cb, slot, reps, ns, 0); break;
      case 1: rc = launch_update_bench<1>(P, ctas, ct, cb, slot, reps, ns, 0); break;
      case 2: rc = launch_update_bench<2>(P, ctas, ct, cb, slot, reps, ns, 0); break;
      case 3: rc = launch_update_bench<3>(P, ctas, ct, cb, slot, reps, ns, 0); break;
      case 4: rc = launch_update_bench<4>(P, ctas, ct, cb, slot, reps, ns, 0); break;
      case 6: rc = launch_update_bench<6>(P, ctas, ct, cb, slot, reps, ns, 0); break;
      case 9: rc = launch_update_bench<9>(P, ctas, ct, cb, slot, reps, ns, 0); break;
      case 11: rc = launch_update_bench<11>(P, ctas, ct, cb, slot, reps, ns, 0); break;
      case 15: rc = launch_update_bench<15>(P, ctas, ct, cb, slot, reps, ns, 0); break;
      case 17: rc = launch_update_bench<17>(P, ctas, ct, cb, slot, reps, ns, 0); break;
      default: rc = launch_update_bench<19>(P, ctas, ct, cb, slot, reps, ns, 0); break;
    }
    if (rc) break;
    cudaEventRecord(e1);
    if ((rc = blr_cuda_check(cudaEventSynchronize(e1), "k_tc_update_bench"))) break;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    std::vector<unsigned long long> h(ctas);
    cudaMemcpy(h.data(), ns, sizeof(unsigned long long) * ctas, cudaMemcpyDeviceToHost);
    int s = 0;
    cudaMemcpy(&s, status, sizeof(int), cudaMemcpyDeviceToHost);
    if ((rc = blr_cuda_check(cudaGetLastError(), "bench readback"))) break;
    if (s & ST_TIMEOUT) { blr_set_error("blr_tc_update_bench: a tensor-core wait ran out"); rc = BLR_ERR_TIMEOUT; break; }
    double sum = 0.0;
    for (unsigned long long v : h) sum += (double)v;
    *ms_per_update = sum / ctas / reps * 1e-6;
    // algorithmic flops of one update: 2 b^3 (Z and Cb -= Y W) + b^3 / 2 (W), times two
    if (aggregate_tflops) *aggregate_tflops = 2.0 * 2.5 * (double)b * b * b * ctas * reps / (ms * 1e-3) / 1e12;
  } while (0);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(ct);
  cudaFree(scratch);
  cudaFree(slot);
  cudaFree(status);
  cudaFree(ns);
  if (phase) cudaFree(phase);
  return rc;
}
