// Host side of blr_qr: builds the scheduler state of the tile DAG of
// Algorithm 4 and launches the persistent kernel (blr_factor_fp64.cu,
// blr_factor_mixed.cu); plus the host-only check of the DAG formulas.
#include <cstdio>
#include <cstdlib>
#include <algorithm>
#include <vector>
#include "blr_internal.h"
#include "blr_dag.h"

// ---------------------------------------------------------------------------
// Host side of blr_qr
// ---------------------------------------------------------------------------
int blr_launch_factor(blr_factor* f, const blr_opts* o, cudaStream_t st) {
  blr_matrix& A = f->a;
  const int p = A.p, q = A.q, b = A.b;
  std::vector<int> offL(q + 1), offS(q + 1), offP(q + 1);
  const int n_tasks = dag_offsets(p, q, offL.data(), offS.data(), offP.data());
  DagShape d{p, q, offL.data(), offS.data(), offP.data()};
  std::vector<int> deps(n_tasks);
  for (int id = 0; id < n_tasks; id++) {
    int i, j, k;
    int t = dag_decode(d, id, &i, &j, &k);
    deps[id] = dag_indegree(t, i, j, k);
  }
  std::vector<long long> toff(q);
  long long acc = 0;
  for (int k = 0; k < q; k++) { toff[k] = acc; acc += p - k; }

  const int nsm = blr_num_sms();
  int ctas = o->sched_ctas > 0 ? o->sched_ctas : nsm;
  const size_t slab = (size_t)(o->scratch_b2 > 0 ? o->scratch_b2 : BLR_SLAB_B2) * b * b;

  // one device block for all scheduler state
  size_t bytes = 0;
  auto take = [&](size_t n) { size_t off = bytes; bytes += (n + 255) & ~(size_t)255; return off; };
  const size_t o_offL = take(sizeof(int) * (q + 1)), o_offS = take(sizeof(int) * (q + 1)),
               o_offP = take(sizeof(int) * (q + 1)), o_toff = take(sizeof(long long) * q),
               o_deps = take(sizeof(int) * n_tasks), o_qbuf = take(sizeof(int) * (size_t)BLR_NQ * n_tasks),
               o_qh = take(sizeof(int) * 32 * BLR_NQ), o_qt = take(sizeof(int) * 32 * BLR_NQ),
               o_done = take(sizeof(int)), o_status = take(sizeof(int)),
               o_prog = take(sizeof(unsigned long long)), o_flops = take(sizeof(double) * 4),
               o_ntask = take(sizeof(unsigned long long) * 4), o_tns = take(sizeof(unsigned long long) * 4),
               o_nvar = take(sizeof(unsigned long long) * 8), o_tvar = take(sizeof(unsigned long long) * 8),
               o_fvar = take(sizeof(double) * 8), o_peak = take(sizeof(unsigned long long));
  char* base = nullptr;
  double* scratch = nullptr;
  if (cudaMalloc(&base, bytes) != cudaSuccess) { blr_set_error("blr_qr: out of device memory (scheduler state)"); return BLR_ERR_OOM; }
  if (cudaMalloc(&scratch, sizeof(double) * slab * ctas) != cudaSuccess) {
    cudaFree(base);
    blr_set_error("blr_qr: out of device memory (scratch %zu MB)", sizeof(double) * slab * ctas >> 20);
    return BLR_ERR_OOM;
  }
  // mixed path: tensor-core operands of every dense reflector block, one
  // slot per (i,k) with i >= k (the T layout), 6 x Rp x b floats each; if the
  // device cannot hold them the updates stage their operands themselves
  float* prep = nullptr;
  const int prep_rp = (b + 127) / 128 * 128;
  if (o->precision == BLR_PREC_MIXED) {
    const size_t pbytes = (size_t)f->nt * 6 * prep_rp * b * sizeof(float);
    if (cudaMalloc(&prep, pbytes) != cudaSuccess) {
      prep = nullptr;
      cudaGetLastError();
    }
  }
  int rc = BLR_OK;
  SchedParams P{};
#ifdef BLR_PHASE_TIMING
  cudaMalloc(&P.phase, 16 * sizeof(unsigned long long));
  cudaMemset(P.phase, 0, 16 * sizeof(unsigned long long));
#endif
  P.prep = prep;
  P.prep_rp = prep_rp;
  P.p = p; P.q = q; P.b = b; P.cap = A.cap;
  P.dense_rank = (o->dense_rank > 0 && o->dense_rank <= A.cap) ? o->dense_rank : A.cap;
  P.precision = o->precision;
  P.rec_tol = o->rec_tol > 0 ? o->rec_tol : o->tol;
  P.tiles = A.tiles; P.rank = A.rank; P.t = f->t;
  P.toff_dev = (const long long*)(base + o_toff);
  P.off_larfb = (const int*)(base + o_offL);
  P.off_tsqrt = (const int*)(base + o_offS);
  P.off_tpmqrt = (const int*)(base + o_offP);
  P.n_tasks = n_tasks;
  P.deps = (int*)(base + o_deps);
  P.qbuf = (int*)(base + o_qbuf);
  P.qhead = (int*)(base + o_qh);
  P.qtail = (int*)(base + o_qt);
  P.done = (int*)(base + o_done);
  P.status = (int*)(base + o_status);
  P.progress_ns = (unsigned long long*)(base + o_prog);
  P.watchdog_ns = (long long)(o->watchdog_ms > 0 ? o->watchdog_ms : 20000) * 1000000ll;
  P.scratch = scratch;
  P.slab = slab;
  P.flops = (double*)(base + o_flops);
  P.ntask = (unsigned long long*)(base + o_ntask);
  P.tns = (unsigned long long*)(base + o_tns);
  P.nvar = (unsigned long long*)(base + o_nvar);
  P.tvar = (unsigned long long*)(base + o_tvar);
  P.fvar = (double*)(base + o_fvar);
  P.slab_peak = (unsigned long long*)(base + o_peak);

  cudaEvent_t e0 = nullptr, e1 = nullptr;
  do {
    if ((rc = blr_cuda_check(cudaMemsetAsync(base, 0, bytes, st), "memset scheduler"))) break;
    if ((rc = blr_cuda_check(cudaMemsetAsync(P.qbuf, 0xff, sizeof(int) * (size_t)BLR_NQ * n_tasks, st), "memset queues"))) break;
    if ((rc = blr_cuda_check(cudaMemcpyAsync((void*)P.off_larfb, offL.data(), sizeof(int) * (q + 1), cudaMemcpyHostToDevice, st), "copy offsets"))) break;
    if ((rc = blr_cuda_check(cudaMemcpyAsync((void*)P.off_tsqrt, offS.data(), sizeof(int) * (q + 1), cudaMemcpyHostToDevice, st), "copy offsets"))) break;
    if ((rc = blr_cuda_check(cudaMemcpyAsync((void*)P.off_tpmqrt, offP.data(), sizeof(int) * (q + 1), cudaMemcpyHostToDevice, st), "copy offsets"))) break;
    if ((rc = blr_cuda_check(cudaMemcpyAsync((void*)P.toff_dev, toff.data(), sizeof(long long) * q, cudaMemcpyHostToDevice, st), "copy T offsets"))) break;
    if ((rc = blr_cuda_check(cudaMemcpyAsync(P.deps, deps.data(), sizeof(int) * n_tasks, cudaMemcpyHostToDevice, st), "copy deps"))) break;
    // the only initially ready task: GEQRT(0) in queue 0
    int first = 0, one = 1;
    if ((rc = blr_cuda_check(cudaMemcpyAsync(P.qbuf, &first, sizeof(int), cudaMemcpyHostToDevice, st), "seed queue"))) break;
    if ((rc = blr_cuda_check(cudaMemcpyAsync(P.qtail, &one, sizeof(int), cudaMemcpyHostToDevice, st), "seed queue"))) break;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0, st);
    rc = (P.precision == BLR_PREC_MIXED) ? blr_run_factor_mixed(P, ctas, st) : blr_run_factor_fp64(P, ctas, st);
    if (rc) break;
    cudaEventRecord(e1, st);
    if ((rc = blr_cuda_check(cudaStreamSynchronize(st), "k_factor"))) break;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    f->seconds = ms * 1e-3;
    int status = 0, done = 0;
    double fl[4];
    unsigned long long nt[4], tns[4];
    cudaMemcpy(tns, P.tns, sizeof(tns), cudaMemcpyDeviceToHost);
    cudaMemcpy(&status, P.status, sizeof(int), cudaMemcpyDeviceToHost);
    cudaMemcpy(&done, P.done, sizeof(int), cudaMemcpyDeviceToHost);
    cudaMemcpy(fl, P.flops, sizeof(fl), cudaMemcpyDeviceToHost);
    cudaMemcpy(nt, P.ntask, sizeof(nt), cudaMemcpyDeviceToHost);
    unsigned long long nv[8], tv[8];
    double fv[8];
    cudaMemcpy(nv, P.nvar, sizeof(nv), cudaMemcpyDeviceToHost);
    cudaMemcpy(tv, P.tvar, sizeof(tv), cudaMemcpyDeviceToHost);
    cudaMemcpy(fv, P.fvar, sizeof(fv), cudaMemcpyDeviceToHost);
    unsigned long long peak = 0;
    cudaMemcpy(&peak, P.slab_peak, sizeof(peak), cudaMemcpyDeviceToHost);
    f->scratch_peak_bytes = (long long)(peak * sizeof(double));
    f->scratch_bytes = (long long)(sizeof(double) * slab * ctas);
    for (int v = 0; v < 8; v++) {
      f->tpmqrt_kind[v] = (long long)nv[v];
      f->tpmqrt_kind_seconds[v] = tv[v] * 1e-9;
      f->tpmqrt_kind_flops[v] = fv[v];
    }
    f->flops[4] = 0;
    for (int t = 0; t < 4; t++) {
      f->flops[t] = fl[t];
      f->flops[4] += fl[t];
      f->tasks[t] = (long long)nt[t];
      f->task_seconds[t] = tns[t] * 1e-9;
    }
    if (status & ST_TIMEOUT) { blr_set_error("blr_qr: scheduler watchdog expired (%d of %d tasks done)", done, n_tasks); rc = BLR_ERR_TIMEOUT; break; }
    if (status & ST_NUMERIC) { blr_set_error("blr_qr: non-finite Householder coefficient"); rc = BLR_ERR_NUMERIC; break; }
    if (status & ST_RANK) { blr_set_error("blr_qr: scratch slab exceeded"); rc = BLR_ERR_RANK_OVERFLOW; break; }
    if (status != 0 || done != n_tasks) { blr_set_error("blr_qr: scheduler ended with status %d, %d of %d tasks", status, done, n_tasks); rc = BLR_ERR_CUDA; break; }
  } while (0);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(scratch);
  cudaFree(base);
  if (prep) cudaFree(prep);
#ifdef BLR_PHASE_TIMING
  {
    unsigned long long ph[16];
    cudaMemcpy(ph, P.phase, sizeof(ph), cudaMemcpyDeviceToHost);
    fprintf(stderr, "blr_qr phases (CTA-s):");
    for (int i2 = 0; i2 < 16; i2++) fprintf(stderr, " %d:%.2f", i2, ph[i2] * 1e-9);
    fprintf(stderr, "\n");
    cudaFree(P.phase);
  }
#endif
  return rc;
}

// Host-side check of the DAG formulas (no device work): builds the DAG from
// dag_successors, checks every in-degree against dag_indegree, and runs the
// counter protocol in a seeded random order, checking that each task runs
// exactly once, after all of its predecessors, and that the per-tile writer
// chains of Algorithm 4 are respected.  Returns 0 on success, or a positive
// code naming the first failed check.
extern "C" int blr_dag_selfcheck(int p, int q, unsigned seed) {
  if (p < 1 || q < 1 || q > p) return 100;
  std::vector<int> offL(q + 1), offS(q + 1), offP(q + 1);
  const int n = dag_offsets(p, q, offL.data(), offS.data(), offP.data());
  DagShape d{p, q, offL.data(), offS.data(), offP.data()};
  std::vector<int> indeg(n, 0), deps(n), order_done(n, -1);
  int bad = 0;
  for (int id = 0; id < n; id++) {
    int i, j, k;
    int t = dag_decode(d, id, &i, &j, &k);
    if (t < 0) return 1;
    if (t == 0 && dag_id_geqrt(d, k) != id) return 11;
    if (t == 1 && dag_id_larfb(d, k, j) != id) return 11;
    if (t == 2 && dag_id_tsqrt(d, i, k) != id) return 11;
    if (t == 3 && dag_id_tpmqrt(d, i, j, k) != id) return 11;
    dag_for_each_successor(d, t, i, j, k, [&](int sid) {
      if (sid < 0 || sid >= n) bad = 1;
      else indeg[sid]++;
    });
    if (bad) return 2;
  }
  for (int id = 0; id < n; id++) {
    int i, j, k;
    int t = dag_decode(d, id, &i, &j, &k);
    if (indeg[id] != dag_indegree(t, i, j, k)) return 3;
    deps[id] = indeg[id];
  }
  // random-order execution of the counter protocol
  std::vector<int> ready;
  for (int id = 0; id < n; id++) if (deps[id] == 0) ready.push_back(id);
  unsigned st = seed * 2654435761u + 12345u;
  // tile version counters: number of writes each tile has seen
  std::vector<int> ver((size_t)p * q, 0);
  int executed = 0;
  while (!ready.empty()) {
    st = st * 1664525u + 1013904223u;
    size_t pick = st % ready.size();
    int id = ready[pick];
    ready[pick] = ready.back();
    ready.pop_back();
    int i, j, k;
    int t = dag_decode(d, id, &i, &j, &k);
    // Algorithm 4 writer chain: before step k's write, tile (a,c) has been
    // written once per earlier step that touched it (min(a,c,k) steps), plus
    // for R_kj / R_kk the earlier i of this step.
    auto expect = [&](int a, int c2) { return std::min(std::min(a, c2), k); };
    if (t == 0) { if (ver[(size_t)k * p + k] != expect(k, k)) return 4; ver[(size_t)k * p + k]++; }
    if (t == 1) {
      if (ver[(size_t)j * p + k] != expect(k, j)) return 5;
      if (ver[(size_t)k * p + k] < k + 1) return 12;                  // reads Y_kk after GEQRT(k)
      ver[(size_t)j * p + k]++;
    }
    if (t == 2) {
      if (ver[(size_t)k * p + i] != expect(i, k)) return 6;
      ver[(size_t)k * p + i]++;
      if (ver[(size_t)k * p + k] != k + 1 + (i - k - 1)) return 7;   // R_kk after GEQRT and i-k-1 TSQRTs
      ver[(size_t)k * p + k]++;
    }
    if (t == 3) {
      if (ver[(size_t)k * p + i] != k + 1) return 13;                 // reads Y~_ik after TSQRT(i,k)
      if (ver[(size_t)j * p + i] != expect(i, j)) return 8;
      ver[(size_t)j * p + i]++;
      if (ver[(size_t)j * p + k] != k + 1 + (i - k - 1)) return 9;   // R_kj after LARFB and i-k-1 updates
      ver[(size_t)j * p + k]++;
    }
    order_done[id] = executed++;
    dag_for_each_successor(d, t, i, j, k, [&](int sid) {
      if (--deps[sid] == 0) ready.push_back(sid);
    });
  }
  if (executed != n) return 10;
  return 0;
}
