// Host side of blr_qr and blr_qr_batched: builds the scheduler state of the
// tile DAGs of Algorithm 4 (one or several matrices), launches the
// persistent kernel (blr_factor_fp64.cu, blr_factor_mixed.cu) and reads its
// status back; the capturable launch plans; and the host-only check of the
// DAG formulas.
#include <cstdio>
#include <cstdlib>
#include <algorithm>
#include <vector>
#include "blr_internal.h"
#include "blr_dag.h"

// ---------------------------------------------------------------------------
// Host side: a launch plan for one persistent scheduler launch over the tile
// DAGs of one or several matrices (a batch).  The plan holds every device
// buffer the launch needs; plan_launch only resets state with device-side
// copies and memsets and launches the kernel (no allocation, no host
// synchronisation), so it can be captured in a CUDA graph; plan_finish reads
// the status back.
// ---------------------------------------------------------------------------
struct blr_batch_plan {
  int count = 0;
  blr_opts opts{};
  std::vector<blr_factor*> fac;           // the factors (storage the launch writes)
  std::vector<const blr_matrix*> src;     // graph mode: tiles restored from these at each launch
  bool owns_factors = false;
  char* base = nullptr;                   // device: static part, then the state reset per launch
  size_t dyn_off = 0, dyn_bytes = 0;
  int* deps0 = nullptr;                   // device: initial dependency counters
  int* seed = nullptr;                    // device: the count initially ready tasks, then count
  double* scratch = nullptr;
  float* prep = nullptr;                  // pool of prepared tensor-core operands (mixed path)
  int* prep_state = nullptr;              // pool state: per-slot counters, search start, misses, then slot_of
  size_t prep_state_zero = 0;             // bytes of prep_state reset to 0 per launch (the rest to -1)
  size_t prep_state_bytes = 0;
  int nslot = 0;
  blr_trace_event* trace = nullptr;       // opts.trace events (device)
  SchedParams P{};
  int ctas = 0, n_tasks = 0;
  size_t slab = 0;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
};

static void plan_free(blr_batch_plan* pl) {
  if (!pl) return;
  if (pl->e0) cudaEventDestroy(pl->e0);
  if (pl->e1) cudaEventDestroy(pl->e1);
  if (pl->scratch) cudaFree(pl->scratch);
  if (pl->prep) cudaFree(pl->prep);
  if (pl->prep_state) cudaFree(pl->prep_state);
  if (pl->trace) cudaFree(pl->trace);
  if (pl->base) cudaFree(pl->base);
#ifdef BLR_PHASE_TIMING
  if (pl->P.phase) cudaFree(pl->P.phase);
#endif
  if (pl->owns_factors)
    for (blr_factor* f : pl->fac) blr_destroy_factor(f);
  delete pl;
}

// Builds the plan for factors whose storage (tiles, ranks, T) exists.
static int plan_build(blr_factor* const* fs, int count, const blr_opts* o, blr_batch_plan** out) {
  blr_batch_plan* pl = new blr_batch_plan;
  pl->count = count;
  pl->opts = *o;
  pl->fac.assign(fs, fs + count);
  struct Mat {
    int p, q, b, nt;
    std::vector<int> offL, offS, offP;
    std::vector<long long> toff;
    size_t o_offL, o_offS, o_offP, o_toff, slot_of_off, chain_off;
    int base;
  };
  std::vector<Mat> M(count);
  int total = 0, bmax = 0;
  size_t slot_floats = 0, nt_total = 0, chain_total = 0;
  for (int m = 0; m < count; m++) {
    const blr_matrix& A = fs[m]->a;
    Mat& x = M[m];
    x.p = A.p; x.q = A.q; x.b = A.b; x.nt = fs[m]->nt;
    x.offL.resize(x.q + 1); x.offS.resize(x.q + 1); x.offP.resize(x.q + 1);
    x.base = total;
    total += dag_offsets(x.p, x.q, x.offL.data(), x.offS.data(), x.offP.data());
    x.toff.resize(x.q);
    long long acc = 0;
    for (int k = 0; k < x.q; k++) { x.toff[k] = acc; acc += x.p - k; }
    bmax = std::max(bmax, x.b);
    x.chain_off = chain_total;
    chain_total += (size_t)x.nt;
    x.slot_of_off = nt_total;
    nt_total += (size_t)x.nt;
    slot_floats = std::max(slot_floats, (size_t)6 * ((x.b + 127) / 128 * 128) * x.b);
  }
  pl->n_tasks = total;
  std::vector<int> deps(total);
  for (int m = 0; m < count; m++) {
    Mat& x = M[m];
    DagShape d{x.p, x.q, x.offL.data(), x.offS.data(), x.offP.data()};
    const int nm = (m + 1 < count ? M[m + 1].base : total) - x.base;
    for (int id = 0; id < nm; id++) {
      int i, j, k;
      const int t = dag_decode(d, id, &i, &j, &k);
      deps[x.base + id] = dag_indegree(t, i, j, k);
    }
  }
  // device layout: [static: per-matrix offsets, params, bases, deps0, seed][state]
  size_t bytes = 0;
  auto take = [&](size_t n) { size_t off = bytes; bytes += (n + 255) & ~(size_t)255; return off; };
  for (int m = 0; m < count; m++) {
    M[m].o_offL = take(sizeof(int) * (M[m].q + 1));
    M[m].o_offS = take(sizeof(int) * (M[m].q + 1));
    M[m].o_offP = take(sizeof(int) * (M[m].q + 1));
    M[m].o_toff = take(sizeof(long long) * M[m].q);
  }
  const size_t o_mats = take(sizeof(SchedParams) * count), o_mbase = take(sizeof(int) * (count + 1)),
               o_deps0 = take(sizeof(int) * total), o_seed = take(sizeof(int) * (count + 1));
  pl->dyn_off = bytes;
  const size_t o_deps = take(sizeof(int) * total), o_qbuf = take(sizeof(int) * (size_t)BLR_NQ * total),
               o_qh = take(sizeof(int) * 32 * BLR_NQ), o_qt = take(sizeof(int) * 32 * BLR_NQ),
               o_done = take(sizeof(int)), o_status = take(sizeof(int)), o_prog = take(sizeof(unsigned long long)),
               o_flops = take(sizeof(double) * 4), o_ntask = take(sizeof(unsigned long long) * 4),
               o_tns = take(sizeof(unsigned long long) * 4), o_nvar = take(sizeof(unsigned long long) * 8),
               o_tvar = take(sizeof(unsigned long long) * 8), o_fvar = take(sizeof(double) * 8),
               o_peak = take(sizeof(unsigned long long)), o_tracen = take(sizeof(unsigned int)),
               o_chain = take(sizeof(int) * chain_total);
  pl->dyn_bytes = bytes - pl->dyn_off;
  const int nsm = blr_num_sms();
  pl->ctas = o->sched_ctas > 0 ? o->sched_ctas : nsm;
  pl->slab = (size_t)(o->scratch_b2 > 0 ? o->scratch_b2 : BLR_SLAB_B2) * bmax * bmax;
  if (cudaMalloc(&pl->base, bytes) != cudaSuccess) {
    plan_free(pl);
    blr_set_error("blr_qr: out of device memory (scheduler state)");
    return BLR_ERR_OOM;
  }
  if (cudaMalloc(&pl->scratch, sizeof(double) * pl->slab * pl->ctas) != cudaSuccess) {
    const size_t mb = sizeof(double) * pl->slab * pl->ctas >> 20;
    plan_free(pl);
    blr_set_error("blr_qr: out of device memory (scratch %zu MB)", mb);
    return BLR_ERR_OOM;
  }
  // mixed path: a pool of slots for the tensor-core operands of reflector
  // blocks, one per block when the device has room (or opts.prep_slots); a
  // block that finds no free slot is applied from its stored factors
  if (o->precision == BLR_PREC_MIXED) {
    size_t want = nt_total;
    if (o->prep_slots > 0) {
      want = std::min(want, (size_t)o->prep_slots);
    } else {
      size_t fr = 0, tot = 0;
      const size_t reserve = (size_t)4 << 30;
      if (cudaMemGetInfo(&fr, &tot) == cudaSuccess)
        want = std::min(want, fr > reserve ? (fr - reserve) / (slot_floats * sizeof(float)) : (size_t)0);
      cudaGetLastError();
    }
    while (want > 0 && cudaMalloc(&pl->prep, sizeof(float) * slot_floats * want) != cudaSuccess) {
      pl->prep = nullptr;
      cudaGetLastError();
      want /= 2;
    }
    pl->nslot = pl->prep ? (int)want : 0;
    if (pl->prep) {
      pl->prep_state_zero = (sizeof(int) * want + sizeof(unsigned long long) * 2 + 255) & ~(size_t)255;
      pl->prep_state_bytes = pl->prep_state_zero + sizeof(int) * nt_total;
      if (cudaMalloc(&pl->prep_state, pl->prep_state_bytes) != cudaSuccess) {
        plan_free(pl);
        blr_set_error("blr_qr: out of device memory (prepared-operand pool state)");
        return BLR_ERR_OOM;
      }
    }
  }
  if (o->trace > 0 && cudaMalloc(&pl->trace, sizeof(blr_trace_event) * (size_t)o->trace) != cudaSuccess) {
    plan_free(pl);
    blr_set_error("blr_qr: out of device memory (trace of %d events)", o->trace);
    return BLR_ERR_OOM;
  }
  char* base = pl->base;
  SchedParams& P = pl->P;
  P.trace = pl->trace;
  P.trace_cap = pl->trace ? o->trace : 0;
  P.trace_n = (unsigned int*)(base + o_tracen);
  P.withhold = o->test_withhold > 0 ? o->test_withhold - 1 : -1;
  P.precision = o->precision;
  P.rec_tol = o->rec_tol > 0 ? o->rec_tol : o->tol;
  P.n_tasks = total;
  P.deps = (int*)(base + o_deps);
  P.qbuf = (int*)(base + o_qbuf);
  P.qhead = (int*)(base + o_qh);
  P.qtail = (int*)(base + o_qt);
  P.done = (int*)(base + o_done);
  P.status = (int*)(base + o_status);
  P.progress_ns = (unsigned long long*)(base + o_prog);
  P.watchdog_ns = (long long)(o->watchdog_ms > 0 ? o->watchdog_ms : 20000) * 1000000ll;
  P.scratch = pl->scratch;
  P.slab = pl->slab;
  P.flops = (double*)(base + o_flops);
  P.ntask = (unsigned long long*)(base + o_ntask);
  P.tns = (unsigned long long*)(base + o_tns);
  P.nvar = (unsigned long long*)(base + o_nvar);
  P.tvar = (unsigned long long*)(base + o_tvar);
  P.fvar = (double*)(base + o_fvar);
  P.slab_peak = (unsigned long long*)(base + o_peak);
#ifdef BLR_PHASE_TIMING
  cudaMalloc(&P.phase, 32 * sizeof(unsigned long long));
  cudaMemset(P.phase, 0, 32 * sizeof(unsigned long long));
#endif
  std::vector<SchedParams> mats(count, P);
  std::vector<int> mbase(count + 1), seed(count + 1);
  int rc = BLR_OK;
  for (int m = 0; m < count && !rc; m++) {
    const blr_matrix& A = fs[m]->a;
    SchedParams& Q = mats[m];
    Q.p = A.p; Q.q = A.q; Q.b = A.b; Q.cap = A.cap;
    Q.dense_rank = (o->dense_rank > 0 && o->dense_rank <= A.cap) ? o->dense_rank : A.cap;
    Q.tiles = A.tiles; Q.rank = A.rank; Q.t = fs[m]->t;
    Q.toff_dev = (const long long*)(base + M[m].o_toff);
    Q.off_larfb = (const int*)(base + M[m].o_offL);
    Q.off_tsqrt = (const int*)(base + M[m].o_offS);
    Q.off_tpmqrt = (const int*)(base + M[m].o_offP);
    Q.prep = pl->prep;
    Q.prep_rp = (A.b + 127) / 128 * 128;
    Q.prep_nslot = pl->nslot;
    Q.prep_slot_floats = slot_floats;
    if (pl->prep) {
      char* ps = reinterpret_cast<char*>(pl->prep_state);
      Q.prep_ref = reinterpret_cast<int*>(ps);
      Q.prep_next = reinterpret_cast<unsigned int*>(ps + sizeof(int) * pl->nslot);
      Q.prep_miss = reinterpret_cast<unsigned long long*>(
          ps + ((sizeof(int) * pl->nslot + sizeof(unsigned int) + 7) & ~(size_t)7));
      Q.prep_slot_of = reinterpret_cast<int*>(ps + pl->prep_state_zero) + M[m].slot_of_off;
    }
    Q.task_base = M[m].base;
    Q.mat_index = m;
    Q.chain = reinterpret_cast<int*>(base + o_chain) + M[m].chain_off;
    mbase[m] = M[m].base;
    seed[m] = M[m].base;   // GEQRT(0) of every matrix is ready at the start
    rc = blr_cuda_check(cudaMemcpy(base + M[m].o_offL, M[m].offL.data(), sizeof(int) * (M[m].q + 1), cudaMemcpyHostToDevice), "copy offsets");
    if (!rc) rc = blr_cuda_check(cudaMemcpy(base + M[m].o_offS, M[m].offS.data(), sizeof(int) * (M[m].q + 1), cudaMemcpyHostToDevice), "copy offsets");
    if (!rc) rc = blr_cuda_check(cudaMemcpy(base + M[m].o_offP, M[m].offP.data(), sizeof(int) * (M[m].q + 1), cudaMemcpyHostToDevice), "copy offsets");
    if (!rc) rc = blr_cuda_check(cudaMemcpy(base + M[m].o_toff, M[m].toff.data(), sizeof(long long) * M[m].q, cudaMemcpyHostToDevice), "copy T offsets");
  }
  mbase[count] = total;
  seed[count] = count;
  for (int m = 0; m < count; m++) {
    mats[m].nmat = count;
    mats[m].mats = (const SchedParams*)(base + o_mats);
    mats[m].mat_base = (const int*)(base + o_mbase);
  }
  if (count == 1) {
    P = mats[0];
    P.nmat = 1;
  } else {
    // batch-level parameters: matrix 0's shape (unused: every task looks up its own)
    SchedParams shared = mats[0];
    P = shared;
  }
  if (!rc) rc = blr_cuda_check(cudaMemcpy(base + o_mats, mats.data(), sizeof(SchedParams) * count, cudaMemcpyHostToDevice), "copy params");
  if (!rc) rc = blr_cuda_check(cudaMemcpy(base + o_mbase, mbase.data(), sizeof(int) * (count + 1), cudaMemcpyHostToDevice), "copy bases");
  if (!rc) rc = blr_cuda_check(cudaMemcpy(base + o_deps0, deps.data(), sizeof(int) * total, cudaMemcpyHostToDevice), "copy deps");
  if (!rc) rc = blr_cuda_check(cudaMemcpy(base + o_seed, seed.data(), sizeof(int) * (count + 1), cudaMemcpyHostToDevice), "copy seed");
  pl->deps0 = (int*)(base + o_deps0);
  pl->seed = (int*)(base + o_seed);
  if (!rc) rc = blr_cuda_check(cudaEventCreate(&pl->e0), "event");
  if (!rc) rc = blr_cuda_check(cudaEventCreate(&pl->e1), "event");
  if (rc) {
    plan_free(pl);
    return rc;
  }
  *out = pl;
  return BLR_OK;
}

// Capturable: device-side resets and the kernel launch only.
static int plan_launch(blr_batch_plan* pl, cudaStream_t st) {
  int rc = BLR_OK;
  for (size_t m = 0; m < pl->src.size() && !rc; m++) {
    const blr_matrix& S = *pl->src[m];
    blr_matrix& A = pl->fac[m]->a;
    rc = blr_cuda_check(cudaMemcpyAsync(A.tiles, S.tiles, sizeof(double) * (size_t)A.p * A.q * A.b * A.b,
                                        cudaMemcpyDeviceToDevice, st), "restore tiles");
    if (!rc) rc = blr_cuda_check(cudaMemcpyAsync(A.rank, S.rank, sizeof(int) * A.p * A.q, cudaMemcpyDeviceToDevice, st),
                                 "restore ranks");
  }
  SchedParams& P = pl->P;
  if (!rc) rc = blr_cuda_check(cudaMemsetAsync(pl->base + pl->dyn_off, 0, pl->dyn_bytes, st), "reset scheduler");
  if (!rc && pl->prep_state) {
    rc = blr_cuda_check(cudaMemsetAsync(pl->prep_state, 0, pl->prep_state_zero, st), "reset operand pool");
    if (!rc)
      rc = blr_cuda_check(cudaMemsetAsync(reinterpret_cast<char*>(pl->prep_state) + pl->prep_state_zero, 0xff,
                                          pl->prep_state_bytes - pl->prep_state_zero, st), "reset operand slots");
  }
  if (!rc) rc = blr_cuda_check(cudaMemcpyAsync(P.deps, pl->deps0, sizeof(int) * pl->n_tasks, cudaMemcpyDeviceToDevice, st), "reset deps");
  if (!rc) rc = blr_cuda_check(cudaMemsetAsync(P.qbuf, 0xff, sizeof(int) * (size_t)BLR_NQ * pl->n_tasks, st), "reset queues");
  if (!rc) rc = blr_cuda_check(cudaMemcpyAsync(P.qbuf, pl->seed, sizeof(int) * pl->count, cudaMemcpyDeviceToDevice, st), "seed queue");
  if (!rc) rc = blr_cuda_check(cudaMemcpyAsync(P.qtail, pl->seed + pl->count, sizeof(int), cudaMemcpyDeviceToDevice, st), "seed queue");
  if (!rc) rc = blr_cuda_check(cudaEventRecord(pl->e0, st), "event");
  if (!rc) rc = (P.precision == BLR_PREC_MIXED) ? blr_run_factor_mixed(P, pl->ctas, st) : blr_run_factor_fp64(P, pl->ctas, st);
  if (!rc) rc = blr_cuda_check(cudaEventRecord(pl->e1, st), "event");
  return rc;
}

// Waits for the launch, reads its status and statistics into every factor.
static int plan_finish(blr_batch_plan* pl, cudaStream_t st) {
  int rc = blr_cuda_check(cudaStreamSynchronize(st), "k_factor");
  if (rc) return rc;
  SchedParams& P = pl->P;
  float ms = 0.f;
  if (cudaEventElapsedTime(&ms, pl->e0, pl->e1) != cudaSuccess) {
    ms = 0.f;                 // no device time (e.g. the launch ran as part of a CUDA graph)
    cudaGetLastError();
  }
  int status = 0, done = 0;
  double fl[4];
  unsigned long long nt[4], tns[4], nv[8], tv[8], peak = 0;
  double fv[8];
  cudaMemcpy(&status, P.status, sizeof(int), cudaMemcpyDeviceToHost);
  cudaMemcpy(&done, P.done, sizeof(int), cudaMemcpyDeviceToHost);
  cudaMemcpy(fl, P.flops, sizeof(fl), cudaMemcpyDeviceToHost);
  cudaMemcpy(nt, P.ntask, sizeof(nt), cudaMemcpyDeviceToHost);
  cudaMemcpy(tns, P.tns, sizeof(tns), cudaMemcpyDeviceToHost);
  cudaMemcpy(nv, P.nvar, sizeof(nv), cudaMemcpyDeviceToHost);
  cudaMemcpy(tv, P.tvar, sizeof(tv), cudaMemcpyDeviceToHost);
  cudaMemcpy(fv, P.fvar, sizeof(fv), cudaMemcpyDeviceToHost);
  cudaMemcpy(&peak, P.slab_peak, sizeof(peak), cudaMemcpyDeviceToHost);
  unsigned long long misses = 0;
  if (P.prep) cudaMemcpy(&misses, P.prep_miss, sizeof(misses), cudaMemcpyDeviceToHost);
  unsigned int tn = 0;
  std::vector<blr_trace_event> trace;
  if (P.trace) {
    cudaMemcpy(&tn, P.trace_n, sizeof(tn), cudaMemcpyDeviceToHost);
    trace.resize(std::min<size_t>(tn, (size_t)P.trace_cap));
    if (!trace.empty())
      cudaMemcpy(trace.data(), P.trace, sizeof(blr_trace_event) * trace.size(), cudaMemcpyDeviceToHost);
  }
  rc = blr_cuda_check(cudaGetLastError(), "read status");
  if (rc) return rc;
  // statistics of the whole launch (a batch reports the batch in every factor)
  for (blr_factor* f : pl->fac) {
    f->trace = trace;
    f->trace_total = tn;
    f->prep_slots = pl->nslot;
    f->prep_misses = (long long)misses;
    f->seconds = ms * 1e-3;
    f->scratch_peak_bytes = (long long)(peak * sizeof(double));
    f->scratch_bytes = (long long)(sizeof(double) * pl->slab * pl->ctas);
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
  }
#ifdef BLR_PHASE_TIMING
  {
    unsigned long long ph[32];
    cudaMemcpy(ph, P.phase, sizeof(ph), cudaMemcpyDeviceToHost);
    fprintf(stderr, "blr_qr phases (CTA-s):");
    for (int i2 = 0; i2 < 32; i2++) fprintf(stderr, " %d:%.2f", i2, ph[i2] * 1e-9);
    fprintf(stderr, "\n");
  }
#endif
  const int n_tasks = pl->n_tasks;
  if (status & ST_TIMEOUT) { blr_set_error("blr_qr: scheduler watchdog expired (%d of %d tasks done)", done, n_tasks); return BLR_ERR_TIMEOUT; }
  if (status & ST_NUMERIC) { blr_set_error("blr_qr: non-finite Householder coefficient"); return BLR_ERR_NUMERIC; }
  if (status & ST_RANK) { blr_set_error("blr_qr: scratch slab exceeded"); return BLR_ERR_RANK_OVERFLOW; }
  if (status != 0 || done != n_tasks) { blr_set_error("blr_qr: scheduler ended with status %d, %d of %d tasks", status, done, n_tasks); return BLR_ERR_CUDA; }
  return BLR_OK;
}

int blr_launch_factors(blr_factor* const* fs, int count, const blr_opts* o, cudaStream_t st) {
  blr_batch_plan* pl = nullptr;
  int rc = plan_build(fs, count, o, &pl);
  if (rc) return rc;
  rc = plan_launch(pl, st);
  if (!rc) rc = plan_finish(pl, st);
  else cudaStreamSynchronize(st);
  plan_free(pl);
  return rc;
}

int blr_launch_factor(blr_factor* f, const blr_opts* o, cudaStream_t st) { return blr_launch_factors(&f, 1, o, st); }

// ---- C ABI of launch plans (graph capture) --------------------------------
extern "C" int blr_batch_plan_create(blr_matrix* const* a, int count, const blr_opts* opts, blr_batch_plan** out,
                                     void* stream) {
  if (!a || !opts || !out || count < 1) { blr_set_error("NULL argument or count < 1"); return BLR_ERR_INVALID; }
  *out = nullptr;
  int rc = blr_check_qr_opts(opts);
  if (rc) return rc;
  for (int m = 0; m < count; m++)
    if (!a[m]) { blr_set_error("matrix %d is NULL", m); return BLR_ERR_INVALID; }
  std::vector<blr_factor*> fs;
  for (int m = 0; m < count && !rc; m++) {
    blr_factor* f = nullptr;
    rc = blr_factor_alloc_like(a[m], opts, &f);
    if (!rc) fs.push_back(f);
  }
  blr_batch_plan* pl = nullptr;
  if (!rc) rc = plan_build(fs.data(), count, opts, &pl);
  if (rc) {
    for (blr_factor* f : fs) blr_destroy_factor(f);
    return rc;
  }
  pl->owns_factors = true;
  pl->src.assign(a, a + count);
  (void)stream;
  *out = pl;
  return BLR_OK;
}

extern "C" int blr_batch_plan_launch(blr_batch_plan* plan, void* stream) {
  if (!plan) { blr_set_error("NULL plan"); return BLR_ERR_INVALID; }
  return plan_launch(plan, (cudaStream_t)stream);
}

extern "C" int blr_batch_plan_finish(blr_batch_plan* plan, void* stream) {
  if (!plan) { blr_set_error("NULL plan"); return BLR_ERR_INVALID; }
  return plan_finish(plan, (cudaStream_t)stream);
}

extern "C" const blr_factor* blr_batch_plan_factor(const blr_batch_plan* plan, int i) {
  if (!plan || i < 0 || i >= plan->count) return nullptr;
  return plan->fac[i];
}

extern "C" void blr_batch_plan_destroy(blr_batch_plan* plan) { plan_free(plan); }

// Host-side check of a batch's task numbering (no device work): the DAGs of
// matrices of shapes (p[t], q[t]) numbered consecutively as a launch plan
// does, every task located by dag_find_matrix as the scheduler kernel does,
// and the dependency-counter protocol run over the whole batch in a seeded
// random order, releasing successors at task_base + local id.  Checks that
// every task runs once, after all its predecessors, that tasks of different
// matrices never depend on each other, and that each matrix's GEQRT(0) is
// the only initially ready task of that matrix.  0 on success.
extern "C" int blr_batch_selfcheck(const int* p, const int* q, int count, unsigned seed) {
  if (!p || !q || count < 1) return 100;
  std::vector<int> base(count + 1, 0);
  std::vector<std::vector<int>> offL(count), offS(count), offP(count);
  for (int t = 0; t < count; t++) {
    if (p[t] < 1 || q[t] < 1 || q[t] > p[t]) return 100;
    offL[t].resize(q[t] + 1); offS[t].resize(q[t] + 1); offP[t].resize(q[t] + 1);
    base[t + 1] = base[t] + dag_offsets(p[t], q[t], offL[t].data(), offS[t].data(), offP[t].data());
  }
  const int n = base[count];
  std::vector<int> deps(n, 0), runs(n, 0);
  auto shape = [&](int t) { return DagShape{p[t], q[t], offL[t].data(), offS[t].data(), offP[t].data()}; };
  for (int id = 0; id < n; id++) {
    const int t = dag_find_matrix(base.data(), count, id);
    if (id < base[t] || id >= base[t + 1]) return 1;
    const DagShape d = shape(t);
    int i, j, k;
    const int ty = dag_decode(d, id - base[t], &i, &j, &k);
    if (ty < 0) return 2;
    deps[id] = dag_indegree(ty, i, j, k);
    if ((deps[id] == 0) != (id == base[t])) return 3;          // only GEQRT(0) starts ready
  }
  std::vector<int> ready;
  for (int t = 0; t < count; t++) ready.push_back(base[t]);
  unsigned st = seed * 2654435761u + 7u;
  int executed = 0;
  while (!ready.empty()) {
    st = st * 1664525u + 1013904223u;
    const size_t pick = st % ready.size();
    const int id = ready[pick];
    ready[pick] = ready.back();
    ready.pop_back();
    if (deps[id] != 0 || runs[id]++) return 4;
    executed++;
    const int t = dag_find_matrix(base.data(), count, id);
    const DagShape d = shape(t);
    int i, j, k;
    const int ty = dag_decode(d, id - base[t], &i, &j, &k);
    int bad = 0;
    dag_for_each_successor(d, ty, i, j, k, [&](int sid) {
      const int gid = base[t] + sid;
      if (gid < base[t] || gid >= base[t + 1]) bad = 1;          // stays inside its matrix
      else if (--deps[gid] == 0) ready.push_back(gid);
    });
    if (bad) return 5;
  }
  return executed == n ? 0 : 6;
}

// Host-side check of the DAG formulas (no device work): builds the DAG from
// dag_successors, checks every in-degree against dag_indegree, and runs the
// counter protocol in a seeded random order, checking that each task runs
// exactly once, after all of its predecessors, and that the per-tile writer
// chains of Algorithm 4 are respected.  Returns 0 on success, or a positive
// code naming the first failed check.
extern "C" int blr_dag_task(int p, int q, int id, int* task, int* succ, int cap) {
  if (p < 1 || q < 1 || q > p || !task || !succ || cap < q + 1) {
    blr_set_error("blr_dag_task: bad shape (p=%d, q=%d), NULL pointer or cap=%d < q+1", p, q, cap);
    return -1;
  }
  std::vector<int> offL(q + 1), offS(q + 1), offP(q + 1);
  const int n = dag_offsets(p, q, offL.data(), offS.data(), offP.data());
  if (id < 0 || id >= n) {
    blr_set_error("blr_dag_task: id %d outside [0, %d)", id, n);
    return -1;
  }
  DagShape d{p, q, offL.data(), offS.data(), offP.data()};
  int i, j, k;
  const int t = dag_decode(d, id, &i, &j, &k);
  task[0] = t; task[1] = i; task[2] = j; task[3] = k;
  int ns = 0;
  dag_for_each_successor(d, t, i, j, k, [&](int sid) {
    if (ns < cap) succ[ns] = sid;
    ns++;
  });
  return ns;
}

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
