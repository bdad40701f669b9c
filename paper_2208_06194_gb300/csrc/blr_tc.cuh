// Fifth-generation tensor-core (tcgen05) building blocks for sm_103a: TMEM
// allocation, shared-memory matrix descriptors, TF32 MMAs with FP32
// accumulation in TMEM, completion through an mbarrier, and TMEM loads.
//
// Operand layout.  Both operands of D = A B^T are "K-major": row r of A
// (M x K) and row n of B (N x K) hold consecutive K elements.  In shared
// memory a K chunk of KC (= TC_KC) elements is stored in the no-swizzle
// canonical layout: 8-row x 16-byte core matrices; element (r, k) of a chunk
// at byte (r / 8) * SBO + (k / 4) * 128 + (r % 8) * 16 + (k % 4) * 4, with
// SBO = KC / 4 * 128 (the 8-row groups follow each other) and the K-direction
// core-matrix stride (LBO) 128 bytes.  One MMA consumes K = 8 (two core
// matrices), so its descriptor start advances by 256 bytes per K step.
//
// Precision: every FP32 operand x is split as x = hi + lo with hi = tf32(x)
// and lo = tf32(x - hi); the product uses hi*hi + hi*lo + lo*hi (three MMAs
// accumulated in FP32, "3xTF32"), which keeps about FP32 accuracy.
//
// Accumulation.  Measured on GB300: each kind::tf32 MMA rounds its FP32
// accumulation toward zero (a positive dot product of length K comes out
// low by about 1.05e-8 K relative, the whole error a bias).  So the error
// grows with the number of MMAs that feed one accumulator.  The small cross
// terms hi*lo + lo*hi (about 2^-11 of the result) go to a second
// accumulator TC_XCOL TMEM columns to the right, which takes two thirds of
// the MMAs off the main one; the epilogue adds the two with round-to-nearest.
// A product of N <= 256 columns uses TMEM columns [col0, col0 + N) and
// [col0 + TC_XCOL, col0 + TC_XCOL + N).
#pragma once
#include <stdint.h>
#include "blr_device.cuh"

#define TC_KC 32                        // K elements per staged chunk
#define TC_SBO (TC_KC / 4 * 128)        // bytes between 8-row groups of a chunk
#define TC_M 128                        // rows per MMA (cta_group::1)
#define TC_XCOL 256                     // TMEM column offset of the cross-term accumulator
#define TC_STAGE_BYTES (2 * (2 * TC_M * TC_KC + 2 * 256 * TC_KC) * 4)   // double-buffered staging, N <= 256

namespace {

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ unsigned long long tc_gtimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// ---- TMEM ------------------------------------------------------------------
// Called by one whole warp.  Writes the TMEM base address to *dst (shared).
__device__ __forceinline__ void tmem_alloc(uint32_t* dst, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst)),
               "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
// Generic-proxy shared-memory writes become visible to the tensor core.
__device__ __forceinline__ void fence_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
// Generic-proxy global writes become visible to bulk copies (TMA reads).
__device__ __forceinline__ void fence_async_global() {
  asm volatile("fence.proxy.async.global;" ::: "memory");
}

// ---- mbarrier --------------------------------------------------------------
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Waits until the phase with the given parity has completed; gives up after
// limit_ns and returns false (the caller flags a timeout, never traps).
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, unsigned long long limit_ns) {
  const uint32_t a = smem_u32(bar);
  const unsigned long long t0 = tc_gtimer();
  while (true) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
    if (tc_gtimer() - t0 > limit_ns) return false;
  }
}

// ---- descriptors -------------------------------------------------------------
// Shared-memory matrix descriptor, no swizzle, K-major canonical layout.
__device__ __forceinline__ uint64_t tc_desc(uint32_t saddr) {
  uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)(128u >> 4) << 16;          // K-direction core-matrix stride
  d |= (uint64_t)(TC_SBO >> 4) << 32;        // 8-row group stride
  d |= (uint64_t)1 << 46;                    // descriptor version for tcgen05
  return d;                                  // base offset 0, no swizzle
}

// Instruction descriptor: kind::tf32, D = F32, A = B = TF32, both K-major,
// M x N (M = 128, N a multiple of 16 up to 256).
__device__ __forceinline__ uint32_t tc_idesc(int m, int n) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

// One thread issues D (+)= A B^T for one K = 8 step.
__device__ __forceinline__ void tc_mma(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}

// The mbarrier receives one arrival when every MMA issued so far by this
// thread has completed.
__device__ __forceinline__ void tc_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   smem_u32(bar))
               : "memory");
}

// 32 lanes x 16 consecutive 32-bit columns: thread t of the warp receives
// lane (taddr.lane + t), columns taddr.col .. +15.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; i++) v[i] = __uint_as_float(r[i]);
}

// The same load issued without waiting; tmem_wait_ld() waits for all of a
// thread's outstanding TMEM loads (several loads then share one wait).
__device__ __forceinline__ void tmem_ld16_nowait(uint32_t taddr, uint32_t* r) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// ---- operand staging ----------------------------------------------------------
__device__ __forceinline__ float tf32_hi(float x) {
  uint32_t u;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(u) : "f"(x));
  return __uint_as_float(u);
}

// x = hi + lo with hi = tf32(x) and lo = tf32(x - hi) (x - hi is exact in
// FP32).  FP64 operands are first rounded to FP32: the dropped part is below
// what the three products resolve, and the split then needs no FP64 work.
__device__ __forceinline__ void tc_split(float x, float& hi, float& lo) {
  hi = tf32_hi(x);
  lo = tf32_hi(x - hi);
}

template <class G>
__device__ __forceinline__ G tc_ld(const G* p) { return __ldcg(p); }

// Stages rows [0, rows) x K columns [k0, k0 + TC_KC) of a strided global
// operand (element (r, k) at p[r * sr + k * sc], element type G) into a
// chunk pair (hi, lo) in the canonical layout above; rows >= nrow and
// columns >= kmax are zero.  rows must be a multiple of 8.
template <class G>
__device__ void tc_stage(float* hi, float* lo, const G* p, long long sr, long long sc, int rows, int nrow,
                         int k0, int kmax) {
  const int groups = rows * (TC_KC / 4);       // (row, 4-column group) pairs
  if (sc == 1) {
    // K contiguous in global: eight consecutive threads take eight rows of
    // one 4-column group (a 128-byte run of shared memory, no conflicts).
    for (int e = threadIdx.x; e < groups; e += BLR_NT) {
      const int r8 = e & 7, kq = (e >> 3) % (TC_KC / 4), rg = e / (8 * (TC_KC / 4));
      const int r = rg * 8 + r8, k = k0 + kq * 4;
      float h[4], l[4];
#pragma unroll
      for (int i = 0; i < 4; i++) {
        G v = G(0);
        if (r < nrow && k + i < kmax) v = tc_ld(p + (long long)r * sr + (k + i));
        tc_split(cvt<float>(v), h[i], l[i]);
      }
      const int off = (rg * TC_SBO + kq * 128 + r8 * 16) >> 2;
      *reinterpret_cast<float4*>(hi + off) = make_float4(h[0], h[1], h[2], h[3]);
      *reinterpret_cast<float4*>(lo + off) = make_float4(l[0], l[1], l[2], l[3]);
    }
  } else {
    // rows contiguous in global: consecutive threads take consecutive rows.
    for (int e = threadIdx.x; e < groups; e += BLR_NT) {
      const int r = e % rows, kq = e / rows;
      const int k = k0 + kq * 4;
      float h[4], l[4];
#pragma unroll
      for (int i = 0; i < 4; i++) {
        G v = G(0);
        if (r < nrow && k + i < kmax) v = tc_ld(p + (long long)r * sr + (long long)(k + i) * sc);
        tc_split(cvt<float>(v), h[i], l[i]);
      }
      const int off = ((r >> 3) * TC_SBO + kq * 128 + (r & 7) * 16) >> 2;
      *reinterpret_cast<float4*>(hi + off) = make_float4(h[0], h[1], h[2], h[3]);
      *reinterpret_cast<float4*>(lo + off) = make_float4(l[0], l[1], l[2], l[3]);
    }
  }
}

// Shared state of the tensor-core GEMM inside a CTA.
struct TcCtx {
  uint32_t tmem;        // TMEM base (lane 0, first allocated column)
  uint64_t* bar;        // two mbarriers (one per staging buffer)
  uint32_t* phase;      // their next parity bits (shared, 2 words)
  float* buf;           // staging: 2 buffers x (A hi, A lo, B hi, B lo)
  int bcap;             // row capacity of the B staging (<= 256)
  int* status;
  unsigned long long limit_ns;
  int* unsafe;          // shared flag: set when an issued copy or MMA could not be waited for, so
                        // the kernel must not release TMEM or reuse the staging buffers
};

__device__ __forceinline__ size_t tc_chunk_floats(int rows) { return (size_t)rows * TC_KC; }

// D (TC_M x ncol, TMEM columns [col0, col0 + ncol)) = sum over K of
// A[r, k] * B[n, k], for r < TC_M (rows >= mrow read as zero), n < ncol
// (a multiple of 16, <= t.bcap; rows >= nrow of B read as zero), k < K.  3xTF32 products, FP32
// accumulation.  Called by all threads; returns with the result complete in
// TMEM (and false if a wait ran out, after flagging ST_TIMEOUT).
template <class GA, class GB>
__device__ bool tc_gemm_tile(TcCtx& t, uint32_t col0, const GA* A, long long sar, long long sak, int mrow,
                             const GB* B, long long sbn, long long sbk, int nrow, int ncol, int K) {
  const size_t fa = tc_chunk_floats(TC_M), fb = tc_chunk_floats(t.bcap);
  const size_t per = 2 * fa + 2 * fb;
  const uint32_t idesc = tc_idesc(TC_M, ncol);
  const int nchunk = (K + TC_KC - 1) / TC_KC;
  __shared__ int fail_sh;
  __syncthreads();
  if (threadIdx.x == 0) fail_sh = (*(volatile int*)t.status & ST_TIMEOUT) != 0;
  __syncthreads();
  if (fail_sh) return false;      // an earlier wait ran out: do no more tensor-core work
  bool pend[2] = {false, false};  // thread 0: a commit on bar[s] not yet waited for
  for (int c = 0; c < nchunk; c++) {
    const int s = c & 1;
    float* ah = t.buf + s * per;
    float* al = ah + fa;
    float* bh = al + fa;
    float* bl = bh + fb;
    // the buffer was last read by the MMAs of chunk c - 2
    if (c >= 2) {
      if (threadIdx.x == 0) {
        if (mbar_wait(t.bar + s, t.phase[s], t.limit_ns)) {
          t.phase[s] ^= 1u;
          pend[s] = false;
        } else {
          fail_sh = 1;
        }
      }
      __syncthreads();
      if (fail_sh) break;         // stage nothing more into a buffer an MMA may still read
    }
    tc_stage(ah, al, A, sar, sak, TC_M, mrow, c * TC_KC, K);
    tc_stage(bh, bl, B, sbn, sbk, ncol, nrow, c * TC_KC, K);
    fence_async_smem();
    __syncthreads();
    if (threadIdx.x == 0) {
      tc_fence_after();
      const uint32_t a0 = smem_u32(ah), a1 = smem_u32(al), b0 = smem_u32(bh), b1 = smem_u32(bl);
#pragma unroll
      for (int ks = 0; ks < TC_KC / 8; ks++) {
        const uint32_t o = ks * 256;
        const uint32_t acc = (c > 0 || ks > 0) ? 1u : 0u;
        tc_mma(t.tmem + col0 + TC_XCOL, tc_desc(a1 + o), tc_desc(b0 + o), idesc, acc);
        tc_mma(t.tmem + col0 + TC_XCOL, tc_desc(a0 + o), tc_desc(b1 + o), idesc, 1u);
        tc_mma(t.tmem + col0, tc_desc(a0 + o), tc_desc(b0 + o), idesc, acc);
      }
      tc_commit(t.bar + s);
      pend[s] = true;
    }
  }
  // drain every commit not yet waited for, also after a failed wait, so that
  // no MMA still reads the staging buffers or writes TMEM after the return
  if (threadIdx.x == 0) {
    for (int s = 0; s < 2; s++) {
      if (!pend[s]) continue;
      if (mbar_wait(t.bar + s, t.phase[s], t.limit_ns)) {
        t.phase[s] ^= 1u;
      } else {
        fail_sh = 1;
        *t.unsafe = 1;
      }
    }
    if (fail_sh) atomicOr(t.status, ST_TIMEOUT);
  }
  __syncthreads();
  tc_fence_after();
  return fail_sh == 0;
}


// ---- operands in global memory, pre-split, in the canonical chunk order ----
// An operand of R rows (R a multiple of 8) and K columns (a multiple of
// TC_KC) is stored as two float arrays (hi, lo), each a sequence of K chunks
// of R x TC_KC elements in the shared-memory layout above, so that rows
// [r0, r0 + n) of chunk c are one contiguous run of n * TC_KC floats at
// c * R * TC_KC + r0 * TC_KC.  Staging then is a plain bulk copy (the TMA
// engine), with no per-element work on the SM.

__device__ __forceinline__ size_t canon_index(int R, int r, int k) {
  return (size_t)(k / TC_KC) * R * TC_KC + (size_t)(r >> 3) * (TC_SBO / 4) + ((k % TC_KC) >> 2) * 32 + (r & 7) * 4 +
         (k & 3);
}

// Writes element (r, k) = src[r * sr + k * sc] (element type G) for r < nrow,
// k < kvalid into the canonical (hi, lo) pair of an R x K operand; the
// padding (rows [nrow, R), columns [kvalid, K)) is zero.  All threads.
template <class G>
__device__ void tc_canon(float* hi, float* lo, int R, int K, const G* src, long long sr, long long sc, int nrow,
                         int kvalid) {
  // four (row, 4-column) groups per thread per pass, all loads issued first
  constexpr int U = 4;
  const int kq4 = K / 4;
  const int groups = R * kq4;
  for (int base = 0; base < groups; base += BLR_NT * U) {
    G v[U][4];
    int rr[U], kk[U];
#pragma unroll
    for (int u = 0; u < U; u++) {
      const int e = base + u * BLR_NT + threadIdx.x;
      int r, k;
      if (sc == 1) {   // eight consecutive threads: eight rows of one 4-column group
        const int r8 = e & 7, kq = (e >> 3) % kq4, rg = (e >> 3) / kq4;
        r = rg * 8 + r8;
        k = kq * 4;
      } else {         // consecutive threads: consecutive rows
        r = e % R;
        k = (e / R) * 4;
      }
      rr[u] = r;
      kk[u] = k;
#pragma unroll
      for (int i = 0; i < 4; i++) {
        v[u][i] = G(0);
        if (e < groups && r < nrow && k + i < kvalid) v[u][i] = tc_ld(src + (long long)r * sr + (long long)(k + i) * sc);
      }
    }
#pragma unroll
    for (int u = 0; u < U; u++) {
      if (base + u * BLR_NT + (int)threadIdx.x >= groups) continue;
      float h[4], l[4];
#pragma unroll
      for (int i = 0; i < 4; i++) tc_split(cvt<float>(v[u][i]), h[i], l[i]);
      const size_t off = canon_index(R, rr[u], kk[u]);
      *reinterpret_cast<float4*>(hi + off) = make_float4(h[0], h[1], h[2], h[3]);
      *reinterpret_cast<float4*>(lo + off) = make_float4(l[0], l[1], l[2], l[3]);
    }
  }
}

// The same for a single value written by the thread that holds it (an
// epilogue that produces an operand of the next product).
__device__ __forceinline__ void tc_canon_put(float* hi, float* lo, int R, int r, int k, float v) {
  const size_t off = canon_index(R, r, k);
  float h, l;
  tc_split(v, h, l);
  hi[off] = h;
  lo[off] = l;
}

// ---- bulk (TMA) copies -----------------------------------------------------
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

// dst (shared) <- src (global), bytes a multiple of 16, both 16-byte aligned;
// completion is counted on the mbarrier.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

// D (TC_M x n, TMEM columns [col0, col0 + n)) = sum over the nchunk K chunks
// of A(r, k) B(c, k) for operands in the canonical global order: chunk c of A
// is the TC_M rows at a_hi + c * a_cs (floats; same offsets in a_lo), chunk c
// of B the n rows at b_hi + c * b_cs.  n a multiple of 16, <= 256.  Thread 0
// runs the copy / MMA pipeline (two stages: full barriers signalled by the
// TMA engine, empty barriers by tcgen05.commit); every thread returns after
// the products are complete.  On a wait that runs out the status gets
// ST_TIMEOUT and false is returned.
struct TcBulk {
  uint64_t* full;   // 2 mbarriers
  uint64_t* empty;  // 2 mbarriers
  uint32_t* ph;     // 4 parity bits: full[0], full[1], empty[0], empty[1]
};

__device__ bool tc_gemm_bulk(TcCtx& t, const TcBulk& q, uint32_t col0, const float* a_hi, const float* a_lo,
                             size_t a_cs, const float* b_hi, const float* b_lo, size_t b_cs, int n, int nchunk) {
  __shared__ int ok_sh;
  if (threadIdx.x == 0) {
    bool ok = (*(volatile int*)t.status & ST_TIMEOUT) == 0;   // after a timeout, no more work
    asm volatile("fence.proxy.async.global;" ::: "memory");    // generic writes -> bulk-copy reads
    const uint32_t abytes = TC_M * TC_KC * 4, bbytes = (uint32_t)n * TC_KC * 4;
    const size_t per = 2 * (size_t)TC_M * TC_KC + 2 * (size_t)256 * TC_KC;   // floats per stage
    const uint32_t idesc = tc_idesc(TC_M, n);
    bool full_pend[2] = {false, false};    // copies issued into stage s, not yet waited for
    bool empty_pend[2] = {false, false};   // MMAs committed on stage s, not yet waited for
    auto load = [&](int c, int s) {
      float* ah = t.buf + s * per;
      float* al = ah + TC_M * TC_KC;
      float* bh = al + TC_M * TC_KC;
      float* bl = bh + 256 * TC_KC;
      mbar_expect_tx(q.full + s, 2 * abytes + 2 * bbytes);
      bulk_g2s(ah, a_hi + c * a_cs, abytes, q.full + s);
      bulk_g2s(al, a_lo + c * a_cs, abytes, q.full + s);
      bulk_g2s(bh, b_hi + c * b_cs, bbytes, q.full + s);
      bulk_g2s(bl, b_lo + c * b_cs, bbytes, q.full + s);
      full_pend[s] = true;
    };
    const int nc_run = ok ? nchunk : 0;
    for (int c = 0; c < nc_run && c < 2; c++) load(c, c);
    for (int c = 0; c < nc_run; c++) {
      const int s = c & 1;
      if (!mbar_wait(q.full + s, q.ph[s], t.limit_ns)) { ok = false; break; }
      q.ph[s] ^= 1u;
      full_pend[s] = false;
      tc_fence_after();
      const uint32_t a0 = smem_u32(t.buf + s * per), a1 = a0 + abytes, b0 = a1 + abytes, b1 = b0 + 256 * TC_KC * 4;
#pragma unroll
      for (int ks = 0; ks < TC_KC / 8; ks++) {
        const uint32_t o = ks * 256;
        const uint32_t acc = (c > 0 || ks > 0) ? 1u : 0u;
        tc_mma(t.tmem + col0 + TC_XCOL, tc_desc(a1 + o), tc_desc(b0 + o), idesc, acc);
        tc_mma(t.tmem + col0 + TC_XCOL, tc_desc(a0 + o), tc_desc(b1 + o), idesc, 1u);
        tc_mma(t.tmem + col0, tc_desc(a0 + o), tc_desc(b0 + o), idesc, acc);
      }
      tc_commit(q.empty + s);
      empty_pend[s] = true;
      // refill this stage with chunk c + 2 once its MMAs are done (measured
      // faster than refilling the other stage behind still-queued MMAs)
      if (c + 2 < nchunk) {
        if (!mbar_wait(q.empty + s, q.ph[2 + s], t.limit_ns)) { ok = false; break; }
        q.ph[2 + s] ^= 1u;
        empty_pend[s] = false;
        load(c + 2, s);
      }
    }
    // drain: every commit and copy not yet waited for (normally the last one
    // or two commits; after a failed wait, whatever is still in flight), so
    // that nothing writes the staging buffers or TMEM after the return
    bool drained = true;
    for (int s = 0; s < 2; s++) {
      if (empty_pend[s]) {
        if (mbar_wait(q.empty + s, q.ph[2 + s], t.limit_ns)) q.ph[2 + s] ^= 1u;
        else drained = false;
      }
      if (full_pend[s]) {
        if (mbar_wait(q.full + s, q.ph[s], t.limit_ns)) q.ph[s] ^= 1u;
        else drained = false;
      }
    }
    if (!drained) {
      ok = false;
      *t.unsafe = 1;
    }
    if (!ok) atomicOr(t.status, ST_TIMEOUT);
    ok_sh = ok && nc_run == nchunk;
  }
  __syncthreads();
  tc_fence_after();
  return ok_sh != 0;
}

// Reads the TC_M x ncol accumulator 16 columns at a time and calls
// f(row, col0, v) with v[0..15] = columns col0 .. col0 + 15 of that row
// (each element once); lets the caller batch its global accesses.
template <class F>
__device__ void tc_epilogue16(const TcCtx& t, uint32_t col0, int ncol, F f) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int quarter = warp & 3, half = warp >> 2;
  const int row = quarter * 32 + lane;
  const int nblk = ncol / 16;
  for (int cb = half; cb < nblk; cb += 2) {
    float v[16], x[16];
    const uint32_t a = t.tmem + ((uint32_t)(quarter * 32) << 16) + col0 + cb * 16;
    tmem_ld16(a, v);
    tmem_ld16(a + TC_XCOL, x);
#pragma unroll
    for (int i = 0; i < 16; i++) v[i] += x[i];
    f(row, cb * 16, v);
  }
  tc_fence_before();
  __syncthreads();
}

// As tc_epilogue16, with a caller's global loads for the same 16 columns
// issued before the accumulator is read, so that the global and the TMEM
// latencies overlap: pre(row, col, g) fills g[0..15] (type G), then
// post(row, col, v, g) receives the accumulator values v[0..15].  Both are
// called by every thread (rows past the product included: they must take
// part in warp-wide exchanges).
template <class G, class Pre, class Post>
__device__ void tc_epilogue16_pf(const TcCtx& t, uint32_t col0, int ncol, Pre pre, Post post) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int quarter = warp & 3, half = warp >> 2;
  const int row = quarter * 32 + lane;
  const int nblk = ncol / 16;
  for (int cb = half; cb < nblk; cb += 2) {
    G g[16];
    pre(row, cb * 16, g);
    uint32_t rv[16], rx[16];
    const uint32_t a = t.tmem + ((uint32_t)(quarter * 32) << 16) + col0 + cb * 16;
    tmem_ld16_nowait(a, rv);
    tmem_ld16_nowait(a + TC_XCOL, rx);
    tmem_wait_ld();
    float v[16];
#pragma unroll
    for (int i = 0; i < 16; i++) v[i] = __uint_as_float(rv[i]) + __uint_as_float(rx[i]);
    post(row, cb * 16, v, g);
  }
  tc_fence_before();
  __syncthreads();
}

// Elements (n, a) = v[u] for n = nbase + u (u < 16) of a canonical (hi, lo)
// operand of R rows, one tile row a per lane, lanes of a warp on
// consecutive a with a % 4 == lane % 4.  The four lanes of a's group of four
// exchange their values (four shuffle rounds per four columns) so that each
// stores the 16-byte run (n, a0 .. a0 + 3) of one column: full 32-byte
// sectors instead of 4-byte pieces.  Columns u >= nvalid and groups whose
// rows are past the operand (avalid false) are not stored; every lane of the
// warp must call this.
__device__ __forceinline__ void tc_canon_put16(float* hi, float* lo, int R, int nbase, int a, const float* v,
                                               int nvalid, bool avalid) {
  const int lane = threadIdx.x & 31, j = lane & 3, a0 = a & ~3;
#pragma unroll
  for (int qb = 0; qb < 4; qb++) {
    float w[4];
#pragma unroll
    for (int k = 0; k < 4; k++) {
      // round k: this lane sends its value of column 4 qb + ((j - k) & 3) and
      // receives from lane (j + k) & 3 of its group that lane's value of
      // column 4 qb + j, i.e. row a0 + ((j + k) & 3) of this lane's column
      const int si = (j - k) & 3;
      const float sv = si == 0 ? v[4 * qb] : si == 1 ? v[4 * qb + 1] : si == 2 ? v[4 * qb + 2] : v[4 * qb + 3];
      w[k] = __shfl_sync(FULLMASK, sv, (lane & ~3) | ((j + k) & 3));
    }
    // rows a0 + i: w[(i - j) & 3]
    float rowv[4];
#pragma unroll
    for (int i = 0; i < 4; i++) {
      const int kk = (i - j) & 3;
      rowv[i] = kk == 0 ? w[0] : kk == 1 ? w[1] : kk == 2 ? w[2] : w[3];
    }
    const int u = 4 * qb + j;
    if (avalid && u < nvalid) {
      float h[4], l[4];
#pragma unroll
      for (int i = 0; i < 4; i++) tc_split(rowv[i], h[i], l[i]);
      const size_t off = canon_index(R, nbase + u, a0);
      *reinterpret_cast<float4*>(hi + off) = make_float4(h[0], h[1], h[2], h[3]);
      *reinterpret_cast<float4*>(lo + off) = make_float4(l[0], l[1], l[2], l[3]);
    }
  }
}

// tc_canon for a source whose K index is contiguous (element (r, k) at
// src[r * sr + k]): a warp takes a tile of 32 consecutive k (one per lane)
// by 16 rows, so that each of its 16 loads reads 32 consecutive elements,
// and stores the tile through the four-lane exchange of tc_canon_put16 as
// 16-byte runs.  Padding rows and columns are written as zeros.
// exchange: stores through tc_canon_put16 (16-byte runs) or one element
// at a time (tc_canon_put).
template <class G>
__device__ void tc_canon_kmajor(float* hi, float* lo, int R, int K, const G* src, long long sr, int nrow,
                                int kvalid, bool exchange) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int tk = K / 32, tiles = tk * ((R + 15) / 16);
  for (int t = warp; t < tiles; t += BLR_NWARP) {
    const int k = (t % tk) * 32 + lane, r0 = (t / tk) * 16;
    float v[16];
    G g[16];
#pragma unroll
    for (int u = 0; u < 16; u++) g[u] = (r0 + u < nrow && k < kvalid) ? tc_ld(src + (long long)(r0 + u) * sr + k) : G(0);
#pragma unroll
    for (int u = 0; u < 16; u++) v[u] = cvt<float>(g[u]);
    if (exchange) {
      tc_canon_put16(hi, lo, R, r0, k, v, R - r0, true);
    } else {
#pragma unroll
      for (int u = 0; u < 16; u++)
        if (r0 + u < R) tc_canon_put(hi, lo, R, r0 + u, k, v[u]);
    }
  }
}

// Reads the TC_M x ncol accumulator at TMEM columns [col0, col0 + ncol)
// and calls f(row, col, value) for every element (each once).  Warps w and
// w + 4 share TMEM lanes 32 (w % 4) .. + 31 and split the columns.
template <class F>
__device__ void tc_epilogue(const TcCtx& t, uint32_t col0, int ncol, F f) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int quarter = warp & 3, half = warp >> 2;
  const int row = quarter * 32 + lane;
  const int nblk = ncol / 16;
  for (int cb = half; cb < nblk; cb += 2) {
    float v[16], x[16];
    const uint32_t a = t.tmem + ((uint32_t)(quarter * 32) << 16) + col0 + cb * 16;
    tmem_ld16(a, v);
    tmem_ld16(a + TC_XCOL, x);
#pragma unroll
    for (int i = 0; i < 16; i++) f(row, cb * 16 + i, v[i] + x[i]);
  }
  tc_fence_before();
  __syncthreads();
}

}  // namespace
