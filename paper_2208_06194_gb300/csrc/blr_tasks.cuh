// Tiled Householder BLR-QR (Algorithm 4 with the BLR tile kernels of
// Section 3.4) as one persistent device-side task scheduler (Section 4.3).
//
// Storage: tile (i,j) owns b*b doubles; a dense tile is b x b column-major;
// a low-rank tile of rank r keeps U (b x r) at offset 0 and V (b x r) at
// offset b*(b/2).  After the factorization tile (i,k), i > k, holds
// Y~_ik = U_ik Y_ik with Y_ik^T in the V slot (Section 3.4.3), or a dense
// Y_ik.  Every reflector block is kept in compact-WY form with inner
// blocking: the T of each 32 consecutive reflectors (Eq. 3, Eq. 21).
#pragma once
#include "blr_device.cuh"
#include "blr_dag.h"
#include "blr_tc.cuh"

// Optional per-phase timing of the task bodies (a build with
// -DBLR_PHASE_TIMING; summed CTA time per phase, printed by blr_qr).
#ifdef BLR_PHASE_TIMING
#define PH(id, ...)                                                              \
  do {                                                                           \
    __syncthreads();                                                             \
    const unsigned long long ph_t0_ = tc_gtimer();                               \
    __VA_ARGS__;                                                                 \
    __syncthreads();                                                             \
    if (threadIdx.x == 0) atomicAdd(env.P->phase + (id), tc_gtimer() - ph_t0_); \
  } while (0)
#define PH_BEGIN()                       \
  __syncthreads();                       \
  const unsigned long long ph_b0_ = tc_gtimer();
#define PH_END(id)                                                               \
  __syncthreads();                                                               \
  if (threadIdx.x == 0) atomicAdd(env.P->phase + (id), tc_gtimer() - ph_b0_);
// a second, independently named pair for regions that share a scope
#define PH_BEGIN2()                      \
  __syncthreads();                       \
  const unsigned long long ph_b2_ = tc_gtimer();
#define PH_END2(id)                                                              \
  __syncthreads();                                                               \
  if (threadIdx.x == 0) atomicAdd(env.P->phase + (id), tc_gtimer() - ph_b2_);
#define PH_BEGIN3()                      \
  __syncthreads();                       \
  const unsigned long long ph_b3_ = tc_gtimer();
#define PH_END3(id)                                                              \
  __syncthreads();                                                               \
  if (threadIdx.x == 0) atomicAdd(env.P->phase + (id), tc_gtimer() - ph_b3_);
#else
#define PH(id, ...) \
  do {              \
    __VA_ARGS__;    \
  } while (0)
#define PH_BEGIN()
#define PH_END(id)
#define PH_BEGIN2()
#define PH_END2(id)
#define PH_BEGIN3()
#define PH_END3(id)
#endif

// The variant of the dense prepared update the factorization runs (see
// tc_apply_prepared; chosen by measurement with blr_tc_update_bench).
#ifndef BLR_TC_UPDATE_VARIANT
#define BLR_TC_UPDATE_VARIANT 17
#endif

namespace {

// Bump allocator over the CTA's private scratch slab.  The slab holds
// BLR_SLAB_B2 * b^2 doubles, more than any task needs, and no single request
// exceeds 2 b^2; should the total ever run over, the request is served from
// the slab's start (still in bounds) and the overflow flag fails the call.
struct TaskEnv {
  const SchedParams* P;
  double* slab;
  size_t used;
  bool overflow;
  TcCtx* tc;          // tensor-core state (mixed path), else nullptr
  const TcBulk* tq;   // its bulk-copy pipeline barriers
  const DagShape* dag;
  int skip_succ;      // a successor the task body has already released (-1: none)
  const float* prep_slot;   // mixed: prepared operands of the current update's low-rank reflector block
  size_t peak;        // high-water mark of used (doubles)
  __device__ double* alloc(size_t n) {
    const size_t nn = (n + 31) & ~(size_t)31;   // 256-byte granules
    if (used + nn > P->slab) {
      overflow = true;
      return slab;
    }
    double* p = slab + used;
    used += nn;
    if (used > peak) peak = used;
    return p;
  }
};

__device__ __forceinline__ double* tile_ptr(const SchedParams& P, int i, int j) {
  return P.tiles + ((size_t)j * P.p + i) * (size_t)P.b * P.b;
}
__device__ __forceinline__ int* rank_ptr(const SchedParams& P, int i, int j) {
  return P.rank + (size_t)j * P.p + i;
}
__device__ __forceinline__ double* t_ptr(const SchedParams& P, int i, int k) {
  return P.t + (size_t)(P.toff_dev[k] + (i - k)) * BLR_NB * P.b;
}
__device__ __forceinline__ int ld_rank(const int* p) { return __ldcg(p); }

__device__ void q_push(const SchedParams& P, int qi, int task);

// Thread 0: one dependency of task sid is satisfied; queue it when ready.
// sid is the task's id within its matrix (P, d); dependency counters and
// queues hold batch-wide ids, task_base + sid.
__device__ void release_task(const SchedParams& P, const DagShape& d, int sid) {
  const int gid = P.task_base + sid;
  if (atomicSub(P.deps + gid, 1) == 1) {
    __threadfence();
    int si, sj, sk;
    const int st = dag_decode(d, sid, &si, &sj, &sk);
    q_push(P, dag_queue(st, si, sj, sk), gid);
  }
}

// The pool of prepared tensor-core operands (mixed path).  Reflector block
// (i,k) has index toff[k] + i - k in prep_slot_of; a slot is
// prep_slot_floats floats.
__device__ __forceinline__ int prep_block(const SchedParams& P, int i, int k) {
  return (int)(P.toff_dev[k] + (i - k));
}
__device__ __forceinline__ float* prep_at(const SchedParams& P, int slot) {
  return P.prep + (size_t)slot * P.prep_slot_floats;
}
// Thread 0: a free slot, marked as being prepared (-1), or -1 when a bounded
// search finds none (the block's updates then use its stored factors).
__device__ int prep_acquire(const SchedParams& P) {
  const int tries = P.prep_nslot < 64 ? P.prep_nslot : 64;
  for (int a = 0; a < tries; a++) {
    const int s = (int)(atomicAdd(P.prep_next, 1u) % (unsigned)P.prep_nslot);
    if (atomicCAS(P.prep_ref + s, 0, -1) == 0) return s;
  }
  atomicAdd(P.prep_miss, 1ull);
  return -1;
}

// ---------------------------------------------------------------------------
// TSQRT panel: Householder on [Rp (w x w upper, ld NB); Bp (ry x w, ld ldb)],
// reflector j = [e_j; y_j] (Section 3.4.3).  Always FP64.
// ---------------------------------------------------------------------------
__device__ void ts_panel_qr(double* Rp, double* Bp, int ldb, int ry, int w, double* tau, Ctx& c) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  for (int j = 0; j < w; j++) {
    double part = 0.0;
    for (int s = threadIdx.x; s < ry; s += BLR_NT) {
      double x = Bp[s + j * ldb];
      part += x * x;
    }
    double sig2 = block_sum(part, c.s.red);
    if (threadIdx.x == 0) {
      double beta, tj, sc;
      house(Rp[j + j * BLR_NB], sig2, beta, tj, sc);
      flag_numeric(c, beta);
      flag_numeric(c, tj);
      c.s.scal[0] = beta;
      c.s.scal[1] = tj;
      c.s.scal[2] = sc;
    }
    __syncthreads();
    const double tj = c.s.scal[1], sc = c.s.scal[2];
    for (int s = threadIdx.x; s < ry; s += BLR_NT) Bp[s + j * ldb] *= sc;
    __syncthreads();
    for (int l = j + 1 + warp; l < w; l += BLR_NWARP) {
      double acc = 0.0;
      for (int s = lane; s < ry; s += 32) acc += Bp[s + j * ldb] * Bp[s + l * ldb];
      acc = warp_sum(acc);
      double wl = (__shfl_sync(FULLMASK, Rp[j + l * BLR_NB], 0) + acc) * tj;
      if (lane == 0) Rp[j + l * BLR_NB] -= wl;
      for (int s = lane; s < ry; s += 32) Bp[s + l * ldb] -= wl * Bp[s + j * ldb];
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      Rp[j + j * BLR_NB] = c.s.scal[0];
      tau[j] = tj;
    }
    __syncthreads();
  }
  c.fma += (double)ry * w * w;
}

// ---------------------------------------------------------------------------
// Rounded addition (Algorithm 6) for C = Uf H0^T where H has already been
// QR-factored in place (R_H in its top s x s, reflectors below, T blocks TH):
// QR(Uf) = Q_U R_U, core M = R_U R_H^T (s x s), then a truncated
// column-pivoted QR of the core, M P = Q_M R_M, stopped at the smallest r
// with ||R_M(r:,r:)||_F <= eps ||M||_F.  Because ||C - C_r||_F equals the
// core's truncation error, the result meets Algorithm 6's bound
// ||C - U_C V_C^T||_F <= eps ||C||_F; U_C = Q_U Q_M [I_r; 0] is orthonormal
// and V_C = Q_H [P R_M(0:r,:)^T; 0].  (Algorithm 6 truncates the core's SVD;
// the pivoted QR reaches the same error bound in O(s^2 r) work instead of
// O(s^3) per Jacobi sweep, with a rank that can exceed the optimal one by a
// few.)  Uf is overwritten.  The result goes to dest in tile layout (U at 0,
// V at b*cap); one whose rank would exceed dense_rank is written dense as
// the product Uf0 H0^T.  Arithmetic in S.
// ---------------------------------------------------------------------------
template <class S>
__device__ void recompress_side(TaskEnv& env, S* Uf, int ldu, const S* H, const S* TH, const S* H0, int s,
                                S* dest, int* dest_rank, Ctx& c) {
  const SchedParams& P = *env.P;
  const int b = P.b;
  const size_t mark = env.used;
  if (s == 0) {
    if (threadIdx.x == 0) *dest_rank = 0;
    __syncthreads();
    return;
  }
  S* U0 = (S*)env.alloc(((size_t)b * s * sizeof(S) + 7) / 8);
  copy_mat(U0, b, Uf, ldu, b, s);
  S* TU = (S*)env.alloc(((size_t)BLR_NB * s * sizeof(S) + 7) / 8);
  __syncthreads();
  PH(9, geqrf(Uf, ldu, b, s, TU, c));
  S* RU = (S*)env.alloc(((size_t)s * s * sizeof(S) + 7) / 8);
  S* RH = (S*)env.alloc(((size_t)s * s * sizeof(S) + 7) / 8);
  for (int e = threadIdx.x; e < s * s; e += BLR_NT) {
    int a = e % s, l = e / s;
    RU[e] = (a <= l) ? ldg(Uf + a + (size_t)l * ldu) : S(0);
    RH[e] = (a <= l) ? ldg(H + a + (size_t)l * b) : S(0);
  }
  __syncthreads();
  S* M = (S*)env.alloc(((size_t)s * s * sizeof(S) + 7) / 8);
  gemm(s, s, s, S(1), RU, s, false, RH, s, true, S(0), M, s, c);
  double part = 0.0;
  for (int e = threadIdx.x; e < s * s; e += BLR_NT) part += (double)M[e] * (double)M[e];
  const double nrm2 = block_sum(part, c.s.red);
  const double tol2 = P.rec_tol * P.rec_tol * nrm2;
  S* tauM = (S*)env.alloc(((size_t)s * sizeof(S) + 7) / 8);
  int* perm = c.s.ivec;
  int r = 0;
  if ((size_t)s * s * sizeof(S) <= (size_t)BLR_SM_PNL * sizeof(double)) {
    // the core fits in shared memory (the panel buffer is idle here): the
    // pivoted QR's many dependent passes then run at shared-memory latency
    S* Ms = as<S>(c.s.pnl);
    __syncthreads();
    copy_mat(Ms, s, M, s, s, s);
    __syncthreads();
    PH(10, r = qrcp(Ms, s, s, s, tol2, P.dense_rank, perm, tauM, c.s.flag + 2, c));
    stage_out(colmajor(M, s), Ms, s, s, s);
    __syncthreads();
  } else {
    PH(10, r = qrcp(M, s, s, s, tol2, P.dense_rank, perm, tauM, c.s.flag + 2, c));
  }
  const int over = c.s.flag[2];
  __syncthreads();
  if (over) {
    gemm(b, b, s, S(1), U0, b, false, H0, b, true, S(0), dest, b, c);
    __syncthreads();
    if (threadIdx.x == 0) *dest_rank = -1;
    __syncthreads();
    env.used = mark;
    return;
  }
  if (r > 0) {
    S* CU = (S*)env.alloc(((size_t)b * r * sizeof(S) + 7) / 8);
    S* CV = (S*)env.alloc(((size_t)b * r * sizeof(S) + 7) / 8);
    zero_mat(CU, b, b, r);
    zero_mat(CV, b, b, r);
    __syncthreads();
    for (int l = threadIdx.x; l < r; l += BLR_NT) CU[l + (size_t)l * b] = S(1);
    for (int e = threadIdx.x; e < s * r; e += BLR_NT) {
      int cc = e % s, l = e / s;
      CV[perm[cc] + (size_t)l * b] = (cc >= l) ? M[l + (size_t)cc * s] : S(0);
    }
    __syncthreads();
    PH(11, apply_q_unblocked(M, s, s, r, tauM, CU, b, r, false, c); apply_q<S>(Uf, ldu, b, s, TU, CU, b, r, false, c);
           apply_q<S>(H, b, b, s, TH, CV, b, r, false, c));
    copy_mat(dest, b, CU, b, b, r);
    copy_mat(dest + (size_t)b * P.cap, b, CV, b, b, r);
  }
  __syncthreads();
  if (threadIdx.x == 0) *dest_rank = r;
  __syncthreads();
  env.used = mark;
}

// ---------------------------------------------------------------------------
// Task bodies.  S is the arithmetic of the trailing compact-WY updates and of
// the recompressions: double on the FP64 path, float on the mixed path.
// Panel factorizations (Householder norms, tau, vectors, T) are FP64 on both.
// ---------------------------------------------------------------------------

__device__ void tc_apply_explicit_group(TaskEnv& env, const double* Yg, long long ldy, int h, int wg,
                                        const double* Tblk, double* C, long long ldc, int nc, float* Tg, float* Zs,
                                        Ctx& c);
__device__ void explicit_reflectors(const double* A, int b, int g0, int wg, double* Yx);

// GEQRT(k): Householder QR of the dense diagonal tile (Section 3.4.1).
template <class S>
__device__ void task_geqrt(TaskEnv& env, int k, Ctx& c) {
  const SchedParams& P = *env.P;
  const int b = P.b;
  double* A = tile_ptr(P, k, k);
  double* Tp = t_ptr(P, k, k);
  if (std::is_same<S, double>::value) {
    PH(21, geqrf(A, b, b, b, Tp, c));
    return;
  }
  double* pnl = c.s.pnl;
  // the panels' updates reach only the columns of their 128-column group;
  // each finished group updates the columns to its right on the tensor
  // cores (tc_apply_explicit_group)
  const bool grouped = env.tc != nullptr && b > 128;
  float *gTg = nullptr, *gZs = nullptr;
  double* gY = nullptr;
  if (grouped) {
    gTg = (float*)env.alloc(128 * 128 / 2);
    gZs = (float*)env.alloc((size_t)128 * b / 2);
    gY = env.alloc((size_t)128 * b);
  }
  for (int c0 = 0; c0 < b; c0 += BLR_NB) {
    const int w = BLR_NB, h = b - c0, ldp = h | 1;
    const int gend = grouped ? min(b, (c0 / 128 + 1) * 128) : b;   // end of this panel's update range
    __syncthreads();
    PH_BEGIN();
    stage_in(pnl, ldp, colmajor(A + c0 + (size_t)c0 * b, b), h, w);
    panel_qr(pnl, ldp, h, w, c.s.tau, c);
    gram_panel(pnl, ldp, h, w, c.s.z, c);
    t_recur(c.s.z, c.s.tau, w, c.s.t, c);
    for (int e = threadIdx.x; e < BLR_NB * BLR_NB; e += BLR_NT) Tp[e + (size_t)c0 * BLR_NB] = c.s.t[e];
    stage_out(colmajor(A + c0 + (size_t)c0 * b, b), pnl, ldp, h, w);
    __syncthreads();
    PH_END(21);
    if (c0 + w < gend) {
      PH_BEGIN();
      const int ldq = stage_panel<S>(A, b, b, c0, w, Tp, c);
      apply_refl_panel(A + c0 + (size_t)(c0 + w) * b, b, h, gend - c0 - w, (const S*)as<S>(c.s.pnl), ldq, w,
                       (const S*)as<S>(c.s.t), true, c);
      PH_END(22);
    }
    __syncthreads();
    if (grouped && c0 + w == gend && gend < b) {
      const int g0 = gend - 128;
      PH_BEGIN();
      explicit_reflectors(A, b, g0, 128, gY);
      tc_apply_explicit_group(env, gY, b - g0, b - g0, 128, Tp + (size_t)g0 * BLR_NB, A + g0 + (size_t)gend * b, b,
                              b - gend, gTg, gZs, c);
      PH_END(28);
    }
  }
}

// LARFB(k,j): R_kj = Q_kk^T A_kj (Section 3.4.2): U <- Q^T U, or the dense tile.
template <class S>
__device__ void task_larfb(TaskEnv& env, int k, int j, Ctx& c) {
  const SchedParams& P = *env.P;
  const int b = P.b;
  const int r = ld_rank(rank_ptr(P, k, j));
  double* C = tile_ptr(P, k, j);
  const int nc = (r < 0) ? b : r;
  if constexpr (std::is_same<S, float>::value) {
    if (r < 0 && env.tc && b > 128) {
      // a dense tile on the mixed path: Q_kk^T C one group of 128 reflectors
      // at a time on the tensor cores (rows g0 .. b of C)
      PH_BEGIN();
      float* gTg = (float*)env.alloc(128 * 128 / 2);
      float* gZs = (float*)env.alloc((size_t)128 * b / 2);
      double* gY = env.alloc((size_t)128 * b);
      const double* A = tile_ptr(P, k, k);
      const double* Tp = t_ptr(P, k, k);
      for (int g0 = 0; g0 < b; g0 += 128) {
        const int wg = min(128, b - g0);
        explicit_reflectors(A, b, g0, wg, gY);
        tc_apply_explicit_group(env, gY, b - g0, b - g0, wg, Tp + (size_t)g0 * BLR_NB, C + g0, b, b, gTg, gZs, c);
      }
      PH_END(23);
      return;
    }
  }
  if (nc > 0) PH(23, apply_q<S>(tile_ptr(P, k, k), b, b, b, t_ptr(P, k, k), C, b, nc, true, c));
}


// ---------------------------------------------------------------------------
// Mixed path: tensor-core operands of a dense reflector block, prepared once
// by TSQRT(i,k) for all the updates TPMQRT(i,j,k) that apply it.  The slot
// holds, each as a pre-split (hi, lo) canonical operand of Rp x b:
//   Yt: rows = reflectors a, K = tile rows   (Y^T, for Z = Y^T C)
//   Yc: rows = tile rows, K = reflectors a   (Y, for C -= Y W)
//   Tt: rows = reflectors a, K = reflectors  (T^T of the whole block, for W = T^T Z)
// where T is the b x b upper triangular factor of the compact WY form of all
// b reflectors (Eq. 3), assembled from the stored 32-reflector blocks and the
// Gram matrix G = Y^T Y of the tails (the identity parts are orthogonal):
// T(0:J, J) = -T(0:J, 0:J) G(0:J, J) T_J, one 32-column block J at a time.
// ---------------------------------------------------------------------------
__device__ void tsqrt_prep(TaskEnv& env, int i, int k, float* slot, Ctx& c) {
  const SchedParams& P = *env.P;
  TcCtx& tc = *env.tc;
  const int b = P.b, Rp = P.prep_rp;
  const size_t op = (size_t)Rp * b;
  float *yt_h = slot, *yt_l = slot + op, *yc_h = slot + 2 * op, *yc_l = slot + 3 * op, *tt_h = slot + 4 * op,
        *tt_l = slot + 5 * op;
  const int r = ld_rank(rank_ptr(P, i, k));
  const double* Tk = t_ptr(P, i, k);
  // the tails: dense Y (b x b) in the tile, or a low-rank tile's Y (r x b)
  // stored transposed in its V slot; Kt = tail length rounded up to a chunk
  const int Kt = r < 0 ? b : (r + TC_KC - 1) / TC_KC * TC_KC;
  PH_BEGIN();
  if (r < 0) {
    const double* Y = tile_ptr(P, i, k);
    tc_canon(yt_h, yt_l, Rp, b, Y, b, 1, b, b);      // (a, s) = Y[s + a b]
    tc_canon(yc_h, yc_l, Rp, b, Y, 1, b, b, b);      // (s, a) = Y[s + a b]
  } else {
    const double* V = tile_ptr(P, i, k) + (size_t)b * P.cap;
    const int Rs = (r + TC_M - 1) / TC_M * TC_M;
    tc_canon(yt_h, yt_l, Rp, Kt, V, 1, b, b, r);     // (a, s) = Y(s, a) = V[a + s b]
    tc_canon(yc_h, yc_l, Rs, b, V, b, 1, r, b);      // (s, a) = V[a + s b]
  }
  fence_async_global();
  __syncthreads();
  PH_END(24);
  PH_BEGIN2();
  // G = Y^T Y (FP32, ld b, upper block triangle)
  float* G = (float*)env.alloc((size_t)b * b / 2);
  float* T = (float*)env.alloc((size_t)b * b / 2);
  const size_t cs = (size_t)Rp * TC_KC;
  for (int m0 = 0; m0 < b; m0 += TC_M) {
    for (int n0 = 0; n0 < b; n0 += 256) {
      if (n0 + 256 <= m0) continue;       // strictly below the diagonal: not needed
      const int nn = min(256, b - n0), nn16 = (nn + 15) & ~15;
      tc_gemm_bulk(tc, *env.tq, 0, yt_h + (size_t)m0 * TC_KC, yt_l + (size_t)m0 * TC_KC, cs,
                   yt_h + (size_t)n0 * TC_KC, yt_l + (size_t)n0 * TC_KC, cs, nn16, Kt / TC_KC);
      tc_epilogue(tc, 0, nn16, [&](int r, int col, float v) {
        if (m0 + r < b && col < nn) G[(m0 + r) + (size_t)(n0 + col) * b] = v;
      });
    }
  }
  c.fma += (double)b * b * Kt / 2;
  PH_END2(25);
  // T from its 32 x 32 diagonal blocks by merging neighbouring blocks of
  // h reflectors into blocks of 2h: for the product of the compact WY forms
  // (I - Y1 T1 Y1^T)(I - Y2 T2 Y2^T) = I - [Y1 Y2] T [Y1 Y2]^T the new
  // off-diagonal block is T12 = -T1 (Y1^T Y2) T2 = -T1 G12 T2 (Eq. 3 for a
  // block of reflectors, the Schreiber-Van Loan recurrence taken a block at
  // a time); each merge is two products on the tensor cores.
  PH_BEGIN3();
  for (int e = threadIdx.x; e < b * b; e += BLR_NT) {
    const int a = e % b, l = e / b;
    T[e] = ((a >> 5) == (l >> 5) && a <= l) ? cvt<float>(ldg(Tk + (size_t)l * BLR_NB + (a & 31))) : 0.f;
  }
  __syncthreads();
  float* X = (float*)env.alloc((size_t)b * b / 4);         // b/2 x b/2 products G12 T2 (ld b/2)
  const int ldx = b / 2;
  for (int h = BLR_NB; h < b; h *= 2) {
    for (int j0 = 0; j0 + h < b; j0 += 2 * h) {
      const int h2 = min(h, b - j0 - h), h216 = (h2 + 15) & ~15;
      // X = G(j0:j0+h, j0+h:j0+h+h2) T(j0+h:j0+h+h2, j0+h:j0+h+h2)
      for (int m0 = 0; m0 < h; m0 += TC_M) {
        const int mrow = min(TC_M, h - m0);
        tc_gemm_tile(tc, 0, (const float*)G + j0 + m0 + (size_t)(j0 + h) * b, 1, b, mrow,
                     (const float*)T + (j0 + h) + (size_t)(j0 + h) * b, b, 1, h2, h216, h2);
        tc_epilogue(tc, 0, h216, [&](int r, int col, float v) {
          if (r < mrow && col < h2) X[(m0 + r) + (size_t)col * ldx] = v;
        });
      }
      // T(j0:j0+h, j0+h:j0+h+h2) = -T(j0:j0+h, j0:j0+h) X
      for (int m0 = 0; m0 < h; m0 += TC_M) {
        const int mrow = min(TC_M, h - m0);
        tc_gemm_tile(tc, 0, (const float*)T + j0 + m0 + (size_t)j0 * b, 1, b, mrow, (const float*)X, ldx, 1, h2,
                     h216, h);
        tc_epilogue(tc, 0, h216, [&](int r, int col, float v) {
          if (r < mrow && col < h2) T[(j0 + m0 + r) + (size_t)(j0 + h + col) * b] = -v;
        });
      }
      c.fma += (double)h * h2 * h2 + (double)h * h2 * h;
    }
  }
  PH_END3(26);
  PH(27, tc_canon(tt_h, tt_l, Rp, b, (const float*)T, b, 1, b, b));   // (a, k) = T(k, a) = T[k + a b]
  fence_async_global();
  __threadfence();
  __syncthreads();
}

// [Ct; Cb] <- Q^T [Ct; Cb] (Ct, Cb: b x b FP64, ld b) for a dense reflector
// block with prepared operands: Z = Ct + Y^T Cb, W = T^T Z, Ct -= W,
// Cb -= Y W, all b reflectors at once (three b x b x b products, the second
// one triangular), on the tensor cores with bulk-copied operands.
// V selects implementation variants of the conversion and the epilogues
// (measured against each other by blr_tc_update_bench): bit 0, Cb is
// converted by K-major tiles with coalesced loads; bit 3 with it, those
// tiles are stored through the four-lane exchange; bit 1, the epilogues
// issue their FP64 loads before reading TMEM; bit 2, the Z and W operands
// are stored through the four-lane exchange; bit 4, the output tiles are
// visited column block by column block (row tiles innermost).
template <int V = 0>
__device__ void tc_apply_prepared(TaskEnv& env, const float* slot, double* Ct, double* Cb, Ctx& c) {
  const SchedParams& P = *env.P;
  TcCtx& tc = *env.tc;
  const TcBulk& q = *env.tq;
  const int b = P.b, Rp = P.prep_rp;
  const size_t op = (size_t)Rp * b, cs = (size_t)Rp * TC_KC;
  const float *yt_h = slot, *yt_l = slot + op, *yc_h = slot + 2 * op, *yc_l = slot + 3 * op, *tt_h = slot + 4 * op,
              *tt_l = slot + 5 * op;
  float* cc_h = (float*)env.alloc(op / 2);    // Cb as an operand (rows = columns n), later W
  float* cc_l = (float*)env.alloc(op / 2);
  float* zc_h = (float*)env.alloc(op / 2);    // Z as an operand (rows = columns n, K = reflectors)
  float* zc_l = (float*)env.alloc(op / 2);
  if constexpr ((V & 1) != 0) {
    PH(12, tc_canon_kmajor(cc_h, cc_l, Rp, b, (const double*)Cb, b, b, b, (V & 8) != 0));
  } else {
    PH(12, tc_canon(cc_h, cc_l, Rp, b, (const double*)Cb, b, 1, b, b));    // (n, r) = Cb[r + n b]
  }
  fence_async_global();
  __syncthreads();
  const int nchunk = b / TC_KC;
  // output tiles of TC_M rows x 256 columns; bit 4 of V runs the row tiles
  // innermost, so that consecutive products share their B operand
  const int mt = (b + TC_M - 1) / TC_M, nt = (b + 255) / 256, ntile = mt * nt;
  auto tile_m0 = [&](int t) { return ((V & 16) != 0 ? t % mt : t / nt) * TC_M; };
  auto tile_n0 = [&](int t) { return ((V & 16) != 0 ? t / mt : t % nt) * 256; };
  // Z = Ct + Y^T Cb
  for (int t = 0; t < ntile; t++) {
    {
      const int m0 = tile_m0(t), n0 = tile_n0(t);
      const int nn = min(256, b - n0), nn16 = (nn + 15) & ~15;
      PH(13, tc_gemm_bulk(tc, q, 0, yt_h + (size_t)m0 * TC_KC, yt_l + (size_t)m0 * TC_KC, cs, cc_h + (size_t)n0 * TC_KC,
                   cc_l + (size_t)n0 * TC_KC, cs, nn16, nchunk));
      {
      PH_BEGIN();
      if constexpr ((V & 6) == 0) {
        tc_epilogue16(tc, 0, nn16, [&](int r, int col, const float* v) {
          const int a = m0 + r;
          if (a >= b) return;
          double ct[16];
#pragma unroll
          for (int u = 0; u < 16; u++) ct[u] = (col + u < nn) ? ldg(Ct + a + (size_t)(n0 + col + u) * b) : 0.0;
#pragma unroll
          for (int u = 0; u < 16; u++)
            if (col + u < nn) tc_canon_put(zc_h, zc_l, Rp, n0 + col + u, a, v[u] + cvt<float>(ct[u]));
        });
      } else {
        tc_epilogue16_pf<double>(
            tc, 0, nn16,
            [&](int r, int col, double* ct) {
              const int a = m0 + r;
#pragma unroll
              for (int u = 0; u < 16; u++)
                ct[u] = (a < b && col + u < nn) ? ldg(Ct + a + (size_t)(n0 + col + u) * b) : 0.0;
            },
            [&](int r, int col, const float* v, const double* ct) {
              const int a = m0 + r;
              float z[16];
#pragma unroll
              for (int u = 0; u < 16; u++) z[u] = v[u] + cvt<float>(ct[u]);
              if constexpr ((V & 4) != 0) {
                tc_canon_put16(zc_h, zc_l, Rp, n0 + col, a, z, nn - col, a < b);
              } else if (a < b) {
#pragma unroll
                for (int u = 0; u < 16; u++)
                  if (col + u < nn) tc_canon_put(zc_h, zc_l, Rp, n0 + col + u, a, z[u]);
              }
            });
      }
      PH_END(14);
      }
    }
  }
  fence_async_global();
  __syncthreads();
  // W = T^T Z (T^T lower triangular: rows m0.. need K < m0 + 128); Ct -= W
  for (int t = 0; t < ntile; t++) {
    {
      const int m0 = tile_m0(t), n0 = tile_n0(t);
      const int kch = min(b, m0 + TC_M) / TC_KC;
      const int nn = min(256, b - n0), nn16 = (nn + 15) & ~15;
      PH(13, tc_gemm_bulk(tc, q, 0, tt_h + (size_t)m0 * TC_KC, tt_l + (size_t)m0 * TC_KC, cs, zc_h + (size_t)n0 * TC_KC,
                   zc_l + (size_t)n0 * TC_KC, cs, nn16, kch));
      {
      PH_BEGIN();
      if constexpr ((V & 6) == 0) {
        tc_epilogue16(tc, 0, nn16, [&](int r, int col, const float* v) {
          const int a = m0 + r;
          if (a >= b) return;
          double ct[16];
#pragma unroll
          for (int u = 0; u < 16; u++) ct[u] = (col + u < nn) ? ldg(Ct + a + (size_t)(n0 + col + u) * b) : 0.0;
#pragma unroll
          for (int u = 0; u < 16; u++) {
            if (col + u < nn) {
              Ct[a + (size_t)(n0 + col + u) * b] = ct[u] - cvt<double>(v[u]);
              tc_canon_put(cc_h, cc_l, Rp, n0 + col + u, a, v[u]);    // W as an operand (rows = n, K = a)
            }
          }
        });
      } else {
        tc_epilogue16_pf<double>(
            tc, 0, nn16,
            [&](int r, int col, double* ct) {
              const int a = m0 + r;
#pragma unroll
              for (int u = 0; u < 16; u++)
                ct[u] = (a < b && col + u < nn) ? ldg(Ct + a + (size_t)(n0 + col + u) * b) : 0.0;
            },
            [&](int r, int col, const float* v, const double* ct) {
              const int a = m0 + r;
              if (a < b) {
#pragma unroll
                for (int u = 0; u < 16; u++)
                  if (col + u < nn) Ct[a + (size_t)(n0 + col + u) * b] = ct[u] - cvt<double>(v[u]);
              }
              if constexpr ((V & 4) != 0) {
                tc_canon_put16(cc_h, cc_l, Rp, n0 + col, a, v, nn - col, a < b);
              } else if (a < b) {
#pragma unroll
                for (int u = 0; u < 16; u++)
                  if (col + u < nn) tc_canon_put(cc_h, cc_l, Rp, n0 + col + u, a, v[u]);
              }
            });
      }
      PH_END(14);
      }
    }
  }
  fence_async_global();
  __syncthreads();
  // Cb -= Y W
  for (int t = 0; t < ntile; t++) {
    {
      const int m0 = tile_m0(t), n0 = tile_n0(t);
      const int nn = min(256, b - n0), nn16 = (nn + 15) & ~15;
      PH(13, tc_gemm_bulk(tc, q, 0, yc_h + (size_t)m0 * TC_KC, yc_l + (size_t)m0 * TC_KC, cs, cc_h + (size_t)n0 * TC_KC,
                   cc_l + (size_t)n0 * TC_KC, cs, nn16, nchunk));
      {
      PH_BEGIN();
      if constexpr ((V & 2) == 0) {
        tc_epilogue16(tc, 0, nn16, [&](int r, int col, const float* v) {
          const int rr = m0 + r;
          if (rr >= b) return;
          double cb[16];
#pragma unroll
          for (int u = 0; u < 16; u++) cb[u] = (col + u < nn) ? ldg(Cb + rr + (size_t)(n0 + col + u) * b) : 0.0;
#pragma unroll
          for (int u = 0; u < 16; u++)
            if (col + u < nn) Cb[rr + (size_t)(n0 + col + u) * b] = cb[u] - cvt<double>(v[u]);
        });
      } else {
        tc_epilogue16_pf<double>(
            tc, 0, nn16,
            [&](int r, int col, double* cb) {
              const int rr = m0 + r;
#pragma unroll
              for (int u = 0; u < 16; u++)
                cb[u] = (rr < b && col + u < nn) ? ldg(Cb + rr + (size_t)(n0 + col + u) * b) : 0.0;
            },
            [&](int r, int col, const float* v, const double* cb) {
              const int rr = m0 + r;
              if (rr >= b) return;
#pragma unroll
              for (int u = 0; u < 16; u++)
                if (col + u < nn) Cb[rr + (size_t)(n0 + col + u) * b] = cb[u] - cvt<double>(v[u]);
            });
      }
      PH_END(14);
      }
    }
  }
  c.fma += 2.0 * b * b * b + (double)b * b * b / 2;
}

__device__ void tc_apply_ts_group(TaskEnv& env, const double* Yg, long long ldy, int wg, const double* Tblk,
                                  double* Ct, long long ldt, double* Cb, long long ldb, int nc, float* Tg,
                                  float* Zs, Ctx& c);


// [Ct; Cb] <- Q^T [Ct; Cb] for a LOW-RANK reflector block (tails Y, ry x b,
// prepared by its TSQRT) with Ct the dense b x b top (FP32, ld b) and Cb the
// ry x b reduced bottom P = U^T A_ij (FP32, ld ry) of the trapezoidal update:
// Z = Ct + Y^T Cb, W = T^T Z (the whole block's T), Ct -= W, Cb -= Y W, on
// the tensor cores.  The same operator as the 32-reflector panel sweep; its
// products are b x b x ry, b x b x b (triangular) and ry x b x b.
__device__ void tc_apply_lr_prepared(TaskEnv& env, const float* slot, int ry, float* Ct, float* Cb, Ctx& c) {
  const SchedParams& P = *env.P;
  TcCtx& tc = *env.tc;
  const TcBulk& q = *env.tq;
  const int b = P.b, Rp = P.prep_rp;
  const int Kt = (ry + TC_KC - 1) / TC_KC * TC_KC, Rs = (ry + TC_M - 1) / TC_M * TC_M;
  const size_t op = (size_t)Rp * b, cs = (size_t)Rp * TC_KC, cs_s = (size_t)Rs * TC_KC;
  const float *yt_h = slot, *yt_l = slot + op, *yc_h = slot + 2 * op, *yc_l = slot + 3 * op, *tt_h = slot + 4 * op,
              *tt_l = slot + 5 * op;
  float* pc_h = (float*)env.alloc((size_t)Rp * Kt / 2);   // Cb as an operand (rows = columns n, K = s)
  float* pc_l = (float*)env.alloc((size_t)Rp * Kt / 2);
  float* zc_h = (float*)env.alloc(op / 2);                // Z, then W (rows = columns n, K = reflectors)
  float* zc_l = (float*)env.alloc(op / 2);
  float* wc_h = (float*)env.alloc(op / 2);
  float* wc_l = (float*)env.alloc(op / 2);
  tc_canon(pc_h, pc_l, Rp, Kt, (const float*)Cb, ry, 1, b, ry);      // (n, s) = Cb[s + n ry]
  fence_async_global();
  __syncthreads();
  // Z = Ct + Y^T Cb
  for (int m0 = 0; m0 < b; m0 += TC_M) {
    for (int n0 = 0; n0 < b; n0 += 256) {
      const int nn = min(256, b - n0), nn16 = (nn + 15) & ~15;
      tc_gemm_bulk(tc, q, 0, yt_h + (size_t)m0 * TC_KC, yt_l + (size_t)m0 * TC_KC, cs, pc_h + (size_t)n0 * TC_KC,
                   pc_l + (size_t)n0 * TC_KC, cs, nn16, Kt / TC_KC);
      tc_epilogue16(tc, 0, nn16, [&](int r, int col, const float* v) {
        const int a = m0 + r;
        if (a >= b) return;
        float ct[16];
#pragma unroll
        for (int u = 0; u < 16; u++) ct[u] = (col + u < nn) ? ldg(Ct + a + (size_t)(n0 + col + u) * b) : 0.f;
#pragma unroll
        for (int u = 0; u < 16; u++)
          if (col + u < nn) tc_canon_put(zc_h, zc_l, Rp, n0 + col + u, a, v[u] + ct[u]);
      });
    }
  }
  fence_async_global();
  __syncthreads();
  // W = T^T Z; Ct -= W
  for (int m0 = 0; m0 < b; m0 += TC_M) {
    const int kch = min(b, m0 + TC_M) / TC_KC;
    for (int n0 = 0; n0 < b; n0 += 256) {
      const int nn = min(256, b - n0), nn16 = (nn + 15) & ~15;
      tc_gemm_bulk(tc, q, 0, tt_h + (size_t)m0 * TC_KC, tt_l + (size_t)m0 * TC_KC, cs, zc_h + (size_t)n0 * TC_KC,
                   zc_l + (size_t)n0 * TC_KC, cs, nn16, kch);
      tc_epilogue16(tc, 0, nn16, [&](int r, int col, const float* v) {
        const int a = m0 + r;
        if (a >= b) return;
        float ct[16];
#pragma unroll
        for (int u = 0; u < 16; u++) ct[u] = (col + u < nn) ? ldg(Ct + a + (size_t)(n0 + col + u) * b) : 0.f;
#pragma unroll
        for (int u = 0; u < 16; u++) {
          if (col + u < nn) {
            Ct[a + (size_t)(n0 + col + u) * b] = ct[u] - v[u];
            tc_canon_put(wc_h, wc_l, Rp, n0 + col + u, a, v[u]);
          }
        }
      });
    }
  }
  fence_async_global();
  __syncthreads();
  // Cb -= Y W
  for (int m0 = 0; m0 < ry; m0 += TC_M) {
    for (int n0 = 0; n0 < b; n0 += 256) {
      const int nn = min(256, b - n0), nn16 = (nn + 15) & ~15;
      tc_gemm_bulk(tc, q, 0, yc_h + (size_t)m0 * TC_KC, yc_l + (size_t)m0 * TC_KC, cs_s, wc_h + (size_t)n0 * TC_KC,
                   wc_l + (size_t)n0 * TC_KC, cs, nn16, b / TC_KC);
      tc_epilogue16(tc, 0, nn16, [&](int r, int col, const float* v) {
        const int s = m0 + r;
        if (s >= ry) return;
#pragma unroll
        for (int u = 0; u < 16; u++)
          if (col + u < nn) Cb[s + (size_t)(n0 + col + u) * ry] -= v[u];
      });
    }
  }
  c.fma += 2.0 * b * b * ry + (double)b * b * b / 2;
}

// TSQRT(i,k): QR([R_kk; A^V_ik]) with A^V = V^T (low-rank) or the dense tile
// (Section 3.4.3, Eqs. 19-21); Y_ik overwrites A^V in place.  The panel
// factorization is FP64; the update of the trailing columns runs in S.
// The update QRs TSQRT(k+1,k), TSQRT(k+2,k), ... of column k form a chain
// through R_kk, but each 128-column group of a TSQRT touches only the rows
// of R_kk of that group, which are final once the previous TSQRT of the
// chain has finished the same group.  So a TSQRT releases its successor
// after its first group and publishes the number of groups it has done in
// chain[toff[k] + i - k] (one counter per update QR, written by it alone,
// so it only grows); the successor waits for each group before it starts
// it (bounded by the watchdog).  One shared counter per column would not
// do: a slower predecessor's later write could lower it under a waiter's
// target for good.
__device__ __forceinline__ int chain_groups(int b) { return (b + 127) / 128; }

// All threads: waits until *flag >= target.  False when the wait ran out
// (ST_TIMEOUT set) or another error stopped the factorization.
__device__ bool chain_wait(const SchedParams& P, const int* flag, int target) {
  __shared__ int ok_sh;
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned long long t0 = tc_gtimer();
    int ok = 1;
    while (*(volatile const int*)flag < target) {
      if (*(volatile int*)P.status != 0) { ok = 0; break; }
      if (tc_gtimer() - t0 > (unsigned long long)P.watchdog_ns) {
        atomicOr(P.status, ST_TIMEOUT);
        ok = 0;
        break;
      }
      __nanosleep(128);
    }
    __threadfence();
    ok_sh = ok;
  }
  __syncthreads();
  return ok_sh != 0;
}

// All threads: group g of TSQRT(i,k) is done; the first group also releases
// the next TSQRT of the chain.
__device__ void chain_publish(TaskEnv& env, int i, int k, int g) {
  const SchedParams& P = *env.P;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    atomicExch(P.chain + P.toff_dev[k] + (i - k), g + 1);
    if (g == 0 && i + 1 < P.p && env.skip_succ < 0 && P.task_base + dag_id_tsqrt(*env.dag, i, k) != P.withhold) {
      const int sid = dag_id_tsqrt(*env.dag, i + 1, k);
      release_task(P, *env.dag, sid);
      env.skip_succ = sid;
    }
  }
  __syncthreads();
}

template <class S>
__device__ void task_tsqrt(TaskEnv& env, int i, int k, Ctx& c) {
  const SchedParams& P = *env.P;
  const int b = P.b;
  const int r = ld_rank(rank_ptr(P, i, k));
  double* R = tile_ptr(P, k, k);
  double* Tk = t_ptr(P, i, k);
  double* B = tile_ptr(P, i, k);
  const int ry = (r < 0) ? b : r;
  View<double> Bv = (r < 0) ? colmajor(B, b) : rowmajor(B + (size_t)b * P.cap, b);
  const int ng = chain_groups(b);
  const bool has_pred = P.chain != nullptr && i > k + 1;
  const int* pred = has_pred ? P.chain + P.toff_dev[k] + (i - 1 - k) : nullptr;   // TSQRT(i-1,k)'s groups done
  if (ry == 0) {
    // a rank-0 tail leaves R_kk as it is: wait for the predecessor to finish
    // it, then pass it on as done
    for (int e = threadIdx.x; e < BLR_NB * b; e += BLR_NT) Tk[e] = 0.0;
    __syncthreads();
    if (P.chain) {
      if (has_pred && !chain_wait(P, pred, ng)) return;
      chain_publish(env, i, k, ng - 1);
    }
    return;
  }
  // mixed path, dense tail: the panels' updates reach only the columns of
  // their 128-column group; each finished group updates the columns to its
  // right on the tensor cores (whole-group T, tc_apply_ts_group)
  const bool grouped = std::is_same<S, float>::value && r < 0 && env.tc != nullptr && b > 128;
  float* gTg = nullptr;
  float* gZs = nullptr;
  if (grouped) {
    gTg = (float*)env.alloc(128 * 128 / 2);
    gZs = (float*)env.alloc((size_t)128 * b / 2);
  }
  for (int c0 = 0; c0 < b; c0 += BLR_NB) {
    const int w = BLR_NB;
    const int ldb = ry | 1;
    const int gend = grouped ? min(b, (c0 / 128 + 1) * 128) : b;   // end of this panel's update range
    // the rows of R_kk of this group are final once the previous update QR
    // of the chain has finished the group
    if (has_pred && c0 % 128 == 0 && !chain_wait(P, pred, c0 / 128 + 1)) return;
    __syncthreads();
    for (int e = threadIdx.x; e < w * w; e += BLR_NT) {
      int a = e % w, l = e / w;
      c.s.rp[a + l * BLR_NB] = (a <= l) ? ldg(R + (c0 + a) + (size_t)(c0 + l) * b) : 0.0;
    }
    View<double> Bp = Bv.shifted(0, c0);
    PH(16, stage_in(c.s.pnl, ldb, Bp, ry, w));
    PH(17, ts_panel_qr(c.s.rp, c.s.pnl, ldb, ry, w, c.s.tau, c));
    PH_BEGIN();
    gram_dense(c.s.pnl, ldb, ry, w, c.s.z, c);
    t_recur(c.s.z, c.s.tau, w, c.s.t, c);
    for (int e = threadIdx.x; e < BLR_NB * BLR_NB; e += BLR_NT) Tk[e + (size_t)c0 * BLR_NB] = c.s.t[e];
    for (int e = threadIdx.x; e < w * w; e += BLR_NT) {
      int a = e % w, l = e / w;
      if (a <= l) R[(c0 + a) + (size_t)(c0 + l) * b] = c.s.rp[a + l * BLR_NB];
    }
    stage_out(Bp, c.s.pnl, ldb, ry, w);
    __syncthreads();
    PH_END(18);
    if (c0 + w < gend) {
      PH_BEGIN();
      View<double> Cb = Bv.shifted(0, c0 + w);
      if (std::is_same<S, double>::value) {
        apply_refl_ts(R + c0 + (size_t)(c0 + w) * b, b, Cb, ry, gend - c0 - w, c.s.pnl, ldb, w, c.s.t, true, c);
      } else {
        const int ldy = stage_reflector_panel<S>(Bv, ry, c0, w, Tk, c);
        apply_refl_ts(R + c0 + (size_t)(c0 + w) * b, b, Cb, ry, gend - c0 - w, (const S*)as<S>(c.s.pnl), ldy, w,
                      (const S*)as<S>(c.s.t), true, c);
      }
      PH_END(19);
    }
    __syncthreads();
    if (grouped && c0 + w == gend && gend < b) {
      const int g0 = gend - 128;
      PH(20, tc_apply_ts_group(env, B + (size_t)g0 * b, b, 128, Tk + (size_t)g0 * BLR_NB, R + g0 + (size_t)gend * b,
                               b, B + (size_t)gend * b, b, b - gend, gTg, gZs, c));
    }
    if (P.chain && ((c0 + w) % 128 == 0 || c0 + w == b)) chain_publish(env, i, k, c0 / 128);
  }
  if constexpr (std::is_same<S, float>::value) {
    if (r != 0 && P.prep && env.tc && k + 1 < P.q) {
      // release the next update QR of this column now (it needs only R_kk),
      // then prepare the tensor-core operands for the updates TPMQRT(i,.,k)
      // in a slot of the pool
      __shared__ int slot_sh;
      __threadfence();
      __syncthreads();
      if (threadIdx.x == 0) {
        if (i + 1 < P.p && env.skip_succ < 0 && P.task_base + dag_id_tsqrt(*env.dag, i, k) != P.withhold) {
          const int sid = dag_id_tsqrt(*env.dag, i + 1, k);
          release_task(P, *env.dag, sid);
          env.skip_succ = sid;
        }
        slot_sh = prep_acquire(P);
      }
      __syncthreads();
      const int slot = slot_sh;
      if (slot >= 0) {
        PH(7, tsqrt_prep(env, i, k, prep_at(P, slot), c));
        if (threadIdx.x == 0) {
          // the q-k-1 updates TPMQRT(i,.,k) each release the slot once; they
          // run after this task ends, so they see the slot it records
          atomicExch(P.prep_ref + slot, P.q - k - 1);
          atomicExch(P.prep_slot_of + prep_block(P, i, k), slot);
          __threadfence();
        }
        __syncthreads();
      }
    }
  }
}

// TPMQRT(i,j,k): [R_kj; A_ij] <- Q_ik^T [R_kj; A_ij] with
// Q_ik = I - [I; Y~] T [I; Y~]^T (Section 3.4.4).  With Y~ = U_ik Y_ik the
// operator acts on A_ij only through P = U_ik^T A_ij, so it is applied to
// the reduced pair [R_kj; P] (rows b + r_Y) and A_ij += U_ik (P' - P).  When
// R_kj and A_ij are low-rank the pair is kept factored, [R; P] = G H^T, the
// reflector is applied to G, and both results are recompressed by the
// rounded addition of Algorithm 6 (sharing the QR of H).
//
// Operands are tile-layout buffers of type S (U at 0, V at b*cap, or dense
// b x b); rY/rR/rA are their ranks (-1 dense); new ranks go to *nR, *nA.
template <class S>
__device__ void tpmqrt_core(TaskEnv& env, S* Yt, int rY, const S* Tik, S* Rt, int rR, S* At, int rA, int* nR,
                            int* nA, Ctx& c) {
  const SchedParams& P = *env.P;
  const int b = P.b, cap = P.cap;
  auto alloc = [&](size_t n) { return (S*)env.alloc((n * sizeof(S) + 7) / 8); };
  const bool ylr = rY >= 0;
  if (ylr && rY == 0) return;           // the reflector is the identity
  const int ry = ylr ? rY : b;
  S* Uy = Yt;
  View<S> Yr = ylr ? rowmajor(Yt + (size_t)b * cap, b) : colmajor(Yt, b);

  if (rR >= 0 && (rA >= 0 || ylr)) {
    // ---------------- factored paths -----------------
    const bool adense = rA < 0;         // A dense, Y low-rank
    const int s2 = adense ? ry : rA;    // columns of the P part
    const int s = rR + s2;
    if (s == 0) return;
    const int ldG = b + ry;
    S* G = alloc((size_t)ldG * s);
    S* H = alloc((size_t)b * s);
    S* H0 = alloc((size_t)b * s);
    S* PU0 = alloc((size_t)ry * s2);
    zero_mat(G, ldG, ldG, s);
    __syncthreads();
    copy_mat(G, ldG, Rt, b, b, rR);                              // U_R
    copy_mat(H, b, Rt + (size_t)b * cap, b, b, rR);              // V_R
    if (!adense) {
      if (ylr) PH(2, gemm(ry, rA, b, S(1), Uy, b, true, At, b, false, S(0), G + b + (size_t)rR * ldG, ldG, c));
      else copy_mat(G + b + (size_t)rR * ldG, ldG, At, b, b, rA);
      copy_mat(H + (size_t)rR * b, b, At + (size_t)b * cap, b, b, rA);
    } else {
      PH(2, gemm(b, ry, b, S(1), At, b, true, Uy, b, false, S(0), H + (size_t)rR * b, b, c));
      __syncthreads();
      for (int e = threadIdx.x; e < ry; e += BLR_NT) G[b + e + (size_t)(rR + e) * ldG] = S(1);
    }
    __syncthreads();
    copy_mat(PU0, ry, G + b + (size_t)rR * ldG, ldG, ry, s2);
    copy_mat(H0, b, H, b, b, s);
    __syncthreads();
    PH(3, apply_ts_reflector<S>(Yr, ry, b, Tik, G, ldG, colmajor(G + b, ldG), s, true, c));
    for (int e = threadIdx.x; e < ry * s2; e += BLR_NT) {
      int a = e % ry, l = e / ry;
      G[b + a + (size_t)(rR + l) * ldG] -= PU0[e];
    }
    __syncthreads();
    S* TH = alloc((size_t)BLR_NB * s);
    if (!adense) {
      S* UfA = alloc((size_t)b * s);
      if (ylr) PH(2, gemm(b, s, ry, S(1), Uy, b, false, G + b, ldG, false, S(0), UfA, b, c));
      else copy_mat(UfA, b, G + b, ldG, b, s);
      __syncthreads();
      for (int e = threadIdx.x; e < b * rA; e += BLR_NT) {
        int a = e % b, l = e / b;
        UfA[a + (size_t)(rR + l) * b] += ldg(At + a + (size_t)l * b);
      }
      __syncthreads();
      PH(4, geqrf(H, b, b, s, TH, c));
      PH(5, recompress_side(env, G, ldG, H, TH, H0, s, Rt, nR, c));
      PH(5, recompress_side(env, UfA, b, H, TH, H0, s, At, nA, c));
    } else {
      S* M1 = alloc((size_t)b * s);
      PH(2, gemm(b, s, ry, S(1), Uy, b, false, G + b, ldG, false, S(0), M1, b, c));
      PH(2, gemm(b, b, s, S(1), M1, b, false, H0, b, true, S(1), At, b, c));
      PH(4, geqrf(H, b, b, s, TH, c));
      PH(5, recompress_side(env, G, ldG, H, TH, H0, s, Rt, nR, c));
    }
    return;
  }

  // ---------------- dense path: R_kj dense (or becomes dense) -----------------
  S* Rd;
  bool r_scratch = false;
  if (rR < 0) {
    Rd = Rt;
  } else {
    Rd = alloc((size_t)b * b);
    if (rR > 0) PH(2, gemm(b, b, rR, S(1), Rt, b, false, Rt + (size_t)b * cap, b, true, S(0), Rd, b, c));
    else zero_mat(Rd, b, b, b);
    r_scratch = true;
  }
  S* Pm;
  int ldp;
  S* P0 = nullptr;
  bool a_inplace = false;
  if (ylr) {
    ldp = ry;
    Pm = alloc((size_t)ry * b);
    if (rA < 0) {
      PH(2, gemm(ry, b, b, S(1), Uy, b, true, At, b, false, S(0), Pm, ry, c));
    } else if (rA == 0) {
      zero_mat(Pm, ry, ry, b);
    } else {
      S* PU = alloc((size_t)ry * rA);
      PH(2, gemm(ry, rA, b, S(1), Uy, b, true, At, b, false, S(0), PU, ry, c));
      PH(2, gemm(ry, b, rA, S(1), PU, ry, false, At + (size_t)b * cap, b, true, S(0), Pm, ry, c));
    }
    P0 = alloc((size_t)ry * b);
    __syncthreads();
    copy_mat(P0, ry, Pm, ry, ry, b);
  } else {
    ldp = b;
    if (rA < 0) {
      Pm = At;
      a_inplace = true;
    } else {
      Pm = alloc((size_t)b * b);
      if (rA > 0) PH(2, gemm(b, b, rA, S(1), At, b, false, At + (size_t)b * cap, b, true, S(0), Pm, b, c));
      else zero_mat(Pm, b, b, b);
    }
  }
  __syncthreads();
  if constexpr (std::is_same<S, float>::value) {
    if (ylr && env.prep_slot && env.tc) {
      // low-rank reflector block with prepared tensor-core operands
      PH(3, tc_apply_lr_prepared(env, env.prep_slot, ry, Rd, Pm, c));
    } else {
      PH(3, apply_ts_reflector<S>(Yr, ry, b, Tik, Rd, b, colmajor(Pm, ldp), b, true, c));
    }
  } else {
    PH(3, apply_ts_reflector<S>(Yr, ry, b, Tik, Rd, b, colmajor(Pm, ldp), b, true, c));
  }
  if (r_scratch) {
    copy_mat(Rt, b, Rd, b, b, b);
    __syncthreads();
    if (threadIdx.x == 0) *nR = -1;
  }
  __syncthreads();
  if (!ylr) {
    if (!a_inplace) {
      copy_mat(At, b, Pm, b, b, b);
      __syncthreads();
      if (threadIdx.x == 0) *nA = -1;
    }
    __syncthreads();
    return;
  }
  for (int e = threadIdx.x; e < ry * b; e += BLR_NT) Pm[e] -= P0[e];
  __syncthreads();
  if (rA < 0) {
    PH(2, gemm(b, b, ry, S(1), Uy, b, false, Pm, ry, false, S(1), At, b, c));
    return;
  }
  const int s = rA + ry;
  S* Uf = alloc((size_t)b * s);
  S* H = alloc((size_t)b * s);
  S* H0 = alloc((size_t)b * s);
  copy_mat(Uf, b, At, b, b, rA);
  copy_mat(Uf + (size_t)rA * b, b, Uy, b, b, ry);
  copy_mat(H, b, At + (size_t)b * cap, b, b, rA);
  __syncthreads();
  for (int e = threadIdx.x; e < b * ry; e += BLR_NT) {
    int a = e % b, l = e / b;
    H[a + (size_t)(rA + l) * b] = Pm[l + (size_t)a * ldp];
  }
  __syncthreads();
  copy_mat(H0, b, H, b, b, s);
  S* TH = alloc((size_t)BLR_NB * s);
  __syncthreads();
  PH(4, geqrf(H, b, b, s, TH, c));
  PH(5, recompress_side(env, Uf, b, H, TH, H0, s, At, nA, c));
}


// ---------------------------------------------------------------------------
// Mixed path on the tensor cores: the dense trapezoidal update.
// ---------------------------------------------------------------------------

// D (b x b, FP64, ld b) = U V^T for a low-rank tile (U, V: b x r in tile
// layout) on the tensor cores.
__device__ void tc_densify(TaskEnv& env, const double* Tl, int r, double* D, Ctx& c) {
  TcCtx& tc = *env.tc;
  const int b = env.P->b, cap = env.P->cap;
  if (r == 0) {
    zero_mat(D, b, b, b);
    __syncthreads();
    return;
  }
  const double* U = Tl;
  const double* V = Tl + (size_t)b * cap;
  for (int r0 = 0; r0 < b; r0 += TC_M) {
    const int mrow = min(TC_M, b - r0);
    for (int n0 = 0; n0 < b; n0 += 256) {
      const int nn = min(256, b - n0), nn16 = (nn + 15) & ~15;
      tc_gemm_tile(tc, 0, U + r0, 1, b, mrow, V + n0, 1, b, nn, nn16, r);
      tc_epilogue(tc, 0, nn16, [&](int rr, int cc, float v) {
        if (rr < mrow && cc < nn) D[(r0 + rr) + (size_t)(n0 + cc) * b] = cvt<double>(v);
      });
    }
  }
  c.fma += (double)b * b * r;
}

// T of a group of wg <= 128 consecutive reflectors (Eq. 3's compact WY form
// of their product) from the stored inner 32-reflector blocks and the Gram
// matrix G = Y_g^T Y_g of their tails (the identity parts are mutually
// orthogonal): T(0:J, J) = -T(0:J, 0:J) G(0:J, J) T_J, block column by
// block column.  Gs, Ts (ld 128) and X (ld 128, 32 columns) are shared
// memory; Ts receives the wg x wg upper triangle (zeros elsewhere).
__device__ void tc_group_t(const double* Tblk, int wg, const float* Gs, float* Ts, float* X, Ctx& c) {
  for (int e = threadIdx.x; e < 128 * 128; e += BLR_NT) {
    const int a = e & 127, l = e >> 7;
    float v = 0.f;
    if (a < wg && l < wg && (a >> 5) == (l >> 5) && a <= l) v = cvt<float>(ldg(Tblk + (size_t)l * BLR_NB + (a & 31)));
    Ts[e] = v;
  }
  __syncthreads();
  for (int J = 1; J * BLR_NB < wg; J++) {
    const int top = J * BLR_NB;
    for (int e = threadIdx.x; e < top * BLR_NB; e += BLR_NT) {
      const int a = e % top, m = e / top;
      float s = 0.f;
      for (int l = 0; l <= m; l++) s += Gs[a + (top + l) * 128] * Ts[(top + l) + (top + m) * 128];
      X[a + m * 128] = s;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < top * BLR_NB; e += BLR_NT) {
      const int a = e % top, m = e / top;
      float s = 0.f;
      for (int l = a; l < top; l++) s += Ts[a + l * 128] * X[l + m * 128];
      Ts[a + (top + m) * 128] = -s;
    }
    __syncthreads();
    c.fma += (double)top * BLR_NB * BLR_NB / 2 + (double)top * top * BLR_NB / 2;
  }
}

// [Ct (b x nc, ld ldt); Cb (b x nc, ld ldb)] <- Q^T [Ct; Cb] for the dense
// reflector block of a TSQRT, Q = I - [I; Y] T [I; Y]^T with Y b x b dense
// (Section 3.4.4, Eq. 21), in groups of 128 reflectors:
//   Z = Ct(g rows) + Y_g^T Cb;  W = T_g^T Z;  Ct(g rows) -= W;  Cb -= Y_g W.
// Products on the tensor cores (3xTF32, FP32 accumulation); the tiles stay
// FP64 and receive FP64 updates.
// One group of wg <= 128 consecutive reflectors [e_a; y_a] of a dense block
// (tails Yg, b x wg, ld ldy; inner T blocks at Tblk) applied to [Ct; Cb] on
// the tensor cores, Ct the wg rows of the top that the group's identity part
// touches (ld ldt) and Cb the b x nc bottom (ld ldb):
//   Z = Ct + Y_g^T Cb;  W = T_g^T Z;  Ct -= W;  Cb -= Y_g W
// with T_g assembled from the inner blocks and G = Y_g^T Y_g.  Tg (128 x 128)
// and Zs (128 x nc) are global scratch.
__device__ void tc_apply_ts_group(TaskEnv& env, const double* Yg, long long ldy, int wg, const double* Tblk,
                                  double* Ct, long long ldt, double* Cb, long long ldb, int nc, float* Tg,
                                  float* Zs, Ctx& c) {
  TcCtx& tc = *env.tc;
  const int b = env.P->b;
  float* Gsm = tc.buf;                                   // staging area, idle between products
  float* Tsm = tc.buf + 128 * 128;
  float* Xsm = tc.buf + 2 * 128 * 128;
  // G = Y_g^T Y_g
  tc_gemm_tile(tc, 0, Yg, ldy, 1, wg, Yg, ldy, 1, wg, wg, b);
  tc_epilogue(tc, 0, wg, [&](int r, int col, float v) { Gsm[r + col * 128] = v; });
  c.fma += (double)wg * wg * b / 2;
  tc_group_t(Tblk, wg, Gsm, Tsm, Xsm, c);
  for (int e = threadIdx.x; e < 128 * 128; e += BLR_NT) Tg[e] = Tsm[e];
  __syncthreads();
  // Z = Ct + Y_g^T Cb
  for (int n0 = 0; n0 < nc; n0 += 256) {
    const int nn = min(256, nc - n0), nn16 = (nn + 15) & ~15;
    tc_gemm_tile(tc, 0, Yg, ldy, 1, wg, Cb + (size_t)n0 * ldb, ldb, 1, nn, nn16, b);
    tc_epilogue(tc, 0, nn16, [&](int r, int col, float v) {
      if (r < wg && col < nn) {
        const size_t n = n0 + col;
        Zs[r + n * 128] = v + cvt<float>(ldg(Ct + r + n * ldt));
      }
    });
  }
  // W = T_g^T Z; Ct -= W
  for (int n0 = 0; n0 < nc; n0 += 256) {
    const int nn = min(256, nc - n0), nn16 = (nn + 15) & ~15;
    tc_gemm_tile(tc, 0, (const float*)Tg, 128, 1, wg, (const float*)Zs + (size_t)n0 * 128, 128, 1, nn, nn16, wg);
    tc_epilogue(tc, 0, nn16, [&](int r, int col, float v) {
      if (r < wg && col < nn) {
        const size_t n = n0 + col;
        double* p = Ct + r + n * ldt;
        *p = ldg(p) - cvt<double>(v);
        Zs[r + n * 128] = v;
      }
    });
  }
  // Cb -= Y_g W
  for (int r0 = 0; r0 < b; r0 += TC_M) {
    const int mrow = min(TC_M, b - r0);
    for (int n0 = 0; n0 < nc; n0 += 256) {
      const int nn = min(256, nc - n0), nn16 = (nn + 15) & ~15;
      tc_gemm_tile(tc, 0, Yg + r0, 1, ldy, mrow, (const float*)Zs + (size_t)n0 * 128, 128, 1, nn, nn16, wg);
      tc_epilogue(tc, 0, nn16, [&](int r, int col, float v) {
        if (r < mrow && col < nn) {
          double* p = Cb + (r0 + r) + (size_t)(n0 + col) * ldb;
          *p = ldg(p) - cvt<double>(v);
        }
      });
    }
  }
  c.fma += (double)wg * nc * b + (double)wg * nc * wg / 2 + (double)b * nc * wg;
}

// C (h x nc, FP64, ld ldc) <- Q_g^T C for a group of wg <= 128 consecutive
// reflectors of a diagonal-tile QR (Section 3.4.1) whose vectors are given
// explicitly, unit diagonal and zeros above it included (Yg, h x wg FP64,
// ld ldy), with their inner 32-reflector T blocks at Tblk:
//   Z = Y_g^T C;  W = T_g^T Z;  C -= Y_g W
// on the tensor cores (3xTF32), T_g assembled from the inner blocks and the
// Gram matrix G = Y_g^T Y_g.  Tg (128 x 128) and Zs (128 x nc) are global
// scratch.
__device__ void tc_apply_explicit_group(TaskEnv& env, const double* Yg, long long ldy, int h, int wg,
                                        const double* Tblk, double* C, long long ldc, int nc, float* Tg, float* Zs,
                                        Ctx& c) {
  TcCtx& tc = *env.tc;
  float* Gsm = tc.buf;                                   // staging area, idle between products
  float* Tsm = tc.buf + 128 * 128;
  float* Xsm = tc.buf + 2 * 128 * 128;
  // G = Y_g^T Y_g
  tc_gemm_tile(tc, 0, Yg, ldy, 1, wg, Yg, ldy, 1, wg, (wg + 15) & ~15, h);
  tc_epilogue(tc, 0, (wg + 15) & ~15, [&](int r, int col, float v) {
    if (r < 128 && col < 128) Gsm[r + col * 128] = v;
  });
  c.fma += (double)wg * wg * h / 2;
  tc_group_t(Tblk, wg, Gsm, Tsm, Xsm, c);
  for (int e = threadIdx.x; e < 128 * 128; e += BLR_NT) Tg[e] = Tsm[e];
  __syncthreads();
  for (int n0 = 0; n0 < nc; n0 += 256) {
    const int nn = min(256, nc - n0), nn16 = (nn + 15) & ~15;
    // Z = Y_g^T C
    tc_gemm_tile(tc, 0, Yg, ldy, 1, wg, C + (size_t)n0 * ldc, ldc, 1, nn, nn16, h);
    tc_epilogue(tc, 0, nn16, [&](int r, int col, float v) {
      if (r < wg && col < nn) Zs[r + (size_t)(n0 + col) * 128] = v;
    });
    // W = T_g^T Z
    tc_gemm_tile(tc, 0, (const float*)Tg, 128, 1, wg, (const float*)Zs + (size_t)n0 * 128, 128, 1, nn, nn16, wg);
    tc_epilogue(tc, 0, nn16, [&](int r, int col, float v) {
      if (r < wg && col < nn) Zs[r + (size_t)(n0 + col) * 128] = v;
    });
    // C -= Y_g W
    for (int r0 = 0; r0 < h; r0 += TC_M) {
      const int mrow = min(TC_M, h - r0);
      tc_gemm_tile(tc, 0, Yg + r0, 1, ldy, mrow, (const float*)Zs + (size_t)n0 * 128, 128, 1, nn, nn16, wg);
      tc_epilogue(tc, 0, nn16, [&](int r, int col, float v) {
        if (r < mrow && col < nn) {
          double* p = C + (r0 + r) + (size_t)(n0 + col) * ldc;
          *p = ldg(p) - cvt<double>(v);
        }
      });
    }
  }
  c.fma += (double)wg * nc * h + (double)wg * nc * wg / 2 + (double)h * nc * wg;
}

// The explicit vectors of the reflectors g0 .. g0 + wg - 1 of a diagonal
// tile's QR (stored below the diagonal of tile A, b x b, ld b): rows g0 .. b
// of those columns with the unit diagonal and zeros above it, into Yx
// (b - g0 rows, ld b - g0).
__device__ void explicit_reflectors(const double* A, int b, int g0, int wg, double* Yx) {
  const int h = b - g0;
  for (int e = threadIdx.x; e < h * wg; e += BLR_NT) {
    const int r = e % h, l = e / h;
    double v = 0.0;
    if (r > l) v = ldg(A + (g0 + r) + (size_t)(g0 + l) * b);
    else if (r == l) v = 1.0;
    Yx[e] = v;
  }
  __syncthreads();
}

// [Ct (b x nc, ld ldt); Cb (b x nc, ld ldb)] <- Q^T [Ct; Cb] for the dense
// reflector block of a TSQRT, Q = I - [I; Y] T [I; Y]^T with Y b x b dense
// (Section 3.4.4, Eq. 21), in groups of 128 reflectors.  Products on the
// tensor cores (3xTF32, FP32 accumulation); the tiles stay FP64 and receive
// FP64 updates.
__device__ void tc_apply_ts_dense(TaskEnv& env, const double* Y, const double* Tik, double* Ct, long long ldt,
                                  double* Cb, long long ldb, int nc, Ctx& c) {
  const int b = env.P->b;
  float* Tg = (float*)env.alloc(128 * 128 / 2);          // global copy of T_g (A operand of W)
  float* Zs = (float*)env.alloc((size_t)128 * nc / 2);   // Z, then W (ld 128)
  for (int c0 = 0; c0 < b; c0 += 128) {
    const int wg = min(128, b - c0);
    tc_apply_ts_group(env, Y + (size_t)c0 * b, b, wg, Tik + (size_t)c0 * BLR_NB, Ct + c0, ldt, Cb, ldb, nc, Tg, Zs,
                      c);
  }
}

// TPMQRT(i,j,k) with a dense reflector block and a dense R_kj or A_ij, on
// the tensor cores: a low-rank operand is densified (it becomes dense, as
// OP1 of Section 3.1 makes it), then the block reflector is applied.
__device__ void tpmqrt_tc_dense(TaskEnv& env, const double* Yt, const double* Tik, const float* prep, double* Rt,
                                int rR, double* At, int rA, int* nR, int* nA, Ctx& c) {
  const int b = env.P->b;
  double* Rd = Rt;
  double* Ad = At;
  if (rR >= 0) {
    Rd = env.alloc((size_t)b * b);
    PH(15, tc_densify(env, Rt, rR, Rd, c));
  }
  if (rA >= 0) {
    Ad = env.alloc((size_t)b * b);
    PH(15, tc_densify(env, At, rA, Ad, c));
  }
  if (prep) tc_apply_prepared<BLR_TC_UPDATE_VARIANT>(env, prep, Rd, Ad, c);
  else tc_apply_ts_dense(env, Yt, Tik, Rd, b, Ad, b, b, c);
  if (rR >= 0) copy_mat(Rt, b, Rd, b, b, b);
  if (rA >= 0) copy_mat(At, b, Ad, b, b, b);
  __syncthreads();
  if (threadIdx.x == 0) {
    if (rR >= 0) *nR = -1;
    if (rA >= 0) *nA = -1;
  }
  __syncthreads();
}

// Copies the live part of a tile (rank r: U and V columns; -1: dense) between
// storage types.
template <class D, class Src>
__device__ void copy_tile(D* dst, const Src* src, int r, int b, int cap) {
  if (r < 0) {
    copy_mat(dst, b, src, b, b, b);
  } else if (r > 0) {
    copy_mat(dst, b, src, b, b, r);
    copy_mat(dst + (size_t)b * cap, b, src + (size_t)b * cap, b, b, r);
  }
}

template <class S>
__device__ void task_tpmqrt(TaskEnv& env, int i, int j, int k, Ctx& c) {
  const SchedParams& P = *env.P;
  const int b = P.b, cap = P.cap;
  const int rY = ld_rank(rank_ptr(P, i, k));
  const int rR = ld_rank(rank_ptr(P, k, j));
  const int rA = ld_rank(rank_ptr(P, i, j));
  double* Yt = tile_ptr(P, i, k);
  double* Rt = tile_ptr(P, k, j);
  double* At = tile_ptr(P, i, j);
  const double* Tik = t_ptr(P, i, k);
  if (std::is_same<S, double>::value) {
    tpmqrt_core<double>(env, Yt, rY, Tik, Rt, rR, At, rA, rank_ptr(P, k, j), rank_ptr(P, i, j), c);
    return;
  }
  if (rY == 0) return;
  // the operands the TSQRT prepared for this reflector block, if it found a slot
  const int slot = P.prep ? __ldcg(P.prep_slot_of + prep_block(P, i, k)) : -1;
  const float* prep = slot >= 0 ? prep_at(P, slot) : nullptr;
  if (rY < 0 && (rR < 0 || rA < 0) && env.tc) {
    PH(6, tpmqrt_tc_dense(env, Yt, Tik, prep, Rt, rR, At, rA, rank_ptr(P, k, j), rank_ptr(P, i, j), c));
    return;
  }
  // a low-rank reflector block whose TSQRT prepared tensor-core operands
  env.prep_slot = (env.tc && rY > 0) ? prep : nullptr;
  // mixed: FP32 copies of the operands, FP32 arithmetic, results back to FP64
  float* Yf = (float*)env.alloc((size_t)b * b / 2);
  float* Tf = (float*)env.alloc((size_t)BLR_NB * b / 2);
  float* Rf = (float*)env.alloc((size_t)b * b / 2);
  float* Af = (float*)env.alloc((size_t)b * b / 2);
  PH(0, copy_tile(Yf, Yt, rY, b, cap); copy_mat(Tf, BLR_NB, Tik, BLR_NB, BLR_NB, b);
        copy_tile(Rf, Rt, rR, b, cap); copy_tile(Af, At, rA, b, cap));
  __shared__ int newr[2];
  if (threadIdx.x == 0) { newr[0] = rR; newr[1] = rA; }
  __syncthreads();
  tpmqrt_core<float>(env, Yf, rY, Tf, Rf, rR, Af, rA, &newr[0], &newr[1], c);
  __syncthreads();
  const int r1 = newr[0], r2 = newr[1];
  PH(1, copy_tile(Rt, Rf, r1, b, cap); copy_tile(At, Af, r2, b, cap));
  __syncthreads();
  if (threadIdx.x == 0) {
    *rank_ptr(P, k, j) = r1;
    *rank_ptr(P, i, j) = r2;
  }
  __syncthreads();
}

// ---------------------------------------------------------------------------
// Persistent scheduler
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long gtimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ void q_push(const SchedParams& P, int qi, int task) {
  int pos = atomicAdd(P.qtail + qi * 32, 1);
  atomicExch(P.qbuf + (size_t)qi * P.n_tasks + pos, task);
}

// Thread 0 only.  Returns a task id, or -1 when the factorization is done
// or aborted.  Every wait is bounded by the watchdog budget.
__device__ int q_pop(const SchedParams& P) {
  unsigned ns = 64;
  while (true) {
    if (*(volatile int*)P.status != 0) return -1;
    for (int qi = 0; qi < BLR_NQ; qi++) {
      volatile int* head = P.qhead + qi * 32;
      volatile int* tail = P.qtail + qi * 32;
      while (true) {
        int h = *head, t = *tail;
        if (h >= t) break;
        if (atomicCAS((int*)head, h, h + 1) == h) {
          volatile int* slot = P.qbuf + (size_t)qi * P.n_tasks + h;
          int v;
          unsigned long long t0 = gtimer();
          while ((v = *slot) < 0) {
            if (gtimer() - t0 > (unsigned long long)P.watchdog_ns) {
              atomicOr(P.status, ST_TIMEOUT);
              return -1;
            }
            __nanosleep(32);
          }
          __threadfence();
          return v;
        }
      }
    }
    if (*(volatile int*)P.done >= P.n_tasks) return -1;
    unsigned long long now = gtimer();
    unsigned long long last = *(volatile unsigned long long*)P.progress_ns;
    if (last == 0ull) {
      atomicCAS(P.progress_ns, 0ull, now);
    } else if (now > last && now - last > (unsigned long long)P.watchdog_ns) {
      atomicOr(P.status, ST_TIMEOUT);
      return -1;
    }
    __nanosleep(ns);
    if (ns < 8192) ns <<= 1;
  }
}

// The scheduler loop.  S is the arithmetic of the trailing updates and
// recompressions (double: FP64 path; float: mixed path); the two
// instantiations live in separate translation units.
template <class S>
__global__ void __launch_bounds__(BLR_NT, 1) k_factor(SchedParams P) {
  extern __shared__ double smem[];
  __shared__ int task_sh;
  Ctx c;
  c.s = sm_carve(smem);
  c.status = P.status;
  DagShape d{P.p, P.q, P.off_larfb, P.off_tsqrt, P.off_tpmqrt};
  TaskEnv env{&P, P.scratch + (size_t)blockIdx.x * P.slab, 0, false, nullptr, nullptr, &d, -1, nullptr, 0};
  const SchedParams* Pm = &P;       // the parameters of the current task's matrix
  constexpr bool kTensor = std::is_same<S, float>::value;
  static_assert(BLR_SMEM_BYTES >= TC_STAGE_BYTES && TC_STAGE_BYTES >= 3 * 128 * 128 * 4, "staging area");
  __shared__ uint64_t tc_bars[2];
  __shared__ uint32_t tc_phase[2];
  __shared__ uint32_t tc_tmem;
  __shared__ uint64_t tq_full[2], tq_empty[2];
  __shared__ uint32_t tq_ph[4];
  __shared__ int tc_unsafe;
  TcCtx tcx;
  TcBulk tq{tq_full, tq_empty, tq_ph};
  if (kTensor) {
    // the mixed path's tensor-core state: all 512 TMEM columns (one CTA per
    // SM), two mbarriers for the double-buffered operand staging
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
    tcx.tmem = tc_tmem;
    tcx.bar = tc_bars;
    tcx.phase = tc_phase;
    tcx.buf = reinterpret_cast<float*>(smem);
    tcx.bcap = 256;
    tcx.status = P.status;
    tcx.limit_ns = (unsigned long long)P.watchdog_ns;
    tcx.unsafe = &tc_unsafe;
    env.tc = &tcx;
    env.tq = &tq;
  }
  while (true) {
    if (threadIdx.x == 0) task_sh = q_pop(P);
    __syncthreads();
    const int task = task_sh;
    __syncthreads();
    if (task < 0) break;
    // a batch (several matrices in one launch): find the task's matrix
    if (P.nmat > 1) {
      int lo = 0, hi = P.nmat - 1;
      while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(P.mat_base + mid) <= task) lo = mid;
        else hi = mid - 1;
      }
      Pm = P.mats + lo;   // the search of dag_find_matrix (blr_dag.h), checked on the host by blr_batch_selfcheck
      d = DagShape{Pm->p, Pm->q, Pm->off_larfb, Pm->off_tsqrt, Pm->off_tpmqrt};
      env.P = Pm;
    }
    const int local = task - Pm->task_base;
    int i, j, k;
    const int type = dag_decode(d, local, &i, &j, &k);
    const unsigned long long t_start = gtimer();
    c.fma = 0.0;
    env.used = 0;
    env.overflow = false;
    env.skip_succ = -1;
    env.prep_slot = nullptr;
    // operand kinds of an update, for the statistics: 4 (Y dense) + 2 (R dense) + (A dense)
    int variant = 0;
    if (type == TASK_TPMQRT && threadIdx.x == 0)
      variant = (ld_rank(rank_ptr(*Pm, i, k)) < 0) * 4 + (ld_rank(rank_ptr(*Pm, k, j)) < 0) * 2 +
                (ld_rank(rank_ptr(*Pm, i, j)) < 0);
    switch (type) {
      case TASK_GEQRT: task_geqrt<S>(env, k, c); break;
      case TASK_LARFB: task_larfb<S>(env, k, j, c); break;
      case TASK_TSQRT: task_tsqrt<S>(env, i, k, c); break;
      case TASK_TPMQRT: task_tpmqrt<S>(env, i, j, k, c); break;
      default:
        if (threadIdx.x == 0) atomicOr(P.status, ST_BADTASK);
        break;
    }
    if (env.overflow && threadIdx.x == 0) atomicOr(P.status, ST_RANK);
    if (threadIdx.x == 0) atomicMax(P.slab_peak, (unsigned long long)env.peak);
    __threadfence();
    __syncthreads();
    // an update has finished with its reflector block's prepared operands
    // (every read of them completed inside the body): return the slot once
    if (kTensor && type == TASK_TPMQRT && threadIdx.x == 0 && Pm->prep) {
      const int slot = __ldcg(Pm->prep_slot_of + prep_block(*Pm, i, k));
      if (slot >= 0) atomicSub(Pm->prep_ref + slot, 1);
    }
    if (threadIdx.x == 0 && type >= 0) {
      const unsigned long long t_end = gtimer();
      if (P.trace) {
        const unsigned slot = atomicAdd(P.trace_n, 1u);
        if (slot < (unsigned)P.trace_cap) {
          unsigned smid;
          asm volatile("mov.u32 %0, %%smid;" : "=r"(smid));
          blr_trace_event ev;
          ev.type = type;
          ev.i = i;
          ev.j = j;
          ev.k = k;
          ev.matrix = Pm->mat_index;
          ev.cta = (int)blockIdx.x;
          ev.sm = (int)smid;
          ev.reserved = 0;
          ev.t_start_ns = (long long)t_start;
          ev.t_end_ns = (long long)t_end;
          P.trace[slot] = ev;
        }
      }
      // the test hook withholds every release of one task: the DAG stalls
      // and the watchdog ends the launch
      if (task != P.withhold) {
        dag_for_each_successor(d, type, i, j, k, [&](int sid) {
          if (sid != env.skip_succ) release_task(*Pm, d, sid);
        });
      }
      const unsigned long long dt = t_end - t_start;
      atomicAdd(P.flops + type, 2.0 * c.fma);
      atomicAdd(P.ntask + type, 1ull);
      atomicAdd(P.tns + type, dt);
      if (type == TASK_TPMQRT) {
        atomicAdd(P.nvar + variant, 1ull);
        atomicAdd(P.tvar + variant, dt);
        atomicAdd(P.fvar + variant, 2.0 * c.fma);
      }
      atomicExch(P.progress_ns, gtimer());
      __threadfence();
      atomicAdd(P.done, 1);
    }
  }
  if (kTensor) {
    tc_fence_before();
    __syncthreads();
    // an MMA or copy that could not be waited for may still use TMEM: keep it
    // (the status already reports the timeout)
    if (threadIdx.x < 32 && !tc_unsafe) tmem_dealloc(tc_tmem, 512);
  }
}

}  // namespace
