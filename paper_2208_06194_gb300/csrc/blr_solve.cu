// Uses of the factor: Q^T B and Q B (Algorithm 5, reflectors applied exactly
// in factorization order or its reverse), R X, R^{-1} C, R^{-T} C, A~ X,
// least squares x = R^{-1} (Q^T B)(1:n) with optional refinement (QR for
// least squares, Section 1) and its adjoint.  Every kernel gives each CTA a
// group of right-hand-side columns; the reflector sequence is applied in
// order inside the CTA.
#include <algorithm>
#include <mutex>
#include <cstdio>
#include <vector>
#include "blr_device.cuh"

namespace {

constexpr int kColsPerCta = 8;

struct FactorView {
  int p, q, b, cap;
  const double* tiles;
  const int* rank;
  const double* t;
  const long long* toff;   // device, per k
  int* status;
  double* scratch;
  size_t slab;
};

__device__ __forceinline__ const double* ftile(const FactorView& F, int i, int j) {
  return F.tiles + ((size_t)j * F.p + i) * (size_t)F.b * F.b;
}
__device__ __forceinline__ const double* ft(const FactorView& F, int i, int k) {
  return F.t + (size_t)(F.toff[k] + (i - k)) * BLR_NB * F.b;
}

// [Ck; Ci] <- Q_ik^T [Ck; Ci] (trans) or Q_ik [Ck; Ci]; Ck, Ci are b x nc, ld ldc.
__device__ void apply_ts_tile(const FactorView& F, int i, int k, double* Ck, double* Ci, long long ldc,
                              int nc, bool trans, double* scr, Ctx& c) {
  const int b = F.b;
  const int r = __ldcg(F.rank + (size_t)k * F.p + i);
  const double* Y = ftile(F, i, k);
  const double* T = ft(F, i, k);
  if (r == 0) return;
  if (r < 0) {
    apply_ts_reflector<double>(colmajor(const_cast<double*>(Y), b), b, b, T, Ck, ldc, colmajor(Ci, (int)ldc), nc,
                       trans, c);
    return;
  }
  double* Pm = scr;
  double* P0 = scr + (size_t)r * nc;
  gemm(r, nc, b, 1.0, Y, b, true, Ci, ldc, false, 0.0, Pm, r, c);
  copy_mat(P0, r, Pm, r, r, nc);
  __syncthreads();
  apply_ts_reflector<double>(rowmajor(const_cast<double*>(Y) + (size_t)b * F.cap, b), r, b, T, Ck, ldc,
                     colmajor(Pm, r), nc, trans, c);
  for (int e = threadIdx.x; e < r * nc; e += BLR_NT) Pm[e] -= P0[e];
  __syncthreads();
  gemm(b, nc, r, 1.0, Y, b, false, Pm, r, false, 1.0, Ci, ldc, c);
}

__global__ void __launch_bounds__(BLR_NT, 1) k_apply_q(FactorView F, double* B, long long ldb, int nrhs,
                                                        int trans, int cpc) {
  extern __shared__ double smem[];
  Ctx c;
  c.s = sm_carve(smem);
  c.status = F.status;
  c.fma = 0.0;
  const int c0 = blockIdx.x * cpc;
  const int nc = min(cpc, nrhs - c0);
  if (nc <= 0) return;
  double* Bc = B + (size_t)c0 * ldb;
  double* scr = F.scratch + (size_t)blockIdx.x * F.slab;
  const int b = F.b;
  if (trans) {
    for (int k = 0; k < F.q; k++) {
      apply_q<double>(ftile(F, k, k), b, b, b, ft(F, k, k), Bc + (size_t)k * b, ldb, nc, true, c);
      for (int i = k + 1; i < F.p; i++)
        apply_ts_tile(F, i, k, Bc + (size_t)k * b, Bc + (size_t)i * b, ldb, nc, true, scr, c);
    }
  } else {
    for (int k = F.q - 1; k >= 0; k--) {
      for (int i = F.p - 1; i > k; i--)
        apply_ts_tile(F, i, k, Bc + (size_t)k * b, Bc + (size_t)i * b, ldb, nc, false, scr, c);
      apply_q<double>(ftile(F, k, k), b, b, b, ft(F, k, k), Bc + (size_t)k * b, ldb, nc, false, c);
    }
  }
}

// ---------------------------------------------------------------------------
// Q^T B and Q B as a pipeline over the 32-reflector blocks of each update QR.
// k_apply_q gives one CTA a group of columns and walks every reflector in
// order, so a few right-hand sides use a few SMs.  Here the S = b/32
// reflector blocks of each TSQRT(i,k) are split over S CTAs: CTA s applies
// block s of every TSQRT, which touches rows [32 s, 32 s + 32) of B_k and
// all of B_i.  Rows of B_k stay with one CTA; the order of the steps on each
// B_i is kept by a counter per (column group, i) that counts the steps done
// on it as the lower block (the order of Algorithm 5: column k ascending,
// then i, then block s; reversed for Q B), and a flag per k marks the
// diagonal block's reflectors (GEQRT(k)) as applied.  A step waits until its
// B_i counter reaches the number of steps on B_i that precede it, so the
// CTAs run as a wavefront down the columns with up to S steps in flight.
// Each element sees exactly the arithmetic of k_apply_q.  A low-rank
// reflector block acts on P = U_ik^T B_i (Eqs. 19-21): its first step forms
// P and P0 = P in a buffer per (group, i), the others update P, the last
// adds U (P - P0) to B_i.  Waits are bounded (the status gets ST_TIMEOUT).
// ---------------------------------------------------------------------------
struct WaveState {
  int* prog;       // [groups][p]: steps done on B_i as the lower block
  int* geq;        // [groups][q]: 1 once GEQRT(k)'s reflectors are applied to B_k
  double* pbuf;    // [groups][p][2 cap cpc]: P and P0 of a low-rank step
  unsigned long long limit_ns;
};

__device__ __forceinline__ unsigned long long wave_timer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Thread 0 waits until *flag >= target; every thread returns whether it got
// there (false after the limit or once another CTA has timed out).
__device__ bool wave_wait(const int* flag, int target, const WaveState& W, int* status) {
  __shared__ int ok_sh;
  if (threadIdx.x == 0) {
    int ok = 1;
    const unsigned long long t0 = wave_timer();
    while (*(volatile const int*)flag < target) {
      if ((*(volatile int*)status & ST_TIMEOUT) || wave_timer() - t0 > W.limit_ns) {
        atomicOr(status, ST_TIMEOUT);
        ok = 0;
        break;
      }
      __nanosleep(200);
    }
    __threadfence();
    ok_sh = ok;
  }
  __syncthreads();
  return ok_sh != 0;
}

// Makes this CTA's global writes visible, then sets *flag = value.
__device__ void wave_publish(int* flag, int value) {
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) atomicExch(flag, value);
}

// Step (i, k, s): reflector block s of TSQRT(i,k) on [B_k rows 32 s..; B_i].
__device__ void wave_step(const FactorView& F, int i, int k, int s, double* Bk, double* Bi, long long ldb, int nc,
                          bool trans, double* pb, int cpc, Ctx& c) {
  const int b = F.b, S = b / BLR_NB;
  const int r = __ldcg(F.rank + (size_t)k * F.p + i);
  if (r == 0) return;
  const double* Y = ftile(F, i, k);
  const double* T = ft(F, i, k);
  const int c0 = s * BLR_NB;
  if (r < 0) {
    const int ldy = stage_reflector_panel<double>(colmajor(const_cast<double*>(Y), b), b, c0, BLR_NB, T, c);
    apply_refl_ts(Bk + c0, ldb, colmajor(Bi, (int)ldb), b, nc, (const double*)as<double>(c.s.pnl), ldy, BLR_NB,
                  (const double*)as<double>(c.s.t), trans, c);
    return;
  }
  double* Pm = pb;
  double* P0 = pb + (size_t)F.cap * cpc;
  const bool first = trans ? s == 0 : s == S - 1, last = trans ? s == S - 1 : s == 0;
  if (first) {
    gemm(r, nc, b, 1.0, Y, b, true, Bi, ldb, false, 0.0, Pm, r, c);
    __syncthreads();
    copy_mat(P0, r, Pm, r, r, nc);
  }
  const int ldy = stage_reflector_panel<double>(rowmajor(const_cast<double*>(Y) + (size_t)b * F.cap, b), r, c0,
                                                BLR_NB, T, c);
  apply_refl_ts(Bk + c0, ldb, colmajor(Pm, r), r, nc, (const double*)as<double>(c.s.pnl), ldy, BLR_NB,
                (const double*)as<double>(c.s.t), trans, c);
  if (last) {
    __syncthreads();
    for (int e = threadIdx.x; e < r * nc; e += BLR_NT) Pm[e] = ldg(Pm + e) - ldg(P0 + e);
    __syncthreads();
    gemm(b, nc, r, 1.0, Y, b, false, Pm, r, false, 1.0, Bi, ldb, c);
  }
}

__global__ void __launch_bounds__(BLR_NT, 1) k_apply_q_wave(FactorView F, WaveState W, double* B, long long ldb,
                                                             int nrhs, int trans, int cpc, int g0) {
  extern __shared__ double smem[];
  Ctx c;
  c.s = sm_carve(smem);
  c.status = F.status;
  c.fma = 0.0;
  const int S = F.b / BLR_NB;
  const int g = g0 + blockIdx.x / S, s = blockIdx.x % S;
  const int col0 = g * cpc;
  const int nc = min(cpc, nrhs - col0);
  if (nc <= 0) return;
  double* Bc = B + (size_t)col0 * ldb;
  int* prog = W.prog + (size_t)g * F.p;
  int* geq = W.geq + (size_t)g * F.q;
  double* pbuf = W.pbuf + (size_t)g * F.p * 2 * F.cap * cpc;
  const size_t pstride = (size_t)2 * F.cap * cpc;
  const int b = F.b, p = F.p, q = F.q;
  if (trans) {
    for (int k = 0; k < q; k++) {
      double* Bk = Bc + (size_t)k * b;
      if (s == 0) {
        if (!wave_wait(prog + k, S * k, W, F.status)) return;
        apply_q<double>(ftile(F, k, k), b, b, b, ft(F, k, k), Bk, ldb, nc, true, c);
        wave_publish(geq + k, 1);
      } else if (!wave_wait(geq + k, 1, W, F.status)) {
        return;
      }
      for (int i = k + 1; i < p; i++) {
        if (!wave_wait(prog + i, S * k + s, W, F.status)) return;
        wave_step(F, i, k, s, Bk, Bc + (size_t)i * b, ldb, nc, true, pbuf + i * pstride, cpc, c);
        wave_publish(prog + i, S * k + s + 1);
      }
    }
  } else {
    for (int k = q - 1; k >= 0; k--) {
      double* Bk = Bc + (size_t)k * b;
      for (int i = p - 1; i > k; i--) {
        // steps on B_i before this one: blocks S-1 .. s+1 of column k, and
        // every block of the columns k+1 .. min(i, q)-1 processed before it;
        // for i < q, GEQRT(i) (processed with column i) comes first too
        const int target = S * (min(i, q) - 1 - k) + (S - 1 - s);
        if (i < q && !wave_wait(geq + i, 1, W, F.status)) return;
        if (!wave_wait(prog + i, target, W, F.status)) return;
        wave_step(F, i, k, s, Bk, Bc + (size_t)i * b, ldb, nc, false, pbuf + i * pstride, cpc, c);
        wave_publish(prog + i, target + 1);
      }
      if (s == 0) {
        // block 0 is the last of every step on B_k's rows in this column:
        // after CTA 0's own step (k+1, k, 0) every other CTA's rows of B_k
        // are final (they precede it on B_{k+1}'s counter)
        apply_q<double>(ftile(F, k, k), b, b, b, ft(F, k, k), Bk, ldb, nc, false, c);
        wave_publish(geq + k, 1);
      }
    }
  }
}

// X = R^{-1} C (n x nrhs), back substitution by block rows.
__global__ void __launch_bounds__(BLR_NT, 1) k_solve_r(FactorView F, const double* C, long long ldc,
                                                        double* X, long long ldx, int nrhs, int cpc) {
  extern __shared__ double smem[];
  Ctx c;
  c.s = sm_carve(smem);
  c.status = F.status;
  c.fma = 0.0;
  const int c0 = blockIdx.x * cpc;
  const int nc = min(cpc, nrhs - c0);
  if (nc <= 0) return;
  const int b = F.b;
  double* scr = F.scratch + (size_t)blockIdx.x * F.slab;
  double* rhs = scr;                              // b x nc
  double* tmp = scr + (size_t)b * cpc;            // cap x nc
  double* xs = c.s.vec;                           // nc values of the current row
  for (int k = F.q - 1; k >= 0; k--) {
    copy_mat(rhs, b, C + (size_t)k * b + (size_t)c0 * ldc, ldc, b, nc);
    __syncthreads();
    for (int j = k + 1; j < F.q; j++) {
      const double* Rkj = ftile(F, k, j);
      const int r = __ldcg(F.rank + (size_t)j * F.p + k);
      const double* Xj = X + (size_t)j * b + (size_t)c0 * ldx;
      if (r < 0) {
        gemm(b, nc, b, -1.0, Rkj, b, false, Xj, ldx, false, 1.0, rhs, b, c);
      } else if (r > 0) {
        gemm(r, nc, b, 1.0, Rkj + (size_t)b * F.cap, b, true, Xj, ldx, false, 0.0, tmp, r, c);
        gemm(b, nc, r, -1.0, Rkj, b, false, tmp, r, false, 1.0, rhs, b, c);
      }
    }
    const double* Rkk = ftile(F, k, k);
    for (int a = b - 1; a >= 0; a--) {
      if (threadIdx.x < nc) {
        const double d = __ldcg(Rkk + a + (size_t)a * b);
        if (d == 0.0 || !isfinite(d)) atomicOr(F.status, ST_NUMERIC);
        xs[threadIdx.x] = rhs[a + (size_t)threadIdx.x * b] / d;
      }
      __syncthreads();
      for (int e = threadIdx.x; e < a * nc; e += BLR_NT) {
        int row = e % a, col = e / a;
        rhs[row + (size_t)col * b] -= __ldcg(Rkk + row + (size_t)a * b) * xs[col];
      }
      if (threadIdx.x < nc) rhs[a + (size_t)threadIdx.x * b] = xs[threadIdx.x];
      __syncthreads();
    }
    copy_mat(X + (size_t)k * b + (size_t)c0 * ldx, ldx, rhs, b, b, nc);
    __syncthreads();
  }
}

// X = R^{-T} C (n x nrhs), forward substitution by block columns of R:
// (R^T)_{kj} = R_jk^T for j <= k, so X_k = R_kk^{-T} (C_k - sum_{j<k} R_jk^T X_j).
__global__ void __launch_bounds__(BLR_NT, 1) k_solve_rt(FactorView F, const double* C, long long ldc,
                                                         double* X, long long ldx, int nrhs, int cpc) {
  extern __shared__ double smem[];
  Ctx c;
  c.s = sm_carve(smem);
  c.status = F.status;
  c.fma = 0.0;
  const int c0 = blockIdx.x * cpc;
  const int nc = min(cpc, nrhs - c0);
  if (nc <= 0) return;
  const int b = F.b;
  double* scr = F.scratch + (size_t)blockIdx.x * F.slab;
  double* rhs = scr;                              // b x nc
  double* tmp = scr + (size_t)b * cpc;            // cap x nc
  double* xs = c.s.vec;
  for (int k = 0; k < F.q; k++) {
    copy_mat(rhs, b, C + (size_t)k * b + (size_t)c0 * ldc, ldc, b, nc);
    __syncthreads();
    for (int j = 0; j < k; j++) {
      const double* Rjk = ftile(F, j, k);
      const int r = __ldcg(F.rank + (size_t)k * F.p + j);
      const double* Xj = X + (size_t)j * b + (size_t)c0 * ldx;
      if (r < 0) {
        gemm(b, nc, b, -1.0, Rjk, b, true, Xj, ldx, false, 1.0, rhs, b, c);
      } else if (r > 0) {
        // (U V^T)^T X_j = V (U^T X_j)
        gemm(r, nc, b, 1.0, Rjk, b, true, Xj, ldx, false, 0.0, tmp, r, c);
        gemm(b, nc, r, -1.0, Rjk + (size_t)b * F.cap, b, false, tmp, r, false, 1.0, rhs, b, c);
      }
    }
    const double* Rkk = ftile(F, k, k);
    for (int a = 0; a < b; a++) {
      if (threadIdx.x < nc) {
        const double d = __ldcg(Rkk + a + (size_t)a * b);
        if (d == 0.0 || !isfinite(d)) atomicOr(F.status, ST_NUMERIC);
        xs[threadIdx.x] = rhs[a + (size_t)threadIdx.x * b] / d;
      }
      __syncthreads();
      const int rest = b - a - 1;
      for (int e = threadIdx.x; e < rest * nc; e += BLR_NT) {
        const int row = a + 1 + e % rest, col = e / rest;
        rhs[row + (size_t)col * b] -= __ldcg(Rkk + a + (size_t)row * b) * xs[col];
      }
      if (threadIdx.x < nc) rhs[a + (size_t)threadIdx.x * b] = xs[threadIdx.x];
      __syncthreads();
    }
    copy_mat(X + (size_t)k * b + (size_t)c0 * ldx, ldx, rhs, b, b, nc);
    __syncthreads();
  }
}

// Gradient of a loss through x = argmin ||A~ x - B|| with respect to the
// storage of tile (i,j) of A~ (same layout as the tiles): with Abar =
// r z^T - (A~ z) x^T (r = B - A~ x, z = (A~^T A~)^{-1} xbar), a dense tile
// gets Abar_ij, a low-rank tile U V^T gets Ubar = Abar_ij V in its U slot and
// Vbar = Abar_ij^T U in its V slot; the unused part of the tile is zero.
// Each CTA handles tiles blockIdx.x, blockIdx.x + gridDim.x, ...
__device__ void lstsq_grad_tile(const FactorView& A, int i, int j, const double* rres, long long ldr,
                                const double* az, long long ldaz, const double* z, long long ldz, const double* x,
                                long long ldxx, int nrhs, double* grad, double* scr, Ctx& c) {
  const int b = A.b, cap = A.cap;
  const double* T = ftile(A, i, j);
  double* G = grad + ((size_t)j * A.p + i) * (size_t)b * b;
  const int r = __ldcg(A.rank + (size_t)j * A.p + i);
  const double* ri = rres + (size_t)i * b;
  const double* ai = az + (size_t)i * b;
  const double* zj = z + (size_t)j * b;
  const double* xj = x + (size_t)j * b;
  zero_mat(G, b, b, b);
  __syncthreads();
  if (r < 0) {
    gemm(b, b, nrhs, 1.0, ri, ldr, false, zj, ldz, true, 0.0, G, b, c);
    gemm(b, b, nrhs, -1.0, ai, ldaz, false, xj, ldxx, true, 1.0, G, b, c);
    return;
  }
  if (r == 0) return;
  double* s1 = scr;                         // V^T z_j  (r x nrhs)
  double* s2 = s1 + (size_t)cap * nrhs;     // V^T x_j
  double* t1 = s2 + (size_t)cap * nrhs;     // U^T r_i
  double* t2 = t1 + (size_t)cap * nrhs;     // U^T (A z)_i
  const double* U = T;
  const double* V = T + (size_t)b * cap;
  gemm(r, nrhs, b, 1.0, V, b, true, zj, ldz, false, 0.0, s1, r, c);
  gemm(r, nrhs, b, 1.0, V, b, true, xj, ldxx, false, 0.0, s2, r, c);
  gemm(r, nrhs, b, 1.0, U, b, true, ri, ldr, false, 0.0, t1, r, c);
  gemm(r, nrhs, b, 1.0, U, b, true, ai, ldaz, false, 0.0, t2, r, c);
  // Ubar = r_i s1^T - (A z)_i s2^T ; Vbar = z_j t1^T - x_j t2^T
  gemm(b, r, nrhs, 1.0, ri, ldr, false, s1, r, true, 0.0, G, b, c);
  gemm(b, r, nrhs, -1.0, ai, ldaz, false, s2, r, true, 1.0, G, b, c);
  gemm(b, r, nrhs, 1.0, zj, ldz, false, t1, r, true, 0.0, G + (size_t)b * cap, b, c);
  gemm(b, r, nrhs, -1.0, xj, ldxx, false, t2, r, true, 1.0, G + (size_t)b * cap, b, c);
}

__global__ void __launch_bounds__(BLR_NT, 1) k_lstsq_grad(FactorView A, const double* rres, long long ldr,
                                                           const double* az, long long ldaz, const double* z,
                                                           long long ldz, const double* x, long long ldxx, int nrhs,
                                                           double* grad) {
  extern __shared__ double smem[];
  Ctx c;
  c.s = sm_carve(smem);
  c.status = A.status;
  c.fma = 0.0;
  double* scr = A.scratch + (size_t)blockIdx.x * A.slab;
  for (int t = blockIdx.x; t < A.p * A.q; t += gridDim.x) {
    __syncthreads();
    lstsq_grad_tile(A, t % A.p, t / A.p, rres, ldr, az, ldaz, z, ldz, x, ldxx, nrhs, grad, scr, c);
  }
}

// Y = A~ X (mode 0, BLR matrix, p block rows) or Y = R X (mode 1, factor).
__global__ void __launch_bounds__(BLR_NT, 1) k_matmul(FactorView F, int mode, const double* X, long long ldx,
                                                       double* Y, long long ldy, int nrhs) {
  extern __shared__ double smem[];
  Ctx c;
  c.s = sm_carve(smem);
  c.status = F.status;
  c.fma = 0.0;
  const int rows = (mode == 0) ? F.p : F.q;
  const int i = blockIdx.x % rows;
  const int cg = blockIdx.x / rows;
  const int c0 = cg * kColsPerCta;
  const int nc = min(kColsPerCta, nrhs - c0);
  if (nc <= 0) return;
  const int b = F.b;
  double* scr = F.scratch + (size_t)blockIdx.x * F.slab;
  double* acc = scr;                        // b x nc
  double* tmp = scr + (size_t)b * kColsPerCta;
  double* rkk = tmp + (size_t)b * kColsPerCta;   // b x b (mode 1)
  zero_mat(acc, b, b, nc);
  __syncthreads();
  const int j0 = (mode == 0) ? 0 : i;
  for (int j = j0; j < F.q; j++) {
    const double* A = ftile(F, i, j);
    const int r = __ldcg(F.rank + (size_t)j * F.p + i);
    const double* Xj = X + (size_t)j * b + (size_t)c0 * ldx;
    if (mode == 1 && j == i) {
      for (int e = threadIdx.x; e < b * b; e += BLR_NT) {
        int a = e % b, l = e / b;
        rkk[e] = (a <= l) ? __ldcg(A + e) : 0.0;
      }
      __syncthreads();
      gemm(b, nc, b, 1.0, rkk, b, false, Xj, ldx, false, 1.0, acc, b, c);
    } else if (r < 0) {
      gemm(b, nc, b, 1.0, A, b, false, Xj, ldx, false, 1.0, acc, b, c);
    } else if (r > 0) {
      gemm(r, nc, b, 1.0, A + (size_t)b * F.cap, b, true, Xj, ldx, false, 0.0, tmp, r, c);
      gemm(b, nc, r, 1.0, A, b, false, tmp, r, false, 1.0, acc, b, c);
    }
  }
  copy_mat(Y + (size_t)i * b + (size_t)c0 * ldy, ldy, acc, b, b, nc);
}

struct Scratch {
  double* scratch = nullptr;
  long long* toff = nullptr;
  int* status = nullptr;
  int* flags = nullptr;
  ~Scratch() {
    if (scratch) cudaFree(scratch);
    if (toff) cudaFree(toff);
    if (status) cudaFree(status);
    if (flags) cudaFree(flags);
  }
};

int make_view(const blr_matrix& a, const double* t, int q_for_toff, FactorView* F, Scratch* S,
              int nctas, size_t slab, cudaStream_t st) {
  F->p = a.p; F->q = a.q; F->b = a.b; F->cap = a.cap;
  F->tiles = a.tiles; F->rank = a.rank; F->t = t;
  F->slab = slab;
  int rc = blr_cuda_check(cudaMalloc(&S->scratch, sizeof(double) * slab * nctas), "solve scratch");
  if (rc) return rc;
  rc = blr_cuda_check(cudaMalloc(&S->status, sizeof(int)), "solve status");
  if (rc) return rc;
  rc = blr_cuda_check(cudaMemsetAsync(S->status, 0, sizeof(int), st), "memset");
  if (rc) return rc;
  F->scratch = S->scratch;
  F->status = S->status;
  F->toff = nullptr;
  if (q_for_toff > 0) {
    std::vector<long long> toff(q_for_toff);
    long long acc = 0;
    for (int k = 0; k < q_for_toff; k++) { toff[k] = acc; acc += a.p - k; }
    rc = blr_cuda_check(cudaMalloc(&S->toff, sizeof(long long) * q_for_toff), "toff");
    if (rc) return rc;
    rc = blr_cuda_check(cudaMemcpy(S->toff, toff.data(), sizeof(long long) * q_for_toff, cudaMemcpyHostToDevice), "toff");
    if (rc) return rc;
    F->toff = S->toff;
  }
  return BLR_OK;
}

int finish(const FactorView& F, cudaStream_t st, const char* what) {
  int rc = blr_cuda_check(cudaStreamSynchronize(st), what);
  if (rc) return rc;
  int s = 0;
  rc = blr_cuda_check(cudaMemcpy(&s, F.status, sizeof(int), cudaMemcpyDeviceToHost), what);
  if (rc) return rc;
  if (s & ST_NUMERIC) {
    blr_set_error("%s: zero or non-finite diagonal entry of R", what);
    return BLR_ERR_NUMERIC;
  }
  if (s & ST_TIMEOUT) {
    blr_set_error("%s: a device wait between CTAs ran out", what);
    return BLR_ERR_TIMEOUT;
  }
  return BLR_OK;
}

// The dynamic shared-memory opt-in is a per-device attribute of each kernel:
// set it once for every device that runs these kernels (with that device
// current), under a lock.
std::mutex g_smem_mu;
bool g_smem_done[64];

int set_smem() {
  int dev = 0;
  int rc = blr_cuda_check(cudaGetDevice(&dev), "cudaGetDevice");
  if (rc) return rc;
  if (dev < 0 || dev >= 64) {
    blr_set_error("device ordinal %d out of range", dev);
    return BLR_ERR_INVALID;
  }
  std::lock_guard<std::mutex> lock(g_smem_mu);
  if (g_smem_done[dev]) return BLR_OK;
  rc = blr_cuda_check(cudaFuncSetAttribute(k_apply_q, cudaFuncAttributeMaxDynamicSharedMemorySize, BLR_SMEM_BYTES), "smem");
  if (!rc) rc = blr_cuda_check(cudaFuncSetAttribute(k_apply_q_wave, cudaFuncAttributeMaxDynamicSharedMemorySize, BLR_SMEM_BYTES), "smem");
  if (!rc) rc = blr_cuda_check(cudaFuncSetAttribute(k_solve_r, cudaFuncAttributeMaxDynamicSharedMemorySize, BLR_SMEM_BYTES), "smem");
  if (!rc) rc = blr_cuda_check(cudaFuncSetAttribute(k_matmul, cudaFuncAttributeMaxDynamicSharedMemorySize, BLR_SMEM_BYTES), "smem");
  if (!rc) rc = blr_cuda_check(cudaFuncSetAttribute(k_solve_rt, cudaFuncAttributeMaxDynamicSharedMemorySize, BLR_SMEM_BYTES), "smem");
  if (!rc) rc = blr_cuda_check(cudaFuncSetAttribute(k_lstsq_grad, cudaFuncAttributeMaxDynamicSharedMemorySize, BLR_SMEM_BYTES), "smem");
  if (!rc) g_smem_done[dev] = true;
  return rc;
}

// Right-hand-side columns per CTA (kColsPerCta) of the kernels that give
// each CTA its own columns (k_apply_q of the no-allocation entry, the R
// solves).  Each CTA streams every block of the factor for its columns, so
// the traffic grows with the number of CTAs: measured for k_apply_q at
// 65536 x 32768 with 16 right-hand sides, 8 columns per CTA (2 CTAs) took
// 6 s per Q application, 1 column per CTA (16 CTAs) 23 s.
int cols_per_cta(int) { return kColsPerCta; }

// Right-hand-side columns per group of the pipelined Q application: each
// group's b/32 CTAs read every reflector block once.
constexpr int kWaveCols = 16;
// Bound of each wait between the pipeline's CTAs.
constexpr unsigned long long kWaveLimitNs = 20ull * 1000 * 1000 * 1000;

int apply_q_launch(const blr_factor* f, double* B, int ldb, int nrhs, int trans, cudaStream_t st) {
  const blr_matrix& a = f->a;
  const int S = a.b / BLR_NB, cpc = kWaveCols;
  const int groups = (nrhs + cpc - 1) / cpc;
  int dev = 0, nsm = 0;
  int rc = blr_cuda_check(cudaGetDevice(&dev), "cudaGetDevice");
  if (!rc) rc = blr_cuda_check(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev), "SM count");
  if (rc) return rc;
  // the CTAs of a group wait on one another, so every CTA of a launch must
  // be resident at once: one per SM (the shared-memory footprint), so at
  // most nsm / S groups per launch, the rest in further launches
  const int per_launch = std::max(1, nsm / S);
  if (S > nsm) {
    blr_set_error("blr_apply_qt: %d reflector blocks per tile exceed the %d SMs", S, nsm);
    return BLR_ERR_INVALID;
  }
  FactorView F{};
  Scratch Sc;
  rc = set_smem();
  if (!rc) rc = make_view(a, f->t, a.q, &F, &Sc, 1, (size_t)groups * a.p * 2 * a.cap * cpc + 64, st);
  if (rc) return rc;
  const size_t nflags = (size_t)groups * (a.p + a.q);
  rc = blr_cuda_check(cudaMalloc(&Sc.flags, sizeof(int) * nflags), "apply flags");
  if (!rc) rc = blr_cuda_check(cudaMemsetAsync(Sc.flags, 0, sizeof(int) * nflags, st), "memset");
  if (rc) return rc;
  WaveState W{Sc.flags, Sc.flags + (size_t)groups * a.p, F.scratch, kWaveLimitNs};
  for (int g0 = 0; g0 < groups; g0 += per_launch) {
    const int n = std::min(per_launch, groups - g0);
    k_apply_q_wave<<<n * S, BLR_NT, BLR_SMEM_BYTES, st>>>(F, W, B, ldb, nrhs, trans, cpc, g0);
    rc = blr_cuda_check(cudaGetLastError(), "launch k_apply_q_wave");
    if (rc) return rc;
  }
  return finish(F, st, "blr_apply_qt");
}

int solve_r_launch(const blr_factor* f, const double* C, int ldc, double* X, int ldx, int nrhs, cudaStream_t st) {
  FactorView F{};
  Scratch S;
  const int cpc = cols_per_cta(nrhs);
  const int nct = (nrhs + cpc - 1) / cpc;
  int rc = set_smem();
  if (!rc) rc = make_view(f->a, f->t, 0, &F, &S, nct, (size_t)(f->a.b + f->a.cap) * cpc + 64, st);
  if (rc) return rc;
  k_solve_r<<<nct, BLR_NT, BLR_SMEM_BYTES, st>>>(F, C, ldc, X, ldx, nrhs, cpc);
  rc = blr_cuda_check(cudaGetLastError(), "launch k_solve_r");
  if (rc) return rc;
  return finish(F, st, "blr_lstsq");
}

int solve_rt_launch(const blr_factor* f, const double* C, int ldc, double* X, int ldx, int nrhs, cudaStream_t st) {
  FactorView F{};
  Scratch S;
  const int cpc = cols_per_cta(nrhs);
  const int nct = (nrhs + cpc - 1) / cpc;
  int rc = set_smem();
  if (!rc) rc = make_view(f->a, f->t, 0, &F, &S, nct, (size_t)(f->a.b + f->a.cap) * cpc + 64, st);
  if (rc) return rc;
  k_solve_rt<<<nct, BLR_NT, BLR_SMEM_BYTES, st>>>(F, C, ldc, X, ldx, nrhs, cpc);
  rc = blr_cuda_check(cudaGetLastError(), "launch k_solve_rt");
  if (rc) return rc;
  return finish(F, st, "blr_solve_r");
}

int matmul_launch(const blr_matrix& a, int mode, const double* X, int ldx, double* Y, int ldy, int nrhs,
                  cudaStream_t st) {
  FactorView F{};
  Scratch S;
  const int ncg = (nrhs + kColsPerCta - 1) / kColsPerCta;
  const int rows = mode == 0 ? a.p : a.q;
  int rc = set_smem();
  if (!rc) rc = make_view(a, nullptr, 0, &F, &S, rows * ncg, (size_t)2 * a.b * kColsPerCta + (size_t)a.b * a.b + 64, st);
  if (rc) return rc;
  k_matmul<<<rows * ncg, BLR_NT, BLR_SMEM_BYTES, st>>>(F, mode, X, ldx, Y, ldy, nrhs);
  rc = blr_cuda_check(cudaGetLastError(), "launch k_matmul");
  if (rc) return rc;
  return finish(F, st, "blr_matmul");
}

__global__ void k_axpby(double* y, long long ldy, const double* x, long long ldx, int rows, int cols,
                        double alpha, double beta) {
  long long tot = (long long)rows * cols;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
    int r = (int)(e % rows), c = (int)(e / rows);
    y[r + c * ldy] = alpha * x[r + c * ldx] + beta * y[r + c * ldy];
  }
}

}  // namespace

extern "C" int blr_apply_qt(const blr_factor* f, double* b_dev, int ldb, int nrhs, int trans, void* stream) {
  if (!f || !b_dev) { blr_set_error("NULL argument"); return BLR_ERR_INVALID; }
  if (ldb < f->a.m || nrhs < 0) { blr_set_error("bad ldb or nrhs"); return BLR_ERR_INVALID; }
  if (nrhs == 0) return BLR_OK;
  return apply_q_launch(f, b_dev, ldb, nrhs, trans ? 0 : 1, (cudaStream_t)stream);
}

extern "C" int blr_apply_r(const blr_factor* f, const double* x_dev, int ldx, double* y_dev, int ldy, int nrhs,
                           void* stream) {
  if (!f || !x_dev || !y_dev) { blr_set_error("NULL argument"); return BLR_ERR_INVALID; }
  if (ldx < f->a.n || ldy < f->a.n || nrhs < 0) { blr_set_error("bad leading dimension"); return BLR_ERR_INVALID; }
  if (nrhs == 0) return BLR_OK;
  return matmul_launch(f->a, 1, x_dev, ldx, y_dev, ldy, nrhs, (cudaStream_t)stream);
}

extern "C" int blr_matmul(const blr_matrix* a, const double* x_dev, int ldx, double* y_dev, int ldy, int nrhs,
                          void* stream) {
  if (!a || !x_dev || !y_dev) { blr_set_error("NULL argument"); return BLR_ERR_INVALID; }
  if (ldx < a->n || ldy < a->m || nrhs < 0) { blr_set_error("bad leading dimension"); return BLR_ERR_INVALID; }
  if (nrhs == 0) return BLR_OK;
  return matmul_launch(*a, 0, x_dev, ldx, y_dev, ldy, nrhs, (cudaStream_t)stream);
}

extern "C" int blr_lstsq(const blr_factor* f, const blr_matrix* a_orig, const double* b_dev, int ldb,
                         double* x_dev, int ldx, int nrhs, int refine_steps, void* stream) {
  if (!f || !b_dev || !x_dev) { blr_set_error("NULL argument"); return BLR_ERR_INVALID; }
  const int m = f->a.m, n = f->a.n;
  if (ldb < m || ldx < n || nrhs < 0 || refine_steps < 0) { blr_set_error("bad leading dimension"); return BLR_ERR_INVALID; }
  if (refine_steps > 0 && (!a_orig || a_orig->m != m || a_orig->n != n || a_orig->b != f->a.b)) {
    blr_set_error("refinement needs the original BLR matrix of the same shape");
    return BLR_ERR_INVALID;
  }
  if (nrhs == 0) return BLR_OK;
  cudaStream_t st = (cudaStream_t)stream;
  double *cbuf = nullptr, *dx = nullptr;
  int rc = blr_cuda_check(cudaMalloc(&cbuf, sizeof(double) * (size_t)m * nrhs), "lstsq buffer");
  if (!rc) rc = blr_cuda_check(cudaMalloc(&dx, sizeof(double) * (size_t)n * nrhs), "lstsq buffer");
  if (!rc) rc = blr_cuda_check(cudaMemcpy2DAsync(cbuf, sizeof(double) * m, b_dev, sizeof(double) * ldb, sizeof(double) * m, nrhs, cudaMemcpyDeviceToDevice, st), "copy B");
  if (!rc) rc = apply_q_launch(f, cbuf, m, nrhs, 1, st);
  if (!rc) rc = solve_r_launch(f, cbuf, m, x_dev, ldx, nrhs, st);
  for (int it = 0; it < refine_steps && !rc; it++) {
    // r = B - A x
    rc = matmul_launch(*a_orig, 0, x_dev, ldx, cbuf, m, nrhs, st);
    if (!rc) {
      k_axpby<<<256, 256, 0, st>>>(cbuf, m, b_dev, ldb, m, nrhs, 1.0, -1.0);
      rc = blr_cuda_check(cudaGetLastError(), "axpby");
    }
    if (!rc) rc = apply_q_launch(f, cbuf, m, nrhs, 1, st);
    if (!rc) rc = solve_r_launch(f, cbuf, m, dx, n, nrhs, st);
    if (!rc) {
      k_axpby<<<256, 256, 0, st>>>(x_dev, ldx, dx, n, n, nrhs, 1.0, 1.0);
      rc = blr_cuda_check(cudaGetLastError(), "axpby");
    }
  }
  if (!rc) rc = blr_cuda_check(cudaStreamSynchronize(st), "blr_lstsq");
  if (cbuf) cudaFree(cbuf);
  if (dx) cudaFree(dx);
  return rc;
}


extern "C" int blr_solve_r(const blr_factor* f, const double* c_dev, int ldc, double* x_dev, int ldx, int nrhs,
                           int trans, void* stream) {
  if (!f || !c_dev || !x_dev) { blr_set_error("NULL argument"); return BLR_ERR_INVALID; }
  if (ldc < f->a.n || ldx < f->a.n || nrhs < 0) { blr_set_error("bad leading dimension"); return BLR_ERR_INVALID; }
  if (nrhs == 0) return BLR_OK;
  cudaStream_t st = (cudaStream_t)stream;
  return trans ? solve_rt_launch(f, c_dev, ldc, x_dev, ldx, nrhs, st) : solve_r_launch(f, c_dev, ldc, x_dev, ldx, nrhs, st);
}

extern "C" int blr_lstsq_backward(const blr_factor* f, const blr_matrix* a_orig, const double* b_dev, int ldb,
                                  const double* x_dev, int ldx, const double* xbar_dev, int ldxb, int nrhs,
                                  double* bbar_dev, int ldbb, double* grad_tiles_dev, void* stream) {
  if (!f || !a_orig || !b_dev || !x_dev || !xbar_dev || !bbar_dev || !grad_tiles_dev) {
    blr_set_error("NULL argument");
    return BLR_ERR_INVALID;
  }
  const int m = f->a.m, n = f->a.n;
  if (a_orig->m != m || a_orig->n != n || a_orig->b != f->a.b) {
    blr_set_error("the BLR matrix does not match the factor");
    return BLR_ERR_INVALID;
  }
  if (ldb < m || ldx < n || ldxb < n || ldbb < m || nrhs < 0) { blr_set_error("bad leading dimension"); return BLR_ERR_INVALID; }
  cudaStream_t st = (cudaStream_t)stream;
  const blr_matrix& A = *a_orig;
  if (nrhs == 0) {
    return blr_cuda_check(cudaMemsetAsync(grad_tiles_dev, 0, sizeof(double) * (size_t)A.p * A.q * A.b * A.b, st),
                          "clear gradient");
  }
  double *y = nullptr, *z = nullptr, *rr = nullptr;
  int rc = blr_cuda_check(cudaMalloc(&y, sizeof(double) * (size_t)n * nrhs), "backward buffer");
  if (!rc) rc = blr_cuda_check(cudaMalloc(&z, sizeof(double) * (size_t)n * nrhs), "backward buffer");
  if (!rc) rc = blr_cuda_check(cudaMalloc(&rr, sizeof(double) * (size_t)m * nrhs), "backward buffer");
  // z = (R^T R)^{-1} xbar = R^{-1} (R^{-T} xbar)
  if (!rc) rc = solve_rt_launch(f, xbar_dev, ldxb, y, n, nrhs, st);
  if (!rc) rc = solve_r_launch(f, y, n, z, n, nrhs, st);
  // Bbar = A~ z
  if (!rc) rc = matmul_launch(A, 0, z, n, bbar_dev, ldbb, nrhs, st);
  // r = B - A~ x
  if (!rc) rc = matmul_launch(A, 0, x_dev, ldx, rr, m, nrhs, st);
  if (!rc) {
    k_axpby<<<256, 256, 0, st>>>(rr, m, b_dev, ldb, m, nrhs, 1.0, -1.0);
    rc = blr_cuda_check(cudaGetLastError(), "axpby");
  }
  if (!rc) {
    FactorView F{};
    Scratch S;
    rc = set_smem();
    int nct = 2 * blr_num_sms();
    if (nct > A.p * A.q) nct = A.p * A.q;
    if (!rc) rc = make_view(A, nullptr, 0, &F, &S, nct, (size_t)4 * A.cap * nrhs + 64, st);
    if (!rc) {
      // (A~ z) is read back from bbar_dev
      k_lstsq_grad<<<nct, BLR_NT, BLR_SMEM_BYTES, st>>>(F, rr, m, bbar_dev, ldbb, z, n, x_dev, ldx, nrhs,
                                                       grad_tiles_dev);
      rc = blr_cuda_check(cudaGetLastError(), "launch k_lstsq_grad");
    }
    if (!rc) rc = finish(F, st, "blr_lstsq_backward");
  }
  if (!rc) rc = blr_cuda_check(cudaStreamSynchronize(st), "blr_lstsq_backward");
  if (y) cudaFree(y);
  if (z) cudaFree(z);
  if (rr) cudaFree(rr);
  return rc;
}

// ---------------------------------------------------------------------------
// blr_apply_qt_noalloc: Q^T B / Q B without any device allocation.
//
// Some callers cannot allocate device memory at call time: applications
// that own all device memory through their own pool and forbid cudaMalloc
// after start-up, and latency-critical solvers that cannot afford the
// allocator's implicit device synchronisation in the middle of an
// iteration.  This entry point runs the same apply kernel as
// blr_apply_qt, with its scratch (status word, per-block-column T offsets,
// per-CTA work slabs) in the fixed array below instead of cudaMalloc'd
// buffers.  The array is a file-scope device variable, so every GPU that
// loads the library holds its 4 MiB until the process exits.  All calls on
// a device share it and it keeps the previous call's contents; the call
// clears the status word itself and every other byte it reads is written
// first.  Calls whose kernels overlap on the GPU (different streams or
// threads at the same time) race on this memory and must be serialised by
// the caller.  The first call on a device looks up the array's device
// address with that device current (cudaGetSymbolAddress), so that first
// call should come before any stream capture.
// ---------------------------------------------------------------------------

#define BLR_NOALLOC_BYTES (4u << 20)
static __device__ __align__(256) double g_apply_scratch[BLR_NOALLOC_BYTES / sizeof(double)];

namespace {

__global__ void k_fill_toff(long long* toff, int p, int q) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < q; k += gridDim.x * blockDim.x)
    toff[k] = (long long)k * p - (long long)k * (k - 1) / 2;   // sum_{k' < k} (p - k')
}

std::mutex g_noalloc_mu;
double* g_noalloc_ptr[64];

// Device address of the static scratch for the current device; looked up
// once per device (with that device current) and cached.
int noalloc_scratch(double** out) {
  int dev = 0;
  int rc = blr_cuda_check(cudaGetDevice(&dev), "cudaGetDevice");
  if (rc) return rc;
  if (dev < 0 || dev >= 64) {
    blr_set_error("device ordinal %d out of range", dev);
    return BLR_ERR_INVALID;
  }
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    double* p = nullptr;
    rc = blr_cuda_check(cudaGetSymbolAddress((void**)&p, g_apply_scratch), "cudaGetSymbolAddress");
    if (rc) return rc;
    g_noalloc_ptr[dev] = p;
  }
  *out = g_noalloc_ptr[dev];
  return BLR_OK;
}

}  // namespace

extern "C" int blr_apply_qt_noalloc(const blr_factor* f, double* b_dev, int ldb, int nrhs, int trans,
                                    void* stream) {
  if (!f || !b_dev) { blr_set_error("NULL argument"); return BLR_ERR_INVALID; }
  if (ldb < f->a.m || nrhs < 0) { blr_set_error("bad ldb or nrhs"); return BLR_ERR_INVALID; }
  if (nrhs == 0) return BLR_OK;
  const blr_matrix& a = f->a;
  const int nct = (nrhs + kColsPerCta - 1) / kColsPerCta;
  const size_t slab = (size_t)2 * a.cap * kColsPerCta + 64;                // doubles per CTA
  const size_t off_toff = 256, toff_bytes = (((size_t)a.q * sizeof(long long)) + 255) & ~(size_t)255;
  const size_t off_slab = off_toff + toff_bytes;
  const size_t need = off_slab + (size_t)nct * slab * sizeof(double);
  if (need > BLR_NOALLOC_BYTES) {
    const size_t max_ct = (BLR_NOALLOC_BYTES - off_slab) / (slab * sizeof(double));
    blr_set_error("blr_apply_qt_noalloc: %d right-hand sides need %zu bytes of the %u-byte static scratch "
                  "(at most %zu columns for b=%d, q=%d)", nrhs, need, BLR_NOALLOC_BYTES,
                  max_ct * kColsPerCta, a.b, a.q);
    return BLR_ERR_INVALID;
  }
  double* base = nullptr;
  int rc = noalloc_scratch(&base);
  if (!rc) rc = set_smem();
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  char* bytes = reinterpret_cast<char*>(base);
  FactorView F{};
  F.p = a.p; F.q = a.q; F.b = a.b; F.cap = a.cap;
  F.tiles = a.tiles; F.rank = a.rank; F.t = f->t;
  F.status = reinterpret_cast<int*>(bytes);
  F.toff = reinterpret_cast<const long long*>(bytes + off_toff);
  F.scratch = reinterpret_cast<double*>(bytes + off_slab);
  F.slab = slab;
  rc = blr_cuda_check(cudaMemsetAsync(F.status, 0, sizeof(int), st), "clear status");
  if (rc) return rc;
  k_fill_toff<<<1, 256, 0, st>>>(const_cast<long long*>(F.toff), a.p, a.q);
  rc = blr_cuda_check(cudaGetLastError(), "launch k_fill_toff");
  if (rc) return rc;
  k_apply_q<<<nct, BLR_NT, BLR_SMEM_BYTES, st>>>(F, b_dev, ldb, nrhs, trans ? 0 : 1, kColsPerCta);
  rc = blr_cuda_check(cudaGetLastError(), "launch k_apply_q");
  if (rc) return rc;
  int s = 0;
  rc = blr_cuda_check(cudaMemcpyAsync(&s, F.status, sizeof(int), cudaMemcpyDeviceToHost, st), "read status");
  if (!rc) rc = blr_cuda_check(cudaStreamSynchronize(st), "blr_apply_qt_noalloc");
  if (rc) return rc;
  if (s & ST_NUMERIC) {
    blr_set_error("blr_apply_qt_noalloc: non-finite value");
    return BLR_ERR_NUMERIC;
  }
  return BLR_OK;
}

// ---------------------------------------------------------------------------
// blr_densify: a dense column-major array from BLR storage (Eq. 7: a tile is
// its dense block or U V^T).  One CTA per tile; consecutive threads take
// consecutive rows of a column, so tile reads and output writes coalesce.
// ---------------------------------------------------------------------------
namespace {

__global__ void __launch_bounds__(BLR_NT) k_densify(const double* tiles, const int* rank, int p, int q, int b,
                                                    int cap, int which, double* out, long long ld) {
  const int t = blockIdx.x;
  const int i = t % p, j = t / p;
  if (which == 1 && i >= q) return;                // R is n x n: tile rows below q are not part of it
  const double* T = tiles + (size_t)t * b * b;
  const int r = rank[t];
  for (int e = threadIdx.x; e < b * b; e += blockDim.x) {
    const int rr = e % b, cc = e / b;
    double v;
    if ((which == 1 && (j < i || (j == i && rr > cc))) || (which == 2 && j > i)) {
      v = 0.0;                                     // below R's diagonal, or above Y~'s
    } else if (which == 2 && i == j) {
      v = rr > cc ? T[rr + (size_t)cc * b] : (rr == cc ? 1.0 : 0.0);   // unit lower triangular Y_kk
    } else if (r < 0) {
      v = T[rr + (size_t)cc * b];
    } else {
      double acc = 0.0;
      for (int l = 0; l < r; l++) acc += T[rr + (size_t)l * b] * T[(size_t)b * cap + cc + (size_t)l * b];
      v = acc;
    }
    out[(size_t)i * b + rr + (size_t)(j * b + cc) * ld] = v;
  }
}

}  // namespace

extern "C" int blr_densify(const void* handle, int handle_is_factor, int which, double* out_dev, int ld,
                           void* stream) {
  if (!handle || !out_dev) { blr_set_error("blr_densify: NULL handle or output"); return BLR_ERR_INVALID; }
  if (which < 0 || which > 2 || (which > 0 && !handle_is_factor)) {
    blr_set_error("blr_densify: which=%d is not valid for a %s handle", which, handle_is_factor ? "factor" : "matrix");
    return BLR_ERR_INVALID;
  }
  const blr_matrix* a = handle_is_factor ? &((const blr_factor*)handle)->a : (const blr_matrix*)handle;
  const int rows = which == 1 ? a->n : a->m;
  if (ld < rows) { blr_set_error("blr_densify: ld=%d < %d rows", ld, rows); return BLR_ERR_INVALID; }
  cudaStream_t st = (cudaStream_t)stream;
  k_densify<<<a->p * a->q, BLR_NT, 0, st>>>(a->tiles, a->rank, a->p, a->q, a->b, a->cap, which, out_dev, ld);
  int rc = blr_cuda_check(cudaGetLastError(), "launch k_densify");
  if (!rc) rc = blr_cuda_check(cudaStreamSynchronize(st), "blr_densify");
  return rc;
}
