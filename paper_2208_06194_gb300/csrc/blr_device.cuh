// CTA-collective building blocks of the BLR-QR kernels.
//
// Every routine is called by all BLR_NT threads of a CTA, starts and ends
// with a barrier, and works on column-major matrices (element (r,c) at
// p[r + c*ld]).  Templates separate the arithmetic type S (shared-memory
// buffers and accumulators: double for the FP64 path, float for the FP32
// trailing updates of the mixed path) from the element types of the global
// operands (tiles are always stored in double); values are converted once
// when staged.  Global operands that other CTAs may have written during a
// persistent launch are read with ld.global.cg (L2, never a stale L1 line);
// CTA-private scratch and shared memory are read with plain loads.
//
// Householder convention (LAPACK's): for x = [alpha; x2], beta =
// -sign(alpha) ||x|| (sign(0) = +1), tau = (beta - alpha)/beta,
// v = [1; x2/(alpha - beta)], so (I - tau v v^T) x = beta e_1; a zero tail
// gives tau = 0.  Blocks of BLR_NB reflectors are kept in compact-WY form
// I - Y T Y^T (Eq. 3), T built by the Schreiber-Van Loan recurrence.
#pragma once
#include <type_traits>
#include "blr_internal.h"

#define FULLMASK 0xffffffffu

namespace {

__device__ __forceinline__ double ldg(const double* p) { return __ldcg(p); }
__device__ __forceinline__ float ldg(const float* p) { return __ldcg(p); }

// FP64 <-> FP32 conversions written from the IEEE 754 binary64 / binary32
// layouts with integer operations: GB300 runs cvt between the two formats on
// its reduced FP64 pipe (about one per clock per SM, measured), the integer
// pipes run these several times faster.  binary64 -> binary32 rounds to
// nearest with ties away from zero, flushes results below the smallest
// normal binary32 (2^-126) to zero, and maps overflow to infinity and NaN to
// NaN; binary32 -> binary64 is exact for normal values and flushes
// subnormals to zero.  The mixed path's data are far from either limit.
__device__ __forceinline__ float d2f_bits(double x) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(x);
  const unsigned hi = (unsigned)(u >> 32), lo = (unsigned)u;
  const unsigned s = hi & 0x80000000u, a = hi & 0x7fffffffu;
  unsigned r;
  if (a < (897u << 20)) {
    r = 0u;                                               // below 2^-126: zero
  } else if (a >= (1151u << 20)) {
    r = (a > 0x7ff00000u || (a == 0x7ff00000u && lo != 0u)) ? 0x7fc00000u : 0x7f800000u;
  } else {
    r = ((a - (896u << 20)) << 3) | (lo >> 29);           // rebias the exponent, keep 23 fraction bits
    r += (lo >> 28) & 1u;                                 // round (a carry may reach infinity)
  }
  return __uint_as_float(s | r);
}

__device__ __forceinline__ double f2d_bits(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned s = u & 0x80000000u, a = u & 0x7fffffffu;
  unsigned hi = 0u, lo = 0u;
  if (a >= 0x7f800000u) {
    hi = 0x7ff00000u | (a & 0x007fffffu ? 0x00080000u : 0u);   // infinity or a quiet NaN
  } else if (a >= 0x00800000u) {
    hi = (a >> 3) + (896u << 20);
    lo = a << 29;
  }
  return __longlong_as_double((long long)(((unsigned long long)(s | hi) << 32) | lo));
}

template <class To, class From>
__device__ __forceinline__ To cvt(From x) { return static_cast<To>(x); }
template <>
__device__ __forceinline__ float cvt<float, double>(double x) { return d2f_bits(x); }
template <>
__device__ __forceinline__ double cvt<double, float>(float x) { return f2d_bits(x); }


// Shared-memory carve-out (sizes in doubles; float users reinterpret).
struct Sm {
  double* pnl;   // BLR_SM_PNL
  double* cs;    // staged block
  double* z;     // NB x CW
  double* w;     // NB x CW
  double* t;     // NB x NB
  double* rp;    // NB x NB
  double* red;   // 8
  double* scal;  // 8
  double* tau;   // 32
  double* vec;   // 512
  int* ivec;     // 512 ints
  int* flag;     // 4 ints
};

struct Ctx {
  Sm s;
  int* status;      // global status word
  double fma;       // fused multiply-adds counted for the current task (same on all threads)
};

template <class S>
__device__ __forceinline__ S* as(double* p) { return reinterpret_cast<S*>(p); }

__device__ __forceinline__ Sm sm_carve(double* base) {
  Sm s;
  s.pnl = base;
  s.cs = s.pnl + BLR_SM_PNL;
  s.z = s.cs + BLR_SM_CS;
  s.w = s.z + BLR_SM_Z;
  s.t = s.w + BLR_SM_W;
  s.rp = s.t + BLR_SM_T;
  double* m = s.rp + BLR_SM_RP;
  s.red = m;
  s.scal = m + 8;
  s.tau = m + 16;
  s.vec = m + 48;
  s.ivec = reinterpret_cast<int*>(m + 48 + 512);
  s.flag = reinterpret_cast<int*>(m + 48 + 512 + 256);
  return s;
}

template <class S>
__device__ __forceinline__ S warp_sum(S v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(FULLMASK, v, o);
  return v;
}

// Sum over the CTA; every thread gets the same value.
template <class S>
__device__ __forceinline__ S block_sum(S v, double* red) {
  v = warp_sum(v);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = (double)v;
  __syncthreads();
  double s = 0.0;
#pragma unroll
  for (int i = 0; i < BLR_NWARP; i++) s += red[i];
  return (S)s;
}

template <class S>
__device__ __forceinline__ void house(S alpha, S sig2, S& beta, S& tau, S& scale) {
  if (sig2 == S(0)) {
    beta = alpha;
    tau = S(0);
    scale = S(0);
    return;
  }
  S nrm = sqrt(alpha * alpha + sig2);
  beta = (alpha >= S(0)) ? -nrm : nrm;
  tau = (beta - alpha) / beta;
  scale = S(1) / (alpha - beta);
}

__device__ __forceinline__ void flag_numeric(Ctx& c, double x) {
  if (!isfinite(x)) atomicOr(c.status, ST_NUMERIC);
}

// ---------------------------------------------------------------------------
// Strided views and staging.  View<T>: element (r,c) at p[r*sr + c*sc].
// ---------------------------------------------------------------------------
template <class T>
struct View {
  T* p;
  long long sr, sc;
  __device__ __forceinline__ T* at(int r, int c) const { return p + r * sr + c * sc; }
  __device__ __forceinline__ View shifted(int r0, int c0) const { return View{p + r0 * sr + c0 * sc, sr, sc}; }
};

template <class T>
__device__ __forceinline__ View<T> colmajor(T* p, long long ld) { return View<T>{p, 1, ld}; }
template <class T>
__device__ __forceinline__ View<T> rowmajor(T* p, long long ld) { return View<T>{p, ld, 1}; }

// Element loops over [0, tot) in CTA-size steps, kMLP elements per thread
// at a time with every load issued before the first use: with one CTA of
// eight warps per SM, a loop that waits on one load at a time is bound by
// memory latency, not bandwidth.
constexpr int kMLP = 4;

// dst (shared, column-major ldd, type S) = src (rows x cols); coalesced along src's unit stride.
template <class S, class G>
__device__ void stage_in(S* dst, int ldd, View<G> src, int rows, int cols) {
  const int tot = rows * cols;
  const bool colwise = src.sr == 1;
  for (int base = 0; base < tot; base += BLR_NT * kMLP) {
    G v[kMLP];
    int off[kMLP];
#pragma unroll
    for (int u = 0; u < kMLP; u++) {
      const int e = base + u * BLR_NT + threadIdx.x;
      int r = 0, c = 0;
      if (e < tot) {
        if (colwise) { r = e % rows; c = e / rows; } else { c = e % cols; r = e / cols; }
      }
      off[u] = r + c * ldd;
      v[u] = (e < tot) ? ldg(src.at(r, c)) : G(0);
    }
#pragma unroll
    for (int u = 0; u < kMLP; u++)
      if (base + u * BLR_NT + (int)threadIdx.x < tot) dst[off[u]] = cvt<S>(v[u]);
  }
}

template <class S, class G>
__device__ void stage_out(View<G> dst, const S* src, int lds, int rows, int cols) {
  const int tot = rows * cols;
  if (dst.sr == 1) {
    for (int e = threadIdx.x; e < tot; e += BLR_NT) {
      int r = e % rows, c = e / rows;
      *dst.at(r, c) = cvt<G>(src[r + c * lds]);
    }
  } else {
    for (int e = threadIdx.x; e < tot; e += BLR_NT) {
      int c = e % cols, r = e / cols;
      *dst.at(r, c) = cvt<G>(src[r + c * lds]);
    }
  }
}

// Global-to-global copy (with conversion) / zero of a rows x cols block.
template <class D, class Src>
__device__ void copy_mat(D* dst, long long ldd, const Src* src, long long lds, int rows, int cols) {
  const int tot = rows * cols;
  for (int base = 0; base < tot; base += BLR_NT * kMLP) {
    Src v[kMLP];
    long long od[kMLP];
#pragma unroll
    for (int u = 0; u < kMLP; u++) {
      const int e = base + u * BLR_NT + threadIdx.x;
      int r = 0, c = 0;
      if (e < tot) { r = e % rows; c = e / rows; }
      od[u] = r + c * ldd;
      v[u] = (e < tot) ? ldg(src + r + c * lds) : Src(0);
    }
#pragma unroll
    for (int u = 0; u < kMLP; u++)
      if (base + u * BLR_NT + (int)threadIdx.x < tot) dst[od[u]] = cvt<D>(v[u]);
  }
}

template <class D>
__device__ void zero_mat(D* dst, long long ldd, int rows, int cols) {
  const int tot = rows * cols;
  for (int e = threadIdx.x; e < tot; e += BLR_NT) {
    const int r = e % rows, c = e / rows;
    dst[r + c * ldd] = D(0);
  }
}

// ---------------------------------------------------------------------------
// Unblocked Householder QR of a panel held in shared memory (h x w, w <= 32):
// R in the upper triangle, v_j below the diagonal, tau[j].
// ---------------------------------------------------------------------------
template <class S>
__device__ void panel_qr(S* P, int ldp, int h, int w, S* tau, Ctx& c) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  S* scal = as<S>(c.s.scal);
  __syncthreads();
  for (int j = 0; j < w && j < h; j++) {
    S part = S(0);
    for (int r = j + 1 + threadIdx.x; r < h; r += BLR_NT) {
      S x = P[r + j * ldp];
      part += x * x;
    }
    S sig2 = block_sum(part, c.s.red);
    if (threadIdx.x == 0) {
      S beta, tj, sc;
      house(P[j + j * ldp], sig2, beta, tj, sc);
      flag_numeric(c, (double)beta);
      flag_numeric(c, (double)tj);
      scal[0] = beta;
      scal[1] = tj;
      scal[2] = sc;
    }
    __syncthreads();
    const S tj = scal[1], sc = scal[2];
    for (int r = j + 1 + threadIdx.x; r < h; r += BLR_NT) P[r + j * ldp] *= sc;
    __syncthreads();
    for (int l = j + 1 + warp; l < w; l += BLR_NWARP) {
      S acc = S(0);
      for (int r = j + 1 + lane; r < h; r += 32) acc += P[r + j * ldp] * P[r + l * ldp];
      acc = warp_sum(acc);
      S wl = (__shfl_sync(FULLMASK, P[j + l * ldp], 0) + acc) * tj;
      if (lane == 0) P[j + l * ldp] -= wl;
      for (int r = j + 1 + lane; r < h; r += 32) P[r + l * ldp] -= wl * P[r + j * ldp];
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      P[j + j * ldp] = scal[0];
      tau[j] = tj;
    }
    __syncthreads();
  }
  for (int j = h + threadIdx.x; j < w; j += BLR_NT) tau[j] = S(0);
  __syncthreads();
  const double hw = (double)h * w - 0.5 * (double)w * w;
  c.fma += hw * w + hw;
}

// T (w x w upper, ld NB) from the Gram matrix G of the reflector vectors
// (G[a + l*NB] for a < l) and tau: T_jj = tau_j, T(0:j,j) = -tau_j T(0:j,0:j) G(0:j,j).
template <class S>
__device__ void t_recur(const S* G, const S* tau, int w, S* T, Ctx& c) {
  __syncthreads();
  if (threadIdx.x < 32) {
    const int a = threadIdx.x;
    for (int j = 0; j < BLR_NB; j++) {
      S v = S(0);
      if (j < w) {
        if (a < j) {
          S s = S(0);
          for (int cc = a; cc < j; cc++) s += T[a + cc * BLR_NB] * G[cc + j * BLR_NB];
          v = -tau[j] * s;
        } else if (a == j) {
          v = tau[j];
        }
      }
      T[a + j * BLR_NB] = v;
      __syncwarp();
    }
  }
  __syncthreads();
  c.fma += (double)w * w * w / 6.0;
}

__device__ __forceinline__ void decode_pair(int e, int& a, int& l) {
  l = 1;
  int base = 0;
  while (base + l <= e) { base += l; l++; }
  a = e - base;
}

// Gram of a panel's unit-lower-trapezoidal reflectors (P from panel_qr), into G (ld NB).
template <class S>
__device__ void gram_panel(const S* P, int ldp, int h, int w, S* G, Ctx& c) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  const int npair = w * (w - 1) / 2;
  for (int e = warp; e < npair; e += BLR_NWARP) {
    int a, l;
    decode_pair(e, a, l);
    S acc = S(0);
    for (int r = l + 1 + lane; r < h; r += 32) acc += P[r + a * ldp] * P[r + l * ldp];
    acc = warp_sum(acc);
    if (lane == 0) G[a + l * BLR_NB] = (l < h ? P[l + a * ldp] : S(0)) + acc;
  }
  __syncthreads();
  c.fma += (double)h * w * w / 2.0;
}

// Gram of dense reflector blocks Bp (ry x w, ld ldb): G[a][l] = Bp(:,a).Bp(:,l).
template <class S>
__device__ void gram_dense(const S* Bp, int ldb, int ry, int w, S* G, Ctx& c) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  const int npair = w * (w - 1) / 2;
  for (int e = warp; e < npair; e += BLR_NWARP) {
    int a, l;
    decode_pair(e, a, l);
    S acc = S(0);
    for (int r = lane; r < ry; r += 32) acc += Bp[r + a * ldb] * Bp[r + l * ldb];
    acc = warp_sum(acc);
    if (lane == 0) G[a + l * BLR_NB] = acc;
  }
  __syncthreads();
  c.fma += (double)ry * w * w / 2.0;
}

// ---------------------------------------------------------------------------
// C (h x nc, global element type G, ldc) <- (I - Y T' Y^T) C with Y the unit
// lower trapezoidal reflectors of a panel in shared memory (P, ldp, h x w,
// type S) and T' = T^T (trans, applies Q^T) or T (applies Q).  Products are
// accumulated in S; the update is subtracted in G.
// ---------------------------------------------------------------------------
template <class S, class G>
__device__ void apply_refl_panel(G* C, long long ldc, int h, int nc, const S* P, int ldp, int w,
                                 const S* T, bool trans, Ctx& c) {
  const int a = threadIdx.x & 31, grp = threadIdx.x >> 5;
  S* Cs = as<S>(c.s.cs);
  const int ldcs = BLR_RB + 1;
  S* Z = as<S>(c.s.z);
  S* W = as<S>(c.s.w);
  constexpr int KPT = BLR_CW / BLR_NWARP;
  for (int c0 = 0; c0 < nc; c0 += BLR_CW) {
    const int cw = min(BLR_CW, nc - c0);
    S acc[KPT];
#pragma unroll
    for (int k = 0; k < KPT; k++) acc[k] = S(0);
    for (int r0 = 0; r0 < h; r0 += BLR_RB) {
      const int rb = min(BLR_RB, h - r0);
      __syncthreads();
      stage_in(Cs, ldcs, colmajor(C + r0 + (long long)c0 * ldc, ldc), rb, cw);
      __syncthreads();
      if (a < w) {
        for (int rr = 0; rr < rb; rr++) {
          const int row = r0 + rr;
          const S y = (row > a) ? P[row + a * ldp] : (row == a ? S(1) : S(0));
#pragma unroll
          for (int k = 0; k < KPT; k++) {
            int ll = grp + BLR_NWARP * k;
            if (ll < cw) acc[k] += y * Cs[rr + ll * ldcs];
          }
        }
      }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < KPT; k++) {
      int ll = grp + BLR_NWARP * k;
      Z[a + ll * BLR_NB] = (a < w && ll < cw) ? acc[k] : S(0);
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < KPT; k++) {
      int ll = grp + BLR_NWARP * k;
      if (ll < cw && a < w) {
        S s = S(0);
        if (trans) {
          for (int cc = 0; cc <= a; cc++) s += T[cc + a * BLR_NB] * Z[cc + ll * BLR_NB];
        } else {
          for (int cc = a; cc < w; cc++) s += T[a + cc * BLR_NB] * Z[cc + ll * BLR_NB];
        }
        W[a + ll * BLR_NB] = s;
      }
    }
    __syncthreads();
    for (long long e = threadIdx.x; e < (long long)h * cw; e += BLR_NT) {
      int row = (int)(e % h), ll = (int)(e / h);
      S s = S(0);
      const int amax = min(w, row + 1);
      for (int aa = 0; aa < amax; aa++) {
        const S y = (row > aa) ? P[row + aa * ldp] : S(1);
        s += y * W[aa + ll * BLR_NB];
      }
      G* cp = C + row + (long long)(c0 + ll) * ldc;
      *cp = ldg(cp) - cvt<G>(s);
    }
    __syncthreads();
  }
  c.fma += (2.0 * h * w + 0.5 * w * w) * nc;
}

// [Ct (w rows, ldt, type GT); Cb (ry x nc view, type GB)] <-
// (I - [I; Yb] T' [I; Yb]^T) [Ct; Cb] for a block of reflectors [e_a; yb_a]
// (Yb in shared memory, ry x w, ldyb, type S).
template <class S, class GT, class GB>
__device__ void apply_refl_ts(GT* Ct, long long ldt, View<GB> Cb, int ry, int nc, const S* Yb, int ldyb,
                              int w, const S* T, bool trans, Ctx& c) {
  const int a = threadIdx.x & 31, grp = threadIdx.x >> 5;
  S* Cs = as<S>(c.s.cs);
  const int ldcs = BLR_RB + 1;
  S* Z = as<S>(c.s.z);
  S* W = as<S>(c.s.w);
  constexpr int KPT = BLR_CW / BLR_NWARP;
  for (int c0 = 0; c0 < nc; c0 += BLR_CW) {
    const int cw = min(BLR_CW, nc - c0);
    S acc[KPT];
#pragma unroll
    for (int k = 0; k < KPT; k++) {
      int ll = grp + BLR_NWARP * k;
      acc[k] = (a < w && ll < cw) ? cvt<S>(ldg(Ct + a + (long long)(c0 + ll) * ldt)) : S(0);
    }
    for (int r0 = 0; r0 < ry; r0 += BLR_RB) {
      const int rb = min(BLR_RB, ry - r0);
      __syncthreads();
      stage_in(Cs, ldcs, Cb.shifted(r0, c0), rb, cw);
      __syncthreads();
      if (a < w) {
        for (int rr = 0; rr < rb; rr++) {
          const S y = Yb[(r0 + rr) + a * ldyb];
#pragma unroll
          for (int k = 0; k < KPT; k++) {
            int ll = grp + BLR_NWARP * k;
            if (ll < cw) acc[k] += y * Cs[rr + ll * ldcs];
          }
        }
      }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < KPT; k++) {
      int ll = grp + BLR_NWARP * k;
      Z[a + ll * BLR_NB] = (a < w && ll < cw) ? acc[k] : S(0);
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < KPT; k++) {
      int ll = grp + BLR_NWARP * k;
      if (ll < cw && a < w) {
        S s = S(0);
        if (trans) {
          for (int cc = 0; cc <= a; cc++) s += T[cc + a * BLR_NB] * Z[cc + ll * BLR_NB];
        } else {
          for (int cc = a; cc < w; cc++) s += T[a + cc * BLR_NB] * Z[cc + ll * BLR_NB];
        }
        W[a + ll * BLR_NB] = s;
      }
    }
    __syncthreads();
    for (int e = threadIdx.x; e < w * cw; e += BLR_NT) {
      int aa = e % w, ll = e / w;
      GT* cp = Ct + aa + (long long)(c0 + ll) * ldt;
      *cp = ldg(cp) - cvt<GT>(W[aa + ll * BLR_NB]);
    }
    if (Cb.sr == 1) {
      for (long long e = threadIdx.x; e < (long long)ry * cw; e += BLR_NT) {
        int rr = (int)(e % ry), ll = (int)(e / ry);
        S s = S(0);
        for (int aa = 0; aa < w; aa++) s += Yb[rr + aa * ldyb] * W[aa + ll * BLR_NB];
        GB* cp = Cb.at(rr, c0 + ll);
        *cp = ldg(cp) - cvt<GB>(s);
      }
    } else {
      for (long long e = threadIdx.x; e < (long long)ry * cw; e += BLR_NT) {
        int ll = (int)(e % cw), rr = (int)(e / cw);
        S s = S(0);
        for (int aa = 0; aa < w; aa++) s += Yb[rr + aa * ldyb] * W[aa + ll * BLR_NB];
        GB* cp = Cb.at(rr, c0 + ll);
        *cp = ldg(cp) - cvt<GB>(s);
      }
    }
    __syncthreads();
  }
  c.fma += (2.0 * ry * w + 0.5 * w * w) * nc;
}

// ---------------------------------------------------------------------------
// C = alpha op(A) op(B) + beta C, global operands of element types GA, GB,
// GC, products accumulated in S.  beta == 0 never reads C.
// ---------------------------------------------------------------------------
template <class S, class GA, class GB, class GC>
__device__ void gemm(int m, int n, int k, S alpha, const GA* A, long long lda, bool ta, const GB* B,
                     long long ldb, bool tb, S beta, GC* C, long long ldc, Ctx& c) {
  S* As = as<S>(c.s.cs);            // 64 x 16, ld 65
  S* Bs = as<S>(c.s.cs) + 65 * 16;  // 16 x 64, ld 64
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  for (int tm = 0; tm < m; tm += 64) {
    for (int tn = 0; tn < n; tn += 64) {
      S acc[4][4];
#pragma unroll
      for (int i = 0; i < 4; i++)
#pragma unroll
        for (int j = 0; j < 4; j++) acc[i][j] = S(0);
      for (int kk = 0; kk < k; kk += 16) {
        __syncthreads();
        for (int e = threadIdx.x; e < 1024; e += BLR_NT) {
          int r, cc;
          if (!ta) { r = e & 63; cc = e >> 6; } else { cc = e & 15; r = e >> 4; }
          int gr = tm + r, gk = kk + cc;
          S v = S(0);
          if (gr < m && gk < k) v = (S)(ta ? ldg(A + gk + (long long)gr * lda) : ldg(A + gr + (long long)gk * lda));
          As[r + cc * 65] = v;
        }
        for (int e = threadIdx.x; e < 1024; e += BLR_NT) {
          int cc, nn;
          if (!tb) { cc = e & 15; nn = e >> 4; } else { nn = e & 63; cc = e >> 6; }
          int gk = kk + cc, gn = tn + nn;
          S v = S(0);
          if (gn < n && gk < k) v = (S)(tb ? ldg(B + gn + (long long)gk * ldb) : ldg(B + gk + (long long)gn * ldb));
          Bs[cc * 64 + nn] = v;
        }
        __syncthreads();
        const int kmax = min(16, k - kk);
        for (int cc = 0; cc < kmax; cc++) {
          S av[4], bv[4];
#pragma unroll
          for (int i = 0; i < 4; i++) av[i] = As[ty + 16 * i + cc * 65];
#pragma unroll
          for (int j = 0; j < 4; j++) bv[j] = Bs[cc * 64 + tx + 16 * j];
#pragma unroll
          for (int i = 0; i < 4; i++)
#pragma unroll
            for (int j = 0; j < 4; j++) acc[i][j] += av[i] * bv[j];
        }
      }
#pragma unroll
      for (int i = 0; i < 4; i++) {
#pragma unroll
        for (int j = 0; j < 4; j++) {
          int gr = tm + ty + 16 * i, gn = tn + tx + 16 * j;
          if (gr < m && gn < n) {
            GC* cp = C + gr + (long long)gn * ldc;
            S v = alpha * acc[i][j];
            if (beta != S(0)) {
              *cp = (GC)v + (GC)beta * ldg(cp);
            } else {
              *cp = (GC)v;
            }
          }
        }
      }
    }
  }
  __syncthreads();
  c.fma += (double)m * n * k;
}

// ---------------------------------------------------------------------------
// Blocked Householder QR of a global m x n matrix (m >= n) in place, all in
// type S; T blocks (one NB x NB per panel) at Tp + c0*NB (ld NB).
// ---------------------------------------------------------------------------
template <class S>
__device__ void geqrf(S* A, long long lda, int m, int n, S* Tp, Ctx& c) {
  S* pnl = as<S>(c.s.pnl);
  S* tau = as<S>(c.s.tau);
  S* Gm = as<S>(c.s.z);
  S* Ts = as<S>(c.s.t);
  for (int c0 = 0; c0 < n; c0 += BLR_NB) {
    const int w = min(BLR_NB, n - c0), h = m - c0;
    if (h <= 0) break;
    const int ldp = h | 1;
    __syncthreads();
    stage_in(pnl, ldp, colmajor(A + c0 + (long long)c0 * lda, lda), h, w);
    panel_qr(pnl, ldp, h, w, tau, c);
    gram_panel(pnl, ldp, h, w, Gm, c);
    t_recur(Gm, tau, w, Ts, c);
    for (int e = threadIdx.x; e < BLR_NB * BLR_NB; e += BLR_NT) {
      int l = e / BLR_NB;
      if (l < w) Tp[e + (long long)c0 * BLR_NB] = Ts[e];
    }
    stage_out(colmajor(A + c0 + (long long)c0 * lda, lda), pnl, ldp, h, w);
    if (c0 + w < n)
      apply_refl_panel(A + c0 + (long long)(c0 + w) * lda, lda, h, n - c0 - w, pnl, ldp, w, Ts, true, c);
    __syncthreads();
  }
}

// Stage panel c0 (rows c0..m-1, w columns) of stored reflectors Y (type GY)
// and its T block (type GT) into shared memory as S; returns the ld.
template <class S, class GY, class GT>
__device__ int stage_panel(const GY* Y, long long ldy, int m, int c0, int w, const GT* Tp, Ctx& c) {
  const int h = m - c0, ldp = h | 1;
  __syncthreads();
  stage_in(as<S>(c.s.pnl), ldp, colmajor(const_cast<GY*>(Y) + c0 + (long long)c0 * ldy, ldy), h, w);
  S* Ts = as<S>(c.s.t);
  for (int e = threadIdx.x; e < BLR_NB * BLR_NB; e += BLR_NT) {
    int l = e / BLR_NB;
    Ts[e] = (l < w) ? cvt<S>(ldg(Tp + e + (long long)c0 * BLR_NB)) : S(0);
  }
  __syncthreads();
  return ldp;
}

// C (m x nc) <- Q^T C (trans) or Q C for Q from geqrf of an m x nref matrix;
// arithmetic in S.
template <class S, class GY, class GT, class GC>
__device__ void apply_q(const GY* Y, long long ldy, int m, int nref, const GT* Tp, GC* C, long long ldc, int nc,
                        bool trans, Ctx& c) {
  const int npan = (nref + BLR_NB - 1) / BLR_NB;
  for (int pi = 0; pi < npan; pi++) {
    const int pp = trans ? pi : npan - 1 - pi;
    const int c0 = pp * BLR_NB, w = min(BLR_NB, nref - c0), h = m - c0;
    if (h <= 0) continue;
    const int ldp = stage_panel<S>(Y, ldy, m, c0, w, Tp, c);
    apply_refl_panel(C + c0, ldc, h, nc, (const S*)as<S>(c.s.pnl), ldp, w, (const S*)as<S>(c.s.t), trans, c);
  }
}

// ---------------------------------------------------------------------------
// Column-pivoted Householder QR of a CTA-private m x n matrix (plain loads),
// stopped at the smallest r whose trailing block has squared Frobenius norm
// <= tol2, or when r reaches maxr (then *over = 1 if the tail is still
// above tol2).  perm (length n) receives the column order; tau the reflector
// scalars.  Column norms are recomputed exactly each step.
// ---------------------------------------------------------------------------
template <class S>
__device__ int qrcp(S* A, long long lda, int m, int n, double tol2, int maxr, int* perm, S* tau, int* over,
                    Ctx& c) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  double* cn = c.s.vec;   // column norms (n <= 512)
  S* scal = as<S>(c.s.scal);
  for (int j = threadIdx.x; j < n; j += BLR_NT) perm[j] = j;
  if (threadIdx.x == 0) *over = 0;
  __syncthreads();
  int r = 0;
  const int kmax = min(m, n);
  while (true) {
    for (int col = r + warp; col < n; col += BLR_NWARP) {
      S acc = S(0);
      const S* ap = A + (long long)col * lda;
      for (int i = r + lane; i < m; i += 32) acc += ap[i] * ap[i];
      acc = warp_sum(acc);
      if (lane == 0) cn[col] = (double)acc;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      double tail = 0.0;
      int piv = r;
      double best = -1.0;
      for (int col = r; col < n; col++) {
        tail += cn[col];
        if (cn[col] > best) { best = cn[col]; piv = col; }
      }
      int stop = 0;
      if (r >= kmax || tail <= tol2) stop = 1;
      else if (r == maxr) { stop = 1; *over = 1; }
      c.s.flag[0] = stop;
      c.s.flag[1] = piv;
    }
    __syncthreads();
    if (c.s.flag[0]) break;
    const int piv = c.s.flag[1];
    c.fma += (double)(m - r) * (n - r);
    if (piv != r) {
      for (int i = threadIdx.x; i < m; i += BLR_NT) {
        S t0 = A[i + (long long)r * lda];
        A[i + (long long)r * lda] = A[i + (long long)piv * lda];
        A[i + (long long)piv * lda] = t0;
      }
      if (threadIdx.x == 0) {
        int t0 = perm[r]; perm[r] = perm[piv]; perm[piv] = t0;
      }
    }
    __syncthreads();
    S* ar = A + (long long)r * lda;
    S part = S(0);
    for (int i = r + 1 + threadIdx.x; i < m; i += BLR_NT) part += ar[i] * ar[i];
    S sig2 = block_sum(part, c.s.red);
    if (threadIdx.x == 0) {
      S beta, tj, sc;
      house(ar[r], sig2, beta, tj, sc);
      flag_numeric(c, (double)beta);
      scal[0] = beta; scal[1] = tj; scal[2] = sc;
    }
    __syncthreads();
    const S tj = scal[1], sc = scal[2];
    for (int i = r + 1 + threadIdx.x; i < m; i += BLR_NT) ar[i] *= sc;
    __syncthreads();
    for (int col = r + 1 + warp; col < n; col += BLR_NWARP) {
      S* ap = A + (long long)col * lda;
      S acc = S(0);
      for (int i = r + 1 + lane; i < m; i += 32) acc += ar[i] * ap[i];
      acc = warp_sum(acc);
      S wl = (__shfl_sync(FULLMASK, ap[r], 0) + acc) * tj;
      if (lane == 0) ap[r] -= wl;
      for (int i = r + 1 + lane; i < m; i += 32) ap[i] -= wl * ar[i];
    }
    __syncthreads();
    if (threadIdx.x == 0) { ar[r] = scal[0]; tau[r] = tj; }
    __syncthreads();
    c.fma += 2.0 * (m - r) * (n - r);
    r++;
  }
  __syncthreads();
  return r;
}

// C (m x nc, CTA-private) <- Q C (trans = false) or Q^T C for the first nr
// unblocked reflectors stored below the diagonal of A (from qrcp).
template <class S>
__device__ void apply_q_unblocked(const S* A, long long lda, int m, int nr, const S* tau, S* C, long long ldc,
                                  int nc, bool trans, Ctx& c) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int jj = 0; jj < nr; jj++) {
    const int j = trans ? jj : nr - 1 - jj;
    const S* v = A + (long long)j * lda;
    const S tj = tau[j];
    __syncthreads();
    if (tj != S(0)) {
      for (int col = warp; col < nc; col += BLR_NWARP) {
        S* cp = C + (long long)col * ldc;
        S acc = S(0);
        for (int i = j + 1 + lane; i < m; i += 32) acc += v[i] * cp[i];
        acc = warp_sum(acc);
        S wl = (__shfl_sync(FULLMASK, cp[j], 0) + acc) * tj;
        if (lane == 0) cp[j] -= wl;
        for (int i = j + 1 + lane; i < m; i += 32) cp[i] -= wl * v[i];
      }
    }
  }
  __syncthreads();
  c.fma += 2.0 * m * nr * nc;
}

// ---------------------------------------------------------------------------
// One-sided (Hestenes) Jacobi on the columns of X (s x s, CTA-private, ld):
// on exit the columns are mutually orthogonal, X = M V.  sig[j] = ||x_j||
// and order[0..s) lists the columns by decreasing norm (ties: lower index).
// Used by the fixed-rank (truncated SVD) compression.
// ---------------------------------------------------------------------------
__device__ void jacobi_svd(double* X, int ldx, int s, double* sig, int* order, Ctx& c) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const double tol = 1e-15;
  double* nrm = sig;
  const int np = (s + 1) & ~1;
  int* pos = order;
  for (int j = threadIdx.x; j < s; j += BLR_NT) {
    double acc = 0.0;
    for (int i = 0; i < s; i++) acc += X[i + j * ldx] * X[i + j * ldx];
    nrm[j] = acc;
  }
  for (int j = threadIdx.x; j < np; j += BLR_NT) pos[j] = j;
  __syncthreads();
  for (int sweeps = 0; sweeps < 40 && s > 1; sweeps++) {
    if (threadIdx.x == 0) c.s.flag[2] = 0;
    __syncthreads();
    for (int round = 0; round < np - 1; round++) {
      for (int pr = warp; pr < np / 2; pr += BLR_NWARP) {
        int p = pos[pr], q = pos[np - 1 - pr];
        if (p >= s || q >= s) continue;
        if (p > q) { int t0 = p; p = q; q = t0; }
        double* xp = X + p * ldx;
        double* xq = X + q * ldx;
        double g = 0.0;
        for (int i = lane; i < s; i += 32) g += xp[i] * xq[i];
        g = warp_sum(g);
        const double al = nrm[p], be = nrm[q];
        if (fabs(g) > tol * sqrt(al * be) && g != 0.0) {
          const double zeta = (be - al) / (2.0 * g);
          const double t = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
          const double cs = 1.0 / sqrt(1.0 + t * t), sn = cs * t;
          for (int i = lane; i < s; i += 32) {
            double u = xp[i], v = xq[i];
            xp[i] = cs * u - sn * v;
            xq[i] = sn * u + cs * v;
          }
          __syncwarp();
          if (lane == 0) {
            nrm[p] = al - t * g;
            nrm[q] = be + t * g;
            c.s.flag[2] = 1;
          }
        }
      }
      __syncthreads();
      if (threadIdx.x == 0) {
        int last = pos[np - 1];
        for (int i = np - 1; i > 1; i--) pos[i] = pos[i - 1];
        pos[1] = last;
      }
      __syncthreads();
    }
    c.fma += 2.5 * (double)s * s * s;
    for (int j = threadIdx.x; j < s; j += BLR_NT) {
      double acc = 0.0;
      for (int i = 0; i < s; i++) acc += X[i + j * ldx] * X[i + j * ldx];
      nrm[j] = acc;
    }
    __syncthreads();
    if (c.s.flag[2] == 0) break;
    __syncthreads();
  }
  for (int j = threadIdx.x; j < s; j += BLR_NT) sig[j] = sqrt(nrm[j]);
  __syncthreads();
  for (int j = threadIdx.x; j < s; j += BLR_NT) {
    int rk = 0;
    for (int i = 0; i < s; i++) rk += (sig[i] > sig[j]) || (sig[i] == sig[j] && i < j);
    order[rk] = j;
  }
  __syncthreads();
}

// ---------------------------------------------------------------------------
// Reduced reflectors of a TSQRT: Q = I - [I; Yr] T [I; Yr]^T with Yr (ry x b,
// view of type GY) and T blocks (32 x b, type GT).
// ---------------------------------------------------------------------------
template <class S, class GY, class GT>
__device__ int stage_reflector_panel(View<GY> Yr, int ry, int c0, int w, const GT* Tik, Ctx& c) {
  const int ldy = ry | 1;
  __syncthreads();
  stage_in(as<S>(c.s.pnl), ldy, Yr.shifted(0, c0), ry, w);
  S* Ts = as<S>(c.s.t);
  for (int e = threadIdx.x; e < BLR_NB * BLR_NB; e += BLR_NT) {
    int l = e / BLR_NB;
    Ts[e] = (l < w) ? cvt<S>(ldg(Tik + e + (size_t)c0 * BLR_NB)) : S(0);
  }
  __syncthreads();
  return ldy;
}

// [Ctop (b x nc, ld ldt); Cbot (ry x nc)] <- Q^T (trans) or Q times it, for
// the b reflectors of a TSQRT in blocks of 32; arithmetic in S.
template <class S, class GY, class GT, class GC, class GB>
__device__ void apply_ts_reflector(View<GY> Yr, int ry, int b, const GT* Tik, GC* Ctop, long long ldt,
                                   View<GB> Cbot, int nc, bool trans, Ctx& c) {
  const int npan = b / BLR_NB;
  for (int pi = 0; pi < npan; pi++) {
    const int pp = trans ? pi : npan - 1 - pi;
    const int c0 = pp * BLR_NB;
    const int ldy = stage_reflector_panel<S>(Yr, ry, c0, BLR_NB, Tik, c);
    apply_refl_ts(Ctop + c0, ldt, Cbot, ry, nc, (const S*)as<S>(c.s.pnl), ldy, BLR_NB, (const S*)as<S>(c.s.t),
                  trans, c);
  }
}

}  // namespace
