// Tile DAG of Algorithm 4 (tiled Householder QR) as closed formulas, shared by
// the device scheduler and the host-side checker.
//
// Tasks: GEQRT(k); LARFB(k,j), j > k (apply block reflector, Section 3.4.2);
// TSQRT(i,k), i > k (update QR, Section 3.4.3); TPMQRT(i,j,k), i,j > k (apply
// trapezoidal block reflector, Section 3.4.4).  Every tile has one chain of
// writers, so the DAG (Section 4.3) follows from which task last wrote each
// tile read:
//   GEQRT(k)      <- TPMQRT(k,k,k-1)
//   LARFB(k,j)    <- GEQRT(k), TPMQRT(k,j,k-1)
//   TSQRT(i,k)    <- GEQRT(k) if i == k+1 else TSQRT(i-1,k); TPMQRT(i,k,k-1)
//   TPMQRT(i,j,k) <- TSQRT(i,k); LARFB(k,j) if i == k+1 else TPMQRT(i-1,j,k);
//                    TPMQRT(i,j,k-1)
// (terms with k-1 exist only for k > 0).  Ids: GEQRT first, then LARFB,
// TSQRT and TPMQRT blocks, each ordered by k.
#pragma once

#ifdef __CUDACC__
#define BLR_HD __host__ __device__ __forceinline__
#else
#define BLR_HD inline
#endif

struct DagShape {
  int p, q;
  const int* off_larfb;   // q+1 entries
  const int* off_tsqrt;   // q+1 entries
  const int* off_tpmqrt;  // q+1 entries
};

BLR_HD int dag_id_geqrt(const DagShape& d, int k) { return k; }
BLR_HD int dag_id_larfb(const DagShape& d, int k, int j) { return d.off_larfb[k] + (j - k - 1); }
BLR_HD int dag_id_tsqrt(const DagShape& d, int i, int k) { return d.off_tsqrt[k] + (i - k - 1); }
BLR_HD int dag_id_tpmqrt(const DagShape& d, int i, int j, int k) {
  return d.off_tpmqrt[k] + (i - k - 1) * (d.q - k - 1) + (j - k - 1);
}

// Decode a task id; returns the type (0..3), or -1 for an id out of range.
BLR_HD int dag_decode(const DagShape& d, int id, int* i, int* j, int* k) {
  const int q = d.q;
  if (id < 0) return -1;
  if (id < q) { *k = id; *i = id; *j = id; return 0; }
  if (id < d.off_larfb[q]) {
    int kk = 0;
    while (d.off_larfb[kk + 1] <= id) kk++;
    *k = kk; *i = kk; *j = kk + 1 + (id - d.off_larfb[kk]);
    return 1;
  }
  if (id < d.off_tsqrt[q]) {
    int kk = 0;
    while (d.off_tsqrt[kk + 1] <= id) kk++;
    *k = kk; *j = kk; *i = kk + 1 + (id - d.off_tsqrt[kk]);
    return 2;
  }
  if (id < d.off_tpmqrt[q]) {
    int kk = 0;
    while (d.off_tpmqrt[kk + 1] <= id) kk++;
    int r = id - d.off_tpmqrt[kk], w = q - kk - 1;
    *k = kk; *i = kk + 1 + r / w; *j = kk + 1 + r % w;
    return 3;
  }
  return -1;
}

BLR_HD int dag_indegree(int type, int i, int j, int k) {
  const int prev = (k > 0) ? 1 : 0;
  switch (type) {
    case 0: return prev;
    case 1: return 1 + prev;
    case 2: return 1 + prev;
    default: return 2 + prev;
  }
}

// Calls f(id) for each successor of a task (at most q+1 of them).
template <typename F>
BLR_HD void dag_for_each_successor(const DagShape& d, int type, int i, int j, int k, F f) {
  const int p = d.p, q = d.q;
  switch (type) {
    case 0:
      for (int jj = k + 1; jj < q; jj++) f(dag_id_larfb(d, k, jj));
      if (k + 1 < p) f(dag_id_tsqrt(d, k + 1, k));
      break;
    case 1:
      if (k + 1 < p) f(dag_id_tpmqrt(d, k + 1, j, k));
      break;
    case 2:
      if (i + 1 < p) f(dag_id_tsqrt(d, i + 1, k));
      for (int jj = k + 1; jj < q; jj++) f(dag_id_tpmqrt(d, i, jj, k));
      break;
    default: {
      if (i + 1 < p) f(dag_id_tpmqrt(d, i + 1, j, k));
      const int k1 = k + 1;
      if (i == k1 && j == k1) f(dag_id_geqrt(d, k1));
      else if (i == k1) f(dag_id_larfb(d, k1, j));
      else if (j == k1) f(dag_id_tsqrt(d, i, k1));
      else f(dag_id_tpmqrt(d, i, j, k1));
      break;
    }
  }
}

// Ready-queue priority (0 = highest): panel factorizations first (the paper
// ranks GEQRT > TSQRT > updates by out-degree), then updates of the next
// block column (they feed the next panel), then the rest.
BLR_HD int dag_queue(int type, int i, int j, int k) {
  if (type == 0 || type == 2) return 0;
  if (j == k + 1) return 1;
  return 2;
}

// A batch numbers the tasks of several matrices consecutively: matrix t's
// tasks are [base[t], base[t+1]).  Returns the matrix of a batch-wide task id
// (nmat >= 1, base[0] = 0 <= task < base[nmat]).
BLR_HD int dag_find_matrix(const int* base, int nmat, int task) {
  int lo = 0, hi = nmat - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (base[mid] <= task) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// Fills the offset tables (q+1 entries each) and returns the task count.
BLR_HD int dag_offsets(int p, int q, int* off_larfb, int* off_tsqrt, int* off_tpmqrt) {
  int id = q;
  for (int k = 0; k <= q; k++) {
    off_larfb[k] = id;
    if (k < q) id += q - k - 1;
  }
  for (int k = 0; k <= q; k++) {
    off_tsqrt[k] = id;
    if (k < q) id += p - k - 1;
  }
  for (int k = 0; k <= q; k++) {
    off_tpmqrt[k] = id;
    if (k < q) id += (p - k - 1) * (q - k - 1);
  }
  return id;
}
