// C ABI of the BLR-QR library: handles, validation, import/export, stats.
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <cmath>
#include <algorithm>
#include <vector>
#include "blr_internal.h"

static thread_local char g_err[512] = "";

void blr_set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}

int blr_cuda_check(cudaError_t e, const char* what) {
  if (e == cudaSuccess) return BLR_OK;
  blr_set_error("%s: %s", what, cudaGetErrorString(e));
  return e == cudaErrorMemoryAllocation ? BLR_ERR_OOM : BLR_ERR_CUDA;
}

int blr_num_sms() {
  int dev = 0, n = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 1;
  if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 1;
  return n > 0 ? n : 1;
}

extern "C" const char* blr_last_error(void) { return g_err; }

extern "C" void blr_opts_default(blr_opts* o) {
  if (!o) return;
  memset(o, 0, sizeof(*o));
  o->b = 512;
  o->tol = 1e-8;
  o->precision = BLR_PREC_FP64;
  o->watchdog_ms = 20000;
}

static int check_device() {
  int n = 0;
  cudaError_t e = cudaGetDeviceCount(&n);
  if (e != cudaSuccess || n == 0) {
    blr_set_error("no usable CUDA device (%s)", e == cudaSuccess ? "none found" : cudaGetErrorString(e));
    return BLR_ERR_CUDA;
  }
  return BLR_OK;
}

static int check_shape(int m, int n, int b) {
  if (b < 32 || b > BLR_BMAX || b % 32 != 0) {
    blr_set_error("tile size b=%d must be a multiple of 32 in [32, %d]", b, BLR_BMAX);
    return BLR_ERR_INVALID;
  }
  if (m <= 0 || n <= 0 || m % b != 0 || n % b != 0) {
    blr_set_error("m=%d and n=%d must be positive multiples of b=%d", m, n, b);
    return BLR_ERR_INVALID;
  }
  if (m < n) {
    blr_set_error("A = QR needs m >= n (m=%d, n=%d)", m, n);
    return BLR_ERR_INVALID;
  }
  return BLR_OK;
}

static int alloc_matrix(blr_matrix* a, int m, int n, int b) {
  a->m = m; a->n = n; a->b = b; a->p = m / b; a->q = n / b; a->cap = b / 2;
  a->tiles = nullptr; a->rank = nullptr;
  const size_t nt = (size_t)a->p * a->q;
  a->bytes = nt * b * b * sizeof(double) + nt * sizeof(int);
  if (cudaMalloc(&a->tiles, nt * b * b * sizeof(double)) != cudaSuccess) {
    blr_set_error("out of device memory for %zu MB of tiles", (nt * b * b * sizeof(double)) >> 20);
    return BLR_ERR_OOM;
  }
  if (cudaMalloc(&a->rank, nt * sizeof(int)) != cudaSuccess) {
    cudaFree(a->tiles);
    a->tiles = nullptr;
    blr_set_error("out of device memory for ranks");
    return BLR_ERR_OOM;
  }
  return BLR_OK;
}

static void free_matrix_storage(blr_matrix* a) {
  if (a->tiles) cudaFree(a->tiles);
  if (a->rank) cudaFree(a->rank);
  a->tiles = nullptr;
  a->rank = nullptr;
}

static int check_opts(const blr_opts* o) {
  if (!o) { blr_set_error("opts is NULL"); return BLR_ERR_INVALID; }
  if (o->fixed_rank < 0 || o->tol < 0 || o->rec_tol < 0 || o->dense_rank < 0 || o->scratch_b2 < 0 || o->eta < 0) {
    blr_set_error("negative option value");
    return BLR_ERR_INVALID;
  }
  if (o->fixed_rank == 0 && o->tol <= 0) {
    blr_set_error("either fixed_rank > 0 or tol > 0 is required");
    return BLR_ERR_INVALID;
  }
  if (o->precision != BLR_PREC_FP64 && o->precision != BLR_PREC_MIXED) {
    blr_set_error("unknown precision %d", o->precision);
    return BLR_ERR_INVALID;
  }
  return BLR_OK;
}

extern "C" int blr_compress_kernel(const double* x_host, const double* y_host, int dim, int m, int n,
                                   int kernel_id, const double* col_scale, const blr_opts* opts,
                                   blr_matrix** out, void* stream) {
  int rc;
  if (!out || !x_host || !y_host) { blr_set_error("NULL argument"); return BLR_ERR_INVALID; }
  *out = nullptr;
  if ((rc = check_opts(opts))) return rc;
  if ((rc = check_shape(m, n, opts->b))) return rc;
  if (kernel_id < 0 || kernel_id > 2) { blr_set_error("unknown kernel id %d", kernel_id); return BLR_ERR_INVALID; }
  const int want_dim = kernel_id == BLR_KERNEL_INV1D ? 1 : 3;
  if (dim != want_dim) { blr_set_error("kernel %d needs dim=%d, got %d", kernel_id, want_dim, dim); return BLR_ERR_INVALID; }
  if (opts->fixed_rank > opts->b / 2) { blr_set_error("fixed_rank must be <= b/2"); return BLR_ERR_INVALID; }
  if ((rc = check_device())) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  blr_matrix* a = new blr_matrix;
  if ((rc = alloc_matrix(a, m, n, opts->b))) { delete a; return rc; }
  double *xd = nullptr, *yd = nullptr, *sd = nullptr;
  unsigned char* adm = nullptr;
  do {
    if (opts->eta > 0) {
      // strong admissibility: tile (i,j) is inadmissible (kept dense) when
      // the bounding boxes of its row and column clusters are closer than
      // eta times the larger box diameter (a larger eta keeps more dense)
      const int p = m / opts->b, q = n / opts->b, b = opts->b;
      std::vector<double> bx((size_t)p * 2 * dim), by((size_t)q * 2 * dim);
      auto boxes = [&](const double* pts, int nclust, std::vector<double>& box) {
        for (int c = 0; c < nclust; c++)
          for (int d = 0; d < dim; d++) {
            double lo = pts[d + (size_t)c * b * dim], hi = lo;
            for (int e = 0; e < b; e++) {
              const double v = pts[d + ((size_t)c * b + e) * dim];
              lo = v < lo ? v : lo;
              hi = v > hi ? v : hi;
            }
            box[((size_t)c * 2 + 0) * dim + d] = lo;
            box[((size_t)c * 2 + 1) * dim + d] = hi;
          }
      };
      boxes(x_host, p, bx);
      boxes(y_host, q, by);
      std::vector<unsigned char> flags((size_t)p * q);
      for (int j = 0; j < q; j++)
        for (int i = 0; i < p; i++) {
          double dist2 = 0.0, di2 = 0.0, dj2 = 0.0;
          for (int d = 0; d < dim; d++) {
            const double ilo = bx[((size_t)i * 2) * dim + d], ihi = bx[((size_t)i * 2 + 1) * dim + d];
            const double jlo = by[((size_t)j * 2) * dim + d], jhi = by[((size_t)j * 2 + 1) * dim + d];
            const double gap = jlo > ihi ? jlo - ihi : (ilo > jhi ? ilo - jhi : 0.0);
            dist2 += gap * gap;
            di2 += (ihi - ilo) * (ihi - ilo);
            dj2 += (jhi - jlo) * (jhi - jlo);
          }
          const double diam = sqrt(di2 > dj2 ? di2 : dj2);
          flags[(size_t)j * p + i] = sqrt(dist2) < opts->eta * diam ? 1 : 0;
        }
      if ((rc = blr_cuda_check(cudaMalloc(&adm, flags.size()), "alloc admissibility"))) break;
      if ((rc = blr_cuda_check(cudaMemcpy(adm, flags.data(), flags.size(), cudaMemcpyHostToDevice), "copy admissibility"))) break;
    }
    if ((rc = blr_cuda_check(cudaMalloc(&xd, sizeof(double) * dim * m), "alloc points"))) break;
    if ((rc = blr_cuda_check(cudaMalloc(&yd, sizeof(double) * dim * n), "alloc points"))) break;
    if ((rc = blr_cuda_check(cudaMemcpyAsync(xd, x_host, sizeof(double) * dim * m, cudaMemcpyHostToDevice, st), "copy x"))) break;
    if ((rc = blr_cuda_check(cudaMemcpyAsync(yd, y_host, sizeof(double) * dim * n, cudaMemcpyHostToDevice, st), "copy y"))) break;
    if (col_scale) {
      if ((rc = blr_cuda_check(cudaMalloc(&sd, sizeof(double) * n), "alloc scale"))) break;
      if ((rc = blr_cuda_check(cudaMemcpyAsync(sd, col_scale, sizeof(double) * n, cudaMemcpyHostToDevice, st), "copy scale"))) break;
    }
    rc = blr_compress_impl(nullptr, 0, xd, yd, dim, kernel_id, sd, m, n, opts, a, st, adm);
  } while (0);
  cudaStreamSynchronize(st);
  if (adm) cudaFree(adm);
  if (xd) cudaFree(xd);
  if (yd) cudaFree(yd);
  if (sd) cudaFree(sd);
  if (rc) { free_matrix_storage(a); delete a; return rc; }
  *out = a;
  return BLR_OK;
}

extern "C" int blr_compress_dense(const double* a_dev, int lda, int m, int n, const blr_opts* opts,
                                  blr_matrix** out, void* stream) {
  int rc;
  if (!out || !a_dev) { blr_set_error("NULL argument"); return BLR_ERR_INVALID; }
  *out = nullptr;
  if ((rc = check_opts(opts))) return rc;
  if ((rc = check_shape(m, n, opts->b))) return rc;
  if (lda < m) { blr_set_error("lda=%d < m=%d", lda, m); return BLR_ERR_INVALID; }
  if (opts->fixed_rank > opts->b / 2) { blr_set_error("fixed_rank must be <= b/2"); return BLR_ERR_INVALID; }
  if ((rc = check_device())) return rc;
  blr_matrix* a = new blr_matrix;
  if ((rc = alloc_matrix(a, m, n, opts->b))) { delete a; return rc; }
  rc = blr_compress_impl(a_dev, lda, nullptr, nullptr, 0, 0, nullptr, m, n, opts, a, (cudaStream_t)stream);
  if (rc) { free_matrix_storage(a); delete a; return rc; }
  *out = a;
  return BLR_OK;
}

static int import_tiles(int m, int n, int b, const int* ranks_host, const double* tiles_host, cudaMemcpyKind kind,
                        blr_matrix** out, void* stream) {
  int rc;
  if (!out || !ranks_host || !tiles_host) { blr_set_error("NULL argument"); return BLR_ERR_INVALID; }
  *out = nullptr;
  if ((rc = check_shape(m, n, b))) return rc;
  const int p = m / b, q = n / b;
  for (int t = 0; t < p * q; t++) {
    if (ranks_host[t] < -1 || ranks_host[t] > b / 2) {
      blr_set_error("tile %d: rank %d outside [-1, b/2]", t, ranks_host[t]);
      return BLR_ERR_INVALID;
    }
  }
  if ((rc = check_device())) return rc;
  blr_matrix* a = new blr_matrix;
  if ((rc = alloc_matrix(a, m, n, b))) { delete a; return rc; }
  cudaStream_t st = (cudaStream_t)stream;
  rc = blr_cuda_check(cudaMemcpyAsync(a->tiles, tiles_host, sizeof(double) * (size_t)p * q * b * b, kind, st), "import tiles");
  if (!rc) rc = blr_cuda_check(cudaMemcpyAsync(a->rank, ranks_host, sizeof(int) * p * q, cudaMemcpyHostToDevice, st), "import ranks");
  if (!rc) rc = blr_cuda_check(cudaStreamSynchronize(st), "import");
  if (rc) { free_matrix_storage(a); delete a; return rc; }
  *out = a;
  return BLR_OK;
}

extern "C" int blr_matrix_import(int m, int n, int b, const int* ranks_host, const double* tiles_host,
                                 blr_matrix** out, void* stream) {
  return import_tiles(m, n, b, ranks_host, tiles_host, cudaMemcpyHostToDevice, out, stream);
}

extern "C" int blr_matrix_import_device(int m, int n, int b, const int* ranks_host, const double* tiles_dev,
                                        blr_matrix** out, void* stream) {
  return import_tiles(m, n, b, ranks_host, tiles_dev, cudaMemcpyDeviceToDevice, out, stream);
}

extern "C" int blr_matrix_export(const void* handle, int handle_is_factor, int* ranks_host,
                                 double* tiles_host, void* stream) {
  if (!handle) { blr_set_error("NULL handle"); return BLR_ERR_INVALID; }
  const blr_matrix* a = handle_is_factor ? &((const blr_factor*)handle)->a : (const blr_matrix*)handle;
  cudaStream_t st = (cudaStream_t)stream;
  int rc = BLR_OK;
  if (ranks_host)
    rc = blr_cuda_check(cudaMemcpyAsync(ranks_host, a->rank, sizeof(int) * a->p * a->q, cudaMemcpyDeviceToHost, st), "export ranks");
  if (!rc && tiles_host)
    rc = blr_cuda_check(cudaMemcpyAsync(tiles_host, a->tiles, sizeof(double) * (size_t)a->p * a->q * a->b * a->b, cudaMemcpyDeviceToHost, st), "export tiles");
  if (!rc) rc = blr_cuda_check(cudaStreamSynchronize(st), "export");
  return rc;
}

extern "C" int blr_matrix_clone(const blr_matrix* a, blr_matrix** out, void* stream) {
  if (!a || !out) { blr_set_error("NULL argument"); return BLR_ERR_INVALID; }
  *out = nullptr;
  blr_matrix* c = new blr_matrix;
  int rc = alloc_matrix(c, a->m, a->n, a->b);
  if (rc) { delete c; return rc; }
  cudaStream_t st = (cudaStream_t)stream;
  rc = blr_cuda_check(cudaMemcpyAsync(c->tiles, a->tiles, sizeof(double) * (size_t)a->p * a->q * a->b * a->b, cudaMemcpyDeviceToDevice, st), "clone tiles");
  if (!rc) rc = blr_cuda_check(cudaMemcpyAsync(c->rank, a->rank, sizeof(int) * a->p * a->q, cudaMemcpyDeviceToDevice, st), "clone ranks");
  if (!rc) rc = blr_cuda_check(cudaStreamSynchronize(st), "clone");
  if (rc) { free_matrix_storage(c); delete c; return rc; }
  *out = c;
  return BLR_OK;
}

int blr_check_qr_opts(const blr_opts* opts) {
  if (!opts) { blr_set_error("opts is NULL"); return BLR_ERR_INVALID; }
  if (opts->trace < 0 || opts->test_withhold < 0 || opts->prep_slots < 0) {
    blr_set_error("negative trace, test_withhold or prep_slots option");
    return BLR_ERR_INVALID;
  }
  if (opts->rec_tol < 0 || (opts->rec_tol == 0 && opts->tol <= 0)) {
    blr_set_error("blr_qr needs rec_tol > 0 or tol > 0");
    return BLR_ERR_INVALID;
  }
  if (opts->precision != BLR_PREC_FP64 && opts->precision != BLR_PREC_MIXED) {
    blr_set_error("unknown precision %d", opts->precision);
    return BLR_ERR_INVALID;
  }
  return BLR_OK;
}

// A factor that takes over a's storage (a is deleted) and owns new T blocks.
static int factor_adopt(blr_matrix* a, const blr_opts* opts, blr_factor** out) {
  blr_factor* F = new blr_factor();
  F->a = *a;
  delete a;   // the factor now owns the tiles
  F->opts = *opts;
  const int p = F->a.p, q = F->a.q, b = F->a.b;
  F->nt = 0;
  for (int k = 0; k < q; k++) F->nt += p - k;
  int rc = blr_cuda_check(cudaMalloc(&F->t, sizeof(double) * (size_t)F->nt * BLR_NB * b), "alloc T blocks");
  if (rc) {
    free_matrix_storage(&F->a);
    delete F;
    return rc;
  }
  F->a.bytes += sizeof(double) * (size_t)F->nt * BLR_NB * b;
  *out = F;
  return BLR_OK;
}

int blr_factor_alloc_like(const blr_matrix* a, const blr_opts* opts, blr_factor** out) {
  blr_matrix* w = new blr_matrix;
  int rc = alloc_matrix(w, a->m, a->n, a->b);
  if (rc) { delete w; return rc; }
  return factor_adopt(w, opts, out);
}

extern "C" int blr_qr(blr_matrix* a, const blr_opts* opts, blr_factor** f, void* stream) {
  int rc;
  if (!a || !f) { blr_set_error("NULL argument"); return BLR_ERR_INVALID; }
  *f = nullptr;
  if ((rc = blr_check_qr_opts(opts))) { free_matrix_storage(a); delete a; return rc; }
  blr_factor* F = nullptr;
  if ((rc = factor_adopt(a, opts, &F))) return rc;
  rc = blr_launch_factor(F, opts, (cudaStream_t)stream);
  if (rc) {
    blr_destroy_factor(F);
    return rc;
  }
  *f = F;
  return BLR_OK;
}

extern "C" int blr_qr_batched(blr_matrix** a, int count, const blr_opts* opts, blr_factor** f, void* stream) {
  if (!a || !f || count < 1) { blr_set_error("NULL argument or count < 1"); return BLR_ERR_INVALID; }
  int rc = blr_check_qr_opts(opts);
  for (int m = 0; m < count && !rc; m++)
    if (!a[m]) { blr_set_error("matrix %d is NULL", m); rc = BLR_ERR_INVALID; }
  std::vector<blr_factor*> fs;
  for (int m = 0; m < count; m++) {
    f[m] = nullptr;
    if (!a[m]) continue;
    if (rc) { free_matrix_storage(a[m]); delete a[m]; continue; }
    blr_factor* F = nullptr;
    rc = factor_adopt(a[m], opts, &F);
    if (!rc) fs.push_back(F);
  }
  if (!rc) rc = blr_launch_factors(fs.data(), count, opts, (cudaStream_t)stream);
  if (rc) {
    for (blr_factor* F : fs) blr_destroy_factor(F);
    return rc;
  }
  for (int m = 0; m < count; m++) f[m] = fs[m];
  return BLR_OK;
}

extern "C" int blr_factor_export_t(const blr_factor* f, double* t_host, void* stream) {
  if (!f || !t_host) { blr_set_error("NULL argument"); return BLR_ERR_INVALID; }
  cudaStream_t st = (cudaStream_t)stream;
  int rc = blr_cuda_check(cudaMemcpyAsync(t_host, f->t, sizeof(double) * (size_t)f->nt * BLR_NB * f->a.b, cudaMemcpyDeviceToHost, st), "export T");
  if (!rc) rc = blr_cuda_check(cudaStreamSynchronize(st), "export T");
  return rc;
}

extern "C" int blr_stats(const void* handle, int handle_is_factor, blr_stats_t* out) {
  if (!handle || !out) { blr_set_error("NULL argument"); return BLR_ERR_INVALID; }
  memset(out, 0, sizeof(*out));
  const blr_matrix* a = handle_is_factor ? &((const blr_factor*)handle)->a : (const blr_matrix*)handle;
  std::vector<int> r((size_t)a->p * a->q);
  int rc = blr_cuda_check(cudaMemcpy(r.data(), a->rank, sizeof(int) * r.size(), cudaMemcpyDeviceToHost), "stats ranks");
  if (rc) return rc;
  out->m = a->m; out->n = a->n; out->b = a->b; out->p = a->p; out->q = a->q;
  long long nlr = 0, sum = 0;
  for (int v : r) {
    if (v < 0) out->n_dense++;
    else { nlr++; sum += v; if (v > out->max_rank) out->max_rank = v; }
  }
  out->mean_rank = nlr ? (double)sum / nlr : 0.0;
  out->device_bytes = (long long)a->bytes;
  if (handle_is_factor) {
    const blr_factor* f = (const blr_factor*)handle;
    for (int t = 0; t < 5; t++) out->flops[t] = f->flops[t];
    for (int t = 0; t < 4; t++) out->tasks[t] = f->tasks[t];
    for (int t = 0; t < 4; t++) out->task_seconds[t] = f->task_seconds[t];
    out->seconds = f->seconds;
    out->scratch_peak_bytes = f->scratch_peak_bytes;
    out->scratch_bytes = f->scratch_bytes;
    out->prep_slots = f->prep_slots;
    out->prep_misses = f->prep_misses;
    for (int v = 0; v < 8; v++) {
      out->tpmqrt_kind[v] = f->tpmqrt_kind[v];
      out->tpmqrt_kind_seconds[v] = f->tpmqrt_kind_seconds[v];
      out->tpmqrt_kind_flops[v] = f->tpmqrt_kind_flops[v];
    }
  }
  return BLR_OK;
}

extern "C" int blr_trace_export(const blr_factor* f, blr_trace_event* events_host, int cap, long long* total) {
  if (!f || (cap > 0 && !events_host) || cap < 0) {
    blr_set_error("blr_trace_export: NULL factor, or NULL events with cap > 0");
    return -1;
  }
  const int n = (int)std::min<size_t>((size_t)cap, f->trace.size());
  if (n > 0) memcpy(events_host, f->trace.data(), sizeof(blr_trace_event) * (size_t)n);
  if (total) *total = f->trace_total;
  return n;
}

extern "C" void blr_destroy_matrix(blr_matrix* a) {
  if (!a) return;
  free_matrix_storage(a);
  delete a;
}

extern "C" void blr_destroy_factor(blr_factor* f) {
  if (!f) return;
  if (f->t) cudaFree(f->t);
  free_matrix_storage(&f->a);
  delete f;
}
