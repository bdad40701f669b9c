/*
 * blr.h -- C ABI of the GB300 tiled Householder BLR-QR library (libblrqr.so).
 *
 * Method: Apriansyah & Yokota, "Parallel QR Factorization of Block Low-Rank
 * Matrices".  A (m x n, m >= n) is tiled into p x q square tiles of size b
 * (p = m/b, q = n/b, Section 2); each tile is dense or U V^T with U
 * orthonormal (Eq. 7, Section 3.1).  blr_qr computes the tiled Householder
 * factorization of Algorithm 4 with the BLR tile kernels of Section 3.4, so
 * that A~ = Q R with Q stored as compact-WY reflectors (Eq. 3, Eq. 21).
 *
 * Conventions for every entry point:
 *  - Matrices are column-major doubles.  "device" pointers are CUDA device
 *    memory of the current device, "host" pointers are ordinary host memory.
 *  - Every call returns an int status: BLR_OK (0) or one of the BLR_ERR_*
 *    codes below; blr_last_error() gives a message for the calling thread.
 *  - Calls are ordered on the given stream (cudaStream_t passed as void*,
 *    NULL = legacy default stream) and return after the work has finished,
 *    because each reads back a device status word.
 *  - Handles (blr_matrix, blr_factor) own device memory allocated by the
 *    library; the caller owns every buffer it passes in.
 *  - Pointers, sizes and options are checked on the host before any CUDA
 *    call: a bad argument gives BLR_ERR_INVALID on any machine.
 *  - Nothing here falls back to the CPU: without a usable CUDA device every
 *    call with valid arguments fails with BLR_ERR_CUDA.
 */
#ifndef BLR_H
#define BLR_H

#ifdef __cplusplus
extern "C" {
#endif

#define BLR_OK 0
#define BLR_ERR_INVALID 1        /* bad sizes, pointers or options */
#define BLR_ERR_OOM 2            /* device allocation failed */
#define BLR_ERR_CUDA 3           /* a CUDA runtime call failed */
#define BLR_ERR_TIMEOUT 4        /* the device scheduler made no progress within its budget */
#define BLR_ERR_NUMERIC 5        /* NaN/Inf met, or a zero pivot in a triangular solve */
#define BLR_ERR_RANK_OVERFLOW 6  /* a rank exceeded the tile's factor capacity */

#define BLR_PREC_FP64 0          /* every step in FP64 */
#define BLR_PREC_MIXED 1         /* trailing updates and recompression in FP32; panels FP64 */

#define BLR_KERNEL_INV1D 0       /* 1/(|x-y| + 1e-3), 1D points */
#define BLR_KERNEL_YUKAWA3D 1    /* exp(-r)/(r + 1e-3), 3D points */
#define BLR_KERNEL_LAPLACE3D 2   /* 1/(r + 1e-3), 3D points */

typedef struct blr_matrix blr_matrix; /* opaque BLR matrix (device tiles + ranks) */
typedef struct blr_factor blr_factor; /* opaque factor: in-place R/Y~ tiles + T panels */
typedef struct blr_batch_plan blr_batch_plan; /* opaque launch plan for one or several matrices */

/*
 * Options.  Zero-initialise, then set what you need (blr_opts_default fills
 * the defaults).
 *  b            tile size; a multiple of 32 in [32, 512] (larger tiles are
 *               rejected with BLR_ERR_INVALID: the shared-memory panel
 *               buffer holds 513 x 32 doubles); m and n must be multiples
 *               of b (Section 2 tiling).
 *  tol          compression tolerance: per tile, the smallest rank r with
 *               ||A_ij - U V^T||_F <= tol ||A_ij||_F (Section 3.1), found by
 *               truncated pivoted QR; ignored when fixed_rank > 0.
 *  fixed_rank   > 0: every off-diagonal tile is its best rank-fixed_rank
 *               approximation (truncated SVD).
 *  rec_tol      relative tolerance of the rounded additions (Algorithm 6)
 *               inside blr_qr; 0 means "use tol".
 *  dense_rank   a low-rank tile whose rank would exceed this is stored
 *               dense (Section 3.1 fallback); 0 means b/2, the maximum.
 *  precision    BLR_PREC_FP64 or BLR_PREC_MIXED.
 *  sched_ctas   persistent scheduler CTAs; 0 = one per SM.
 *  watchdog_ms  the scheduler gives up (BLR_ERR_TIMEOUT) after this many
 *               milliseconds without any task completing; 0 = 20000.
 *  eta          blr_compress_kernel only: 0 = weak admissibility (only the
 *               diagonal tiles are dense); eta > 0 = strong admissibility
 *               (Section 3.1): tile (i,j) is also kept dense when the
 *               bounding boxes of its row points and column points are
 *               closer than eta times the larger box diameter, so a larger
 *               eta keeps more tiles dense.
 *  scratch_b2   private scratch per scheduler CTA, in units of b*b doubles;
 *               0 = 20 (ample for every rank up to b/2).  A task that needs
 *               more fails the call with BLR_ERR_RANK_OVERFLOW (blr_stats
 *               reports the largest use, scratch_peak_bytes).
 *  trace        blr_qr / blr_qr_batched: > 0 records one blr_trace_event per
 *               task (type, tiles, CTA, SM, start and end time), keeping the
 *               first `trace` of them (blr_trace_export); 0 = no trace.
 *  test_withhold  test hook, 0 = off: 1 + the id of one task (numbered as
 *               blr_dag_task numbers them; in a batch, ids of matrix t start
 *               after all tasks of matrices 0..t-1) whose successors are
 *               never released, so the scheduler stalls and the watchdog
 *               ends the call with BLR_ERR_TIMEOUT.  Only a device wait that
 *               runs out: nothing faults.
 *  prep_slots   mixed path: slots in the pool of prepared tensor-core
 *               operands (6 x b_r x b floats each, b_r = b rounded up to 128:
 *               6 MB at b = 512).  An update QR takes a free slot for its
 *               reflector block and the slot returns to the pool when the
 *               last update of that block has used it; a block that finds no
 *               free slot is applied from its stored factors instead (same
 *               result, slower).  0 = automatic: one slot per reflector
 *               block when the device has room, else as many as fit while
 *               4 GB stay free.
 */
typedef struct blr_opts {
  int b;
  int fixed_rank;
  double tol;
  double rec_tol;
  int dense_rank;
  int precision;
  int sched_ctas;
  int watchdog_ms;
  int scratch_b2;
  int trace;
  double eta;
  int test_withhold;
  int prep_slots;
  int reserved[2];
} blr_opts;

/* One task of a traced factorization (blr_trace_export). */
typedef struct blr_trace_event {
  int type;                 /* 0 GEQRT, 1 LARFB, 2 TSQRT, 3 TPMQRT */
  int i, j, k;              /* its 0-based tile indices (as blr_dag_task gives them) */
  int matrix;               /* matrix of a batched launch (0 for blr_qr) */
  int cta;                  /* scheduler CTA that ran it */
  int sm;                   /* SM that CTA ran on */
  int reserved;
  long long t_start_ns;     /* device global timer at the task's start */
  long long t_end_ns;       /* ... at its end, before it released its successors */
} blr_trace_event;

/* Statistics of a handle (host struct filled by blr_stats). */
typedef struct blr_stats_t {
  int m, n, b, p, q;
  int n_dense;              /* dense tiles (diagonal included) */
  int max_rank;             /* largest low-rank tile rank */
  double mean_rank;         /* mean rank over low-rank tiles */
  long long device_bytes;   /* device memory held by the handle */
  double flops[5];          /* factor only: counted FP ops per task type
                               (GEQRT, LARFB, TSQRT, TPMQRT, total) */
  long long tasks[4];       /* factor only: tasks executed per type */
  double task_seconds[4];   /* factor only: summed task durations per type (CTA-seconds) */
  double seconds;           /* factor only: device time of the factorization kernel (0 when
                               the launch ran inside a CUDA graph) */
  long long tpmqrt_kind[8]; /* factor only: trapezoidal updates by operand kinds, index
                               4 (Y~_ik dense) + 2 (R_kj dense) + (A_ij dense) at task start */
  double tpmqrt_kind_seconds[8]; /* factor only: their summed durations (CTA-seconds) */
  double tpmqrt_kind_flops[8];   /* factor only: their counted FP ops */
  long long scratch_peak_bytes;  /* factor only: largest per-CTA scratch use of any task */
  long long scratch_bytes;       /* factor only: per-CTA scratch slabs allocated (all CTAs) */
  long long prep_slots;          /* factor only, mixed path: slots in the prepared-operand pool */
  long long prep_misses;         /* factor only, mixed path: reflector blocks that found no free slot */
} blr_stats_t;

/* Fills *opts with the defaults (b = 512, tol = 1e-8, FP64). */
void blr_opts_default(blr_opts* opts);

/* Message of the last failing call on this thread ("" if none). */
const char* blr_last_error(void);

/*
 * blr_compress_kernel -- build the BLR matrix of a kernel matrix
 * A(i,j) = K(|x_i - y_j|) * col_scale[j] (Section 3.1, Eq. 7) on the device.
 *  x_host      host, dim x m (column i = point x_i), already ordered.
 *  y_host      host, dim x n.
 *  dim         1 or 3 (must match kernel_id).
 *  col_scale   host, n doubles, or NULL for no scaling.
 *  kernel_id   BLR_KERNEL_*.
 * Diagonal tiles (i == j) are dense (weak admissibility); every other tile
 * is compressed per opts (tol or fixed_rank) and kept dense when its rank
 * exceeds the dense threshold.  *out receives a new handle.
 * Errors: BLR_ERR_INVALID (m < n, sizes not multiples of b, bad dim/kernel),
 * BLR_ERR_OOM, BLR_ERR_CUDA.
 */
int blr_compress_kernel(const double* x_host, const double* y_host, int dim, int m, int n,
                        int kernel_id, const double* col_scale, const blr_opts* opts,
                        blr_matrix** out, void* stream);

/*
 * blr_compress_dense -- BLR matrix of a dense device matrix A (m x n,
 * leading dimension lda >= m), compressed as in blr_compress_kernel.
 * A is only read.  Errors as above.
 */
int blr_compress_dense(const double* a_dev, int lda, int m, int n, const blr_opts* opts,
                       blr_matrix** out, void* stream);

/*
 * blr_matrix_import -- BLR matrix from explicit host tiles in the library's
 * layout: tiles_host holds p*q blocks of b*b doubles, block (i,j) at offset
 * (j*p + i)*b*b; a dense tile is b x b column-major; a low-rank tile of
 * rank r stores U (b x r, orthonormal columns) in its first b*r doubles and
 * V (b x r) from offset b*(b/2).  ranks_host[(j*p)+i] is r, or -1 for dense.
 * Errors: BLR_ERR_INVALID (rank > b/2), BLR_ERR_OOM, BLR_ERR_CUDA.
 */
int blr_matrix_import(int m, int n, int b, const int* ranks_host, const double* tiles_host,
                      blr_matrix** out, void* stream);

/*
 * blr_matrix_import_device -- as blr_matrix_import, with the tiles in device
 * memory (tiles_dev, p*q*b*b doubles in the same layout; copied, not
 * adopted).  ranks_host is host memory.
 */
int blr_matrix_import_device(int m, int n, int b, const int* ranks_host, const double* tiles_dev,
                             blr_matrix** out, void* stream);

/*
 * blr_matrix_export -- copy tiles and ranks of a matrix, or of a factor's
 * in-place storage, to host buffers of p*q*b*b doubles and p*q ints (same
 * layout as blr_matrix_import).  handle_is_factor selects the handle type.
 */
int blr_matrix_export(const void* handle, int handle_is_factor, int* ranks_host,
                      double* tiles_host, void* stream);

/* Deep copy of a BLR matrix (e.g. to keep A~ for refinement). */
int blr_matrix_clone(const blr_matrix* a, blr_matrix** out, void* stream);

/*
 * blr_qr -- tiled Householder BLR-QR (Algorithm 4 with Section 3.4's
 * GEQRT / apply-block-reflector / update-QR / apply-trapezoidal-reflector,
 * rounded additions of Algorithm 6), run as one persistent device-side task
 * scheduler over the tile DAG (Section 4.3).
 *  a       consumed: its tiles become the factor's in-place storage and the
 *          handle is invalidated (do not use or destroy it afterwards; the
 *          factor owns the memory).  Clone it first to keep A~.
 *  opts    rec_tol (0: tol), dense_rank, precision, sched_ctas, watchdog_ms
 *          and scratch_b2 are used; b comes from the matrix.
 *  f       receives the factor.  Tile (k,k) holds R_kk (upper) and Y_kk
 *          (strictly lower, unit diagonal implied); tile (k,j), j > k, holds
 *          R_kj; tile (i,k), i > k, holds Y~_ik = U_ik Y_ik (low-rank: U slot
 *          = U_ik, V slot = Y_ik^T) or a dense Y_ik.
 * Errors: BLR_ERR_INVALID, BLR_ERR_OOM, BLR_ERR_CUDA, BLR_ERR_TIMEOUT,
 * BLR_ERR_NUMERIC (NaN/Inf in a reflector), BLR_ERR_RANK_OVERFLOW.  On error
 * the factor is not created and the consumed matrix is freed.
 */
int blr_qr(blr_matrix* a, const blr_opts* opts, blr_factor** f, void* stream);

/*
 * blr_qr_batched -- blr_qr of count independent matrices (each with its own
 * m, n, b, ranks) in ONE persistent scheduler launch: the tile DAGs of all
 * matrices share the ready queues, so small matrices fill the SMs together.
 * Every a[i] is consumed exactly as by blr_qr (also on error) and f[i]
 * receives its factor.  opts applies to all (precision, tolerances, dense
 * threshold (capped at each matrix's b/2), scheduler width, watchdog); the
 * statistics of every factor describe the whole launch.  Results are the
 * same as count separate blr_qr calls (each tile's writer order is fixed by
 * its own DAG).  Errors as blr_qr.
 */
int blr_qr_batched(blr_matrix** a, int count, const blr_opts* opts, blr_factor** f, void* stream);

/*
 * Launch plans: the same factorization(s) split so that the launch itself can
 * be captured in a CUDA graph and replayed.
 *  blr_batch_plan_create  allocates everything one launch over the matrices
 *                         a[0..count) needs (factor storage, T blocks,
 *                         scheduler state, scratch) and uploads the static
 *                         scheduler state.  The matrices are NOT consumed: each
 *                         launch restores the factor storage from them, so
 *                         they must stay alive and unchanged while the plan
 *                         is used.
 *  blr_batch_plan_launch  device-side copies and memsets, then the persistent
 *                         kernel, ordered on the stream: no allocation and no
 *                         host synchronisation (capturable; replaying the
 *                         graph re-factors the same inputs).
 *  blr_batch_plan_finish  waits for the stream and reads the device status
 *                         (BLR_ERR_TIMEOUT, BLR_ERR_NUMERIC, ... as blr_qr).
 *  blr_batch_plan_factor  the plan-owned factor i (valid until destroy; its
 *                         content is the last finished launch's), usable
 *                         with every function taking a const blr_factor*.
 * Calls on one plan must not overlap on the GPU.
 * Errors of blr_batch_plan_create: BLR_ERR_INVALID (NULL array or plan,
 * count < 1, a NULL matrix, options blr_qr rejects), BLR_ERR_OOM,
 * BLR_ERR_CUDA; on error *plan is NULL and nothing stays allocated.
 */
int blr_batch_plan_create(blr_matrix* const* a, int count, const blr_opts* opts, blr_batch_plan** plan,
                          void* stream);
int blr_batch_plan_launch(blr_batch_plan* plan, void* stream);
int blr_batch_plan_finish(blr_batch_plan* plan, void* stream);
const blr_factor* blr_batch_plan_factor(const blr_batch_plan* plan, int i);
void blr_batch_plan_destroy(blr_batch_plan* plan);

/*
 * blr_apply_qt -- in place on a device matrix B (m x nrhs, ldb >= m):
 * trans = 0: B <- Q^T B (reflectors in factorization order);
 * trans = 1: B <- Q B (reverse order; Algorithm 5 read with the "I -" of
 * Eq. 21's reflector).  Exact application of the stored reflectors.
 * Columns run in groups of 16; the b/32 blocks of 32 reflectors of each
 * update QR are applied by b/32 CTAs as a pipeline that keeps Algorithm
 * 5's order on every block row, as many groups per launch as the SMs hold
 * at once.  Its CTAs wait on one another with a bounded wait: a wait that
 * runs out (only if the GPU cannot keep all of a launch's CTAs resident)
 * ends the call with BLR_ERR_TIMEOUT.  Errors: BLR_ERR_INVALID, BLR_ERR_OOM,
 * BLR_ERR_CUDA, BLR_ERR_TIMEOUT.
 */
int blr_apply_qt(const blr_factor* f, double* b_dev, int ldb, int nrhs, int trans,
                 void* stream);

/*
 * blr_apply_qt_noalloc -- the same operation as blr_apply_qt, for callers
 * that cannot allocate device memory during the call (an application that
 * owns all device memory through its own pool and forbids cudaMalloc after
 * start-up, or a latency-critical solver that cannot afford the allocator's
 * implicit device synchronisation).  The paper has no counterpart: this is
 * an interface variant of the Algorithm 5 apply.  Nothing is allocated: the
 * scratch is a 4 MiB static device array inside the library, held by every
 * GPU that loads it until the process exits.  Limit: the scratch must hold
 * 256 bytes + q*8 bytes (rounded up to 256) + ceil(nrhs/8) * (16 (b/2) + 64)
 * * 8 bytes; larger nrhs is rejected with BLR_ERR_INVALID (at b = 512, q = 64:
 * up to 1008 right-hand sides).  The first call on a device looks up the
 * array's device address (with that device current), so make it before any
 * stream capture.  Every call shares the array: calls whose kernels overlap
 * on the GPU race and must be serialised by the caller.  Arguments, layout
 * and errors as blr_apply_qt.
 */
int blr_apply_qt_noalloc(const blr_factor* f, double* b_dev, int ldb, int nrhs, int trans,
                         void* stream);

/*
 * blr_lstsq -- least squares min ||A~ X - B||_F via the factor (QR used for
 * least squares, Section 1): X = R^{-1} (Q^T B)(1:n), then refine_steps
 * steps of X += R^{-1} Q_1^T (B - A X) with A = a_orig (BLR, FP64).
 *  b_dev   device, m x nrhs (ldb), read only.   x_dev  device, n x nrhs (ldx).
 *  a_orig  may be NULL when refine_steps == 0.
 * Errors: BLR_ERR_NUMERIC for a zero or non-finite diagonal of R.
 */
int blr_lstsq(const blr_factor* f, const blr_matrix* a_orig, const double* b_dev, int ldb,
              double* x_dev, int ldx, int nrhs, int refine_steps, void* stream);

/*
 * blr_solve_r -- X = R^{-1} C (trans = 0, back substitution) or X = R^{-T} C
 * (trans = 1, forward substitution) with the factor's n x n upper triangular
 * BLR R (C, X device n x nrhs).  Errors: BLR_ERR_NUMERIC for a zero or
 * non-finite diagonal entry of R.
 */
int blr_solve_r(const blr_factor* f, const double* c_dev, int ldc, double* x_dev, int ldx, int nrhs, int trans,
                void* stream);

/*
 * blr_lstsq_backward -- adjoint of x = argmin ||A~ x - B||_F (the least
 * squares use of A = QR, Section 1) for a loss L(x): given xbar = dL/dx
 * (device n x nrhs) and the forward's B (m x nrhs) and x (n x nrhs), with
 * z = (A~^T A~)^{-1} xbar = R^{-1} R^{-T} xbar (the stored R of f) and
 * r = B - A~ x (A~ = a_orig, the matrix that was factored):
 *   bbar = dL/dB = A~ z                              (device m x nrhs, ldbb)
 *   dL/dA~ = r z^T - (A~ z) x^T, projected on the storage of a_orig:
 *   grad_tiles (device, p*q*b*b doubles, the tile layout of
 *   blr_matrix_import) receives for a dense tile (i,j) the b x b block of
 *   dL/dA~, and for a low-rank tile U V^T the gradients dL/dU = (dL/dA~)_ij V
 *   in its U slot and dL/dV = (dL/dA~)_ij^T U in its V slot; the rest of
 *   each tile is zero.
 * Every product runs on the device (triangular solves with the factor, BLR
 * matrix products, one CTA per tile for the projection).
 * Errors: BLR_ERR_INVALID (shapes), BLR_ERR_NUMERIC, BLR_ERR_OOM, BLR_ERR_CUDA.
 */
int blr_lstsq_backward(const blr_factor* f, const blr_matrix* a_orig, const double* b_dev, int ldb,
                       const double* x_dev, int ldx, const double* xbar_dev, int ldxb, int nrhs,
                       double* bbar_dev, int ldbb, double* grad_tiles_dev, void* stream);

/* Y = A~ X for a BLR matrix (X device n x nrhs, Y device m x nrhs). */
int blr_matmul(const blr_matrix* a, const double* x_dev, int ldx, double* y_dev, int ldy,
               int nrhs, void* stream);

/* Y = R X for the factor's n x n upper triangular BLR R (X, Y device n x nrhs). */
int blr_apply_r(const blr_factor* f, const double* x_dev, int ldx, double* y_dev, int ldy,
                int nrhs, void* stream);

/*
 * blr_factor_export_t -- copy the compact-WY T panels to the host.  For the
 * reflector block of tile (i,k) (i >= k) the library stores T_ik as b/32
 * diagonal 32 x 32 upper-triangular blocks (inner blocking, each the T of 32
 * consecutive reflectors), laid out 32 x b column-major; blocks appear in
 * column-major order of (i,k), i = k..p-1 for each k.  t_host holds
 * (sum_k (p-k)) * 32 * b doubles.
 */
int blr_factor_export_t(const blr_factor* f, double* t_host, void* stream);

/* Statistics of a matrix or factor handle. */
int blr_stats(const void* handle, int handle_is_factor, blr_stats_t* out);

/*
 * blr_trace_export -- the per-task trace of the launch that made f (opts.trace
 * > 0; the execution traces of Section 5.1 for the device scheduler).  Copies
 * min(cap, recorded) events into events_host (host, cap entries) in the order
 * the tasks finished; *total (host, may be NULL) receives the number of tasks
 * the launch ran (more than recorded when the trace capacity was smaller).
 * A factor of a batched launch holds the whole batch's trace.  Returns the
 * number copied, or -1 (BLR_ERR_INVALID, message in blr_last_error) for a
 * NULL factor or events_host with cap > 0.
 */
int blr_trace_export(const blr_factor* f, blr_trace_event* events_host, int cap, long long* total);

/*
 * blr_densify -- a dense m x n (or n x n) column-major device array from BLR
 * storage, for checks and for callers that need the explicit matrix
 * (Eq. 7: a tile is its dense block or U V^T).
 *  which = 0: every tile as stored (a matrix: A~; a factor: its in-place
 *             storage, R above and reflector tails below the diagonal),
 *             m x n;
 *  which = 1: a factor's R (upper triangular, n x n);
 *  which = 2: a factor's reflector tails Y~ (m x n: unit lower triangular
 *             Y_kk on the diagonal tiles, Y~_ik = U_ik Y_ik below, zero above).
 *  out_dev    device, ld >= m (which 0, 2) or >= n (which 1); the caller owns it.
 * Errors: BLR_ERR_INVALID (NULL handle or out_dev, ld too small, which out
 * of range, which 1 or 2 with a matrix handle), BLR_ERR_CUDA.
 */
int blr_densify(const void* handle, int handle_is_factor, int which, double* out_dev, int ld, void* stream);

void blr_destroy_matrix(blr_matrix* a);
void blr_destroy_factor(blr_factor* f);

/* ---- diagnostics ------------------------------------------------------- */

/*
 * blr_dag_selfcheck -- host only, no device work: builds the tile DAG of
 * Algorithm 4 (Section 4.3) for p x q tiles from the scheduler's closed
 * formulas, checks every in-degree, and runs the dependency-counter protocol
 * in a seeded random order, checking that each task runs once, after its
 * predecessors, and in each tile's writer order.  Returns 0 on success, or a
 * positive code naming the first failed check (100: q > p or p, q < 1).
 */
int blr_dag_selfcheck(int p, int q, unsigned seed);

/*
 * blr_batch_selfcheck -- host only, no device work: the tile DAGs of count
 * matrices of p[t] x q[t] tiles numbered consecutively as a batched launch
 * numbers them, each task located the way the scheduler kernel locates it,
 * and the dependency-counter protocol run over the whole batch in a seeded
 * random order.  Returns 0 when every task runs exactly once after its
 * predecessors and no dependency crosses matrices; a positive code
 * otherwise (100: bad shapes).
 */
int blr_batch_selfcheck(const int* p, const int* q, int count, unsigned seed);

/*
 * blr_dag_task -- host only, no device work: task `id` of the p x q tile DAG
 * of Algorithm 4 as the device scheduler numbers and releases it (the
 * formulas the scheduler kernel runs).  task[0..3] (host, 4 ints) receives
 * the type (0 GEQRT, 1 LARFB, 2 TSQRT, 3 TPMQRT) and the 0-based tile
 * indices i, j, k; succ (host, cap ints, cap >= q + 1) receives the ids of
 * the tasks it releases.  Returns the number of successors, or -1 (message
 * in blr_last_error) for q > p, p or q < 1, an id outside the DAG, NULL
 * pointers or cap < q + 1.
 */
int blr_dag_task(int p, int q, int id, int* task, int* succ, int cap);

/*
 * blr_tc_gemm_selftest -- D = A B (device, column-major, FP64 in and out:
 * A m x k, lda >= m; B k x n, ldb >= k; D m x n, ldd >= m) through the
 * tensor-core building block of the mixed-precision updates (tcgen05 TF32
 * MMAs on hi/lo splits of the operands, "3xTF32", FP32 accumulation in
 * TMEM), one 128 x 256 tile of D per CTA.  The result has FP32 accuracy.
 * Errors: BLR_ERR_INVALID, BLR_ERR_CUDA, BLR_ERR_TIMEOUT (a completion wait
 * ran out; the kernel returns instead of hanging).
 */
int blr_tc_gemm_selftest(const double* a_dev, int lda, const double* b_dev, int ldb, double* d_dev,
                         int ldd, int m, int n, int k, void* stream);

/*
 * blr_tc_update_bench -- diagnostic timing of the dense prepared trapezoidal
 * update on its own (Section 3.4.4 with a dense reflector block and dense
 * tiles; the mixed path's tensor-core body, 2.5 b^3 multiply-adds): ctas
 * CTAs each repeat the update reps times on their own b x b tiles with one
 * shared slot of prepared operands, filled with synthetic bounded values.
 * variant selects an implementation variant of its conversion and
 * epilogues and its tile order (0, 1, 2, 3, 4, 6, 9, 11, 15, 17 or 19; the
 * factorization uses the fastest measured at b = 512 on 152 CTAs).
 * *ms_per_update (host) receives the mean device time of one update per
 * CTA; *aggregate_tflops (host, may be NULL) the algorithmic rate of the
 * whole launch.  Errors: BLR_ERR_INVALID (b not a multiple of 128 in
 * [128, 512], ctas or reps < 1, unknown variant), BLR_ERR_OOM, BLR_ERR_CUDA,
 * BLR_ERR_TIMEOUT.
 */
int blr_tc_update_bench(int b, int ctas, int reps, int variant, double* ms_per_update, double* aggregate_tflops);

#ifdef __cplusplus
}
#endif

#endif /* BLR_H */
