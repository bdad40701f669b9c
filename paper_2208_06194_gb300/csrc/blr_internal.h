// Internal host/device definitions of the BLR-QR library.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <stddef.h>
#include "blr.h"

// CTA shape shared by every kernel in the library.
#define BLR_NT 256                    // threads per CTA
#define BLR_NWARP (BLR_NT / 32)
#define BLR_NB 32                     // reflectors per compact-WY block (inner blocking)
#define BLR_CW 64                     // column chunk of a block-reflector apply
#define BLR_RB 64                     // row block staged in shared memory
#define BLR_BMAX 512                  // largest supported tile size
#define BLR_SLAB_B2 20                // scratch slab per CTA, in units of b*b doubles

// Shared-memory carve-out (doubles) used by the task bodies.
#define BLR_PNL_LD_MAX (BLR_BMAX + 1)
#define BLR_SM_PNL (BLR_PNL_LD_MAX * BLR_NB)          // panel: up to 513 x 32
#define BLR_SM_CS ((BLR_RB + 1) * BLR_CW)             // staged C block
#define BLR_SM_Z (BLR_NB * BLR_CW)                    // Z = Y^T C chunk
#define BLR_SM_W (BLR_NB * BLR_CW)                    // W = T^T Z chunk
#define BLR_SM_T (BLR_NB * BLR_NB)                    // one T block
#define BLR_SM_RP (BLR_NB * BLR_NB)                   // R panel block (TSQRT)
#define BLR_SM_MISC 1408                              // reductions, scalars, taus, norms, perms
#define BLR_SM_DOUBLES (BLR_SM_PNL + BLR_SM_CS + BLR_SM_Z + BLR_SM_W + BLR_SM_T + BLR_SM_RP + BLR_SM_MISC)
#define BLR_SMEM_BYTES (BLR_SM_DOUBLES * 8)

// Task types of the tile DAG (Algorithm 4).
#define TASK_GEQRT 0
#define TASK_LARFB 1
#define TASK_TSQRT 2
#define TASK_TPMQRT 3

#define BLR_NQ 3                      // ready queues by priority

// Device status bits (combined with atomicOr).
#define ST_TIMEOUT 1
#define ST_NUMERIC 2
#define ST_RANK 4
#define ST_BADTASK 8

struct blr_matrix {
  int m, n, b, p, q, cap;
  double* tiles;   // p*q blocks of b*b doubles, block (i,j) at (j*p+i)*b*b
  int* rank;       // p*q, -1 = dense
  size_t bytes;
};

#ifdef __cplusplus
#include <vector>
#endif

struct blr_factor {
  blr_matrix a;    // in-place R / Y~ storage
  double* t;       // T blocks: for each (i,k), i >= k, 32 x b doubles
  long long* toff; // host: offset (in units of 32*b doubles) of column k's first T block
  int nt;          // number of T blocks
  blr_opts opts;
  double flops[5];
  long long tasks[4];
  double task_seconds[4];
  long long tpmqrt_kind[8];
  double tpmqrt_kind_seconds[8];
  double tpmqrt_kind_flops[8];
  long long scratch_peak_bytes;
  long long scratch_bytes;
  long long prep_slots;
  long long prep_misses;
  double seconds;
  std::vector<blr_trace_event> trace;   // host copy of the launch's task trace (opts.trace > 0)
  long long trace_total;                // tasks the traced launch ran
};

// Parameters of the persistent scheduler kernel.
struct SchedParams {
  int p, q, b, cap, dense_rank, precision;
  double rec_tol;
  double* tiles;
  int* rank;
  double* t;
  const long long* toff_dev;    // per k, offset in T blocks
  const int* off_larfb;          // per k: first task id of LARFB(k, .)
  const int* off_tsqrt;          // per k
  const int* off_tpmqrt;         // per k
  int n_tasks;
  int* deps;
  int* qbuf;                     // BLR_NQ * n_tasks
  int* qhead;                    // BLR_NQ, spaced by 32 ints
  int* qtail;
  int* done;
  int* status;
  unsigned long long* progress_ns;
  long long watchdog_ns;
  double* scratch;
  size_t slab;                   // doubles per CTA
  double* flops;                 // 4 counters
  unsigned long long* ntask;     // 4 counters
  unsigned long long* tns;       // 4 counters: summed task durations (ns)
  unsigned long long* nvar;      // 8 counters: updates per operand kind (4 Y dense + 2 R dense + A dense)
  unsigned long long* tvar;      // 8 counters: their summed durations (ns)
  double* fvar;                  // 8 counters: their counted flops
  // mixed path: a pool of slots of prepared tensor-core operands, shared by
  // every matrix of a launch.  An update QR (i,k) takes a free slot and
  // records it in prep_slot_of[toff[k] + i - k]; prep_ref counts the updates
  // still to use it (0 free, -1 being prepared); the last one frees it.
  float* prep;                   // pool base, or NULL
  int prep_rp;                   // rows of the operands (this matrix's b rounded up to 128)
  int prep_nslot;                // slots in the pool
  size_t prep_slot_floats;       // floats per slot (the largest matrix of the launch)
  int* prep_slot_of;             // this matrix's reflector blocks: slot or -1
  int* prep_ref;                 // per slot
  unsigned int* prep_next;       // rotating start of the free-slot search
  unsigned long long* prep_miss; // blocks that found no free slot
  unsigned long long* phase;     // 32 phase-time counters (builds with BLR_PHASE_TIMING only)
  unsigned long long* slab_peak; // largest scratch use of any task (doubles)
  // batches: several matrices in one launch.  Every matrix has its own copy
  // of these parameters (shape, tiles, T, DAG offsets, prepared operands)
  // sharing the scheduler state above; task ids are batch-wide, matrix t's
  // first task is task_base.
  int task_base;
  int nmat;                      // > 1: a batch (mats, mat_base valid)
  const SchedParams* mats;       // device, nmat entries
  const int* mat_base;           // device, nmat + 1 entries (task_base of each, then the total)
  int mat_index;                 // this matrix's position in the batch
  // task trace (opts.trace > 0): trace_cap events; trace_n counts the tasks
  blr_trace_event* trace;
  int trace_cap;
  unsigned int* trace_n;
  int withhold;                  // test hook: batch-wide id of a task that releases nothing, or -1
  int* chain;                    // per reflector block (toff[k] + i - k): groups done by TSQRT(i,k) (reset per launch)
};

// host helpers (blr_api.cu)
void blr_set_error(const char* fmt, ...);
int blr_cuda_check(cudaError_t e, const char* what);
int blr_num_sms();

// kernel launchers implemented in the .cu files
int blr_launch_factor(blr_factor* f, const blr_opts* o, cudaStream_t st);
int blr_launch_factors(blr_factor* const* fs, int count, const blr_opts* o, cudaStream_t st);
// Options check shared by blr_qr, blr_qr_batched and blr_batch_plan_create
// (host only: BLR_ERR_INVALID with a message, no CUDA call).
int blr_check_qr_opts(const blr_opts* opts);
int blr_factor_alloc_like(const blr_matrix* a, const blr_opts* opts, blr_factor** out);
int blr_run_factor_fp64(const SchedParams& P, int ctas, cudaStream_t st);
int blr_run_factor_mixed(const SchedParams& P, int ctas, cudaStream_t st);
int blr_compress_impl(const double* a_dev, int lda, const double* x_dev, const double* y_dev,
                      int dim, int kernel_id, const double* scale_dev, int m, int n,
                      const blr_opts* o, blr_matrix* out, cudaStream_t st,
                      const unsigned char* inadmissible_dev = nullptr);
