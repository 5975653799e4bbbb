/*
 * bsm.h -- C ABI of libbsm: the local filtered block-sparse matrix multiply
 *
 *     C = beta * C + alpha * A . B      (products filtered on block norms)
 *
 * on one GB300 GPU (sm_103a).
 *
 * The operation is the local block multiplication of the paper's Sec. 2: the
 * matrices are stored in blocked compressed sparse row form (elements grouped
 * into blocks by block rows and block columns), the result pattern is not
 * fixed beforehand but determined by the multiplication itself, and a block
 * product A_ik . B_kj is only carried out when the product of the two block
 * norms is not below the threshold eps (on-the-fly filtering). Algorithms 1
 * and 2 call it once per tick as C = C + A . B; alpha and beta generalise this
 * the BLAS way.
 *
 * Conventions shared by every call:
 *   - Every call returns BSM_OK (0) or a negative BSM_ERR_* code. Nothing is
 *     thrown, nothing aborts. bsm_strerror() names a code.
 *   - Handles (bsm_ctx, bsm_mat) belong to the library until *_destroy.
 *     Arrays passed in are copied (host arrays) or only read (device arrays);
 *     the caller keeps ownership of its buffers.
 *   - Block values are column-major inside a block. A matrix is given as a
 *     list of blocks (block row, block column) in any order; the values
 *     argument holds the blocks concatenated in the order of that list.
 *   - Block sizes are >= 1. Block row/column counts and block counts are
 *     below 2^31; value counts may exceed 2^31.
 *   - The canonical block norm is the Frobenius norm accumulated element by
 *     element in column-major order, each multiply and add rounded separately,
 *     followed by a correctly rounded square root. A product (i,k,j) is
 *     dropped iff nrm(A_ik) * nrm(B_kj) < eps (a tie is kept, NaN is kept,
 *     eps <= 0 drops nothing); alpha does not enter the test.
 *   - With beta == 0 the previous contents of C (pattern and values) are
 *     ignored. With beta != 0 the result pattern is the union of the kept
 *     products' pattern and C's previous pattern.
 *   - All device work of a context runs in stream order on the context's
 *     stream (or the stream given in bsm_opts). Getters synchronise.
 */
#ifndef BSM_H
#define BSM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  BSM_OK = 0,
  BSM_ERR_INVALID_ARG = -1,     /* null handle, bad size, bad option, small cap */
  BSM_ERR_DIM_MISMATCH = -2,    /* A's column sizes != B's row sizes, or C not r x c */
  BSM_ERR_DUPLICATE_BLOCK = -3, /* the same (row, col) listed twice */
  BSM_ERR_OUT_OF_RANGE = -4,    /* a block index outside the block grid */
  BSM_ERR_ALIAS = -5,           /* C is the same handle as A or B (A == B is fine) */
  BSM_ERR_NOMEM = -6,           /* device or pinned host allocation failed (also past
                                   the cap BSM_DEVICE_MEMORY_CAP=<bytes> in the environment:
                                   the device bytes the library may hold per device, read
                                   once per process, for simulating a full device) */
  BSM_ERR_CUDA = -7,            /* a CUDA runtime error (details: bsm_last_cuda_error) */
  BSM_ERR_TIMEOUT = -8,         /* a bounded device-side wait gave up */
  BSM_ERR_UNSUPPORTED = -9      /* valid request the library does not handle */
};

/* Arithmetic of the block products (C accumulation is always FP64). */
enum {
  BSM_PREC_FP64 = 0,        /* FP64 FMA throughout */
  BSM_PREC_SPLIT_BF16X3 = 1, /* 3 BF16 slices per operand, 6 slice products, FP32 sums */
  BSM_PREC_SPLIT_TF32X2 = 2  /* 2 TF32 slices per operand, 3 slice products, FP32 sums */
};

/* FP64 numeric kernels. bsm_opts.fp64_kernel = 1 + one of these forces that
 * kernel for every shape class (no autotuning); 0 leaves the choice to the
 * library: the tuned one with autotune, else PK12, or T16_B2 when the last
 * multiply into the same C had fewer than 4 block products per C block (there
 * the per-block setup of PK costs more than its fuller lanes save).
 *   T16: one output element per lane slot, 16 x 16 tiles, 2 or 3 blocks/SM;
 *   T32: 32 x 32 tiles, synchronous staging;
 *   PK12, PK16: packed lane slots (output element, k-group) over the products
 *        of a C block concatenated along k, 16 x 16 tiles, 12 or 16 slots per
 *        lane, 2 blocks/SM;
 *   G8: groups of 4, 6 or 8 lanes, a lane per C column (up to 8 rows at a
 *        time in registers), a C block per group: for tiny blocks with few
 *        products.
 * All give the same result up to the order of the FP64 additions. */
enum {
  BSM_FP64_T16_B2 = 0,
  BSM_FP64_T16_B3 = 1,
  BSM_FP64_T32 = 2,
  BSM_FP64_PK12 = 3,
  BSM_FP64_PK16 = 4,
  BSM_FP64_G8 = 5,
  BSM_FP64_NUM_KERNELS = 6
};

/* Split-precision numeric kernels. bsm_opts.split_kernel = 1 + one of these
 * forces it; 0 leaves the choice to the library (BLOCKS).
 *   PANEL:  one C block row at a time as a dense panel product on the
 *           tcgen05 tensor cores (MMA M = the row's C columns, N = its block
 *           row size x slices, K = A's row), accumulators in tensor memory;
 *   BLOCKS: one C block per warp, its products one after another on mma.sync
 *           tiles, each product's operands streamed through shared memory;
 *   CHUNKS: one C block per warp on mma.sync tiles, its products concatenated
 *           along k and staged into shared memory in chunks of whole products
 *           (C blocks larger than 16 x 16 go to the BLOCKS kernel).
 * All multiply the same slice products; they differ in FP32 rounding only. */
enum { BSM_SPLIT_PANEL = 0, BSM_SPLIT_BLOCKS = 1, BSM_SPLIT_CHUNKS = 2, BSM_SPLIT_NUM_KERNELS = 3 };

/* How the numeric stacks are launched. */
enum {
  BSM_LAUNCH_PERSISTENT = 0, /* one persistent launch over all shape classes */
  BSM_LAUNCH_PER_STACK = 1   /* one launch per (m,n) shape class, generic tiles */
};

typedef struct bsm_ctx_s *bsm_ctx;
typedef struct bsm_mat_s *bsm_mat;

/* Options of one multiply. A NULL bsm_opts* means all defaults (zeroes). */
typedef struct {
  int32_t precision; /* BSM_PREC_* */
  int32_t launch;    /* BSM_LAUNCH_* */
  int32_t blocking;  /* 1: return after the result is complete and checked */
  int32_t autotune;  /* 1: time the FP64 kernel variants on the real data the first
                        time a shape class (per-stack) or class mix (persistent) is
                        met, and use the fastest; the choice is kept per context and,
                        with BSM_AUTOTUNE_CACHE=<file>, across runs */
  void *stream;      /* cudaStream_t to use instead of the context stream, or NULL */
  int32_t graph;     /* 1: capture the multiply's launches in a CUDA graph the first
                        time a given set of arguments is met and replay it after */
  int32_t fp64_kernel; /* 0, or 1 + BSM_FP64_* to force that FP64 kernel (ignored by
                          the split precisions); out of range: BSM_ERR_INVALID_ARG.
                          Without it (and without a tuned choice): PK12, or where
                          C blocks have fewer than 4 products on average, G8 when
                          C's blocks are at most 8 x 8, else T16_B2 */
  double *host_values; /* NULL, or page-locked host memory (cudaHostAlloc /
                          cudaHostRegister, device-mapped) of host_cap doubles that also
                          receives the result's values, in bsm_mat_get_values order,
                          written by the device while the multiply runs (the packed and g8
                          FP64 kernels and the split-precision kernels store each C block
                          there as they complete it; the other kernels are followed by a
                          device copy). Written only if the
                          result has at most host_cap values (bsm_mat_nblocks tells); valid
                          once the result is complete (a getter, bsm_sync or a blocking
                          multiply). Memory that is not device-mapped: BSM_ERR_INVALID_ARG.
                          The caller keeps ownership and must not free it before then. */
  int64_t host_cap;
  int32_t split_kernel; /* 0, or 1 + BSM_SPLIT_* to force that split-precision kernel
                           (ignored by FP64); out of range: BSM_ERR_INVALID_ARG */
  int32_t numeric_slices; /* 0 or 1: the numeric phase in one launch; n > 1 (at most 64):
                             the FP64 persistent launch in n launches over consecutive
                             ranges of the C blocks, so that other streams' kernels can
                             run between them (the request loop slices large requests);
                             out of range: BSM_ERR_INVALID_ARG */
} bsm_opts;

/* Counters of one multiply (filled when bsm_stats* is not NULL; this makes
 * the call blocking). FLOPs count 2*m*n*k per kept block product, the
 * convention of the paper's Table 1. */
typedef struct {
  int64_t candidates; /* block products (i,k,j) with A_ik and B_kj present */
  int64_t kept;       /* products that passed the filter */
  int64_t dropped;    /* candidates - kept */
  int64_t c_blocks;   /* blocks in the result pattern */
  int64_t c_nnz;      /* scalars in the result */
  double flops;       /* sum over kept products of 2*m*n*k */
  float ms_total;     /* device time of the whole multiply (CUDA events) */
  int32_t retries;    /* times the result buffers had to grow and rerun */
  int32_t reserved;
} bsm_stats;

/* Create a context on CUDA device `device` with its own stream and
 * workspace. *out receives the handle. */
int bsm_ctx_create(int device, bsm_ctx *out);

/* Wait for the context's work and free everything it owns, including every
 * matrix still alive on it. */
int bsm_ctx_destroy(bsm_ctx ctx);

/* Create a block-sparse matrix from host arrays (Sec. 2: blocked CSR built
 * from block row sizes, block column sizes and the list of present blocks).
 *   nbrows, row_sizes[nbrows]   block row count and sizes (each >= 1)
 *   nbcols, col_sizes[nbcols]   block column count and sizes (each >= 1)
 *   nblocks, blk_row[], blk_col[]  the present blocks, any order, no duplicates
 *   values   host array of the blocks' values, concatenated in list order,
 *            each block column-major; NULL creates zero blocks.
 * Errors: INVALID_ARG, OUT_OF_RANGE, DUPLICATE_BLOCK, NOMEM, CUDA. The arrays
 * are copied; the call returns once the copy to the device is done. */
int bsm_mat_create(bsm_ctx ctx, int32_t nbrows, const int32_t *row_sizes, int32_t nbcols,
                   const int32_t *col_sizes, int64_t nblocks, const int32_t *blk_row,
                   const int32_t *blk_col, const double *values, bsm_mat *out);

/* Free a matrix (after the work that uses it has finished). */
int bsm_mat_destroy(bsm_mat m);

/* Replaces the pattern and values of m with a new block list over the same
 * block row / column sizes (arguments as in bsm_mat_create; values NULL =
 * zeros). m's device buffers are reused and grown only when too small, so a
 * stream of inputs of similar size costs no device allocation. Work that reads
 * m is finished first; a pending result computed into m is dropped. Work on
 * other matrices is not waited for: the upload runs on a stream of the
 * context's own, so the next input can go to the device while a multiply of
 * other matrices runs. Inputs are copied before the call returns. Errors: BSM_ERR_OUT_OF_RANGE,
 * BSM_ERR_DUPLICATE_BLOCK, BSM_ERR_INVALID_ARG, BSM_ERR_UNSUPPORTED leave m
 * unchanged; BSM_ERR_NOMEM / BSM_ERR_CUDA leave m empty (no blocks).
 * The paper has no counterpart (there the operands are given to each multiply). */
int bsm_mat_assign(bsm_mat m, int64_t nblocks, const int32_t *blk_row, const int32_t *blk_col,
                   const double *values);

/* C = beta*C + alpha*A.B with the on-the-fly filter (Sec. 2, Algorithm 1's
 * local step C_ij = C_ij + A_comp . B_comp).
 *   A: r x s blocks, B: s x c blocks (A's column sizes must equal B's row
 *   sizes), C: r x c blocks; C's pattern is replaced by the result pattern.
 *   eps: filter threshold; opts, stats: may be NULL.
 * C may not be A or B (ALIAS); A may be B. Without opts->blocking and without
 * stats the call only enqueues work; C's result is complete at the next
 * getter, bsm_sync, or use of C as an operand. Inputs must stay alive and
 * unchanged until then. Errors: INVALID_ARG, DIM_MISMATCH, ALIAS, NOMEM,
 * CUDA, UNSUPPORTED; TIMEOUT (from the call when blocking, else from the
 * getter or bsm_sync that completes the result) when a split-precision
 * kernel's bounded wait for an operand copy gave up: C is then left empty. */
int bsm_multiply(bsm_ctx ctx, double alpha, bsm_mat A, bsm_mat B, double beta, bsm_mat C,
                 double eps, const bsm_opts *opts, bsm_stats *stats);

/* Number of stored blocks and scalars of m (synchronises m). */
int bsm_mat_nblocks(bsm_mat m, int64_t *nblocks, int64_t *nnz);

/* The pattern of m sorted by (row, col) into caller arrays of capacity cap
 * (>= nblocks, else INVALID_ARG). Synchronises. */
int bsm_mat_get_pattern(bsm_mat m, int64_t cap, int32_t *blk_row, int32_t *blk_col);

/* The values of m in the order of bsm_mat_get_pattern, each block
 * column-major, into a host array of capacity cap (>= nnz). Synchronises. */
int bsm_mat_get_values(bsm_mat m, int64_t cap, double *values);

/* Post-multiplication filter (Sec. 1: filtering also after each
 * multiplication; Sec. 2: blocks below the threshold are removed after the
 * multiplication): drop every block of m whose canonical norm is below eps
 * (a tie and NaN are kept; eps <= 0 drops nothing). Kept blocks keep their
 * values. Blocking. Errors: INVALID_ARG, NOMEM, CUDA. */
int bsm_mat_filter(bsm_mat m, double eps);

/* Block-sparse accumulation C = beta*C + alpha*A (Algorithm 2: the partial C
 * panels of the last ticks are summed into the final panel). A and C have the
 * same block sizes; the result pattern is A's plus, when beta != 0, C's.
 * Blocking. Errors: INVALID_ARG, DIM_MISMATCH, ALIAS (A == C), NOMEM, CUDA. */
int bsm_mat_add(bsm_ctx ctx, double alpha, bsm_mat A, double beta, bsm_mat C);

/* Device-time profile of the multiplies of a context: CUDA events recorded
 * on the launch stream at the phase boundaries of every multiply (block norms
 * | symbolic count, scan and fill | numeric block products). */
typedef struct {
  double ms_norms;     /* sum over multiplies of the block-norm phase */
  double ms_symbolic;  /* ... of the symbolic phase (count, scan, fill) */
  double ms_numeric;   /* ... of the numeric phase */
  double ms_total;     /* ... of whole multiplies */
  int64_t multiplies;  /* multiplies profiled */
  int64_t launches;    /* kernels launched by this context since profiling started */
  int32_t last_fp64_kernel; /* BSM_FP64_* of the last FP64 numeric launch enqueued by the
                               context (forced, tuned or default), -1 if none */
  int32_t last_split_kernel; /* BSM_SPLIT_* of the last split-precision numeric launch, -1 if
                                none */
} bsm_profile;

/* enable != 0: start profiling (totals reset); enable == 0: stop. */
int bsm_ctx_profile(bsm_ctx ctx, int enable);

/* Totals since the last bsm_ctx_profile(ctx, 1). Synchronises the context. */
int bsm_ctx_profile_read(bsm_ctx ctx, bsm_profile *out);

/* ---------------------------------------------------------------------------
 * Request loop (serving). Independent multiplies C = A.A of square block-sparse
 * systems of different sizes (the application's repeated multiplies, Sec. 1)
 * arrive one by one. The server keeps `slots` lanes, each a context with its
 * own stream, workspace and worker thread. A free lane takes the next batch of
 * queued requests as soon as its device-memory footprint (an upper bound per
 * request, computed at submission) fits the budget beside the requests already
 * held. Admission is earliest deadline first, the deadline being the
 * submission time plus four times the request's estimated run time (from its
 * exact count of unfiltered multiply-adds): small requests pass large ones that
 * arrived shortly before, no request is passed by one that arrives after its
 * deadline, and the earliest-deadline request waits for memory rather than be
 * passed. A large request (estimated at least 8 ms) fills the GPU alone: one
 * runs at a time (two when only large requests, at least two, wait), and a
 * large earliest-deadline request waits only for the running one, while the
 * other lanes take small requests. A large request's
 * numeric phase runs in slices of about 2 ms (bsm_opts.numeric_slices), each
 * launched once the one before has finished and, while small batches are on
 * the device, held back until they finish (at most 4 ms per slice); small
 * batches run on a stream of the highest priority. A small request arriving
 * meanwhile therefore starts at the next slice boundary and finds the SMs
 * free. Latency and deadline count from the start of bsm_server_submit
 * (bsm_server_timing splits it). A small request (estimated at most 4 ms) shares its multiply with the
 * other small queued requests of the same eps (up to 16 requests and 8 ms of
 * estimated work, at most four times the first request's estimate, so that it
 * still makes its deadline): the batch runs as one multiply of the block-diagonal matrix
 * of its requests, one launch sequence over all their blocks, and each request
 * receives its own part of the result, which is bit for bit the result of that
 * request multiplied alone (the kernels compute each C block from its own
 * products only). The lanes run concurrently on the device, at most two of
 * them small batches. Inputs are copied at submission into page-locked host
 * memory (blocks sorted by (row, col); large copies on several threads) and
 * uploaded from there, or, submitted with bsm_server_submit_borrowed,
 * uploaded from the caller's array. Results wait in page-locked host memory
 * until taken (copied out) or released after use in place. Admission needs no call from
 * the caller. The server functions may be called from any thread;
 * bsm_server_destroy only once every other call on the server has returned.
 * ------------------------------------------------------------------------- */
typedef struct bsm_server_s *bsm_server;

typedef struct {
  int32_t slots;      /* requests on the device at once (default 4, at most 64) */
  int32_t precision;  /* BSM_PREC_* of every multiply */
  int64_t hbm_budget; /* device bytes the admitted requests may hold (default 8 GiB) */
} bsm_server_opts;

typedef struct {
  int64_t queued, running, completed;
  int64_t bytes_in_use, bytes_peak, budget;
  int64_t batches; /* multiplies run, each over a batch of one or more requests */
} bsm_server_info;

/* Request states reported by bsm_server_poll. */
enum { BSM_REQ_QUEUED = 0, BSM_REQ_RUNNING = 1, BSM_REQ_DONE = 2, BSM_REQ_FAILED = 3 };

/* Start a request loop on `device` (opts NULL: 4 lanes, FP64, an 8 GiB
 * budget); *out receives the handle, owned by the caller until
 * bsm_server_destroy. INVALID_ARG for slots above 64, an unknown precision or
 * device; NOMEM; CUDA. */
int bsm_server_create(int device, const bsm_server_opts *opts, bsm_server *out);
/* Finish the requests running, drop the queued ones and free everything the
 * server holds, results not yet taken and result views included. Blocking. */
int bsm_server_destroy(bsm_server s);

/* Queue C = A.A for a square matrix given as in bsm_mat_create (block sizes
 * sizes[nbrows] for rows and columns, a block list in any order, column-major
 * values in list order). The arrays are copied. *id receives the request id.
 * OUT_OF_RANGE for an index outside [0, nbrows), DUPLICATE_BLOCK for a block
 * listed twice, NOMEM if the request's footprint bound exceeds the whole budget
 * (or page-locked memory for its copy cannot be had). */
int bsm_server_submit(bsm_server s, int32_t nbrows, const int32_t *sizes, int64_t nblocks,
                      const int32_t *blk_row, const int32_t *blk_col, const double *values,
                      double eps, int64_t *id);

/* As bsm_server_submit, but the values are not copied: the lane uploads them
 * from the caller's array when the request runs, which saves the copy into
 * page-locked memory at submission (part of every request's latency). The
 * caller keeps `values` alive and unchanged until the request is done or
 * failed (bsm_server_poll) or the server is destroyed; the other arrays are
 * copied. The block list must be sorted by (row, col) without duplicates
 * (INVALID_ARG otherwise). Page-locked values upload fastest. */
int bsm_server_submit_borrowed(bsm_server s, int32_t nbrows, const int32_t *sizes,
                               int64_t nblocks, const int32_t *blk_row, const int32_t *blk_col,
                               const double *values, double eps, int64_t *id);

/* Never blocks. *completed: requests finished since the previous call (the
 * lanes admit and run requests by themselves). */
int bsm_server_progress(bsm_server s, int32_t *completed);

/* State of a request; once done (or failed): latency_ms (submit to
 * completion) and the result's block and value counts, else -1, 0, 0. A failed
 * request returns its error code. */
int bsm_server_poll(bsm_server s, int64_t id, int32_t *state, double *latency_ms,
                    int64_t *nblocks, int64_t *nnz);

/* Where a finished (done or failed) request's latency went, in milliseconds:
 * submit_ms inside bsm_server_submit (checks, sorting, the copy into
 * page-locked memory), wait_ms queued until a lane took its batch, run_ms from
 * then until its result was in host memory (upload, multiply, read-back). The
 * three add up to the latency bsm_server_poll reports. Null pointers are
 * skipped. INVALID_ARG if the request is unknown or not finished. */
int bsm_server_timing(bsm_server s, int64_t id, double *submit_ms, double *wait_ms,
                      double *run_ms);

/* Copy a finished request's result (pattern sorted by (row, col), values as
 * bsm_mat_get_values) into the caller's arrays and release it. Null arrays skip
 * a part; capacities below the result's sizes: INVALID_ARG (nothing released). */
int bsm_server_take(bsm_server s, int64_t id, int64_t cap_blk, int32_t *blk_row,
                    int32_t *blk_col, int64_t cap_nnz, double *values);

/* A finished request's result without a copy: pointers into page-locked host
 * memory owned by the server (pattern sorted by (row, col), values as
 * bsm_mat_get_values), valid until bsm_server_release (or bsm_server_take, or
 * bsm_server_destroy). Null pointer arguments are skipped. INVALID_ARG if the
 * request is unknown or not done. */
int bsm_server_result(bsm_server s, int64_t id, const int32_t **blk_row, const int32_t **blk_col,
                      const double **values, int64_t *nblocks, int64_t *nnz);

/* Forget a finished (done or failed) request and return its result memory. */
int bsm_server_release(bsm_server s, int64_t id);

/* The server's counters at the time of the call: requests queued, running and
 * completed, device bytes held by admitted requests now and at most, the
 * budget, and the multiplies (batches) run. */
int bsm_server_get_info(bsm_server s, bsm_server_info *out);

/* ---------------------------------------------------------------------------
 * Allocation-free multiply. The paper has no counterpart: this entry point
 * exists for callers that cannot call cudaMalloc (a framework whose pool owns
 * all device memory, a callback that must not block on the allocator, a
 * process at its allocation limit). The caller passes device buffers for the
 * inputs and the outputs; everything else the multiply needs lives in one
 * fixed array of BSM_NOALLOC_SCRATCH_BYTES that the library image carries on
 * every GPU that loads it, for the life of the process. No context is used.
 * ------------------------------------------------------------------------- */
#define BSM_NOALLOC_SCRATCH_BYTES (32ll << 20)

/* A block-sparse matrix in device memory, blocked CSR: blocks of a row sorted
 * by column, each block's values column-major at vals + blk_off[b]. */
typedef struct {
  int32_t nbr, nbc;
  const int32_t *row_sizes; /* device [nbr] */
  const int32_t *col_sizes; /* device [nbc] */
  const int32_t *row_ptr;   /* device [nbr+1] */
  const int32_t *col_idx;   /* device [nblk] */
  const int64_t *blk_off;   /* device [nblk] */
  const double *values;     /* device [nnz] */
  int64_t nblk;
} bsm_dev_csr;

/* Caller-owned device buffers that receive the result in the same form. */
typedef struct {
  int32_t *row_ptr; /* device [nbr of A + 1] */
  int32_t *col_idx; /* device [cap_blk] */
  int64_t *blk_off; /* device [cap_blk] */
  double *values;   /* device [cap_nnz] */
  int64_t cap_blk, cap_nnz;
} bsm_dev_csr_out;

/* C = alpha * A.B with the on-the-fly filter, FP64, the result written into
 * C's caller buffers; the C pattern and values are the same as bsm_multiply's
 * with beta = 0. sizes (host, 3 words) receives {C blocks, C values, kept
 * products}. Calls no cudaMalloc, cudaFree or allocating library routine.
 * Every call looks up the device address of the scratch array on the current
 * device (cudaGetSymbolAddress, which allocates nothing); the first call on a
 * device also sets a kernel attribute there: make that first call before any
 * stream capture. Calls share the array: calls that overlap on the GPU race.
 * The call enqueues on `stream` (a cudaStream_t, NULL = legacy default) and
 * returns after the work is done.
 * The caller's device arrays are checked on the device before any kernel uses
 * them as indices: row_ptr[0] == 0, row_ptr non-decreasing, row_ptr[nbr] ==
 * nblk, column indices in [0, nbc) and strictly increasing within a row, block
 * sizes >= 1, block offsets >= 0, A's column sizes equal to B's row sizes.
 * Not checked (the library cannot see the allocations' sizes): each block's
 * values, blk_off[b] .. blk_off[b] + rows*cols, lie inside `values`.
 * Scratch use: about 24 bytes per block of A and of B, 56 per block row of A,
 * 20 per block of C's capacity cap_blk, and 8 per kept product; a generous
 * cap_blk therefore leaves less room for the products.
 * Errors: INVALID_ARG (malformed row pointers, unsorted or duplicate columns,
 * a block size below 1, a negative offset; also when C's capacities are too
 * small: sizes[] then holds what is needed), OUT_OF_RANGE (a column index
 * outside the block grid), DIM_MISMATCH, UNSUPPORTED (the problem needs more
 * scratch than BSM_NOALLOC_SCRATCH_BYTES), CUDA. */
int bsm_multiply_noalloc(double alpha, const bsm_dev_csr *A, const bsm_dev_csr *B, double eps,
                         bsm_dev_csr_out *C, int64_t *sizes, void *stream);

/* Wait for all work of the context and complete every pending result. */
int bsm_sync(bsm_ctx ctx);

/* Check of the bounded device-side wait the split-precision kernels use on
 * their copy barriers (an mbarrier in shared memory): one warp on the
 * context's stream waits on a barrier that its own lane 0 completes
 * (never_complete = 0: BSM_OK) or that nothing completes (never_complete = 1:
 * the wait gives up after its limit, about a second, and the call returns
 * BSM_ERR_TIMEOUT with the context still usable). Blocking. */
int bsm_selftest_wait(bsm_ctx ctx, int never_complete);

/* Static text for a BSM_* code. */
const char *bsm_strerror(int code);

/* Text of the last CUDA error seen by this thread ("" if none). */
const char *bsm_last_cuda_error(void);

#ifdef __cplusplus
}
#endif

#endif /* BSM_H */
