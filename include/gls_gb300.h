/*
 * gls_gb300.h -- C ABI of the GB300 (sm_103a) GWAS GLS library.
 *
 * The library computes the sequence of generalized least-squares problems of
 * Eq. 1 of Fabregat-Traver, Aulchenko and Bientinesi, "Solving Sequences of
 * Generalized Least-Squares Problems on Multi-threaded Architectures":
 *
 *     b_i := (X_i^T M^{-1} X_i)^{-1} X_i^T M^{-1} y,   1 <= i <= m,
 *
 * with X_i = (X_L | x_Ri) (Section 1), M an n x n SPD matrix, X_L the n x (p-1)
 * covariates shared by every problem, x_Ri one n x 1 SNP column and y the
 * phenotype.  The calls follow the two phases of Alg. 5 (hp-gwas) and Alg. 8
 * (ooc-hp-gwas): a setup that factors M and whitens X_L and y once
 * (Alg. 5 lines 1, 2, 4, 5, 6), then a loop over blocks of SNP columns
 * (Alg. 5 lines 3, 7-11; Alg. 8 lines 6-16).
 *
 * Conventions for every entry point
 *   - Matrices are column-major with an explicit leading dimension (the
 *     LAPACK convention of Table 1).
 *   - Pointers may be host memory (pageable or pinned) or device memory of the
 *     plan's device; the library finds out which with cudaPointerGetAttributes.
 *     The caller owns every input and output buffer.
 *   - No call throws, aborts or traps: each returns a gls_status_t, and
 *     gls_last_error() gives a one-line description of the last failure on
 *     the calling thread.
 *   - A plan is used by one host thread at a time.
 *   - Ordering of device inputs.  Every call reads its device inputs on the
 *     plan's compute stream (gls_plan_stream), a non-blocking stream that is
 *     not ordered after any stream of the caller.  The caller orders the work
 *     that produces those inputs before the call: either that work has
 *     finished (the producing stream was synchronized), or the caller records
 *     an event after it on the producing stream and passes the event to
 *     gls_plan_wait_event before the call.  Synchronizing some other stream
 *     (for instance a framework's current stream, when the inputs were made on
 *     a side stream) does not order them.
 *   - Lifetime of caller buffers.  Every input and output buffer stays
 *     allocated, and is not reused, until the call that reads or writes it has
 *     finished on the device: until it returns for the synchronous calls, and
 *     until the plan's stream has passed it for gls_solve_block on device
 *     buffers.  A stream-ordered allocator (for instance PyTorch's caching
 *     allocator) recycles a freed block on the stream that allocated it and
 *     knows nothing of the plan's stream.
 */
#ifndef GLS_GB300_H
#define GLS_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct gls_plan* gls_plan_t;

typedef enum {
  GLS_OK = 0,
  GLS_ERR_INVALID_ARG = 1,      /* a size, pointer or leading dimension is invalid          */
  GLS_ERR_NOT_SPD = 2,          /* M is not SPD; *info = 1-based failing pivot (potrf)      */
  GLS_ERR_OOM = 3,              /* device or pinned host allocation failed                  */
  GLS_ERR_CUDA = 4,             /* a CUDA runtime call failed (see gls_last_error)          */
  GLS_ERR_TIMEOUT = 5,          /* a bounded device wait gave up; the result is not valid   */
  GLS_ERR_STATE = 6,            /* call out of order (e.g. solve before factor)             */
  GLS_ERR_UNSUPPORTED = 7,      /* precision or device not supported by this build          */
  GLS_ERR_COVARIATES_SINGULAR = 8, /* X~_L^T X~_L not SPD; *info = 1-based failing pivot    */
  GLS_ERR_IO = 9                /* a genotype file could not be opened or read              */
} gls_status_t;

typedef enum {
  /* Every step in binary64 (the precision of the paper's MKL runs). */
  GLS_PREC_FP64 = 0,
  /* Mixed paths.  The n^2-per-SNP work of the blocked triangular solve runs
   * on tcgen05 tensor cores: each row of L^{-1}, left of its 4 x 4 diagonal
   * block, is held as split_terms 16-bit slices (a fixed-point integer part
   * under a per-row power of two, then floating-point remainders; BF16 or
   * FP16) and multiplied by the exact 16-bit genotype codes with FP32
   * accumulation.  The rest, and its arithmetic:
   *   - the factor of M (Cholesky, L^{-1}, whitening of X_L and y): binary64
   *     values from products of exact 8-bit integer slices on the tensor
   *     cores, each rounded once to binary64, with 64 x 64 diagonal leaves in
   *     binary64 arithmetic (GLS_FLAG_FACTOR_NATIVE: binary64 CUDA-core
   *     kernels throughout);
   *   - the 4 x 4 diagonal blocks of L^{-1}: an integer part (at most 12
   *     bits) under a per-row power of two plus an FP32 low part, together at
   *     least 36 bits of the row's diagonal-block scale, applied in FP32 with
   *     one rounding;
   *   - S_BR = x~^T x~: FP32 squares (each row rounded once) in a
   *     compensated FP32 sum per 128-row block, added across blocks in
   *     binary64;
   *   - S_BL and b_B: the same tensor-core products against the rows of
   *     W^T = (M^{-1} [X_L | y])^T (equal to X~_L^T x~ and y~^T x~ by
   *     associativity), scaled to binary64;
   *   - the p x p assembly and Cholesky solve: binary64.
   * b_i is within 1e-6 relative (2-norm) of the binary64 result on every
   * workload tested.  A GLS_PREC_MIXED_BF16 plan with n < 2048 uses FP16
   * slices instead: BF16 slices fall short of 1e-6 at small n, FP16 slices
   * carry three more bits each at the same tensor rate
   * (gls_plan_operand_precision reports which a plan uses). */
  GLS_PREC_MIXED_BF16 = 1,
  GLS_PREC_MIXED_FP16 = 2
} gls_precision_t;

/* Plan flags (gls_plan_desc_t.flags). */
/* Mixed paths only: split every entry of L^{-1} on its own in floating point
 * (hi/lo terms, no per-row fixed-point hi part).  FP32 accumulation of the hi
 * products is then inexact; kept to measure what the fixed-point hi part buys. */
#define GLS_FLAG_NAIVE_SPLIT 1u
/* Mixed paths factor M (Cholesky, L^{-1}, whitening) with binary64 products
 * evaluated exactly on the tensor cores (integer slices, see gls_factor); this
 * flag selects the plain binary64 CUDA-core kernels instead. */
#define GLS_FLAG_FACTOR_NATIVE 2u
/* FP64 path: factor M with the tensor-core binary64 products instead of the
 * default plain binary64 CUDA-core kernels. */
#define GLS_FLAG_FACTOR_TENSOR 4u
/* Launch every kernel directly.  By default a launch sequence that repeats
 * with the same arguments (the factor of M on a plan, one block of
 * gls_solve_block / gls_solve_stream, one gls_batch_solve round) is captured
 * as a CUDA graph the second time it is seen and replayed from then on (one
 * graph launch instead of up to ~1500 kernel launches for the factor).  Only
 * plans that own their stream (desc.stream == NULL) use graphs; results are
 * the same either way.  For a batch the flag of its first plan decides.
 * While such a call runs, nothing else may enqueue work on the plan's stream
 * (gls_plan_stream) from another thread: a capture would take it in. */
#define GLS_FLAG_EAGER 8u
/* Mixed paths: gls_solve_stream copies pinned int8 blocks to the device with
 * the copy engine (double-buffered on a side stream) instead of reading them
 * in place.  By default the conversion kernel reads each pinned block over the
 * host link itself: the copy engine's rate on this part falls several-fold
 * while kernels run, reading in place does not depend on it.  When the
 * columns start on 16-byte boundaries, block j+1 is then converted beside
 * the solve of block j, on 8 SMs that solve leaves free, into a second
 * operand buffer (2 x max_block_snps x npad bytes more device memory,
 * npad = n rounded up to 128, allocated on the first such call).  Results
 * are the same either way. */
#define GLS_FLAG_STAGED_INPUT 16u

/* Plan description.  Zero-initialise and fill the fields that matter. */
typedef struct {
  int64_t n;               /* number of observations (rows of M, X_L, y, x_Ri), n >= 1       */
  int32_t p;               /* unknowns per problem: cols(X_L) + 1, 1 <= p <= 32              */
  int32_t precision;       /* gls_precision_t                                                */
  int64_t max_block_snps;  /* largest k passed to gls_solve_block; sizes the workspaces      */
  int32_t device;          /* CUDA device ordinal                                            */
  int32_t split_terms;     /* mixed paths: operand slices of L^{-1}, 2 or 3 (0 = default 3)  */
  void* stream;            /* cudaStream_t for compute; NULL = the plan creates its own      */
  uint32_t flags;          /* GLS_FLAG_* bits; 0 for the defaults                            */
  int32_t wait_limit_us;   /* mixed paths: each pipeline wait of the tensor-core solve gives
                              up after this many microseconds (0 = 1 s); see below         */
  int32_t host_wait_ms;    /* each host wait of a call gives up after this many ms
                              (0 = no limit); see below                                    */
  int32_t phenotypes;      /* t: phenotypes per factor the plan holds (0 = 1);
                              p - 1 + t <= 32                                              */
  int32_t reserved[4];     /* must be 0                                                      */
} gls_plan_desc_t;

/*
 * Bounded waits.  Every wait inside the tensor-core kernels polls a clock and
 * gives up after a limit; the kernel then lets its in-flight copies and
 * products finish, frees its tensor memory and returns, so no kernel is left
 * running, and the call (or the next gls_synchronize, for an asynchronous
 * gls_solve_block) returns GLS_ERR_TIMEOUT.  Those results are not valid; the
 * plan stays usable and its next gls_factor clears the error.  wait_limit_us
 * shortens the limit of the blocked solve's waits (the default second is far
 * above any wait of a working pipeline; a short one is for tests of this path).
 * host_wait_ms bounds the host-side waits of gls_factor, the synchronous solve
 * calls, gls_batch_solve (first plan's value) and gls_synchronize: past it they return
 * GLS_ERR_TIMEOUT with the plan's work still queued, so the caller must call
 * gls_synchronize again (or gls_destroy, which always waits to the end) before
 * it reuses or frees any buffer of that call.  Copies between the device and
 * the caller's pageable host memory complete inside the CUDA runtime and are
 * not bounded by it.
 */

/*
 * Creates a plan and allocates its device workspaces (L, L^{-1}, whitened
 * covariates and phenotype, the two double-buffered X_R and b blocks, the
 * Gram partials).  *out receives the plan.  Errors: INVALID_ARG (bad
 * description), UNSUPPORTED (device is not sm_103), OOM, CUDA.
 */
gls_status_t gls_plan_create(const gls_plan_desc_t* desc, gls_plan_t* out);

/*
 * Setup phase of Alg. 5 (lines 1, 2, 4, 5, 6):
 *   L L^T = M (potrf); X~_L = L^{-1} X_L; y~ = L^{-1} y;
 *   S_TL = X~_L^T X~_L; b_T = X~_L^T y~ (Fig. 1), all in binary64.
 * Two implementations give binary64 results: plain FP64 kernels, and (default
 * for the mixed paths, see GLS_FLAG_FACTOR_*) a recursive Cholesky with
 * inverse whose dense products are split into exact 8-bit integer slices and
 * summed exactly on the tensor cores, rounded once to binary64; only its
 * 64 x 64 diagonal blocks use FP64 arithmetic.
 * M   n x n (ldm >= n), only the lower triangle is read.  M == NULL keeps the
 *     factor of the previous call (a new phenotype for the same M).
 * XL  n x (p-1) (ldxl >= n); NULL when p == 1.  With M == NULL, XL == NULL
 *     also keeps the previous X~_L.
 * y   n.
 * info (may be NULL) receives 0, or the 1-based failing pivot when the
 *     status is NOT_SPD or COVARIATES_SINGULAR.
 * Synchronous: returns when the setup has finished on the device.
 */
gls_status_t gls_factor(gls_plan_t plan, const double* M, int64_t ldm, const double* XL,
                        int64_t ldxl, const double* y, int64_t* info);

/*
 * gls_factor for several phenotypes at once: Eq. 1 with the index
 * 1 <= j <= t that the paper comments out, b_ij = (X_i^T M^{-1} X_i)^{-1}
 * X_i^T M^{-1} y_j.  The Gram matrix S_i and its Cholesky factor do not
 * depend on j, so one pass of the blocked solve over X_R serves all t
 * right-hand sides: the whitened block becomes [X~_L | Y~], b_T a
 * (p-1) x t block, and each SNP gets t values b_B_ij = y~_j^T x~_i.
 * Y   n x t (ldy >= n), 1 <= t <= desc.phenotypes.  M, XL and info as for
 *     gls_factor (M == NULL keeps the factor: new phenotypes for the same M).
 * Until the next gls_factor[_y], the SNP calls write b_ij to column
 * i t + j (0-based) of their B (p x (k t)): the t vectors of a SNP are adjacent.
 * gls_factor is gls_factor_y with t = 1 and ldy = n.
 */
gls_status_t gls_factor_y(gls_plan_t plan, const double* M, int64_t ldm, const double* XL,
                          int64_t ldxl, const double* Y, int64_t ldy, int32_t t,
                          int64_t* info);

/*
 * One block of the SNP loop (Alg. 5 lines 3 and 7-11): for the k SNP columns
 * of XR, x~_i = L^{-1} x_Ri (blocked triangular solve), the Gram entries
 * S_BL_i = X~_L^T x~_i, S_BR_i = x~_i^T x~_i, b_B_i = y~^T x~_i, and
 * b_i = S_i^{-1} (b_T; b_B_i) by a Cholesky solve of the p x p system.
 * XR  n x k int8 genotype codes (ldxr >= n); every int8 value is accepted.
 * B   p x k binary64 output (ldb >= p): X_L coefficients first, SNP last;
 *     p x (k t) after gls_factor_y with t phenotypes (column i t + j).
 * snp_status (may be NULL) k int32: 0, or 1 when S_i is not numerically SPD
 *     (its last pivot d <= tau * S_BR_i with tau = 2^-30 for FP64 and 2^-16
 *     for the mixed paths); that b_i is NaN and the call still returns OK.
 * 0 <= k <= max_block_snps.  With every pointer in device memory the call is
 * asynchronous on the plan's stream; with any host pointer it copies and
 * returns after the block is complete.  Errors: STATE (no successful
 * gls_factor yet), INVALID_ARG, CUDA, TIMEOUT.
 */
gls_status_t gls_solve_block(gls_plan_t plan, const int8_t* XR, int64_t ldxr, int64_t k,
                             double* B, int64_t ldb, int32_t* snp_status);

/*
 * The whole SNP stream of Alg. 8 (ooc-hp-gwas): XR holds m SNP columns in host
 * memory (pinned for full overlap; pageable is staged through pinned
 * buffers).  Blocks of up to max_block_snps columns are double-buffered: the
 * copy of block j+1 to the device runs on a side stream while block j is
 * solved, and b of block j is copied back while block j+1 is solved
 * (Section 4.2).  Mixed plans read pinned int8 input in place instead (see
 * GLS_FLAG_STAGED_INPUT).  The first block of host input is smaller so that
 * its unoverlapped load is short (Section 4.3).  B (p x m, or p x (m t) with
 * t phenotypes; ldb >= p) and snp_status (m, may be NULL) are host or device
 * memory.  Synchronous.  Device-resident XR is also accepted: blocks are then
 * max_block_snps columns throughout and only host outputs are copied.
 */
gls_status_t gls_solve_stream(gls_plan_t plan, const int8_t* XR, int64_t ldxr, int64_t m,
                              double* B, int64_t ldb, int32_t* snp_status);

/*
 * gls_solve_block and gls_solve_stream with the genotype codes packed four to
 * a byte, a quarter of the host-to-device bytes of int8 input (the blocked
 * solve of Alg. 5 line 3 on X_R as stored; the storage format is not the
 * paper's, which reads binary64 blocks).  Column j of XP holds ceil(n/4)
 * bytes (ldxp >= ceil(n/4)); genotype i is the 2-bit code in bits
 * 2 (i mod 4) .. 2 (i mod 4) + 1 of byte floor(i/4) of its column (the first
 * sample in the lowest bits), read as the value 0, 1, 2 or 3 (no code means
 * "missing": 2-bit files whose codes mean something else, such as formats
 * with a missing-call code, must be recoded first).  The mixed
 * paths of the stream convert the packed codes straight to their tensor-core
 * operand; otherwise a block is unpacked on the device into the plan's int8
 * staging and solved as an int8 block.  Either way the results equal those of
 * the int8 calls on the same values, bit for bit.  XP may
 * be device, pinned or pageable memory; B and snp_status as for the int8
 * calls.  The first call allocates 2 x ceil(n/4) x max_block_snps bytes of
 * device staging (and as much pinned host memory for pageable input to the
 * stream); an allocation failure returns OOM.  Errors otherwise as for the
 * int8 calls.
 */
gls_status_t gls_solve_block_packed(gls_plan_t plan, const uint8_t* XP, int64_t ldxp, int64_t k,
                                    double* B, int64_t ldb, int32_t* snp_status);
gls_status_t gls_solve_stream_packed(gls_plan_t plan, const uint8_t* XP, int64_t ldxp,
                                     int64_t m, double* B, int64_t ldb, int32_t* snp_status);

/*
 * The disk tier of Alg. 8 (ooc-hp-gwas): the SNP stream read from a file.
 * The file holds m genotype columns from byte `offset` on, column j at
 * offset + j ldx: int8 codes (packed == 0, ldx >= n) or the 2-bit layout of
 * gls_solve_block_packed (packed != 0, ldx >= ceil(n/4)).  Blocks follow the
 * schedule of gls_solve_stream (a short first block, then doubling, Section
 * 4.3).  A background thread reads them with parallel pread calls into a ring
 * of three pinned slots, up to two blocks ahead of the GPU (the async_read of
 * Alg. 8), and the GPU takes each block from its slot as from pinned input to
 * gls_solve_stream.  The slots (3 x ldx x max_block_snps bytes of pinned host
 * memory) stay with the plan for later calls.  B and snp_status as for
 * gls_solve_stream.  Synchronous.  Errors: GLS_ERR_IO when the file cannot be
 * opened, is shorter than offset + m ldx bytes, or a read fails; otherwise
 * as for gls_solve_stream.
 */
gls_status_t gls_solve_file(gls_plan_t plan, const char* path, int64_t offset, int32_t packed,
                            int64_t ldx, int64_t m, double* B, int64_t ldb,
                            int32_t* snp_status);

/*
 * Batched uneven scans: several independent sequences (each its own plan, with
 * its own M, n, p and SNP block) solved by ONE persistent launch of the
 * mixed-precision blocked solve, so that small scans fill the GPU together.
 * All plans must be mixed-precision plans (BF16 and FP16 may be mixed) with
 * the same split_terms, live on the same device, and be factored before
 * gls_batch_solve.  At most 64
 * plans.  The batch keeps pointers to the plans; destroy it before them.
 */
typedef struct gls_batch* gls_batch_t;

gls_status_t gls_batch_create(const gls_plan_t* plans, int32_t nplans, gls_batch_t* out);

/*
 * One block per plan, all in one launch: plan i solves k[i] SNP columns of
 * XR[i] (device memory, n_i x k[i] int8, ldxr[i] >= n_i) into B[i] (device,
 * p_i x (k[i] t_i) for its t_i phenotypes, ldb[i] >= p_i) and snp_status[i]
 * (device, may be NULL; the array
 * snp_status itself may be NULL).  0 <= k[i] <= max_block_snps of plan i.
 * group: pairs of 128-row blocks per L2 rasterization group of the launch (0 = default 3;
 * a tuning knob only, results do not depend on it).  Runs on the first plan's
 * stream after the work already queued on every plan's stream, and returns
 * when the launch has finished.  Errors: INVALID_ARG, STATE, CUDA, TIMEOUT.
 */
gls_status_t gls_batch_solve(gls_batch_t batch, const int8_t* const* XR, const int64_t* ldxr,
                             const int64_t* k, double* const* B, const int64_t* ldb,
                             int32_t* const* snp_status, int32_t group);

gls_status_t gls_batch_destroy(gls_batch_t batch);

/* Waits for all work of the plan (all its streams).  */
gls_status_t gls_synchronize(gls_plan_t plan);

/* The plan's compute stream (a cudaStream_t), for callers that order their
 * own work after an asynchronous gls_solve_block. */
void* gls_plan_stream(gls_plan_t plan);

/*
 * Orders the plan's later work after `event` (a cudaEvent_t the caller
 * recorded on the stream that produced the inputs of its next calls): the
 * plan's compute stream waits for it on the device; the host does not block.
 * It has no counterpart in the paper, whose inputs come from disk.
 * Errors: INVALID_ARG (NULL plan or event), CUDA.
 */
gls_status_t gls_plan_wait_event(gls_plan_t plan, void* event);

/* The gls_precision_t of the plan's tensor-core operands: its description's
 * precision, except GLS_PREC_MIXED_FP16 for a GLS_PREC_MIXED_BF16 plan with
 * n < 2048.  -1 for a NULL plan. */
int32_t gls_plan_operand_precision(gls_plan_t plan);

/* Frees every resource of the plan (after waiting for its work).  NULL is OK. */
gls_status_t gls_destroy(gls_plan_t plan);

/* Device bytes a plan with this description allocates at creation (0 for an
 * invalid one); a mixed plan's first in-place int8 stream adds a second
 * operand buffer (see GLS_FLAG_STAGED_INPUT). */
size_t gls_plan_footprint_bytes(const gls_plan_desc_t* desc);

/* Static, NUL-terminated name of a status code. */
const char* gls_status_string(gls_status_t status);

/* One-line description of the last failure on the calling thread ("" if none). */
const char* gls_last_error(void);

/*
 * Device-time accounting for benchmarks.  With timing enabled, each kernel of
 * the SNP loop and each whole setup phase is bracketed by CUDA events on the
 * plan's stream, so the figures are the kernels' own device times, and each
 * host<->device block copy of gls_solve_stream[_packed] by events on its side
 * stream; launches counts every kernel the plan enqueued.
 * gls_plan_set_timing resets the counters; gls_plan_stats synchronizes the
 * plan's streams and sums.
 */
typedef struct {
  int64_t launches;          /* kernels enqueued since the last reset                 */
  double trsm_ms;            /* blocked triangular solve + Gram epilogue kernels     */
  int64_t trsm_launches;
  double convert_ms;         /* int8 -> 16-bit genotype operand kernels (mixed)      */
  int64_t convert_launches;
  double solve_ms;           /* p x p assembly + Cholesky solve kernels              */
  int64_t solve_launches;
  double factor_ms;          /* whole gls_factor setup phases                        */
  int64_t factor_calls;
  /* genotype blocks copied host -> device and b blocks device -> host by the
   * stream calls, each copy timed on its side stream (while overlapped) */
  double h2d_ms;
  int64_t h2d_bytes;
  int64_t h2d_copies;
  double d2h_ms;
  int64_t d2h_bytes;
  int64_t d2h_copies;
} gls_stats_t;

gls_status_t gls_plan_set_timing(gls_plan_t plan, int32_t enable);
gls_status_t gls_plan_stats(gls_plan_t plan, gls_stats_t* out);

/*
 * Allocation-free FP64 block solve, for callers that cannot call cudaMalloc
 * (code whose device memory belongs to another allocator, such as a
 * framework's caching pool, or loops that must not enter the driver's
 * allocator).  It has no counterpart in the paper: it is gls_solve_block's
 * binary64 path with every buffer supplied by the caller.
 *
 * All pointers are device memory of the current device; the call is
 * asynchronous on `stream` (a cudaStream_t, NULL = legacy default stream).
 *   Zinv  n x n, ldz >= n: L^{-1} with L L^T = M; only the lower triangle is read.
 *   W     n x p, ldw >= n: [L^{-1} X_L | L^{-1} y].
 *   RTL   (p-1) x (p-1) column-major lower Cholesky factor of W[:,0:p-1]^T W[:,0:p-1];
 *   zT    p-1: RTL^{-1} W[:,0:p-1]^T W[:,p-1].  Both may be NULL when p == 1.
 *   XR, B, snp_status as for gls_solve_block (snp_status may be NULL).
 * The only scratch is a 4 MiB array inside the library; every GPU that loads
 * the library holds its own copy until the process exits.  ceil(n/64) *
 * (p+1) * k must not exceed 524288, otherwise GLS_ERR_INVALID_ARG (see
 * gls_last_error).  The first call on a device looks up that device's copy
 * (and again after a device reset, which moves it); make that call before any
 * stream capture.  Calls on the same device share its copy, which keeps the
 * last call's contents: calls whose work can overlap on that GPU (other
 * streams, other threads) race and must be ordered by the caller.  Calls on
 * different devices use different copies.  Nothing is allocated or freed.
 */
gls_status_t gls_solve_block_fp64_static(int64_t n, int32_t p, const double* Zinv, int64_t ldz,
                                         const double* W, int64_t ldw, const double* RTL,
                                         const double* zT, const int8_t* XR, int64_t ldxr,
                                         int64_t k, double* B, int64_t ldb,
                                         int32_t* snp_status, void* stream);

/*
 * Copies the factor of the last successful gls_factor: L (n x n lower
 * triangular, zeros above the diagonal, ldl >= n) and Zinv = L^{-1} (same
 * shape, ldz >= n).  Either pointer may be NULL; host or device memory.
 * Synchronous.  Errors: STATE (no factor yet), INVALID_ARG, CUDA.
 */
gls_status_t gls_plan_get_factor(gls_plan_t plan, double* L, int64_t ldl, double* Zinv,
                                 int64_t ldz);

/*
 * The paper's comparison algorithms for a sequence of GLS problems
 * (Section 2), as binary64 GPU paths for the cost comparison of Table 2:
 *   GLS_ALG_BLACK_BOX (Alg. 3): each problem solved on its own (Cholesky of M,
 *     whitening of X_i = (X_L | x_Ri) and y, X_i^T X_i, X_i^T y, posv):
 *     about n^3 / 3 flops per problem;
 *   GLS_ALG_SEQ_GLS (Alg. 4): the Cholesky of M and y~ once, then per problem
 *     the whitening of the whole X_i: about n^2 p flops per problem;
 *   GLS_ALG_HP_GWAS (Alg. 5): this library's path (gls_factor +
 *     gls_solve_block in blocks of max_block_snps): about n^2 per problem;
 *   GLS_ALG_GWFGLS (Alg. 6, GenABEL's gwfgls): the explicit inverse M^{-1} and
 *     W_L = M^{-1} X_L once, then per problem w = M^{-1} x_Ri with the full
 *     inverse, S_i = (W_L | w)^T X_i formed without its symmetry, and an LU
 *     solve (gesv): about 2 n^2 per problem.
 * Triangular solves with L are applied as products with L^{-1}, which costs
 * the same.  Every path gives b_i of Eq. 1 (B p x k, ldb >= p; snp_status k,
 * may be NULL, 1 where S_i is singular and b_i NaN).  The plan must be a
 * binary64 plan with one phenotype and, except for Alg. 5, p <= 8.  All
 * pointers are device memory (M n x n, X_L n x (p-1), y n, X_R n x k int8).
 * The call is synchronous and allocates its own workspace (cudaMalloc).
 * Alg. 3, 4 and 6 overwrite the plan's factor and leave it without one
 * (gls_factor again before gls_solve_block); Alg. 5 leaves its factor.
 * Errors: INVALID_ARG, NOT_SPD, OOM, CUDA.
 */
typedef enum {
  GLS_ALG_BLACK_BOX = 3,
  GLS_ALG_SEQ_GLS = 4,
  GLS_ALG_HP_GWAS = 5,
  GLS_ALG_GWFGLS = 6
} gls_algorithm_t;

gls_status_t gls_solve_variant(gls_plan_t plan, int32_t algorithm, const double* M, int64_t ldm,
                               const double* XL, int64_t ldxl, const double* y,
                               const int8_t* XR, int64_t ldxr, int64_t k, double* B,
                               int64_t ldb, int32_t* snp_status);

/* Library version as major*10000 + minor*100 + patch. */
int32_t gls_version(void);

#ifdef __cplusplus
}
#endif

#endif /* GLS_GB300_H */
