/*
 * loops.h -- C ABI of the GB300 (sm_103a) LOOPS hybrid SpMM library, libloops.so.
 *
 * The operation is SpMM, C = A . B, with A sparse (CSR on input) and B dense with N columns
 * (Sec. 2.1: c_ij = sum_k a_ik b_kj). A plan splits A into a row-wise CSR part and a
 * vector-wise BCSR part of B_r x 1 tiles (the LOOPS format, Sec. 3.2.1; conversion,
 * Algorithm 1), and the SpMM runs both parts on one GPU: the CSR part on CUDA cores (the
 * AXPY row kernel of Sec. 3.3), the BCSR part on tensor cores (the outer-product tile kernel,
 * Algorithms 2 and 3) -- FP64 DMMA, FP16/BF16 MMA with FP32 accumulation -- or, for FP32, on a
 * register-blocked CUDA-core outer product. Each output row has exactly one writer, so the
 * result is deterministic and needs no atomics (Sec. 3.4).
 *
 * Conventions shared by every entry point:
 *  - Errors are returned as loops_status, never by aborting; loops_last_error() gives a
 *    thread-local message for the last failing call of the calling thread.
 *  - "device" pointers are CUDA global-memory pointers of the current device; "host"
 *    pointers are ordinary CPU memory. Dense matrices are row-major with a leading
 *    dimension (elements between consecutive rows), ld >= number of columns.
 *  - Every GPU call is ordered on the given stream (NULL = legacy default stream) and does
 *    not synchronise the device unless its comment says so.
 *  - Element types per plan dtype:
 *        dtype      A values stored   B, dC      C, dB, dvals   accumulation
 *        LOOPS_F64  f64               f64        f64            f64 (DFMA / DMMA)
 *        LOOPS_F32  f32               f32        f32            f32 (FFMA)
 *        LOOPS_F16  f16 (x s_A)       f16        f32            f32 (HMMA)
 *        LOOPS_BF16 bf16 (x s_A)      bf16       f32            f32 (HMMA)
 *    s_A is a power-of-two plan scale (max|a| * s_A <= 2^14) that the epilogue divides out
 *    exactly; the 16-bit dense operands may carry per-column power-of-two scales.
 *  - Inputs must be finite: a zero slot of a BCSR tile multiplies its B row, and 0 * inf
 *    is NaN under IEEE 754.
 */
#ifndef LOOPS_H
#define LOOPS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* A cudaStream_t (struct CUstream_st*); NULL means the legacy default stream. */
typedef struct CUstream_st* loops_stream_t;

typedef enum {
  LOOPS_OK = 0,
  LOOPS_ERR_INVALID_ARG = 1,  /* null pointer, negative size, bad leading dimension, ... */
  LOOPS_ERR_INVALID_CSR = 2,  /* row_ptr not monotone / wrong ends, column out of range  */
  LOOPS_ERR_UNSUPPORTED = 3,  /* dtype or size the library does not handle              */
  LOOPS_ERR_OOM = 4,          /* a host or device allocation failed                     */
  LOOPS_ERR_CUDA = 5,         /* a CUDA runtime call failed (message in last_error)     */
  LOOPS_ERR_TIMEOUT = 6,      /* a bounded device-side wait gave up (see loops_plan_check) */
  LOOPS_ERR_STATE = 7         /* destroyed / mismatched plan, or wrong call order       */
} loops_status;

typedef enum { LOOPS_F64 = 0, LOOPS_F32 = 1, LOOPS_F16 = 2, LOOPS_BF16 = 3 } loops_dtype;

/* Sparse input A in CSR form; the arrays are borrowed only for the call and live on the HOST
 * (loops_plan, loops_partition_host, loops_plan_batched) or on the DEVICE (loops_plan_device).
 * row_ptr: int64[n_rows + 1], row_ptr[0] = 0, non-decreasing, row_ptr[n_rows] = nnz.
 * col_idx: int32[nnz], 0 <= col < n_cols; columns may be unsorted and may repeat (repeats
 *          are summed). vals: nnz values of type vals_dtype (LOOPS_F64 or LOOPS_F32). */
typedef struct {
  int64_t n_rows;
  int64_t n_cols;
  int64_t nnz;
  const int64_t* row_ptr;
  const int32_t* col_idx;
  const void* vals;
  loops_dtype vals_dtype;
} loops_csr;

/* Plan options; loops_plan_opts_default() fills the defaults.
 * tau: split threshold on row-block density d = nnz_rb / distinct columns of the block
 *      (nnz per B_r x 1 tile, the paper's block density, Sec. 4.2/4.5). A block with
 *      nnz_rb >= tau * distinct_cols goes to the BCSR part. LOOPS_TAU_MODEL (-2): the
 *      performance model picks tau (see LOOPS_TAU_MODEL). Other tau < 0: autotune (time
 *      candidate thresholds on the plan's stream, the L2 flushed before each timed call;
 *      for F32 with block_rows 0 also B_r 8 and 16; then, on the chosen split, the CSR
 *      kernel's vectors per lane and the F16/BF16 BCSR kernel's columns per CTA -- reported
 *      by loops_plan_info); +inf: CSR only (the pure vector-unit configuration of Sec. 4.3);
 *      0: every non-empty block BCSR (pure matrix unit).
 * block_rows: B_r (tile height); 0 = default (8 for F64, 16 otherwise; F32 autotuning tries
 *      both); F64 needs 8, F16/BF16 need 16, F32 accepts 8 or 16.
 * contiguous_split: paper mode (Eq. 1, Algorithm 1): rows [0, r_boundary) rounded up to a
 *      multiple of B_r form the CSR part and every later row block is BCSR; tau ignored.
 *      r_boundary < 0 derives it from Eq. 1: the all-CSR and all-BCSR plans are timed on the
 *      plan's stream (synchronised), each part's throughput is TP = rows / time, and
 *      r_boundary / TP_csr = (n_rows - r_boundary) / TP_bcsr balances the two parts' times.
 * want_backward: also build the transposed plan and keep A's pattern so that
 *      loops_spmm_backward works.
 * tile_min: tile-level split inside BCSR blocks (the dense/sparse-region idea the paper cites,
 *      Sec. 5): tiles holding fewer than tile_min stored entries leave the block, and their
 *      entries join the CSR part, whose rows then add to the C rows the BCSR part wrote
 *      (after it, in a fixed order). 0 or 1: off; -1: the autotuner (tau < 0) also tries 2.
 *      Not available together with want_backward or in batched plans. */
typedef struct {
  double tau;
  int32_t block_rows;
  int32_t contiguous_split;
  int64_t r_boundary;
  int32_t want_backward;
  int32_t split_len;      /* CSR rows longer than this are split in segments; 0 = default */
  int32_t tile_min;
  int32_t reserved[5];
} loops_plan_opts;

typedef struct loops_plan_s* loops_plan_t;

/* tau value selecting the performance model (Sec. 3.5, Eq. 2 and Eq. 3, restated for the GPU):
 * warm-up plans at a few thresholds are timed, the quadratic of Eq. 2 is fitted to their
 * throughput as a function of the CSR-part and BCSR-part work, and the threshold of highest
 * predicted throughput (Eq. 3) is used -- among +inf, 0 and the matrix's block densities. */
#define LOOPS_TAU_MODEL (-2.0)

/* Counts describing a plan (loops_plan_info). */
typedef struct {
  loops_dtype dtype;
  int32_t block_rows;      /* B_r */
  int32_t k_pad;           /* tiles per block are padded to a multiple of this (MMA K) */
  int32_t has_backward;
  int64_t n_rows, n_cols, nnz, N;
  double tau;              /* threshold actually used (after autotuning) */
  double scale;            /* s_A */
  int64_t n_csr_rows, nnz_csr;
  int64_t n_row_blocks, n_tiles, nnz_bcsr;  /* n_tiles includes padding tiles */
  int64_t n_split_rows, n_segments;
  int64_t n_subnormal_vals;/* stored 16-bit A values that are subnormal */
  int64_t device_bytes;    /* device memory owned by the plan */
  int64_t r_boundary;      /* paper mode: the boundary used (Eq. 1 when derived); else -1 */
  int64_t tile_min;        /* tile-level split threshold in effect (0: off) */
  int32_t tau_source;      /* 0 given, 1 timed autotuner, 2 performance model (Eq. 2/3),
                              3 contiguous split (paper mode) */
  int32_t csr_lane_vectors;/* CSR kernel: 16-byte column vectors per lane the autotuner chose
                              (1 or 2); 0: the built-in rule */
  int32_t bcsr_col_tile;   /* F16/BF16 BCSR kernel: columns per CTA the autotuner chose (32, 64,
                              128); 0: the smallest tile covering N */
  int32_t reserved0;
  double model_gflops;     /* tau_source 2: the Eq. 2 prediction for the chosen split; else NaN */
  double model_coef[5];    /* tau_source 2: the fitted a0..a4 of Eq. 2 */
} loops_plan_info;

/* Canonical partition (host arrays, malloc'ed by the library; release with
 * loops_partition_free). csr_rows ascending; each CSR row keeps its entries in input order.
 * rb_ids ascending; tiles of a block ordered by column; tile t of block b holds rows
 * b*B_r .. b*B_r+B_r-1 in tile_val[t*B_r ...]; padding tiles have tile_col = -1 and zero
 * values. Values are the stored (rounded, s_A-scaled) values converted to f64. */
typedef struct {
  int64_t n_rows, n_cols;
  int32_t block_rows, k_pad;
  double scale;
  int64_t n_csr_rows, nnz_csr, n_row_blocks, n_tiles;
  int32_t* csr_rows;
  int64_t* csr_ptr;
  int32_t* csr_col;
  double* csr_val;
  int32_t* rb_ids;
  int64_t* rb_ptr;
  int32_t* tile_col;
  double* tile_val;
} loops_partition;

/* ---------------------------------------------------------------------------------------- */

/* Library version (major * 10000 + minor * 100 + patch). */
int32_t loops_version(void);

/* Static description of a status code. */
const char* loops_status_str(loops_status status);

/* Thread-local message of the last failing call on this thread ("" if none). */
const char* loops_last_error(void);

/* Fill *opts with defaults: tau = 2.0, block_rows = 0, no contiguous split, no backward,
 * tile_min = -1 (tile split only considered when autotuning). */
void loops_plan_opts_default(loops_plan_opts* opts);

/* Host-only partition of A (Algorithm 1 with the structural split) -- no GPU needed.
 * Produces exactly the arrays loops_plan would upload (in canonical order). tau must be
 * >= 0 (no autotuning here). *out must be released with loops_partition_free. */
loops_status loops_partition_host(const loops_csr* A, loops_dtype dtype,
                                  const loops_plan_opts* opts, loops_partition* out);

/* Release the arrays of a partition filled by loops_partition_host / loops_plan_export. */
void loops_partition_free(loops_partition* part);

/* Build a plan for C = A . B with B of N columns in `dtype` (Sec. 3.1 pipeline: choose the
 * split, convert with Algorithm 1, upload). Validates A (LOOPS_ERR_INVALID_CSR). The plan
 * owns all device memory it allocates. With tau < 0 the call times candidate splits on
 * `stream` and synchronises it. On success *out is a new plan; on failure *out is NULL. */
loops_status loops_plan(const loops_csr* A, int64_t N, loops_dtype dtype,
                        const loops_plan_opts* opts, loops_stream_t stream, loops_plan_t* out);

/* Build the same plan as loops_plan from a matrix whose CSR arrays are in DEVICE memory,
 * with every step of the conversion run on the GPU on `stream`: validation, row-block
 * analysis (nnz_rb, distinct columns), the split (Sec. 3.1, Algorithm 1 with the structural
 * or the contiguous Eq. 1 boundary, and the tile-level split), and the packing of both parts
 * (stable radix sorts by (row block, column), so tiles come out in ascending column order
 * and duplicates are summed in input order). The plan equals loops_plan's on the same
 * matrix bit for bit (loops_plan_export) and runs on the same kernels. For re-planning when
 * the pattern changes between calls (dynamic graphs, Sec. 4.5): the matrix never travels to
 * the host. The paper builds its format on the CPU; this on-device build has no counterpart
 * there. Arguments as loops_plan, except: A->row_ptr, A->col_idx and A->vals are device
 * pointers, borrowed for the call. Validation errors are those of loops_plan (the first bad
 * row or entry is reported). The call synchronises `stream` (it reads back a few totals);
 * with tau < 0 it autotunes exactly as loops_plan does. Plans built here (unless they use the
 * tile-level split) also accept loops_plan_set_values without want_backward;
 * loops_plan_update_values refreshes them through the same device maps. */
loops_status loops_plan_device(const loops_csr* A, int64_t N, loops_dtype dtype,
                               const loops_plan_opts* opts, loops_stream_t stream, loops_plan_t* out);

/* Test hook for the error paths (not for production use): the n-th device or pinned-host
 * allocation the library makes from now on (n >= 1) fails as if memory were exhausted, and the
 * call that made it returns LOOPS_ERR_OOM after releasing what it had allocated; n <= 0 disarms.
 * Returns the number of allocations made since the previous call of this hook, so a test can
 * count the allocations of an operation first and then fail each of them in turn. The paper
 * has no counterpart. Process-wide; not meant to be armed while other threads build plans. */
int64_t loops_test_fail_alloc(int64_t n);

/* Test hook for the bounded waits (not for production use): kernels launched from now on give
 * up each shared-memory barrier wait of the F16/BF16 BCSR kernel after `polls` unsuccessful
 * polls (0: at once), instead of the default 2^24. A wait that gives up sets the plan's error
 * word (loops_plan_check then returns LOOPS_ERR_TIMEOUT), lets the copies already in flight
 * into its CTA's shared memory land (with its own bound), and skips that CTA's store: the C
 * rows of its block are then not written (or, for a block cut into several units, are summed
 * from partials this call did not write) and must not be used. polls < 0 restores the
 * default. Returns
 * the previous limit. Process-wide. The paper has no counterpart: it is the failure-detection
 * path of the GPU kernels, exercised without faulting or hanging the device. */
int64_t loops_test_wait_limit(int64_t polls);

/* The performance model of Sec. 3.5 restated for the GPU (host only, no device access).
 * Eq. 2: f(x, y) = a0 + a1 x + a2 y + a3 x^2 + a4 y^2, where x is the CSR-part work (stored
 * entries of the CSR part x N) and y the BCSR-part work (tiles x B_r x N, padding included)
 * of a split. loops_perf_model_fit computes the five coefficients coef[0..4] by least squares
 * over n samples (x[i], y[i], f[i]); samples on a line (one matrix, whose x and y move
 * together) still give a solution (a tiny ridge). LOOPS_ERR_STATE if the system has no finite
 * solution. loops_perf_model_argmax is Eq. 3: the index of the candidate (x[i], y[i]) of
 * highest predicted f, and that prediction. The library's plans fit f to the measured time
 * and take the highest predicted throughput (flops / predicted time): with tau =
 * LOOPS_TAU_MODEL (loops_plan) and in the batched autotuner. */
loops_status loops_perf_model_fit(const double* x, const double* y, const double* perf, int32_t n, double* coef);
loops_status loops_perf_model_argmax(const double* coef, const double* x, const double* y, int32_t n,
                                     int32_t* best, double* best_perf);

/* Release a plan and its device memory (synchronises the device first). NULL is a no-op. A
 * handle that is not a live plan (never returned, or already destroyed) gives
 * LOOPS_ERR_STATE here and in every other call, without its memory being read. */
loops_status loops_plan_destroy(loops_plan_t plan);

/* Counts of the plan (host only, no GPU work). */
loops_status loops_plan_info_get(loops_plan_t plan, loops_plan_info* out);

/* Copy the plan's device arrays back and return them in canonical order (synchronises). */
loops_status loops_plan_export(loops_plan_t plan, loops_partition* out);

/* Replace A's values (same pattern as at plan time; host array of nnz values of
 * vals_dtype, input order) and re-upload both parts (and the transposed plan). The plan
 * scale s_A is kept; values are rounded into the plan dtype. Synchronises `stream`. */
loops_status loops_plan_update_values(loops_plan_t plan, const void* vals, loops_dtype vals_dtype,
                                      loops_stream_t stream);

/* Replace A's values from a DEVICE array (nnz values of vals_dtype, F64 or F32, in A's input
 * order; same pattern) for a plan built with want_backward (or by loops_plan_device without
 * the tile-level split): both parts and the transposed
 * plan are refreshed by a kernel on `stream` (stored value = round(s_A * sum of the entries
 * of a slot, in input order), exactly as the host packer rounds). Stream-ordered; used by
 * the autograd path so that C = A(vals) . B follows the current values. */
loops_status loops_plan_set_values(loops_plan_t plan, const void* vals, loops_dtype vals_dtype,
                                   loops_stream_t stream);

/* C = A . B. B: device, n_cols x N (row-major, ldb); C: device, n_rows x N (ldc); element
 * types per the table above. Overwrites C (no accumulation into it). Stream-ordered. */
loops_status loops_spmm(loops_plan_t plan, const void* B, int64_t ldb, void* C, int64_t ldc,
                        loops_stream_t stream);

/* As loops_spmm, for the 16-bit dtypes with per-column scales: B holds B'[:, j] = B[:, j] / s_j
 * and col_scale (device, f32[N], or NULL for all ones) holds s_j; the epilogue writes
 * C[:, j] = s_j * (A . B')[:, j]. For F64/F32 col_scale must be NULL. */
loops_status loops_spmm_scaled(loops_plan_t plan, const void* B, int64_t ldb,
                               const float* col_scale, void* C, int64_t ldc, loops_stream_t stream);

/* End-to-end SpMM with HOST buffers: copies B (host, ideally pinned) to plan-owned device
 * memory, runs loops_spmm, copies C back to host, and synchronises `stream` before
 * returning. The staging buffers are allocated on the first call and kept by the plan. (The
 * paper's method runs on CPU cores, Sec. 3, where the operands need no transfer; this call
 * has no counterpart there.) */
loops_status loops_spmm_host(loops_plan_t plan, const void* B_host, int64_t ldb, void* C_host,
                             int64_t ldc, loops_stream_t stream);

/* Pipelined end-to-end SpMM with HOST buffers, for a sequence of calls: like loops_spmm_host,
 * but it does not wait. Two plan-owned staging sets alternate between calls; B comes in on one
 * internal stream and C goes back on another, so the copy-in of call k+1 and the SpMM of call
 * k+1 (on `stream`) overlap the copy-out of call k. The C_host of every call made so far is
 * complete once loops_spmm_host_flush(plan, stream) has been called and `stream` has then been
 * synchronised; B_host and C_host must stay valid and unchanged until then. Calls on one plan
 * must use the same `stream`. */
loops_status loops_spmm_host_async(loops_plan_t plan, const void* B_host, int64_t ldb, void* C_host,
                                   int64_t ldc, loops_stream_t stream);

/* Make `stream` wait for the copy-out of the last loops_spmm_host_async call on this plan
 * (stream-ordered, no host wait). No counterpart in the paper, as for loops_spmm_host. */
loops_status loops_spmm_host_flush(loops_plan_t plan, loops_stream_t stream);

/* Backward of C = A . B for a plan built with want_backward:
 *   dB = A^T . dC  (transposed hybrid SpMM; dB device, n_cols x N, lddb; NULL to skip)
 *   dvals[k] = <dC[i_k, :], B[j_k, :]>  (SDDMM on A's pattern, in A's input order;
 *              dvals device, nnz elements of the C type; NULL to skip)
 * dC: device, n_rows x N (lddc), B: device, n_cols x N (ldb), both in the plan dtype.
 * Overwrites dB and dvals. Stream-ordered. */
loops_status loops_spmm_backward(loops_plan_t plan, const void* dC, int64_t lddc, const void* B,
                                 int64_t ldb, void* dB, int64_t lddb, void* dvals,
                                 loops_stream_t stream);

/* Backward with per-column power-of-two scales for the 16-bit dtypes (the precision pattern of
 * loops_spmm_scaled applied to the gradients; the paper's FP16 mode has no backward):
 * the true operands are dC diag(dc_scale) and B diag(b_scale), where dc_scale and b_scale
 * (device f32[N], each optional, NULL = all ones) typically come from loops_cast_scaled, so
 * that small or large gradients keep their precision in F16/BF16. Returns the true gradients:
 *   dB = (A^T . dC) diag(dc_scale)
 *   dvals[k] = sum_n dC[i_k, n] B[j_k, n] dc_scale[n] b_scale[n]  (in f32).
 * Scales with F64/F32 plans give LOOPS_ERR_INVALID_ARG. Otherwise as loops_spmm_backward,
 * which is this call with both scales NULL. */
loops_status loops_spmm_backward_scaled(loops_plan_t plan, const void* dC, int64_t lddc,
                                        const float* dc_scale, const void* B, int64_t ldb,
                                        const float* b_scale, void* dB, int64_t lddb, void* dvals,
                                        loops_stream_t stream);

/* Per-column power-of-two scaling and cast for the 16-bit dtypes:
 *   s_j = 2^ceil(log2 max_i |X_ij|) (1 for an all-zero column), Y_ij = round(X_ij / s_j).
 * X: device f32, rows x cols (ldx); Y: device, y_dtype (LOOPS_F16 or LOOPS_BF16), ldy;
 * col_scale: device f32[cols], written. Rounding is to nearest, ties to even. */
loops_status loops_cast_scaled(const float* X, int64_t rows, int64_t cols, int64_t ldx,
                               loops_dtype y_dtype, void* Y, int64_t ldy, float* col_scale,
                               loops_stream_t stream);

/* Profiling hook: events[0..3] are caller-owned cudaEvent_t handles (timing enabled). Every
 * later loops_spmm* call on this plan records events[0]/events[1] around the CSR-part
 * launches (on the call's stream) and events[2]/events[3] around the BCSR-part launch (on the
 * stream that runs it), back to back when a part is empty. For a batched plan the events are
 * recorded inside its captured graph (which is rebuilt): events[0]/events[1] around the
 * persistent kernel, events[2]/events[3] around the launches that add partial sums. NULL
 * disables the hook. Host only. */
loops_status loops_plan_set_timing_events(loops_plan_t plan, void* const* events);

/* Read and clear the plan's device error word (synchronises `stream`): LOOPS_OK, or
 * LOOPS_ERR_TIMEOUT when a bounded device-side wait gave up in an earlier launch. */
loops_status loops_plan_check(loops_plan_t plan, loops_stream_t stream);

/* Batched plan (the paper runs one matrix at a time; many matrices in one launch has no
 * counterpart there): `count` matrices As[m] (host CSR, as for loops_plan) with their own
 * N = Ns[m], in one dtype
 * (LOOPS_F32, LOOPS_F16 or LOOPS_BF16). Each N must be a multiple of the elements of a 16-byte
 * vector (4 for F32, 8 otherwise) and at most 128. opts->tau < 0 autotunes on `stream`
 * (synchronises it): candidates with one split threshold for all matrices (and, for F32 with
 * block_rows 0, either tile height) are timed as whole batches; then the performance model
 * (Eq. 2 fitted to those timings, Eq. 3 applied per matrix) proposes a threshold and tile
 * height per matrix, which is timed too, and the fastest candidate is kept
 * (loops_plan_batched_stats reports which, with the prediction). The tasks of the batch fall
 * into classes by kind and lane-group width, one persistent kernel each; the launches are
 * captured in a CUDA graph by the first loops_spmm_batched call and replayed by later ones. */
loops_status loops_plan_batched(const loops_csr* As, const int64_t* Ns, int32_t count, loops_dtype dtype,
                                const loops_plan_opts* opts, loops_stream_t stream, loops_plan_t* out);

/* The same batched plan with every matrix's conversion run on the GPU (as loops_plan_device):
 * the CSR arrays of As[m] are DEVICE pointers, borrowed for the call. Each matrix is validated
 * once on the device (errors name the matrix); the sub-plans equal loops_plan_batched's bit for
 * bit, and so does the task list. Synchronises `stream`. No counterpart in the paper. */
loops_status loops_plan_batched_device(const loops_csr* As, const int64_t* Ns, int32_t count,
                                       loops_dtype dtype, const loops_plan_opts* opts,
                                       loops_stream_t stream, loops_plan_t* out);

/* C_m = A_m . B_m for every matrix of a batched plan. Bs, Cs, ldbs, ldcs: HOST arrays of
 * `count` entries holding device pointers / leading dimensions (rows 16-byte aligned);
 * col_scales: NULL, or a host array of `count` device f32[N_m] pointers (16-bit dtypes; NULL
 * entries mean no scaling). The kernels index each B_m with 32-bit element offsets, so
 * n_cols x ldbs[m] must stay below 2^31 (LOOPS_ERR_UNSUPPORTED otherwise). When the pointers
 * differ from the previous call the descriptor table is re-uploaded first (waiting, on the
 * host, for the previous upload to have been read). Stream-ordered otherwise. */
loops_status loops_spmm_batched(loops_plan_t plan, const void* const* Bs, const int64_t* ldbs,
                                void* const* Cs, const int64_t* ldcs, const float* const* col_scales,
                                loops_stream_t stream);

/* End-to-end batched SpMM with HOST buffers: copies every B_m (host, n_cols x N_m, ldbs[m],
 * in the plan dtype; pinned memory makes the copies asynchronous and fast) into one
 * plan-owned device staging area, runs the batch (no column scales), copies every C_m (f32,
 * n_rows x N_m, ldcs[m]) back to the host and synchronises `stream`. The matrices go in up to
 * 16 groups of consecutive matrices (about equal bytes): group g's kernels run on `stream`
 * once its B operands are in, while later groups' B operands are copied in and earlier
 * groups' C results copied out on two plan-owned streams. Matrices whose dense host operands
 * lie back to back in memory (one host arena for all B, one for all C, in matrix order) move
 * in one copy per group and direction, which the CPU-GPU link carries at a higher rate than
 * many small ones; other layouts are copied matrix by matrix, and no byte outside the C_m
 * operands is written. The staging area is allocated on the first call and kept until the
 * plan is destroyed. On an error no copy is left in flight. No counterpart in the paper (its operands never leave
 * the CPU's memory). */
loops_status loops_spmm_batched_host(loops_plan_t plan, const void* const* Bs_host, const int64_t* ldbs,
                                     void* const* Cs_host, const int64_t* ldcs, loops_stream_t stream);

/* Counts of a batched plan: matrices, tasks of the persistent launch, tuned tau and B_r. */
loops_status loops_plan_batched_info(loops_plan_t plan, int32_t* count, int64_t* n_tasks, double* tau,
                                     int32_t* block_rows);

/* Totals of a batched plan (loops_plan_batched_stats). */
typedef struct {
  int32_t count;           /* matrices */
  int32_t block_rows;      /* B_r of the BCSR tasks */
  double tau;              /* the split threshold, or NaN when the matrices use different ones */
  int64_t n_tasks;         /* tasks of the persistent launches */
  int32_t n_kernels;       /* library kernels launched by one loops_spmm_batched call */
  int32_t n_classes;       /* task classes, one persistent kernel each */
  int64_t n_split_rows;    /* CSR rows cut into segments (their sums are a follow-up launch) */
  int64_t n_split_blocks;  /* BCSR blocks cut into units (likewise) */
  int64_t n_rows, nnz, nnz_bcsr;
  int64_t device_bytes;    /* device memory owned by the plan (staging areas included) */
  int32_t tau_source;      /* 0 given; 1 autotuned, one threshold for all matrices; 2 autotuned,
                              a threshold and tile height per matrix from the performance model */
  int32_t reserved0;
  double model_gflops;           /* autotuned: Eq. 2 prediction for the per-matrix choice (NaN if none) */
  double model_measured_gflops;  /* autotuned: that choice, timed (NaN if it equalled a timed one) */
  double timed_best_gflops;      /* autotuned: the best single-threshold candidate, timed */
  int32_t reserved[2];
} loops_batched_info;

/* Totals of a batched plan, for reporting (host only, no device access). */
loops_status loops_plan_batched_stats(loops_plan_t plan, loops_batched_info* out);

/* The loops_plan_info of matrix m (0 <= m < count) of a batched plan: its threshold, tile
 * height and the sizes of its two parts, as the batch's autotuner left them (with the
 * performance model, thresholds and tile heights can differ between matrices). Host only. */
loops_status loops_plan_batched_matrix_info(loops_plan_t plan, int32_t m, loops_plan_info* out);

/* ---------------------------------------------------------------------------------------- */
/* Allocation-free CSR SpMM. The paper has no counterpart: it serves callers that must not
 * allocate device memory at the point where they multiply -- code being recorded into a CUDA
 * graph under the global capture mode, host callbacks and latency-critical paths where an
 * allocation could stall or fail, and services that reserve all device memory up front.
 * loops_plan allocates (it owns the partition on the device), so such callers cannot build a
 * plan; this entry point takes their CSR arrays as they are.
 *
 * Computes C = A . B with A given by DEVICE arrays row_ptr (int64[n_rows + 1]), col_idx
 * (int32[nnz]) and vals (nnz values of `dtype`), B (device, n_cols x N, ldb) and C (device,
 * n_rows x N, ldc) in the element types of the dtype table above (for F16/BF16 the values and
 * B are used as given: no plan scale, no column scale). Rows are split into chunks of 128
 * stored entries; the partial sums of rows that cross chunk boundaries are kept in one static
 * device array of LOOPS_NOALLOC_SCRATCH_BYTES that every GPU loading the library holds until
 * the process exits. The call allocates nothing (no cudaMalloc, no cudaFree, no allocating
 * library routine) and returns LOOPS_ERR_UNSUPPORTED with a message when the problem needs
 * more than that array: 2 * ceil(nnz / 128) * N * (8 for F64, else 4) bytes.
 * Entries whose column lies outside [0, n_cols) are skipped; row_ptr values are clamped to
 * [0, nnz]. The first call on a device looks up the array's device address (a one-time
 * set-up with that device current), so make that first call before any stream capture.
 * Every call uses the same array: calls that overlap on the GPU (for example on two
 * concurrent streams) race and must be serialised by the caller. Stream-ordered. */
#define LOOPS_NOALLOC_SCRATCH_BYTES (16u << 20)
loops_status loops_csr_spmm_noalloc(int64_t n_rows, int64_t n_cols, int64_t nnz,
                                    const int64_t* row_ptr, const int32_t* col_idx,
                                    const void* vals, loops_dtype dtype, const void* B,
                                    int64_t ldb, int64_t N, void* C, int64_t ldc,
                                    loops_stream_t stream);

#ifdef __cplusplus
}
#endif

#endif /* LOOPS_H */
