// Internal declarations shared by the host plan builder, the C-ABI layer and the kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>

#include <string>
#include <vector>

#include "../../include/loops.h"

namespace loops {

// ------------------------------------------------------------------ errors
void set_error(const std::string& msg);
void clear_error();

// Every device (and pinned host) allocation of the library goes through these, so that a test
// can make the n-th one fail (loops_test_fail_alloc) and exercise each error path.
cudaError_t dev_malloc_raw(void** p, size_t bytes);
cudaError_t dev_malloc_async_raw(void** p, size_t bytes, cudaStream_t s);  // stream-ordered (pool)
cudaError_t host_malloc_raw(void** p, size_t bytes);
template <class T>
cudaError_t dev_malloc_async(T** p, size_t bytes, cudaStream_t s) {
  return dev_malloc_async_raw(reinterpret_cast<void**>(p), bytes, s);
}
template <class T>
cudaError_t dev_malloc(T** p, size_t bytes) { return dev_malloc_raw(reinterpret_cast<void**>(p), bytes); }
template <class T>
cudaError_t host_malloc(T** p, size_t bytes) { return host_malloc_raw(reinterpret_cast<void**>(p), bytes); }

// NVTX range in the library's own domain ("loops") for the duration of a scope: plan builds
// and SpMM calls show up in a profiler timeline without touching the caller's default-domain
// ranges. Costs a few nanoseconds when no tool is attached.
class NvtxScope {
 public:
  explicit NvtxScope(const char* name);
  ~NvtxScope();
  NvtxScope(const NvtxScope&) = delete;
  NvtxScope& operator=(const NvtxScope&) = delete;
};

// A device-side wait gave up (bit set in the plan's error word).
constexpr int32_t kErrWaitTimeout = 1;

// Bound on mbarrier polls before a kernel records kErrWaitTimeout and leaves its loop.
constexpr long long kMaxWaitPolls = 1ll << 24;
// The bound kernels launched now use: kMaxWaitPolls, or what loops_test_wait_limit set.
long long wait_poll_limit();

// ------------------------------------------------------------------ dtypes
inline int dense_elem_bytes(loops_dtype d) {  // B / dC element size
  return d == LOOPS_F64 ? 8 : d == LOOPS_F32 ? 4 : 2;
}
inline int out_elem_bytes(loops_dtype d) {    // C / dB / dvals element size
  return d == LOOPS_F64 ? 8 : 4;
}
inline int default_block_rows(loops_dtype d) { return d == LOOPS_F64 ? 8 : 16; }
inline int k_pad_for(loops_dtype d) {  // MMA K of the BCSR kernel (tiles per MMA)
  return d == LOOPS_F64 ? 4 : (d == LOOPS_F32 ? 1 : 16);
}

// Host rounding of binary64 into the storage formats (round to nearest, ties to even).
uint16_t f64_to_f16_bits(double x);
uint16_t f64_to_bf16_bits(double x);
double f16_bits_to_f64(uint16_t h);
double bf16_bits_to_f64(uint16_t h);

// Power of two s with max|a| * s <= 2^14 for 16-bit dtypes, 1 otherwise.
double plan_scale_for(const double* vals, int64_t nnz, loops_dtype d);

// ------------------------------------------------------------------ canonical partition
struct Canon {
  int64_t n_rows = 0, n_cols = 0;
  int32_t br = 8, kpad = 1;
  double scale = 1.0;
  std::vector<int32_t> csr_rows;
  std::vector<int64_t> csr_ptr;   // size n_csr + 1
  std::vector<int32_t> csr_col;
  std::vector<double> csr_val;    // stored values (rounded, scaled) as f64
  std::vector<int32_t> rb_ids;
  std::vector<int64_t> rb_ptr;    // size n_rb + 1 (tile offsets)
  std::vector<int32_t> tile_col;  // -1 for padding tiles
  std::vector<double> tile_val;   // n_tiles * br
  // input-entry -> storage map (for value updates): kind 0 CSR (index into csr_val),
  // 1 BCSR (index into tile_val)
  std::vector<int64_t> src_slot;  // per input entry k: slot index (CSR) or tile*br + r (BCSR)
  std::vector<uint8_t> src_kind;
};

// Validate a CSR input. Returns LOOPS_OK or an error status (message set).
loops_status validate_csr(const loops_csr* A);

// Read A's values as f64 into `out` (host).
void read_vals_f64(const loops_csr* A, std::vector<double>& out);

// Algorithm 1 with the structural split (see partition.cpp).
loops_status build_canon(const loops_csr* A, const double* vals, loops_dtype dtype, int32_t br,
                         double tau, bool contiguous, int64_t r_boundary, int32_t tile_min, Canon& out);

// Round raw f64 values into the dtype after scaling (used by build_canon and updates).
double round_store(double v, double scale, loops_dtype d);

// ------------------------------------------------------------------ device layout
#ifdef __CUDACC__
#define LOOPS_HD __host__ __device__
#else
#define LOOPS_HD
#endif

// Position in the fragment-ordered tile array of (tile t, row r), per dtype:
//   F64  (m8n8k4, K = 4 tiles, B_r = 8):  group g, lane l = 4*row + t -> A[row][t]
//   F16/BF16 (m16n8k16, K = 16, B_r = 16): group g, lane l = 4*q + t, j = 0..7 ->
//        row = q + 8*(j>>1 & 1), tile = 2t + (j & 1) + 8*(j >> 2)
//   F32  (CUDA-core outer product): tile-major, B_r values of a tile contiguous.
LOOPS_HD inline int64_t frag_index(loops_dtype d, int64_t t, int32_t r, int32_t br) {
  if (d == LOOPS_F64) {  // K = 4 tiles per group, 32 lanes x 1 value
    const int64_t g = t / 4;
    const int32_t tt = (int32_t)(t % 4);
    return g * 32 + (int64_t)(r * 4 + tt);
  }
  if (d == LOOPS_F16 || d == LOOPS_BF16) {  // K = 16 tiles per group, 32 lanes x 8 values
    const int64_t g = t / 16;
    const int32_t k = (int32_t)(t % 16);
    const int32_t q = r & 7, hi_r = r >> 3;          // row = q + 8 * hi_r
    const int32_t hi_k = k >> 3, kk = k & 7;         // tile = 2*tq + lo + 8 * hi_k
    const int32_t tq = kk >> 1, lo = kk & 1;
    const int32_t lane = q * 4 + tq;
    const int32_t j = hi_k * 4 + hi_r * 2 + lo;
    return g * 256 + lane * 8 + j;
  }
  return t * br + r;
}
// CSR part work items: item i covers entries [item_ptr[i], item_ptr[i+1]) of col/val and
// writes C row item_row[i] (>= 0) or partial-sum slot -1 - item_row[i] (< 0).
struct CsrDev {
  int64_t n_items = 0, nnz = 0;
  int32_t* item_row = nullptr;
  int64_t* item_ptr = nullptr;
  int32_t* col = nullptr;
  void* val = nullptr;                 // dtype storage type
  int64_t n_split = 0, n_slots = 0;
  int32_t* split_row = nullptr;        // global C row of each split row
  int32_t* split_slot_ptr = nullptr;   // size n_split + 1
  void* scratch = nullptr;             // n_slots x N partial sums (accumulator type)
  // host mirrors used for export
  std::vector<int32_t> h_item_row;
  std::vector<int64_t> h_item_ptr;
  std::vector<int32_t> h_split_row;
  std::vector<int32_t> h_split_slot_ptr;
};

// BCSR part: block b has tiles [rb_ptr[b], rb_ptr[b+1]) (a multiple of k_pad), global row
// block id rb_id[b]. tile_val is stored in the MMA fragment order of the dtype's kernel.
// Work units (longest first) cover a block's tiles [unit_t0, unit_t1); a block with more than
// kBcsrSplitTiles tiles is cut into several units whose partial sums (B_r x N accumulators,
// slot unit_slot) are added in slot order by a second kernel; unit_slot -1 writes C directly.
constexpr int64_t kBcsrSplitTiles = 256;

// CSR work items: 1 = ordered by decreasing length class (longest work first, row order within
// a class), 0 = row order. Both plan builders follow it.
#ifndef LOOPS_CSR_ITEMS_BY_LENGTH
#define LOOPS_CSR_ITEMS_BY_LENGTH 1
#endif
struct BcsrDev {
  int64_t n_rb = 0, n_tiles = 0;
  int32_t* rb_id = nullptr;
  int64_t* rb_ptr = nullptr;
  int32_t* tile_col = nullptr;
  void* tile_val = nullptr;
  int64_t n_units = 0;
  int32_t* unit_block = nullptr;
  int64_t* unit_t0 = nullptr;
  int64_t* unit_t1 = nullptr;
  int32_t* unit_slot = nullptr;
  int64_t n_split = 0, n_slots = 0;
  int32_t* split_block = nullptr;      // block index of each block cut into units
  int32_t* split_slot_ptr = nullptr;   // size n_split + 1
  void* scratch = nullptr;             // n_slots x B_r x N accumulators
  std::vector<int64_t> h_unit_tiles;   // tiles per unit (host, for batched task costs)
};

// csr: rows that no BCSR block covers (written); csr_acc: rows of BCSR blocks whose sparse tiles
// moved to the CSR part (tile-level split), added to C after the BCSR part has written it.
struct PartDev {
  CsrDev csr;
  CsrDev csr_acc;
  BcsrDev bcsr;
  int64_t device_bytes = 0;
};

// Original pattern kept for the SDDMM (dvals in A's input order), split in items.
struct SddmmDev {
  int64_t n_items = 0;
  int32_t* item_row = nullptr;
  int64_t* item_beg = nullptr;         // size n_items + 1 is not used: begin/end pairs
  int64_t* item_end = nullptr;
  int32_t* col = nullptr;              // input order columns (nnz)
};

// Device maps from A's input entries to the stored values, for loops_plan_set_values:
// CSR position p of the device value array takes input entry csr_src[p]; BCSR fragment slot f
// takes the sum (in input order) of input entries bcsr_src[bcsr_ptr[f] .. bcsr_ptr[f+1]).
struct ValueMapDev {
  int64_t n_csr = 0, n_slots = 0;
  int64_t* csr_src = nullptr;
  int64_t* bcsr_ptr = nullptr;
  int64_t* bcsr_src = nullptr;
  int64_t bytes = 0;
};

// Device descriptor of one matrix of a batched plan (pointers into its sub-plan, plus the
// dense operands of the current call).
struct BatchDesc {
  const int32_t* item_row;
  const int64_t* item_ptr;
  const int32_t* col;
  const void* val;
  const int32_t* rb_id;
  const int64_t* rb_ptr;
  const int32_t* tile_col;
  const void* tile_val;
  const int32_t* unit_block;
  const int64_t* unit_t0;
  const int64_t* unit_t1;
  const int32_t* unit_slot;
  void* bscratch;
  const int32_t* bsplit_block;
  const int32_t* bsplit_slot_ptr;
  int32_t br;
  void* scratch;
  const int32_t* split_row;
  const int32_t* split_slot_ptr;
  const void* B;
  void* C;
  const float* col_scale;
  int64_t ldb, ldc, N, n_rows;
  float inv_scale;
};

// One task of a persistent batched kernel: kind 0 CSR items [first, first + count) of
// matrix m, kind 1 F32 BCSR units [first, first + count), kind 2 one F16/BF16 BCSR unit.
struct BatchTask {
  int32_t m;
  int32_t kind;
  int64_t first;
  int32_t count;
  int32_t pad;
};

// A class of tasks: one kind and one lane-group width (G lanes per CSR item or F32 unit, VPL
// 16-byte vectors per lane), run by one persistent kernel specialised for it over the tasks
// [first, first + n_tasks) of the list, with `grid` blocks of 256 threads.
struct BatchClass {
  int32_t kind;
  int32_t G;
  int32_t vpl;
  int32_t br;                          // tile height of an F32 BCSR class (8 or 16)
  int32_t grid;
  int64_t first;
  int64_t n_tasks;
};

struct BatchLaunch {
  const BatchDesc* descs;
  const BatchTask* tasks;
  const BatchClass* classes;           // host array
  int n_classes;
  unsigned long long* counters;        // one task counter per class (device), zeroed per call
  const int2* splits;                  // (matrix, split row) pairs
  int64_t n_splits;
  const int2* bsplits;                 // (matrix, split block) pairs
  int64_t n_bsplits;
  const cudaEvent_t* tev;              // optional timing events: [0]/[1] around the class
                                       // kernels, [2]/[3] around the partial-sum launches
  int n_side;                          // extra branches of the graph (0: one stream)
  const cudaStream_t* side;            // their streams
  cudaEvent_t fork;                    // the branches start after the counters are zeroed
  const cudaEvent_t* join;             // one per extra branch: the call waits for all of them
};

struct BatchState;

// Double-buffered host pipeline of loops_spmm_host_async.
struct HostPipe {
  void* B[2] = {nullptr, nullptr};
  void* C[2] = {nullptr, nullptr};
  int64_t B_bytes = 0, C_bytes = 0;
  cudaStream_t s_in = nullptr, s_out = nullptr;
  cudaEvent_t in_done[2] = {nullptr, nullptr}, compute_done[2] = {nullptr, nullptr},
              out_done[2] = {nullptr, nullptr};
  bool used[2] = {false, false};
  int next = 0;
  int last = -1;                       // buffer set of the last call (for the flush)
};
void destroy_pipe(HostPipe* h);

}  // namespace loops

// Opaque plan handle of the C ABI.
struct loops_plan_s {
  uint64_t magic;
  loops_dtype dtype;
  int64_t n_rows, n_cols, nnz, N;
  int32_t br, kpad;
  double tau;
  double scale;
  int32_t split_len;
  int32_t tile_min;                    // tile-level split threshold in effect (0: off)
  loops_plan_opts opts;
  loops::Canon canon;                  // host copy (canonical order)
  loops::PartDev dev;
  loops_plan_s* transposed;            // plan of A^T for dB (want_backward)
  loops::SddmmDev sddmm;
  loops::ValueMapDev vmap;
  std::vector<int64_t> t_perm;         // A^T entry e comes from input entry t_perm[e]
  int32_t* d_error;                    // device error word
  cudaStream_t side;                   // second stream for the BCSR part
  cudaEvent_t ev_fork, ev_join;
  void* stage_B;                       // loops_spmm_host staging buffers
  void* stage_C;
  int64_t stage_B_bytes, stage_C_bytes;
  loops::HostPipe* pipe;               // loops_spmm_host_async state (lazily created)
  int64_t n_subnormal;
  int64_t nnz_bcsr;
  cudaEvent_t tev[4];                  // optional caller-owned timing events (may be null)
  bool timing;
  loops::BatchState* batch;            // non-null for a batched plan
  int64_t other_bytes;                 // device bytes outside the part arrays
  // partition counts (canonical): CSR-part rows and entries, BCSR blocks and tiles
  int64_t n_csr_rows, nnz_csr, n_rb, n_tiles;
  bool device_built;                   // built by loops_plan_device (no host canonical copy)
  int32_t csr_vpl = 0;                 // CSR kernel: 16-byte vectors per lane (0: heuristic, 1, 2)
  int32_t bcsr_ntile = 0;              // F16/BF16 BCSR kernel: columns per CTA (0: smallest covering N)
  int32_t tau_source = 0;              // 0 given, 1 timed autotuner, 2 Eq. 2/3 model, 3 Eq. 1 / contiguous
  double model_gflops = NAN;           // Eq. 2 prediction for the chosen split (model mode)
  double model_coef[5] = {0, 0, 0, 0, 0};
  bool has_vmap;                       // value maps present (loops_plan_set_values works)
};

namespace loops {

constexpr uint64_t kPlanMagic = 0x4c4f4f5053504c4eull;  // "LOOPSPLN"

// Handles given to callers are registered until loops_plan_destroy, so a destroyed or foreign
// handle is recognised without reading the memory it points to.
void register_plan(const loops_plan_s* p);
void unregister_plan(const loops_plan_s* p);

// Device upload of a canonical partition (partition.cpp). Sets plan->dev.
loops_status upload_part(loops_plan_s* plan, int64_t N);
void free_part(PartDev& d);
// Build and upload the value maps; `remap` (optional) maps the plan's entry order to the
// caller's input order (the transposed plan).
loops_status upload_value_maps(loops_plan_s* plan, const std::vector<int64_t>* remap);
void free_value_maps(ValueMapDev& m);

// ------------------------------------------------------------------ kernel launchers
struct DenseArgs {
  const void* B;
  int64_t ldb;
  void* C;
  int64_t ldc;
  const float* col_scale;   // may be null
  float inv_scale_f;        // 1 / s_A (16-bit)
  double inv_scale_d;
  int64_t N;
  int64_t n_rows;           // rows of C (bounds for BCSR tails)
};

cudaError_t launch_csr(const loops_plan_s* p, const CsrDev& d, const DenseArgs& a, bool accumulate,
                       cudaStream_t s);
cudaError_t launch_bcsr(const loops_plan_s* p, const BcsrDev& d, const DenseArgs& a, cudaStream_t s);
cudaError_t launch_sddmm(const loops_plan_s* p, const void* dC, int64_t lddc, const void* B,
                         int64_t ldb, void* dvals, const float* dc_scale, const float* b_scale, cudaStream_t s);
cudaError_t launch_batched(loops_dtype dtype, const BatchLaunch& L, cudaStream_t s);
// Blocks of a class kernel: resident blocks per SM x SMs, at most one per 8 tasks; 0 if the
// class has no kernel.
int batched_class_grid(loops_dtype dtype, const BatchClass& c);

// Plan construction shared by the single and batched entry points (capi.cpp). `light` plans
// (sub-plans of a batch) get no side stream, events or error word.
loops_status make_plan(const loops_csr* A, const double* vals, int64_t N, loops_dtype dtype,
                       const loops_plan_opts& o, int32_t br, double tau, bool light, loops_plan_s** out);
void destroy_plan(loops_plan_s* p);
loops_status cuda_status(cudaError_t e, const char* what);
loops_status resolve_block_rows(loops_dtype dtype, const loops_plan_opts& o, int32_t* br);
loops_status check_plan(loops_plan_t p);
void destroy_batch(BatchState* b);
int batch_classes(const BatchState* b);
int batch_kernels_per_call(const BatchState* b);
// Fills *out from a plan (single or a batch's sub-plan).
loops_status plan_info_of(const loops_plan_s* p, loops_plan_info* out);
// Timing events of a batched plan (null: none); the captured graph is rebuilt with them.
void batch_set_timing(BatchState* b, const cudaEvent_t* ev);

// ------------------------------------------------------------------ device-side plan build
// A CSR matrix whose arrays are in device memory (values binary64, or binary32 when vals_f32).
struct DevCsrIn {
  int64_t n_rows, n_cols, nnz;
  const int64_t* rp;
  const int32_t* ci;
  const void* vals;
  int vals_f32;
};
// Checks of validate_csr on the device; max_abs = max |a| over finite values.
loops_status validate_csr_device(const DevCsrIn& A, loops_dtype dtype, cudaStream_t s, double* max_abs);
double plan_scale_from_max(double max_abs, loops_dtype d);
// Fills plan->dev (and plan->vmap when want_maps) from A on the device; plan fields dtype, br,
// kpad, scale, split_len and tile_min must be set. `remap` (device, optional) maps A's entries
// to the caller's input order (the transposed plan).
loops_status build_part_device(loops_plan_s* p, const DevCsrIn& A, const int64_t* remap, int64_t N, double tau,
                               bool contiguous, int64_t r_boundary, bool want_maps, cudaStream_t s);
loops_status build_sddmm_device(loops_plan_s* p, const DevCsrIn& A, cudaStream_t s);
loops_status transpose_device(const DevCsrIn& A, int64_t** t_rp, int32_t** t_ci, double** t_vals, int64_t** perm,
                              cudaStream_t s);
// A plan built on the device (capi.cpp); `light` plans (sub-plans of a batch) get no side
// stream, events or error word.
loops_status make_plan_device(const DevCsrIn& A, const int64_t* remap, double scale, int64_t N, loops_dtype dtype,
                              const loops_plan_opts& o, int32_t br, double tau, bool want_maps, bool light,
                              cudaStream_t s, loops_plan_s** out);
// Host copies of the work-item offsets and unit lengths of a device-built plan (the batched
// task list is formed from them on the host).
loops_status download_mirrors(loops_plan_s* p);

// A device buffer whose write evicts the L2 (timed autotuning). Allocation failure leaves it
// empty (run() then does nothing): tuning still works, on a warmer cache.
constexpr size_t kL2FlushBytes = (size_t)256 << 20;
struct L2Flush {
  void* buf = nullptr;
  int n = 0;
  L2Flush();
  ~L2Flush();
  L2Flush(const L2Flush&) = delete;
  L2Flush& operator=(const L2Flush&) = delete;
  cudaError_t run(cudaStream_t s);
};

// ------------------------------------------------------------------ performance model
// Per row block of B_r rows: stored entries and distinct columns (perf_model.cpp).
struct BlockProfile {
  int32_t br = 16;
  std::vector<int64_t> nnz, ucols;
};
struct SplitWork {
  double x, y;  // CSR-part work (entries x N), BCSR-part work (tiles x B_r x N)
};
void block_profile(const loops_csr* A, int32_t br, BlockProfile& out);
SplitWork split_work(const BlockProfile& p, double tau, int32_t kpad, int64_t N);
// Thresholds worth predicting: +inf, the distinct block densities (quantiles if more than
// max_cands), 0.
std::vector<double> tau_grid(const BlockProfile& p, size_t max_cands);
// Eq. 2: perf(x, y) = a0 + a1 x + a2 y + a3 x^2 + a4 y^2, least squares over n samples.
bool fit_perf_model(const double* x, const double* y, const double* perf, int n, double a[5]);
double eval_perf_model(const double a[5], double x, double y);

cudaError_t launch_set_values(const loops_plan_s* p, const void* vals, loops_dtype vd, cudaStream_t s);
cudaError_t launch_cast_scaled(const float* X, int64_t rows, int64_t cols, int64_t ldx,
                               loops_dtype yd, void* Y, int64_t ldy, float* col_scale,
                               cudaStream_t s);

}  // namespace loops
