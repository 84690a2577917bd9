// C-ABI entry points of libloops.so (declared in include/loops.h).
#include <algorithm>
#include <atomic>
#include <mutex>
#include <unordered_set>

#include <nvtx3/nvToolsExt.h>
#include <functional>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <string>

#include "loops_internal.h"

namespace loops {

static thread_local std::string g_last_error;

void set_error(const std::string& msg) { g_last_error = msg; }
void clear_error() { g_last_error.clear(); }

loops_status export_part(const loops_plan_s* p, loops_partition* out);
// Builds a candidate plan for the given options and threshold (host or device builder).
using PlanBuilder = std::function<loops_status(const loops_plan_opts& o, double tau, loops_plan_s** out)>;
struct TunedShape {
  double tau;
  int32_t tile_min, br, csr_vpl, bcsr_ntile;
};
loops_status autotune_tau(const PlanBuilder& build, int64_t n_rows, int64_t n_cols, int64_t nnz, int64_t N,
                          loops_dtype dtype, int32_t split_len, bool try_tile_split, int32_t br, bool try_br,
                          cudaStream_t s, TunedShape* out);

loops_status cuda_status(cudaError_t e, const char* what) {
  if (e == cudaSuccess) return LOOPS_OK;
  set_error(std::string(what) + ": " + cudaGetErrorString(e));
  return e == cudaErrorMemoryAllocation ? LOOPS_ERR_OOM : LOOPS_ERR_CUDA;
}

// ------------------------------------------------------------------ NVTX
static nvtxDomainHandle_t nvtx_domain() {
  static nvtxDomainHandle_t d = nvtxDomainCreateA("loops");
  return d;
}

NvtxScope::NvtxScope(const char* name) {
  nvtxEventAttributes_t a = {};
  a.version = NVTX_VERSION;
  a.size = NVTX_EVENT_ATTRIB_STRUCT_SIZE;
  a.messageType = NVTX_MESSAGE_TYPE_ASCII;
  a.message.ascii = name;
  nvtxDomainRangePushEx(nvtx_domain(), &a);
}

NvtxScope::~NvtxScope() { nvtxDomainRangePop(nvtx_domain()); }

// ------------------------------------------------------------------ allocation hook
static std::atomic<int64_t> g_alloc_countdown{0};  // > 0: this many allocations from now, the last fails
static std::atomic<int64_t> g_alloc_seen{0};       // allocations since the last loops_test_fail_alloc

static bool alloc_should_fail() {
  // LOOPS_FAULT_ALLOC=k in the environment arms the hook once, for the k-th allocation of the
  // process (the same hook as loops_test_fail_alloc)
  static std::once_flag env_once;
  std::call_once(env_once, [] {
    if (const char* v = std::getenv("LOOPS_FAULT_ALLOC")) {
      const long long k = std::atoll(v);
      if (k > 0) g_alloc_countdown.store(k);
    }
  });
  g_alloc_seen.fetch_add(1, std::memory_order_relaxed);
  int64_t c = g_alloc_countdown.load();
  while (c > 0) {
    if (g_alloc_countdown.compare_exchange_weak(c, c - 1)) return c == 1;
  }
  return false;
}

// ------------------------------------------------------------------ wait-bound hook
static std::atomic<int64_t> g_wait_polls{(int64_t)kMaxWaitPolls};

long long wait_poll_limit() { return (long long)g_wait_polls.load(std::memory_order_relaxed); }

cudaError_t dev_malloc_raw(void** p, size_t bytes) {
  if (alloc_should_fail()) {
    *p = nullptr;
    return cudaErrorMemoryAllocation;
  }
  return cudaMalloc(p, bytes);
}

cudaError_t dev_malloc_async_raw(void** p, size_t bytes, cudaStream_t s) {
  if (alloc_should_fail()) {
    *p = nullptr;
    return cudaErrorMemoryAllocation;
  }
  return cudaMallocAsync(p, bytes, s);
}

cudaError_t host_malloc_raw(void** p, size_t bytes) {
  if (alloc_should_fail()) {
    *p = nullptr;
    return cudaErrorMemoryAllocation;
  }
  return cudaMallocHost(p, bytes);
}

// ------------------------------------------------------------------ live handles
static std::mutex g_plans_mu;
static std::unordered_set<const loops_plan_s*> g_plans;

void register_plan(const loops_plan_s* p) {
  std::lock_guard<std::mutex> g(g_plans_mu);
  g_plans.insert(p);
}

void unregister_plan(const loops_plan_s* p) {
  std::lock_guard<std::mutex> g(g_plans_mu);
  g_plans.erase(p);
}

static bool plan_live(const loops_plan_s* p) {
  std::lock_guard<std::mutex> g(g_plans_mu);
  return g_plans.count(p) != 0;
}

static bool valid_dtype(loops_dtype d) {
  return d == LOOPS_F64 || d == LOOPS_F32 || d == LOOPS_F16 || d == LOOPS_BF16;
}

loops_status check_plan(loops_plan_t p) {
  if (!p || !plan_live(p) || p->magic != kPlanMagic) {
    set_error("invalid or destroyed plan handle");
    return LOOPS_ERR_STATE;
  }
  return LOOPS_OK;
}

// A single-matrix plan (not batched).
static loops_status check_single(loops_plan_t p) {
  loops_status st = check_plan(p);
  if (st) return st;
  if (p->batch) {
    set_error("this call needs a single-matrix plan, not a batched one");
    return LOOPS_ERR_STATE;
  }
  return LOOPS_OK;
}

static void fill_partition(const Canon& c, loops_partition* out) {
  std::memset(out, 0, sizeof(*out));
  out->n_rows = c.n_rows;
  out->n_cols = c.n_cols;
  out->block_rows = c.br;
  out->k_pad = c.kpad;
  out->scale = c.scale;
  out->n_csr_rows = (int64_t)c.csr_rows.size();
  out->nnz_csr = (int64_t)c.csr_col.size();
  out->n_row_blocks = (int64_t)c.rb_ids.size();
  out->n_tiles = (int64_t)c.tile_col.size();
  auto dup = [](const void* src, size_t bytes) {
    void* d = std::malloc(bytes ? bytes : 1);
    if (bytes) std::memcpy(d, src, bytes);
    return d;
  };
  out->csr_rows = (int32_t*)dup(c.csr_rows.data(), c.csr_rows.size() * 4);
  out->csr_ptr = (int64_t*)dup(c.csr_ptr.data(), c.csr_ptr.size() * 8);
  out->csr_col = (int32_t*)dup(c.csr_col.data(), c.csr_col.size() * 4);
  out->csr_val = (double*)dup(c.csr_val.data(), c.csr_val.size() * 8);
  out->rb_ids = (int32_t*)dup(c.rb_ids.data(), c.rb_ids.size() * 4);
  out->rb_ptr = (int64_t*)dup(c.rb_ptr.data(), c.rb_ptr.size() * 8);
  out->tile_col = (int32_t*)dup(c.tile_col.data(), c.tile_col.size() * 4);
  out->tile_val = (double*)dup(c.tile_val.data(), c.tile_val.size() * 8);
}

loops_status resolve_block_rows(loops_dtype dtype, const loops_plan_opts& o, int32_t* br) {
  int32_t b = o.block_rows ? o.block_rows : default_block_rows(dtype);
  const bool ok = (dtype == LOOPS_F64 && b == 8) || ((dtype == LOOPS_F16 || dtype == LOOPS_BF16) && b == 16) ||
                  (dtype == LOOPS_F32 && (b == 8 || b == 16));
  if (!ok) {
    set_error("unsupported block_rows " + std::to_string(b) + " for this dtype");
    return LOOPS_ERR_UNSUPPORTED;
  }
  *br = b;
  return LOOPS_OK;
}

void destroy_pipe(HostPipe* h) {
  if (!h) return;
  for (int i = 0; i < 2; ++i) {
    if (h->B[i]) cudaFree(h->B[i]);
    if (h->C[i]) cudaFree(h->C[i]);
    cudaEvent_t evs[] = {h->in_done[i], h->compute_done[i], h->out_done[i]};
    for (cudaEvent_t ev : evs)
      if (ev) cudaEventDestroy(ev);
  }
  if (h->s_in) cudaStreamDestroy(h->s_in);
  if (h->s_out) cudaStreamDestroy(h->s_out);
  delete h;
}

void destroy_plan(loops_plan_s* p) {
  if (!p) return;
  if (p->pipe) destroy_pipe(p->pipe);
  if (p->batch) destroy_batch(p->batch);
  if (p->transposed) destroy_plan(p->transposed);
  free_part(p->dev);
  free_value_maps(p->vmap);
  void* ptrs[] = {p->sddmm.item_row, p->sddmm.item_beg, p->sddmm.item_end, p->sddmm.col,
                  p->d_error, p->stage_B, p->stage_C};
  for (void* q : ptrs)
    if (q) cudaFree(q);
  if (p->side) cudaStreamDestroy(p->side);
  if (p->ev_fork) cudaEventDestroy(p->ev_fork);
  if (p->ev_join) cudaEventDestroy(p->ev_join);
  p->magic = 0;
  delete p;
}

// Builds a single (non-transposed) plan from validated input and f64 values.
// A plan object with its fields set from the arguments and no device part yet.
static loops_plan_s* new_plan(int64_t n_rows, int64_t n_cols, int64_t nnz, int64_t N, loops_dtype dtype,
                              const loops_plan_opts& o, int32_t br, double tau) {
  loops_plan_s* p = new (std::nothrow) loops_plan_s();
  if (!p) { set_error("host allocation failed"); return nullptr; }
  p->magic = kPlanMagic;
  p->dtype = dtype;
  p->n_rows = n_rows;
  p->n_cols = n_cols;
  p->nnz = nnz;
  p->N = N;
  p->br = br;
  p->kpad = k_pad_for(dtype);
  p->tau = tau;
  p->opts = o;
  p->split_len = o.split_len > 0 ? o.split_len : 512;
  p->tile_min = o.tile_min > 1 ? o.tile_min : 0;
  p->transposed = nullptr;
  p->d_error = nullptr;
  p->side = nullptr;
  p->ev_fork = p->ev_join = nullptr;
  p->stage_B = p->stage_C = nullptr;
  p->stage_B_bytes = p->stage_C_bytes = 0;
  p->pipe = nullptr;
  p->timing = false;
  for (auto& ev : p->tev) ev = nullptr;
  p->batch = nullptr;
  p->other_bytes = 0;
  p->n_csr_rows = p->nnz_csr = p->n_rb = p->n_tiles = 0;
  p->device_built = false;
  p->has_vmap = false;
  p->n_subnormal = 0;
  p->nnz_bcsr = 0;
  p->scale = 1.0;
  return p;
}

// Error word, side stream and fork/join events of a plan that runs SpMM calls.
static loops_status plan_runtime(loops_plan_s* p) {
  cudaError_t e = dev_malloc((void**)&p->d_error, sizeof(int32_t));
  if (e == cudaSuccess) e = cudaMemset(p->d_error, 0, sizeof(int32_t));
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&p->side, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->ev_fork, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->ev_join, cudaEventDisableTiming);
  if (e != cudaSuccess) return cuda_status(e, "plan setup");
  p->other_bytes += sizeof(int32_t);
  return LOOPS_OK;
}

loops_status make_plan(const loops_csr* A, const double* vals, int64_t N, loops_dtype dtype,
                       const loops_plan_opts& o, int32_t br, double tau, bool light, loops_plan_s** out) {
  *out = nullptr;
  loops_plan_s* p = new_plan(A->n_rows, A->n_cols, A->nnz, N, dtype, o, br, tau);
  if (!p) return LOOPS_ERR_OOM;
  loops_status st = build_canon(A, vals, dtype, br, tau, o.contiguous_split != 0, o.r_boundary, p->tile_min,
                                p->canon);
  if (st) { destroy_plan(p); return st; }
  p->scale = p->canon.scale;
  p->n_subnormal = 0;
  if (dtype == LOOPS_F16 || dtype == LOOPS_BF16) {
    const double tiny = dtype == LOOPS_F16 ? std::ldexp(1.0, -14) : std::ldexp(1.0, -126);
    for (double v : p->canon.csr_val) p->n_subnormal += (v != 0.0 && std::fabs(v) < tiny);
    for (double v : p->canon.tile_val) p->n_subnormal += (v != 0.0 && std::fabs(v) < tiny);
  }
  p->nnz_bcsr = 0;
  for (uint8_t k : p->canon.src_kind) p->nnz_bcsr += k;
  p->n_csr_rows = (int64_t)p->canon.csr_rows.size();
  p->nnz_csr = (int64_t)p->canon.csr_col.size();
  p->n_rb = (int64_t)p->canon.rb_ids.size();
  p->n_tiles = (int64_t)p->canon.tile_col.size();
  if ((st = upload_part(p, N))) { destroy_plan(p); return st; }
  if (!light && (st = plan_runtime(p))) { destroy_plan(p); return st; }
  *out = p;
  return LOOPS_OK;
}

// The same plan built on the device from a device-resident CSR matrix (plan_device.cu).
loops_status make_plan_device(const DevCsrIn& A, const int64_t* remap, double scale, int64_t N, loops_dtype dtype,
                              const loops_plan_opts& o, int32_t br, double tau, bool want_maps, bool light,
                              cudaStream_t s, loops_plan_s** out) {
  *out = nullptr;
  loops_plan_s* p = new_plan(A.n_rows, A.n_cols, A.nnz, N, dtype, o, br, tau);
  if (!p) return LOOPS_ERR_OOM;
  p->device_built = true;
  p->scale = scale;
  loops_status st = build_part_device(p, A, remap, N, tau, o.contiguous_split != 0, o.r_boundary,
                                      want_maps && p->tile_min == 0, s);
  if (!st && !light) st = plan_runtime(p);
  if (st) { destroy_plan(p); return st; }
  *out = p;
  return LOOPS_OK;
}

// A^T in CSR (stable counting sort by column): entry e of A^T comes from input entry perm[e].
static void transpose_csr(const loops_csr* A, std::vector<int64_t>& rp, std::vector<int32_t>& ci,
                          std::vector<int64_t>& perm) {
  rp.assign((size_t)A->n_cols + 1, 0);
  for (int64_t k = 0; k < A->nnz; ++k) rp[(size_t)A->col_idx[k] + 1]++;
  for (int64_t j = 0; j < A->n_cols; ++j) rp[(size_t)j + 1] += rp[(size_t)j];
  std::vector<int64_t> pos(rp.begin(), rp.end() - 1);
  ci.resize((size_t)A->nnz);
  perm.resize((size_t)A->nnz);
  for (int64_t i = 0; i < A->n_rows; ++i)
    for (int64_t k = A->row_ptr[i]; k < A->row_ptr[i + 1]; ++k) {
      const int64_t e = pos[(size_t)A->col_idx[k]]++;
      ci[(size_t)e] = (int32_t)i;
      perm[(size_t)e] = k;
    }
}

static loops_status build_sddmm(loops_plan_s* p, const loops_csr* A) {
  std::vector<int32_t> row;
  std::vector<int64_t> beg, end;
  struct It { int32_t r; int64_t b, e; };
  std::vector<It> it;
  const int64_t L = p->split_len;
  for (int64_t i = 0; i < A->n_rows; ++i)
    for (int64_t b = A->row_ptr[i]; b < A->row_ptr[i + 1]; b += L)
      it.push_back({(int32_t)i, b, std::min(b + L, A->row_ptr[i + 1])});
  std::stable_sort(it.begin(), it.end(), [](const It& x, const It& y) { return x.e - x.b > y.e - y.b; });
  for (auto& x : it) { row.push_back(x.r); beg.push_back(x.b); end.push_back(x.e); }
  p->sddmm.n_items = (int64_t)it.size();
  auto up = [&](void** dst, const void* src, size_t bytes) -> loops_status {
    if (!bytes) { *dst = nullptr; return LOOPS_OK; }
    cudaError_t e = dev_malloc(dst, bytes);
    if (e == cudaSuccess) e = cudaMemcpy(*dst, src, bytes, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) p->other_bytes += (int64_t)bytes;
    return cuda_status(e, "upload SDDMM pattern");
  };
  loops_status st;
  if ((st = up((void**)&p->sddmm.item_row, row.data(), row.size() * 4))) return st;
  if ((st = up((void**)&p->sddmm.item_beg, beg.data(), beg.size() * 8))) return st;
  if ((st = up((void**)&p->sddmm.item_end, end.data(), end.size() * 8))) return st;
  if ((st = up((void**)&p->sddmm.col, A->col_idx, (size_t)A->nnz * 4))) return st;
  return LOOPS_OK;
}

static loops_status check_dense(const void* ptr, int64_t rows, int64_t N, int64_t ld, const char* name) {
  if (ld < N || ld < 0) {
    set_error(std::string("leading dimension of ") + name + " is smaller than N");
    return LOOPS_ERR_INVALID_ARG;
  }
  if (!ptr && rows > 0 && N > 0) {
    set_error(std::string(name) + " is NULL");
    return LOOPS_ERR_INVALID_ARG;
  }
  return LOOPS_OK;
}

// Run C = A.B on the plan: BCSR part on the side stream, CSR part on `s`, joined by events.
static loops_status run_spmm(loops_plan_s* p, const void* B, int64_t ldb, const float* col_scale,
                             void* C, int64_t ldc, cudaStream_t s) {
  if (p->n_rows == 0 || p->N == 0) return LOOPS_OK;
  DenseArgs a;
  a.B = B;
  a.ldb = ldb;
  a.C = C;
  a.ldc = ldc;
  a.col_scale = col_scale;
  a.inv_scale_d = 1.0 / p->scale;
  a.inv_scale_f = (float)(1.0 / p->scale);
  a.N = p->N;
  a.n_rows = p->n_rows;
  const bool has_csr = p->dev.csr.n_items > 0;
  const bool has_bcsr = p->dev.bcsr.n_rb > 0;
  const bool tm = p->timing;
  auto rec = [&](int i, cudaStream_t st) { return tm ? cudaEventRecord(p->tev[i], st) : cudaSuccess; };
  cudaError_t e = cudaSuccess;
  const bool has_acc = p->dev.csr_acc.n_items > 0;
  if (has_csr && has_bcsr) {
    e = cudaEventRecord(p->ev_fork, s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(p->side, p->ev_fork, 0);
    if (e == cudaSuccess) e = rec(2, p->side);
    if (e == cudaSuccess) e = launch_bcsr(p, p->dev.bcsr, a, p->side);
    if (e == cudaSuccess && !has_acc) e = rec(3, p->side);
    if (e == cudaSuccess) e = rec(0, s);
    if (e == cudaSuccess) e = launch_csr(p, p->dev.csr, a, false, s);
    if (e == cudaSuccess) e = rec(1, s);
    if (e == cudaSuccess) e = cudaEventRecord(p->ev_join, p->side);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, p->ev_join, 0);
  } else {
    if (e == cudaSuccess) e = rec(2, s);
    if (e == cudaSuccess && has_bcsr) e = launch_bcsr(p, p->dev.bcsr, a, s);
    if (e == cudaSuccess && !has_acc) e = rec(3, s);
    if (e == cudaSuccess) e = rec(0, s);
    if (e == cudaSuccess && has_csr) e = launch_csr(p, p->dev.csr, a, false, s);
    if (e == cudaSuccess) e = rec(1, s);
  }
  // tile-level split: rows of BCSR blocks add their moved entries after the BCSR part wrote
  // them (the BCSR timing window then ends after this pass)
  if (e == cudaSuccess && has_acc) {
    e = launch_csr(p, p->dev.csr_acc, a, true, s);
    if (e == cudaSuccess) e = rec(3, s);
  }
  return cuda_status(e, "SpMM launch");
}

// Fill a device buffer with finite values of the dense dtype (timing input only).
static cudaError_t fill_finite(void* p, int64_t bytes, cudaStream_t s) {
  // 0x3C bytes: f16 1.06, bf16 0.0115, f32 0.0115, f64 1.6e-18 -- all finite
  return cudaMemsetAsync(p, 0x3C, (size_t)bytes, s);
}

}  // namespace loops

namespace loops {

// Candidates are timed the way SpMM runs in a sequence of calls on fresh operands: with the
// L2 holding none of them (a write of a buffer twice the L2 size before each timed call).
L2Flush::L2Flush() {
  if (dev_malloc(&buf, kL2FlushBytes) != cudaSuccess) {
    buf = nullptr;
    cudaGetLastError();
  }
}
L2Flush::~L2Flush() {
  if (buf) cudaFree(buf);
}
cudaError_t L2Flush::run(cudaStream_t s) {
  return buf ? cudaMemsetAsync(buf, ++n & 0xff, kL2FlushBytes, s) : cudaSuccess;
}

// Autotuner: times C = A.B for candidate split thresholds (and, for F32, either tile height)
// on synthetic B with the L2 flushed before each timed call, keeps the fastest, then times the
// shapes of its kernels on that plan: the CSR kernel's 16-byte column vectors per lane (1 or
// 2) and, for F16/BF16, the BCSR kernel's columns per CTA (32, 64 or 128). Candidates that give
// the same row-block split as an earlier one are skipped.
loops_status autotune_tau(const PlanBuilder& build, int64_t n_rows, int64_t n_cols, int64_t nnz, int64_t N,
                          loops_dtype dtype, int32_t split_len, bool try_tile_split, int32_t br, bool try_br,
                          cudaStream_t s, TunedShape* out) {
  struct Cand { double tau; int32_t tile_min; int32_t br; };
  std::vector<Cand> cands;
  for (double t : {(double)INFINITY, 8.0, 4.0, 3.0, 2.0, 1.5, 1.25, 0.0}) cands.push_back({t, 0, br});
  if (try_tile_split)  // tile-level split: dense tiles (>= 2 entries) on the BCSR kernel only
    for (double t : {4.0, 2.0, 1.25}) cands.push_back({t, 2, br});
  if (try_br && dtype == LOOPS_F32)
    for (double t : {4.0, 2.0, 1.25}) cands.push_back({t, 0, br == 16 ? 8 : 16});
  *out = TunedShape{2.0, 0, br, 0, 0};
  if (nnz == 0 || N == 0 || n_rows == 0) return LOOPS_OK;
  const int64_t eb = dense_elem_bytes(dtype), ec = out_elem_bytes(dtype);
  void *dB = nullptr, *dC = nullptr;
  cudaError_t e = dev_malloc(&dB, (size_t)std::max<int64_t>(n_cols * N * eb, 16));
  if (e == cudaSuccess) e = dev_malloc(&dC, (size_t)std::max<int64_t>(n_rows * N * ec, 16));
  if (e == cudaSuccess) e = fill_finite(dB, n_cols * N * eb, s);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  loops_status st = cuda_status(e, "autotune setup");
  L2Flush flush;
  // best of 5 timed calls (after 2 warm-up calls), the L2 flushed before each
  auto time_plan = [&](loops_plan_s* p, float* ms_out) {
    float best_ms = INFINITY;
    for (int it = 0; it < 7 && !st; ++it) {
      if ((st = run_spmm(p, dB, N, nullptr, dC, N, s))) break;
      if (it < 2) continue;
      if ((st = cuda_status(flush.run(s), "L2 flush"))) break;
      cudaEventRecord(e0, s);
      st = run_spmm(p, dB, N, nullptr, dC, N, s);
      cudaEventRecord(e1, s);
      if (!st) st = cuda_status(cudaEventSynchronize(e1), "autotune timing");
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      best_ms = std::min(best_ms, ms);
    }
    *ms_out = best_ms;
  };
  float best = INFINITY;
  loops_plan_s* best_p = nullptr;
  std::vector<std::tuple<int64_t, int64_t, int32_t>> seen;
  loops_plan_opts o;
  loops_plan_opts_default(&o);
  o.split_len = split_len;
  for (const Cand& cand : cands) {
    if (st) break;
    o.tile_min = cand.tile_min;
    o.block_rows = cand.br;
    loops_plan_s* p = nullptr;
    if ((st = build(o, cand.tau, &p))) break;
    // a split without BCSR blocks is the same plan for either tile height
    const auto key = std::make_tuple(p->n_rb, p->n_tiles, p->n_rb > 0 ? cand.br : 0);
    if (std::find(seen.begin(), seen.end(), key) != seen.end()) { destroy_plan(p); continue; }
    seen.push_back(key);
    float ms = INFINITY;
    time_plan(p, &ms);
    if (!st && ms < best) {
      best = ms;
      out->tau = cand.tau;
      out->tile_min = cand.tile_min;
      out->br = cand.br;
      if (best_p) destroy_plan(best_p);
      best_p = p;
    } else {
      destroy_plan(p);
    }
  }
  // kernel shapes on the chosen split
  if (!st && best_p) {
    const int64_t nvec = dtype == LOOPS_F64 ? 0 : N / (16 / dense_elem_bytes(dtype));
    if (best_p->dev.csr.n_items > 0 && nvec >= 2 && N % (16 / dense_elem_bytes(dtype)) == 0) {
      for (int v : {1, 2}) {
        best_p->csr_vpl = v;
        float ms = INFINITY;
        time_plan(best_p, &ms);
        if (!st && ms < best) { best = ms; out->csr_vpl = v; }
      }
      best_p->csr_vpl = out->csr_vpl;
    }
    if ((dtype == LOOPS_F16 || dtype == LOOPS_BF16) && best_p->dev.bcsr.n_rb > 0 && N > 32) {
      for (int t : {32, 64, 128}) {
        if (t > 2 * N) break;
        best_p->bcsr_ntile = t;
        float ms = INFINITY;
        time_plan(best_p, &ms);
        if (!st && ms < best) { best = ms; out->bcsr_ntile = t; }
      }
    }
  }
  if (best_p) destroy_plan(best_p);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (dB) cudaFree(dB);
  if (dC) cudaFree(dC);
  return st;
}

// Split threshold from the performance model (Eq. 2 and Eq. 3, restated in perf_model.cpp):
// the warm-up candidates (the timed autotuner's thresholds, each distinct split once) are
// built and timed (L2 flushed before each timed call), Eq. 2 is fitted to their (CSR work,
// BCSR work, time), and Eq. 3 picks the threshold of highest predicted throughput (flops over
// predicted time) among +inf, 0 and the matrix's distinct block densities -- including
// thresholds never timed.
loops_status model_tau(const PlanBuilder& build, const BlockProfile& prof, int64_t n_rows, int64_t n_cols,
                       int64_t nnz, int64_t N, loops_dtype dtype, int32_t split_len, cudaStream_t s,
                       double* tau_out, double* pred_out, double coef[5]) {
  *tau_out = 2.0;
  *pred_out = NAN;
  for (int i = 0; i < 5; ++i) coef[i] = 0.0;
  if (nnz == 0 || N == 0 || n_rows == 0) return LOOPS_OK;
  const int32_t kpad = k_pad_for(dtype);
  const double flops = 2.0 * (double)nnz * (double)N;
  const int64_t eb = dense_elem_bytes(dtype), ec = out_elem_bytes(dtype);
  void *dB = nullptr, *dC = nullptr;
  cudaError_t e = dev_malloc(&dB, (size_t)std::max<int64_t>(n_cols * N * eb, 16));
  if (e == cudaSuccess) e = dev_malloc(&dC, (size_t)std::max<int64_t>(n_rows * N * ec, 16));
  if (e == cudaSuccess) e = fill_finite(dB, n_cols * N * eb, s);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  loops_status st = cuda_status(e, "model setup");
  L2Flush flush;
  std::vector<double> xs, ys, ps;
  loops_plan_opts o;
  loops_plan_opts_default(&o);
  o.split_len = split_len;
  o.tile_min = 0;
  const double warm[] = {(double)INFINITY, 8.0, 4.0, 3.0, 2.0, 1.5, 1.25, 0.0};
  std::vector<double> taus;
  for (double tau : warm) {
    if (st) break;
    const SplitWork w = split_work(prof, tau, kpad, N);
    bool dup = false;
    for (size_t i = 0; i < xs.size(); ++i) dup = dup || (xs[i] == w.x && ys[i] == w.y);
    if (dup) continue;
    loops_plan_s* p = nullptr;
    if ((st = build(o, tau, &p))) break;
    float best_ms = INFINITY;
    for (int it = 0; it < 7 && !st; ++it) {
      if ((st = run_spmm(p, dB, N, nullptr, dC, N, s))) break;  // it 0, 1: warm-up
      if (it < 2) continue;
      if ((st = cuda_status(flush.run(s), "L2 flush"))) break;
      cudaEventRecord(e0, s);
      st = run_spmm(p, dB, N, nullptr, dC, N, s);
      cudaEventRecord(e1, s);
      if (!st) st = cuda_status(cudaEventSynchronize(e1), "model timing");
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      best_ms = std::min(best_ms, ms);
    }
    destroy_plan(p);
    if (st) break;
    xs.push_back(w.x);
    ys.push_back(w.y);
    taus.push_back(tau);
    ps.push_back((double)best_ms);
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (dB) cudaFree(dB);
  if (dC) cudaFree(dC);
  if (st) return st;
  if (!fit_perf_model(xs.data(), ys.data(), ps.data(), (int)xs.size(), coef)) {
    // degenerate samples: the fastest measured threshold
    size_t b = 0;
    for (size_t i = 1; i < ps.size(); ++i)
      if (ps[i] < ps[b]) b = i;
    if (!taus.empty()) *tau_out = taus[b];
    return LOOPS_OK;
  }
  // Eq. 3: the highest predicted throughput, flops / predicted time (predictions of no more
  // than a tenth of the fastest measured time are not trusted: the fit extrapolates there)
  double tmin = INFINITY;
  for (double t : ps) tmin = std::min(tmin, t);
  double best = INFINITY;
  for (double tau : tau_grid(prof, 64)) {
    const SplitWork w = split_work(prof, tau, kpad, N);
    const double t = eval_perf_model(coef, w.x, w.y);
    if (t > 0.1 * tmin && t < best) {
      best = t;
      *tau_out = tau;
    }
  }
  if (best < INFINITY) *pred_out = flops / (best * 1e-3) / 1e9;
  return LOOPS_OK;
}

// Paper mode with the boundary from Eq. 1: time the pure CSR plan (the paper's pure vector-unit
// configuration) and the pure BCSR plan (rows from 0 on in BCSR) on synthetic B, take each
// part's throughput TP = rows / time, and choose r_b so that the two parts, running side by
// side, take the same time: r_b / TP_csr = (n_rows - r_b) / TP_bcsr.
loops_status model_boundary(const PlanBuilder& build, int64_t n_rows, int64_t n_cols, int64_t nnz, int64_t N,
                            loops_dtype dtype, int32_t split_len, cudaStream_t s, int64_t* rb_out) {
  *rb_out = n_rows;
  if (nnz == 0 || N == 0 || n_rows == 0) return LOOPS_OK;
  const int64_t eb = dense_elem_bytes(dtype), ec = out_elem_bytes(dtype);
  void *dB = nullptr, *dC = nullptr;
  cudaError_t e = dev_malloc(&dB, (size_t)std::max<int64_t>(n_cols * N * eb, 16));
  if (e == cudaSuccess) e = dev_malloc(&dC, (size_t)std::max<int64_t>(n_rows * N * ec, 16));
  if (e == cudaSuccess) e = fill_finite(dB, n_cols * N * eb, s);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  loops_status st = cuda_status(e, "model setup");
  L2Flush flush;
  float t[2] = {INFINITY, INFINITY};
  for (int which = 0; which < 2 && !st; ++which) {
    loops_plan_opts o;
    loops_plan_opts_default(&o);
    o.split_len = split_len;
    o.contiguous_split = which;          // 0: tau = inf (all CSR); 1: r_b = 0 (all BCSR)
    o.r_boundary = 0;
    loops_plan_s* p = nullptr;
    if ((st = build(o, INFINITY, &p))) break;
    for (int it = 0; it < 7 && !st; ++it) {
      if (it >= 2) {
        if ((st = cuda_status(flush.run(s), "L2 flush"))) break;
        cudaEventRecord(e0, s);
      }
      st = run_spmm(p, dB, N, nullptr, dC, N, s);
      if (it >= 2) {
        cudaEventRecord(e1, s);
        if (!st) st = cuda_status(cudaEventSynchronize(e1), "model timing");
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        t[which] = std::min(t[which], ms);
      }
    }
    destroy_plan(p);
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (dB) cudaFree(dB);
  if (dC) cudaFree(dC);
  if (st) return st;
  const double tp_csr = (double)n_rows / std::max((double)t[0], 1e-9);
  const double tp_bcsr = (double)n_rows / std::max((double)t[1], 1e-9);
  *rb_out = (int64_t)std::llround((double)n_rows * tp_csr / (tp_csr + tp_bcsr));
  return LOOPS_OK;
}

}  // namespace loops

using namespace loops;

extern "C" {

int32_t loops_version(void) { return 10000; }

const char* loops_status_str(loops_status s) {
  switch (s) {
    case LOOPS_OK: return "LOOPS_OK";
    case LOOPS_ERR_INVALID_ARG: return "LOOPS_ERR_INVALID_ARG";
    case LOOPS_ERR_INVALID_CSR: return "LOOPS_ERR_INVALID_CSR";
    case LOOPS_ERR_UNSUPPORTED: return "LOOPS_ERR_UNSUPPORTED";
    case LOOPS_ERR_OOM: return "LOOPS_ERR_OOM";
    case LOOPS_ERR_CUDA: return "LOOPS_ERR_CUDA";
    case LOOPS_ERR_TIMEOUT: return "LOOPS_ERR_TIMEOUT";
    case LOOPS_ERR_STATE: return "LOOPS_ERR_STATE";
  }
  return "LOOPS_ERR_UNKNOWN";
}

const char* loops_last_error(void) { return g_last_error.c_str(); }

void loops_plan_opts_default(loops_plan_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->tau = 2.0;
  o->tile_min = -1;
}

loops_status loops_partition_host(const loops_csr* A, loops_dtype dtype, const loops_plan_opts* opts,
                                  loops_partition* out) {
  clear_error();
  if (!out) { set_error("out is NULL"); return LOOPS_ERR_INVALID_ARG; }
  std::memset(out, 0, sizeof(*out));
  if (!valid_dtype(dtype)) { set_error("bad dtype"); return LOOPS_ERR_INVALID_ARG; }
  loops_plan_opts o;
  loops_plan_opts_default(&o);
  if (opts) o = *opts;
  loops_status st = validate_csr(A);
  if (st) return st;
  if (!(o.tau >= 0.0)) { set_error("tau must be >= 0 for a host partition"); return LOOPS_ERR_INVALID_ARG; }
  int32_t br;
  if ((st = resolve_block_rows(dtype, o, &br))) return st;
  std::vector<double> vals;
  read_vals_f64(A, vals);
  Canon c;
  if ((st = build_canon(A, vals.data(), dtype, br, o.tau, o.contiguous_split != 0, o.r_boundary,
                        o.tile_min > 1 ? o.tile_min : 0, c)))
    return st;
  fill_partition(c, out);
  return LOOPS_OK;
}

void loops_partition_free(loops_partition* part) {
  if (!part) return;
  void* ptrs[] = {part->csr_rows, part->csr_ptr, part->csr_col, part->csr_val,
                  part->rb_ids, part->rb_ptr, part->tile_col, part->tile_val};
  for (void* q : ptrs) std::free(q);
  std::memset(part, 0, sizeof(*part));
}

loops_status loops_plan(const loops_csr* A, int64_t N, loops_dtype dtype, const loops_plan_opts* opts,
                        loops_stream_t stream, loops_plan_t* out) {
  clear_error();
  NvtxScope nvtx("loops_plan");
  if (!out) { set_error("out is NULL"); return LOOPS_ERR_INVALID_ARG; }
  *out = nullptr;
  if (!valid_dtype(dtype)) { set_error("bad dtype"); return LOOPS_ERR_INVALID_ARG; }
  if (N < 0) { set_error("N < 0"); return LOOPS_ERR_INVALID_ARG; }
  if (N > (1 << 20)) { set_error("N above 2^20 is not supported"); return LOOPS_ERR_UNSUPPORTED; }
  loops_plan_opts o;
  loops_plan_opts_default(&o);
  if (opts) o = *opts;
  if (std::isnan(o.tau)) { set_error("tau is NaN"); return LOOPS_ERR_INVALID_ARG; }
  loops_status st = validate_csr(A);
  if (st) return st;
  int32_t br;
  if ((st = resolve_block_rows(dtype, o, &br))) return st;
  if (o.split_len < 0) { set_error("split_len < 0"); return LOOPS_ERR_INVALID_ARG; }
  if (o.want_backward && o.tile_min > 1) {
    set_error("the tile-level split is not available with want_backward");
    return LOOPS_ERR_UNSUPPORTED;
  }
  std::vector<double> vals;
  read_vals_f64(A, vals);
  double tau = o.tau;
  TunedShape shape{tau, o.tile_min, br, 0, 0};
  int32_t tau_source = o.contiguous_split ? 3 : 0;
  double model_pred = NAN, coef[5] = {0, 0, 0, 0, 0};
  if (tau == LOOPS_TAU_MODEL && !o.contiguous_split) {
    const PlanBuilder host_build = [&](const loops_plan_opts& oc, double t, loops_plan_s** q) {
      return make_plan(A, vals.data(), N, dtype, oc, br, t, false, q);
    };
    BlockProfile prof;
    block_profile(A, br, prof);
    if ((st = model_tau(host_build, prof, A->n_rows, A->n_cols, A->nnz, N, dtype, o.split_len, (cudaStream_t)stream,
                        &tau, &model_pred, coef)))
      return st;
    o.tile_min = 0;
    tau_source = 2;
  } else if (tau < 0.0 && !o.contiguous_split) {
    tau_source = 1;
    const PlanBuilder host_build = [&](const loops_plan_opts& oc, double t, loops_plan_s** q) {
      return make_plan(A, vals.data(), N, dtype, oc, oc.block_rows > 0 ? oc.block_rows : br, t, false, q);
    };
    if ((st = autotune_tau(host_build, A->n_rows, A->n_cols, A->nnz, N, dtype, o.split_len,
                           o.tile_min < 0 && !o.want_backward, br, o.block_rows == 0, (cudaStream_t)stream, &shape)))
      return st;
    tau = shape.tau;
    o.tile_min = shape.tile_min;
    br = o.block_rows = shape.br;
  }
  if (o.contiguous_split && o.r_boundary < 0) {
    const PlanBuilder host_build = [&](const loops_plan_opts& oc, double t, loops_plan_s** q) {
      return make_plan(A, vals.data(), N, dtype, oc, br, t, false, q);
    };
    if ((st = model_boundary(host_build, A->n_rows, A->n_cols, A->nnz, N, dtype, o.split_len,
                             (cudaStream_t)stream, &o.r_boundary)))
      return st;
  }
  loops_plan_s* p = nullptr;
  if ((st = make_plan(A, vals.data(), N, dtype, o, br, tau, false, &p))) return st;
  p->tau_source = tau_source;
  p->csr_vpl = shape.csr_vpl;
  p->bcsr_ntile = shape.bcsr_ntile;
  p->model_gflops = model_pred;
  for (int i = 0; i < 5; ++i) p->model_coef[i] = coef[i];
  if (o.want_backward) {
    std::vector<int64_t> trp;
    std::vector<int32_t> tci;
    transpose_csr(A, trp, tci, p->t_perm);
    std::vector<double> tv((size_t)A->nnz);
    for (size_t e = 0; e < tv.size(); ++e) tv[e] = vals[(size_t)p->t_perm[e]];
    loops_csr At;
    At.n_rows = A->n_cols;
    At.n_cols = A->n_rows;
    At.nnz = A->nnz;
    At.row_ptr = trp.data();
    At.col_idx = tci.data();
    At.vals = tv.data();
    At.vals_dtype = LOOPS_F64;
    loops_plan_opts ot = o;
    ot.want_backward = 0;
    ot.contiguous_split = 0;
    loops_plan_s* pt = nullptr;
    if ((st = make_plan(&At, tv.data(), N, dtype, ot, br, tau, false, &pt))) { destroy_plan(p); return st; }
    p->transposed = pt;
    if ((st = build_sddmm(p, A))) { destroy_plan(p); return st; }
    if ((st = upload_value_maps(p, nullptr))) { destroy_plan(p); return st; }
    if ((st = upload_value_maps(pt, &p->t_perm))) { destroy_plan(p); return st; }
    p->has_vmap = pt->has_vmap = true;
  }
  register_plan(p);
  *out = p;
  return LOOPS_OK;
}

loops_status loops_plan_device(const loops_csr* A, int64_t N, loops_dtype dtype, const loops_plan_opts* opts,
                               loops_stream_t stream, loops_plan_t* out) {
  clear_error();
  NvtxScope nvtx("loops_plan_device");
  if (!out) { set_error("out is NULL"); return LOOPS_ERR_INVALID_ARG; }
  *out = nullptr;
  if (!A) { set_error("A is NULL"); return LOOPS_ERR_INVALID_ARG; }
  if (!valid_dtype(dtype)) { set_error("bad dtype"); return LOOPS_ERR_INVALID_ARG; }
  if (N < 0) { set_error("N < 0"); return LOOPS_ERR_INVALID_ARG; }
  if (N > (1 << 20)) { set_error("N above 2^20 is not supported"); return LOOPS_ERR_UNSUPPORTED; }
  loops_plan_opts o;
  loops_plan_opts_default(&o);
  if (opts) o = *opts;
  if (std::isnan(o.tau)) { set_error("tau is NaN"); return LOOPS_ERR_INVALID_ARG; }
  if (A->vals_dtype != LOOPS_F64 && A->vals_dtype != LOOPS_F32) {
    set_error("A values must be LOOPS_F64 or LOOPS_F32 on input");
    return LOOPS_ERR_UNSUPPORTED;
  }
  loops_status st;
  int32_t br;
  if ((st = resolve_block_rows(dtype, o, &br))) return st;
  if (o.split_len < 0) { set_error("split_len < 0"); return LOOPS_ERR_INVALID_ARG; }
  if (o.want_backward && o.tile_min > 1) {
    set_error("the tile-level split is not available with want_backward");
    return LOOPS_ERR_UNSUPPORTED;
  }
  const cudaStream_t s = (cudaStream_t)stream;
  const DevCsrIn d{A->n_rows, A->n_cols, A->nnz, A->row_ptr, A->col_idx, A->vals, A->vals_dtype == LOOPS_F32};
  double max_abs = 0.0;
  if ((st = validate_csr_device(d, dtype, s, &max_abs))) return st;
  const double scale = plan_scale_from_max(max_abs, dtype);
  const PlanBuilder dev_build = [&](const loops_plan_opts& oc, double t, loops_plan_s** q) {
    return make_plan_device(d, nullptr, scale, N, dtype, oc, oc.block_rows > 0 ? oc.block_rows : br, t, false,
                            false, s, q);
  };
  double tau = o.tau;
  if (tau == LOOPS_TAU_MODEL && !o.contiguous_split) {
    set_error("the performance model (LOOPS_TAU_MODEL) needs host CSR arrays: use loops_plan");
    return LOOPS_ERR_UNSUPPORTED;
  }
  TunedShape shape{tau, o.tile_min, br, 0, 0};
  if (tau < 0.0 && !o.contiguous_split) {
    if ((st = autotune_tau(dev_build, A->n_rows, A->n_cols, A->nnz, N, dtype, o.split_len,
                           o.tile_min < 0 && !o.want_backward, br, o.block_rows == 0, s, &shape)))
      return st;
    tau = shape.tau;
    o.tile_min = shape.tile_min;
    br = o.block_rows = shape.br;
  }
  if (o.contiguous_split && o.r_boundary < 0) {
    if ((st = model_boundary(dev_build, A->n_rows, A->n_cols, A->nnz, N, dtype, o.split_len, s, &o.r_boundary)))
      return st;
  }
  loops_plan_s* p = nullptr;
  if ((st = make_plan_device(d, nullptr, scale, N, dtype, o, br, tau, true, false, s, &p))) return st;
  p->tau_source = o.contiguous_split ? 3 : (o.tau < 0.0 ? 1 : 0);
  p->csr_vpl = shape.csr_vpl;
  p->bcsr_ntile = shape.bcsr_ntile;
  if (o.want_backward) {
    int64_t* trp = nullptr;
    int32_t* tci = nullptr;
    double* tv = nullptr;
    int64_t* perm = nullptr;
    st = transpose_device(d, &trp, &tci, &tv, &perm, s);
    if (!st) {
      const DevCsrIn dt{A->n_cols, A->n_rows, A->nnz, trp, tci, tv, 0};
      loops_plan_opts ot = o;
      ot.want_backward = 0;
      ot.contiguous_split = 0;
      loops_plan_s* pt = nullptr;
      st = make_plan_device(dt, perm, scale, N, dtype, ot, br, tau, true, false, s, &pt);
      p->transposed = pt;
    }
    if (!st) st = build_sddmm_device(p, d, s);
    cudaStreamSynchronize(s);
    void* tmp[] = {trp, tci, tv, perm};
    for (void* q : tmp)
      if (q) cudaFree(q);
    if (st) { destroy_plan(p); return st; }
  }
  cudaError_t e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) { destroy_plan(p); return cuda_status(e, "device plan build"); }
  register_plan(p);
  *out = p;
  return LOOPS_OK;
}

int64_t loops_test_wait_limit(int64_t polls) {
  return g_wait_polls.exchange(polls >= 0 ? polls : (int64_t)kMaxWaitPolls);
}

int64_t loops_test_fail_alloc(int64_t n) {
  const int64_t seen = g_alloc_seen.exchange(0);
  g_alloc_countdown.store(n > 0 ? n : 0);
  return seen;
}

loops_status loops_plan_destroy(loops_plan_t plan) {
  clear_error();
  if (!plan) return LOOPS_OK;
  loops_status st = check_plan(plan);
  if (st) return st;
  unregister_plan(plan);
  cudaDeviceSynchronize();
  destroy_plan(plan);
  return LOOPS_OK;
}

loops_status loops_plan_info_get(loops_plan_t p, loops_plan_info* out) {
  clear_error();
  loops_status st = check_plan(p);
  if (st) return st;
  return plan_info_of(p, out);
}

}  // extern "C"

namespace loops {

loops_status plan_info_of(const loops_plan_s* p, loops_plan_info* out) {
  if (!out) { set_error("out is NULL"); return LOOPS_ERR_INVALID_ARG; }
  std::memset(out, 0, sizeof(*out));
  out->dtype = p->dtype;
  out->block_rows = p->br;
  out->k_pad = p->kpad;
  out->has_backward = p->transposed != nullptr;
  out->n_rows = p->n_rows;
  out->n_cols = p->n_cols;
  out->nnz = p->nnz;
  out->N = p->N;
  out->tau = p->tau;
  out->scale = p->scale;
  out->n_csr_rows = p->n_csr_rows;
  out->nnz_csr = p->nnz_csr;
  out->n_row_blocks = p->n_rb;
  out->n_tiles = p->n_tiles;
  out->nnz_bcsr = p->nnz_bcsr;
  out->n_split_rows = p->dev.csr.n_split;
  out->n_segments = p->dev.csr.n_slots;
  out->n_subnormal_vals = p->n_subnormal;
  out->device_bytes = p->dev.device_bytes + p->other_bytes + p->vmap.bytes;
  out->r_boundary = p->opts.contiguous_split ? p->opts.r_boundary : -1;
  out->tile_min = p->tile_min;
  out->tau_source = p->tau_source;
  out->csr_lane_vectors = p->csr_vpl;
  out->bcsr_col_tile = p->bcsr_ntile;
  out->model_gflops = p->model_gflops;
  for (int i = 0; i < 5; ++i) out->model_coef[i] = p->model_coef[i];
  if (p->transposed)
    out->device_bytes += p->transposed->dev.device_bytes + p->transposed->other_bytes + p->transposed->vmap.bytes;
  return LOOPS_OK;
}

}  // namespace loops

extern "C" {

loops_status loops_plan_export(loops_plan_t p, loops_partition* out) {
  clear_error();
  loops_status st = check_single(p);
  if (st) return st;
  if (!out) { set_error("out is NULL"); return LOOPS_ERR_INVALID_ARG; }
  std::memset(out, 0, sizeof(*out));
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return cuda_status(e, "synchronize before export");
  st = export_part(p, out);
  if (st) loops_partition_free(out);
  return st;
}

loops_status loops_plan_update_values(loops_plan_t p, const void* vals, loops_dtype vd,
                                      loops_stream_t stream) {
  clear_error();
  loops_status st = check_single(p);
  if (st) return st;
  if (!vals && p->nnz) { set_error("vals is NULL"); return LOOPS_ERR_INVALID_ARG; }
  if (vd != LOOPS_F64 && vd != LOOPS_F32) { set_error("vals must be F64 or F32"); return LOOPS_ERR_UNSUPPORTED; }
  if (p->device_built) {  // no host copy of the partition: refresh through the device value maps
    if (!p->has_vmap) {
      set_error("values of a device-built plan with the tile-level split cannot be updated");
      return LOOPS_ERR_UNSUPPORTED;
    }
    const size_t bytes = (size_t)p->nnz * (vd == LOOPS_F64 ? 8 : 4);
    void* dv = nullptr;
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = bytes ? dev_malloc(&dv, bytes) : cudaSuccess;
    if (e == cudaSuccess && bytes) e = cudaMemcpyAsync(dv, vals, bytes, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = launch_set_values(p, dv, vd, s);
    if (e == cudaSuccess && p->transposed) e = launch_set_values(p->transposed, dv, vd, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (dv) cudaFree(dv);
    return cuda_status(e, "value update");
  }
  std::vector<double> v((size_t)p->nnz);
  for (int64_t k = 0; k < p->nnz; ++k) v[(size_t)k] = vd == LOOPS_F64 ? ((const double*)vals)[k] : (double)((const float*)vals)[k];
  cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_status(e, "synchronize before value update");
  auto refresh = [](loops_plan_s* q, const std::vector<double>& vv) -> loops_status {
    Canon& c = q->canon;
    std::fill(c.tile_val.begin(), c.tile_val.end(), 0.0);
    std::vector<double> raw_tile(c.tile_val.size(), 0.0);
    for (size_t k = 0; k < vv.size(); ++k) {
      if (c.src_kind[k] == 0) c.csr_val[(size_t)c.src_slot[k]] = round_store(vv[k], c.scale, q->dtype);
      else raw_tile[(size_t)c.src_slot[k]] += vv[k];
    }
    for (size_t x = 0; x < raw_tile.size(); ++x) c.tile_val[x] = round_store(raw_tile[x], c.scale, q->dtype);
    const int64_t N = q->N;
    free_part(q->dev);
    return upload_part(q, N);
  };
  if ((st = refresh(p, v))) return st;
  if (p->transposed) {
    std::vector<double> tv(v.size());
    for (size_t x = 0; x < tv.size(); ++x) tv[x] = v[(size_t)p->t_perm[x]];
    if ((st = refresh(p->transposed, tv))) return st;
  }
  return LOOPS_OK;
}

loops_status loops_plan_set_values(loops_plan_t p, const void* vals, loops_dtype vd, loops_stream_t stream) {
  clear_error();
  loops_status st = check_single(p);
  if (st) return st;
  if (!p->has_vmap) {
    set_error("plan has no device value maps (built on the host without want_backward, or with the "
              "tile-level split)");
    return LOOPS_ERR_STATE;
  }
  if (vd != LOOPS_F64 && vd != LOOPS_F32) { set_error("vals must be F64 or F32"); return LOOPS_ERR_UNSUPPORTED; }
  if (!vals && p->nnz) { set_error("vals is NULL"); return LOOPS_ERR_INVALID_ARG; }
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = launch_set_values(p, vals, vd, s);
  if (e == cudaSuccess && p->transposed) e = launch_set_values(p->transposed, vals, vd, s);
  return cuda_status(e, "value refresh launch");
}

loops_status loops_spmm(loops_plan_t p, const void* B, int64_t ldb, void* C, int64_t ldc,
                        loops_stream_t stream) {
  return loops_spmm_scaled(p, B, ldb, nullptr, C, ldc, stream);
}

loops_status loops_spmm_scaled(loops_plan_t p, const void* B, int64_t ldb, const float* col_scale,
                               void* C, int64_t ldc, loops_stream_t stream) {
  clear_error();
  NvtxScope nvtx("loops_spmm");
  loops_status st = check_single(p);
  if (st) return st;
  if ((st = check_dense(B, p->n_cols, p->N, ldb, "B"))) return st;
  if ((st = check_dense(C, p->n_rows, p->N, ldc, "C"))) return st;
  if (col_scale && (p->dtype == LOOPS_F64 || p->dtype == LOOPS_F32)) {
    set_error("col_scale is only defined for the 16-bit dtypes");
    return LOOPS_ERR_INVALID_ARG;
  }
  return run_spmm(p, B, ldb, col_scale, C, ldc, (cudaStream_t)stream);
}

loops_status loops_spmm_host(loops_plan_t p, const void* B_host, int64_t ldb, void* C_host, int64_t ldc,
                             loops_stream_t stream) {
  clear_error();
  NvtxScope nvtx("loops_spmm_host");
  loops_status st = check_single(p);
  if (st) return st;
  if ((st = check_dense(B_host, p->n_cols, p->N, ldb, "B"))) return st;
  if ((st = check_dense(C_host, p->n_rows, p->N, ldc, "C"))) return st;
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t eb = dense_elem_bytes(p->dtype), ec = out_elem_bytes(p->dtype);
  const int64_t need_B = p->n_cols * p->N * eb, need_C = p->n_rows * p->N * ec;
  cudaError_t e = cudaSuccess;
  if (need_B > p->stage_B_bytes) {
    if (p->stage_B) cudaFree(p->stage_B);
    p->stage_B = nullptr;
    p->stage_B_bytes = 0;
    e = dev_malloc(&p->stage_B, (size_t)need_B);
    if (e != cudaSuccess) return cuda_status(e, "staging allocation");
    p->stage_B_bytes = need_B;
  }
  if (need_C > p->stage_C_bytes) {
    if (p->stage_C) cudaFree(p->stage_C);
    p->stage_C = nullptr;
    p->stage_C_bytes = 0;
    e = dev_malloc(&p->stage_C, (size_t)need_C);
    if (e != cudaSuccess) return cuda_status(e, "staging allocation");
    p->stage_C_bytes = need_C;
  }
  if (need_B && ldb == p->N)
    e = cudaMemcpyAsync(p->stage_B, B_host, (size_t)need_B, cudaMemcpyHostToDevice, s);
  else if (need_B)
    e = cudaMemcpy2DAsync(p->stage_B, (size_t)(p->N * eb), B_host, (size_t)(ldb * eb), (size_t)(p->N * eb),
                          (size_t)p->n_cols, cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return cuda_status(e, "host-to-device copy");
  if ((st = run_spmm(p, p->stage_B, p->N, nullptr, p->stage_C, p->N, s))) return st;
  if (need_C && ldc == p->N)
    e = cudaMemcpyAsync(C_host, p->stage_C, (size_t)need_C, cudaMemcpyDeviceToHost, s);
  else if (need_C)
    e = cudaMemcpy2DAsync(C_host, (size_t)(ldc * ec), p->stage_C, (size_t)(p->N * ec), (size_t)(p->N * ec),
                          (size_t)p->n_rows, cudaMemcpyDeviceToHost, s);
  if (e != cudaSuccess) return cuda_status(e, "device-to-host copy");
  return cuda_status(cudaStreamSynchronize(s), "synchronize");
}

loops_status loops_spmm_host_async(loops_plan_t p, const void* B_host, int64_t ldb, void* C_host, int64_t ldc,
                                   loops_stream_t stream) {
  clear_error();
  NvtxScope nvtx("loops_spmm_host_async");
  loops_status st = check_single(p);
  if (st) return st;
  if ((st = check_dense(B_host, p->n_cols, p->N, ldb, "B"))) return st;
  if ((st = check_dense(C_host, p->n_rows, p->N, ldc, "C"))) return st;
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t eb = dense_elem_bytes(p->dtype), ec = out_elem_bytes(p->dtype);
  const int64_t need_B = p->n_cols * p->N * eb, need_C = p->n_rows * p->N * ec;
  cudaError_t e = cudaSuccess;
  if (!p->pipe) {
    HostPipe* h = new (std::nothrow) HostPipe();
    if (!h) { set_error("host allocation failed"); return LOOPS_ERR_OOM; }
    e = cudaStreamCreateWithFlags(&h->s_in, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&h->s_out, cudaStreamNonBlocking);
    for (int i = 0; i < 2 && e == cudaSuccess; ++i) {
      e = cudaEventCreateWithFlags(&h->in_done[i], cudaEventDisableTiming);
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->compute_done[i], cudaEventDisableTiming);
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->out_done[i], cudaEventDisableTiming);
      if (e == cudaSuccess) e = dev_malloc(&h->B[i], (size_t)std::max<int64_t>(need_B, 16));
      if (e == cudaSuccess) e = dev_malloc(&h->C[i], (size_t)std::max<int64_t>(need_C, 16));
    }
    if (e != cudaSuccess) { destroy_pipe(h); return cuda_status(e, "host pipeline setup"); }
    h->B_bytes = need_B;
    h->C_bytes = need_C;
    p->pipe = h;
  }
  HostPipe* h = p->pipe;
  const int i = h->next;
  h->next ^= 1;
  // copy in: after the call that last used this buffer set has finished reading it
  if (h->used[i]) e = cudaStreamWaitEvent(h->s_in, h->compute_done[i], 0);
  if (e == cudaSuccess && need_B) {
    if (ldb == p->N)
      e = cudaMemcpyAsync(h->B[i], B_host, (size_t)need_B, cudaMemcpyHostToDevice, h->s_in);
    else
      e = cudaMemcpy2DAsync(h->B[i], (size_t)(p->N * eb), B_host, (size_t)(ldb * eb), (size_t)(p->N * eb),
                            (size_t)p->n_cols, cudaMemcpyHostToDevice, h->s_in);
  }
  if (e == cudaSuccess) e = cudaEventRecord(h->in_done[i], h->s_in);
  // compute on the caller's stream once B is in and the previous copy-out of this C set is done
  if (e == cudaSuccess) e = cudaStreamWaitEvent(s, h->in_done[i], 0);
  if (e == cudaSuccess && h->used[i]) e = cudaStreamWaitEvent(s, h->out_done[i], 0);
  if (e != cudaSuccess) return cuda_status(e, "host pipeline");
  if ((st = run_spmm(p, h->B[i], p->N, nullptr, h->C[i], p->N, s))) return st;
  e = cudaEventRecord(h->compute_done[i], s);
  // copy out on its own stream: the next call's copy-in and SpMM overlap it; the caller's
  // stream waits for it only in loops_spmm_host_flush (or when this C set is reused)
  if (e == cudaSuccess) e = cudaStreamWaitEvent(h->s_out, h->compute_done[i], 0);
  if (e == cudaSuccess && need_C) {
    if (ldc == p->N)
      e = cudaMemcpyAsync(C_host, h->C[i], (size_t)need_C, cudaMemcpyDeviceToHost, h->s_out);
    else
      e = cudaMemcpy2DAsync(C_host, (size_t)(ldc * ec), h->C[i], (size_t)(p->N * ec), (size_t)(p->N * ec),
                            (size_t)p->n_rows, cudaMemcpyDeviceToHost, h->s_out);
  }
  if (e == cudaSuccess) e = cudaEventRecord(h->out_done[i], h->s_out);
  h->used[i] = true;
  h->last = i;
  return cuda_status(e, "host pipeline");
}

loops_status loops_spmm_host_flush(loops_plan_t p, loops_stream_t stream) {
  clear_error();
  loops_status st = check_single(p);
  if (st) return st;
  if (!p->pipe || p->pipe->last < 0) return LOOPS_OK;
  return cuda_status(cudaStreamWaitEvent((cudaStream_t)stream, p->pipe->out_done[p->pipe->last], 0),
                     "host pipeline flush");
}

loops_status loops_spmm_backward_scaled(loops_plan_t p, const void* dC, int64_t lddc, const float* dc_scale,
                                        const void* B, int64_t ldb, const float* b_scale, void* dB, int64_t lddb,
                                        void* dvals, loops_stream_t stream) {
  clear_error();
  NvtxScope nvtx("loops_spmm_backward");
  loops_status st = check_single(p);
  if (st) return st;
  if (!p->transposed) {
    set_error("plan was built without want_backward");
    return LOOPS_ERR_STATE;
  }
  if ((dc_scale || b_scale) && p->dtype != LOOPS_F16 && p->dtype != LOOPS_BF16) {
    set_error("dc_scale and b_scale are only defined for the 16-bit dtypes");
    return LOOPS_ERR_INVALID_ARG;
  }
  if ((st = check_dense(dC, p->n_rows, p->N, lddc, "dC"))) return st;
  cudaStream_t s = (cudaStream_t)stream;
  if (dB) {
    if ((st = check_dense(dB, p->n_cols, p->N, lddb, "dB"))) return st;
    // dB = A^T . (dC diag(dc_scale)) = (A^T . dC) diag(dc_scale): the column scales of the
    // transposed SpMM's epilogue
    if ((st = run_spmm(p->transposed, dC, lddc, dc_scale, dB, lddb, s))) return st;
  }
  if (dvals && p->nnz > 0) {
    if ((st = check_dense(B, p->n_cols, p->N, ldb, "B"))) return st;
    if ((st = cuda_status(launch_sddmm(p, dC, lddc, B, ldb, dvals, dc_scale, b_scale, s), "SDDMM launch")))
      return st;
  }
  return LOOPS_OK;
}

loops_status loops_spmm_backward(loops_plan_t p, const void* dC, int64_t lddc, const void* B, int64_t ldb,
                                 void* dB, int64_t lddb, void* dvals, loops_stream_t stream) {
  return loops_spmm_backward_scaled(p, dC, lddc, nullptr, B, ldb, nullptr, dB, lddb, dvals, stream);
}

loops_status loops_cast_scaled(const float* X, int64_t rows, int64_t cols, int64_t ldx, loops_dtype yd,
                               void* Y, int64_t ldy, float* col_scale, loops_stream_t stream) {
  clear_error();
  if (yd != LOOPS_F16 && yd != LOOPS_BF16) { set_error("y_dtype must be F16 or BF16"); return LOOPS_ERR_UNSUPPORTED; }
  if (rows < 0 || cols < 0 || ldx < cols || ldy < cols) { set_error("bad sizes"); return LOOPS_ERR_INVALID_ARG; }
  if (cols == 0) return LOOPS_OK;
  if (!col_scale || (rows > 0 && (!X || !Y))) { set_error("NULL pointer"); return LOOPS_ERR_INVALID_ARG; }
  return cuda_status(launch_cast_scaled(X, rows, cols, ldx, yd, Y, ldy, col_scale, (cudaStream_t)stream),
                     "cast launch");
}

loops_status loops_plan_set_timing_events(loops_plan_t p, void* const* events) {
  clear_error();
  loops_status st = check_plan(p);
  if (st) return st;
  if (!events) {
    p->timing = false;
    for (auto& ev : p->tev) ev = nullptr;
    if (p->batch) batch_set_timing(p->batch, nullptr);
    return LOOPS_OK;
  }
  for (int i = 0; i < 4; ++i) {
    if (!events[i]) { set_error("timing event is NULL"); return LOOPS_ERR_INVALID_ARG; }
    p->tev[i] = (cudaEvent_t)events[i];
  }
  p->timing = true;
  if (p->batch) batch_set_timing(p->batch, p->tev);
  return LOOPS_OK;
}

loops_status loops_plan_check(loops_plan_t p, loops_stream_t stream) {
  clear_error();
  loops_status st = check_single(p);
  if (st) return st;
  int32_t h = 0;
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = cudaMemcpyAsync(&h, p->d_error, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(p->d_error, 0, sizeof(int32_t), s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_status(e, "read error word");
  if (p->transposed) {
    int32_t ht = 0;
    e = cudaMemcpyAsync(&ht, p->transposed->d_error, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(p->transposed->d_error, 0, sizeof(int32_t), s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_status(e, "read error word");
    h |= ht;
  }
  if (h & kErrWaitTimeout) {
    set_error("a device-side wait exceeded its bound");
    return LOOPS_ERR_TIMEOUT;
  }
  return LOOPS_OK;
}

}  // extern "C"
