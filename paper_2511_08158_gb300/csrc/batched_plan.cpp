// Batched plans: many sparse matrices of uneven size and N behind one plan, executed by one
// persistent kernel launch that is captured in a CUDA graph on the first call and replayed.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <functional>

#include "loops_internal.h"

namespace loops {

struct BatchState {
  std::vector<loops_plan_s*> subs;
  int32_t count = 0;
  loops_dtype dtype = LOOPS_F32;
  int32_t br = 16;
  double tau = 2.0;
  BatchDesc* h_desc = nullptr;        // pinned host copy of the descriptors
  BatchDesc* d_desc = nullptr;
  BatchTask* d_tasks = nullptr;
  int2* d_splits = nullptr;
  int2* d_bsplits = nullptr;
  int64_t n_tasks = 0, n_splits = 0, n_bsplits = 0;
  std::vector<BatchClass> classes;    // task classes, one persistent kernel each
  unsigned long long* d_counters = nullptr;  // one task counter per class
  cudaStream_t cap = nullptr;         // capture stream
  std::vector<cudaStream_t> side;     // extra branches of the captured graph
  std::vector<cudaEvent_t> ev_join;   // one per extra branch
  cudaEvent_t ev_fork = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaEvent_t ev_copied = nullptr;    // the last descriptor upload has read h_desc
  bool copied_once = false;
  int64_t device_bytes = 0;
  int64_t total_nnz = 0, total_rows = 0;
  std::vector<uint8_t> owned;         // subs[m] is owned (freed with the batch) or borrowed
  int32_t tau_source = 0;             // 0 given, 1 timed autotuner, 2 performance model
  double model_gflops = NAN;          // Eq. 2 prediction for the per-matrix choice
  double model_measured_gflops = NAN; // the per-matrix choice, measured
  double timed_best_gflops = NAN;     // the best single-threshold candidate, measured
  cudaEvent_t tev[4] = {nullptr, nullptr, nullptr, nullptr};  // caller's timing events
  cudaGraphNode_t tev_node[4] = {nullptr, nullptr, nullptr, nullptr};  // their nodes in `graph`
  bool timing = false;
  // loops_spmm_batched_host: one device staging area (every B, then every C, dense rows)
  void* stage = nullptr;
  int64_t stage_bytes = 0;
  // host copies of the task list (sorted) and of the partial-sum lists, for the host call's
  // groups of matrices
  std::vector<BatchTask> h_tasks;
  std::vector<int2> h_splits, h_bsplits;
  // loops_spmm_batched_host pipeline: consecutive matrices in groups; group g's copies in,
  // kernels and copies out overlap the neighbouring groups' on three streams
  struct HostGroup {
    int32_t m0 = 0, m1 = 0;           // matrices [m0, m1)
    std::vector<BatchClass> classes;  // the classes' sub-runs of the task list for these matrices
    int64_t split0 = 0, n_splits = 0, bsplit0 = 0, n_bsplits = 0;
    int64_t counter0 = 0;             // first of its task counters in d_gcounters
  };
  std::vector<HostGroup> groups;
  unsigned long long* d_gcounters = nullptr;
  cudaStream_t copy_in = nullptr, copy_out = nullptr;
  cudaEvent_t ev_start = nullptr, ev_fin = nullptr;
  std::vector<cudaEvent_t> ev_in, ev_out;
};

void batch_set_timing(BatchState* b, const cudaEvent_t* ev) {
  // new events for a graph that already records events: point its event nodes at them (the
  // launches already queued keep the old ones), with no capture or instantiation
  if (ev && b->timing && b->exec && b->tev_node[0] && b->tev_node[1] && b->tev_node[2] && b->tev_node[3]) {
    bool ok = true;
    for (int i = 0; i < 4 && ok; ++i) ok = cudaGraphExecEventRecordNodeSetEvent(b->exec, b->tev_node[i], ev[i]) == cudaSuccess;
    if (ok) {
      for (int i = 0; i < 4; ++i) b->tev[i] = ev[i];
      return;
    }
    cudaGetLastError();
  }
  b->timing = ev != nullptr;
  for (int i = 0; i < 4; ++i) {
    b->tev[i] = ev ? ev[i] : nullptr;
    b->tev_node[i] = nullptr;
  }
  // the next call captures the graph again, with or without the event nodes
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->exec = nullptr;
  b->graph = nullptr;
}

namespace {

// The event-record nodes of a captured graph that record the caller's timing events.
void find_timing_nodes(BatchState* b) {
  for (auto& n : b->tev_node) n = nullptr;
  if (!b->timing || !b->graph) return;
  size_t n = 0;
  if (cudaGraphGetNodes(b->graph, nullptr, &n) != cudaSuccess) { cudaGetLastError(); return; }
  std::vector<cudaGraphNode_t> nodes(n);
  if (n && cudaGraphGetNodes(b->graph, nodes.data(), &n) != cudaSuccess) { cudaGetLastError(); return; }
  for (cudaGraphNode_t node : nodes) {
    cudaGraphNodeType t;
    cudaEvent_t e = nullptr;
    if (cudaGraphNodeGetType(node, &t) != cudaSuccess || t != cudaGraphNodeTypeEventRecord) continue;
    if (cudaGraphEventRecordNodeGetEvent(node, &e) != cudaSuccess) continue;
    for (int i = 0; i < 4; ++i)
      if (e == b->tev[i] && !b->tev_node[i]) { b->tev_node[i] = node; break; }
  }
  cudaGetLastError();
}

}  // namespace

void destroy_batch(BatchState* b) {
  if (!b) return;
  for (size_t m = 0; m < b->subs.size(); ++m)
    if (b->subs[m] && (m >= b->owned.size() || b->owned[m])) destroy_plan(b->subs[m]);
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  if (b->h_desc) cudaFreeHost(b->h_desc);
  void* ptrs[] = {b->d_desc, b->d_tasks, b->d_splits, b->d_bsplits, b->d_counters, b->stage, b->d_gcounters};
  for (void* q : ptrs)
    if (q) cudaFree(q);
  if (b->cap) cudaStreamDestroy(b->cap);
  for (cudaStream_t x : b->side)
    if (x) cudaStreamDestroy(x);
  for (cudaEvent_t x : b->ev_join)
    if (x) cudaEventDestroy(x);
  if (b->ev_fork) cudaEventDestroy(b->ev_fork);
  if (b->ev_copied) cudaEventDestroy(b->ev_copied);
  for (cudaStream_t x : {b->copy_in, b->copy_out})
    if (x) cudaStreamDestroy(x);
  for (cudaEvent_t x : {b->ev_start, b->ev_fin})
    if (x) cudaEventDestroy(x);
  for (cudaEvent_t x : b->ev_in)
    if (x) cudaEventDestroy(x);
  for (cudaEvent_t x : b->ev_out)
    if (x) cudaEventDestroy(x);
  delete b;
}

// Library kernels one call launches, and the task classes (one persistent kernel each).
int batch_classes(const BatchState* b) { return (int)b->classes.size(); }
int batch_kernels_per_call(const BatchState* b) {
  return batch_classes(b) + (b->n_splits > 0) + (b->n_bsplits > 0);
}

namespace {

int elems_per_16b(loops_dtype d) { return d == LOOPS_F32 ? 4 : 8; }

// Branches of the captured graph: the class kernels are dealt to this many parallel branches
// (their tails overlap); 1 runs every class in turn on one stream.
#ifndef LOOPS_BATCHED_BRANCHES
#define LOOPS_BATCHED_BRANCHES 4
#endif

int next_pow2(int64_t x) {
  int p = 1;
  while (p < x && p < 32) p <<= 1;
  return p;
}

// Class of a matrix's CSR items: G lanes per item with VPL 16-byte column vectors each. FP32
// rows take two vectors per lane once they have at least LOOPS_BATCHED_CSR_VPL2 of them (fewer
// lanes per item, more items per warp); 16-bit rows (at most 16 vectors) always take one,
// which measured faster (their unpacked vectors double the registers of a second one).
#ifndef LOOPS_BATCHED_CSR_VPL2
#define LOOPS_BATCHED_CSR_VPL2 16
#endif
void csr_shape(loops_dtype dtype, int64_t N, int32_t* G, int32_t* vpl) {
  const int64_t nvec = N / elems_per_16b(dtype);
  *vpl = dtype == LOOPS_F32 && nvec >= LOOPS_BATCHED_CSR_VPL2 ? 2 : 1;
  *G = next_pow2(*vpl == 2 ? (nvec + 1) / 2 : nvec);
}

// Class key: kind, then group width, then vectors per lane (CSR) or tile height (F32 BCSR,
// 8 or 16, stored as 8 -> 8, 16 -> 0 in the low four bits).
int64_t class_key(int32_t kind, int32_t G, int32_t low) { return ((int64_t)kind << 16) | (G << 4) | (low & 0xf); }

// Builds the sub-plan of matrix m for the given options, tile height and threshold.
using SubBuilder = std::function<loops_status(int32_t m, const loops_plan_opts& o, int32_t br, double tau,
                                              loops_plan_s** out)>;

// Build the sub-plans (matrix m with tile height brs[m] and threshold taus[m]; or, with
// `borrowed`, take those sub-plans without owning them), the task list and the descriptor
// tables.
loops_status build_batch(const loops_csr* As, const int64_t* Ns, int32_t count, loops_dtype dtype,
                         const loops_plan_opts& o, const std::vector<int32_t>& brs, const std::vector<double>& taus,
                         const SubBuilder& sub, const std::vector<loops_plan_s*>* borrowed, BatchState** out) {
  *out = nullptr;
  BatchState* b = new (std::nothrow) BatchState();
  if (!b) { set_error("host allocation failed"); return LOOPS_ERR_OOM; }
  b->count = count;
  b->dtype = dtype;
  b->br = count > 0 ? brs[0] : 16;
  b->tau = count > 0 ? taus[0] : 2.0;
  for (int32_t m = 1; m < count; ++m) {
    if (brs[(size_t)m] != b->br) b->br = 0;
    if (!(taus[(size_t)m] == b->tau)) b->tau = NAN;
  }
  loops_status st = LOOPS_OK;
  const int VE = elems_per_16b(dtype);
  std::vector<BatchTask> tasks;
  std::vector<double> cost;
  std::vector<int64_t> cls;                       // class key of each task
  std::vector<int2> splits, bsplits;
  for (int32_t m = 0; m < count && !st; ++m) {
    const int64_t N = Ns[m];
    if (N <= 0 || N % VE != 0 || N > (dtype == LOOPS_F32 ? 32 * VE : 128)) {
      set_error("batched SpMM needs N a positive multiple of " + std::to_string(VE) + " and at most " +
                std::to_string(dtype == LOOPS_F32 ? 32 * VE : 128) + " (matrix " + std::to_string(m) + ")");
      st = LOOPS_ERR_UNSUPPORTED;
      break;
    }
    const int32_t br = brs[(size_t)m];
    loops_plan_s* p = nullptr;
    if (borrowed) {
      p = (*borrowed)[(size_t)m];
    } else {
      loops_plan_opts om = o;
      om.block_rows = br;
      if ((st = sub(m, om, br, taus[(size_t)m], &p))) break;
    }
    b->subs.push_back(p);
    b->owned.push_back(borrowed ? 0 : 1);
    b->total_nnz += As[m].nnz;
    b->total_rows += As[m].n_rows;
    int32_t G = 0, vpl = 0;
    csr_shape(dtype, N, &G, &vpl);
    const int per_round = 32 / G;
    // CSR items: consecutive items (similar length, longest first) up to ~1024 entries
    const CsrDev& c = p->dev.csr;
    for (int64_t i = 0; i < c.n_items;) {
      int64_t j = i, nnz = 0;
      while (j < c.n_items && (j - i) < (int64_t)32 * per_round && (nnz < 1024 || (j - i) < per_round)) {
        nnz += c.h_item_ptr[(size_t)j + 1] - c.h_item_ptr[(size_t)j];
        ++j;
      }
      tasks.push_back({m, 0, i, (int32_t)(j - i), 0});
      cost.push_back((double)(nnz + (j - i)) * (double)N);
      cls.push_back(class_key(0, G, vpl));
      i = j;
    }
    // BCSR units (most tiles first): F32 in groups of G lanes (4 columns each), 16-bit one per warp
    const BcsrDev& bd = p->dev.bcsr;
    if (dtype == LOOPS_F32) {
      const int32_t Gf = next_pow2(N / VE);
      const int rf = 32 / Gf;
      for (int64_t q = 0; q < bd.n_units; q += rf) {
        const int32_t cnt = (int32_t)std::min<int64_t>(rf, bd.n_units - q);
        tasks.push_back({m, 1, q, cnt, 0});
        cost.push_back((double)bd.h_unit_tiles[(size_t)q] * br * (double)N);
        cls.push_back(class_key(1, Gf, br));
      }
    } else {
      for (int64_t q = 0; q < bd.n_units; ++q) {
        tasks.push_back({m, 2, q, 1, 0});
        cost.push_back((double)bd.h_unit_tiles[(size_t)q] * br * (double)N);
        cls.push_back(class_key(2, 0, 0));
      }
    }
    for (int64_t sidx = 0; sidx < bd.n_split; ++sidx) bsplits.push_back(make_int2(m, (int)sidx));
    for (int64_t sidx = 0; sidx < c.n_split; ++sidx) splits.push_back(make_int2(m, (int)sidx));
  }
  if (st) { destroy_batch(b); return st; }
  // Task order: by class (each class is one kernel's contiguous run of the list), then matrix
  // by matrix, and within a matrix by decreasing cost. The warps of a class kernel claim
  // tasks in this order, so they work on one or a few matrices at a time, whose B operands
  // stay in L2 while their rows gather from them.
  std::vector<int64_t> idx(tasks.size());
  for (size_t i = 0; i < idx.size(); ++i) idx[i] = (int64_t)i;
  std::stable_sort(idx.begin(), idx.end(), [&](int64_t x, int64_t y) {
    if (cls[(size_t)x] != cls[(size_t)y]) return cls[(size_t)x] < cls[(size_t)y];
    if (tasks[(size_t)x].m != tasks[(size_t)y].m) return tasks[(size_t)x].m < tasks[(size_t)y].m;
    return cost[(size_t)x] > cost[(size_t)y];
  });
  std::vector<BatchTask> sorted(tasks.size());
  for (size_t i = 0; i < idx.size(); ++i) sorted[i] = tasks[(size_t)idx[i]];
  for (size_t i = 0; i < idx.size();) {
    size_t j = i;
    const int64_t key = cls[(size_t)idx[i]];
    while (j < idx.size() && cls[(size_t)idx[j]] == key) ++j;
    BatchClass bc;
    bc.kind = (int32_t)(key >> 16);
    bc.G = (int32_t)((key >> 4) & 0xfff);
    bc.vpl = bc.kind == 0 ? (int32_t)(key & 0xf) : 1;
    bc.br = (bc.kind == 1 && (key & 0xf) == 8) ? 8 : 16;
    bc.first = (int64_t)i;
    bc.n_tasks = (int64_t)(j - i);
    bc.grid = batched_class_grid(dtype, bc);
    if (bc.grid <= 0) {
      set_error("no batched kernel for a task class (kind " + std::to_string(bc.kind) + ", G " +
                std::to_string(bc.G) + ")");
      destroy_batch(b);
      return LOOPS_ERR_STATE;
    }
    b->classes.push_back(bc);
    i = j;
  }
  b->n_tasks = (int64_t)sorted.size();
  b->n_splits = (int64_t)splits.size();
  b->n_bsplits = (int64_t)bsplits.size();
  // descriptors (static parts now; B/C pointers per call)
  cudaError_t e = host_malloc((void**)&b->h_desc, sizeof(BatchDesc) * (size_t)std::max(count, 1));
  if (e == cudaSuccess) e = dev_malloc((void**)&b->d_desc, sizeof(BatchDesc) * (size_t)std::max(count, 1));
  if (e == cudaSuccess && b->n_tasks) e = dev_malloc((void**)&b->d_tasks, sizeof(BatchTask) * (size_t)b->n_tasks);
  if (e == cudaSuccess && b->n_tasks)
    e = cudaMemcpy(b->d_tasks, sorted.data(), sizeof(BatchTask) * (size_t)b->n_tasks, cudaMemcpyHostToDevice);
  if (e == cudaSuccess && b->n_splits) e = dev_malloc((void**)&b->d_splits, sizeof(int2) * (size_t)b->n_splits);
  if (e == cudaSuccess && b->n_splits)
    e = cudaMemcpy(b->d_splits, splits.data(), sizeof(int2) * (size_t)b->n_splits, cudaMemcpyHostToDevice);
  if (e == cudaSuccess && b->n_bsplits) e = dev_malloc((void**)&b->d_bsplits, sizeof(int2) * (size_t)b->n_bsplits);
  if (e == cudaSuccess && b->n_bsplits)
    e = cudaMemcpy(b->d_bsplits, bsplits.data(), sizeof(int2) * (size_t)b->n_bsplits, cudaMemcpyHostToDevice);
  if (e == cudaSuccess && !b->classes.empty())
    e = dev_malloc((void**)&b->d_counters, sizeof(unsigned long long) * b->classes.size());
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
  const int n_side = std::min<int>(LOOPS_BATCHED_BRANCHES, (int)b->classes.size()) - 1;
  if (e == cudaSuccess && n_side > 0) e = cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming);
  for (int i = 0; i < n_side && e == cudaSuccess; ++i) {
    cudaStream_t x = nullptr;
    cudaEvent_t j = nullptr;
    e = cudaStreamCreateWithFlags(&x, cudaStreamNonBlocking);
    if (e == cudaSuccess) b->side.push_back(x);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&j, cudaEventDisableTiming);
    if (e == cudaSuccess) b->ev_join.push_back(j);
  }
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_copied, cudaEventDisableTiming);
  if (e != cudaSuccess) { st = cuda_status(e, "batched plan setup"); destroy_batch(b); return st; }
  b->device_bytes = (int64_t)(sizeof(BatchDesc) * count + sizeof(BatchTask) * b->n_tasks +
                              sizeof(int2) * (b->n_splits + b->n_bsplits));
  for (int32_t m = 0; m < count; ++m) {
    const loops_plan_s* p = b->subs[(size_t)m];
    BatchDesc& d = b->h_desc[m];
    std::memset(&d, 0, sizeof(d));
    d.item_row = p->dev.csr.item_row;
    d.item_ptr = p->dev.csr.item_ptr;
    d.col = p->dev.csr.col;
    d.val = p->dev.csr.val;
    d.rb_id = p->dev.bcsr.rb_id;
    d.rb_ptr = p->dev.bcsr.rb_ptr;
    d.tile_col = p->dev.bcsr.tile_col;
    d.tile_val = p->dev.bcsr.tile_val;
    d.unit_block = p->dev.bcsr.unit_block;
    d.unit_t0 = p->dev.bcsr.unit_t0;
    d.unit_t1 = p->dev.bcsr.unit_t1;
    d.unit_slot = p->dev.bcsr.unit_slot;
    d.bscratch = p->dev.bcsr.scratch;
    d.bsplit_block = p->dev.bcsr.split_block;
    d.bsplit_slot_ptr = p->dev.bcsr.split_slot_ptr;
    d.br = p->br;
    d.scratch = p->dev.csr.scratch;
    d.split_row = p->dev.csr.split_row;
    d.split_slot_ptr = p->dev.csr.split_slot_ptr;
    d.N = p->N;
    d.n_rows = p->n_rows;
    d.inv_scale = (float)(1.0 / p->scale);
    b->device_bytes += p->dev.device_bytes;
  }
  b->h_tasks = std::move(sorted);
  b->h_splits = std::move(splits);
  b->h_bsplits = std::move(bsplits);
  *out = b;
  return LOOPS_OK;
}

cudaError_t run_batch(BatchState* b, cudaStream_t s) {
  BatchLaunch L;
  L.descs = b->d_desc;
  L.tasks = b->d_tasks;
  L.classes = b->classes.data();
  L.n_classes = (int)b->classes.size();
  L.counters = b->d_counters;
  L.splits = b->d_splits;
  L.n_splits = b->n_splits;
  L.bsplits = b->d_bsplits;
  L.n_bsplits = b->n_bsplits;
  L.tev = b->timing ? b->tev : nullptr;
  L.n_side = (int)b->side.size();
  L.side = b->side.data();
  L.fork = b->ev_fork;
  L.join = b->ev_join.data();
  return launch_batched(b->dtype, L, s);
}

// Refresh the descriptors' dense pointers if they changed: one upload from the pinned copy,
// which is not rewritten before the previous upload has read it.
cudaError_t refresh_descs(BatchState* b, const void* const* Bs, const int64_t* ldbs, void* const* Cs,
                          const int64_t* ldcs, const float* const* col_scales, cudaStream_t s) {
  bool changed = !b->copied_once;
  for (int32_t m = 0; m < b->count && !changed; ++m) {
    const BatchDesc& d = b->h_desc[m];
    const float* cs = col_scales ? col_scales[m] : nullptr;
    changed = d.B != Bs[m] || d.C != Cs[m] || d.ldb != ldbs[m] || d.ldc != ldcs[m] || d.col_scale != cs;
  }
  cudaError_t e = cudaSuccess;
  if (changed) {
    if (b->copied_once) {
      e = cudaEventSynchronize(b->ev_copied);
      if (e != cudaSuccess) return e;
    }
    for (int32_t m = 0; m < b->count; ++m) {
      BatchDesc& d = b->h_desc[m];
      d.B = Bs[m];
      d.C = Cs[m];
      d.ldb = ldbs[m];
      d.ldc = ldcs[m];
      d.col_scale = col_scales ? col_scales[m] : nullptr;
    }
    e = cudaMemcpyAsync(b->d_desc, b->h_desc, sizeof(BatchDesc) * (size_t)b->count, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaEventRecord(b->ev_copied, s);
    if (e != cudaSuccess) return e;
    b->copied_once = true;
  }
  return cudaSuccess;
}

// Per call: refresh the descriptors, then replay the captured graph (the class kernels, plus
// the partial sums if any).
loops_status spmm_batch(BatchState* b, const void* const* Bs, const int64_t* ldbs, void* const* Cs,
                        const int64_t* ldcs, const float* const* col_scales, cudaStream_t s) {
  cudaError_t e = refresh_descs(b, Bs, ldbs, Cs, ldcs, col_scales, s);
  if (e != cudaSuccess) return cuda_status(e, "descriptor upload");
  if (!b->exec) {
    e = cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      cudaError_t e2 = run_batch(b, b->cap);
      e = cudaStreamEndCapture(b->cap, &b->graph);
      if (e2 != cudaSuccess) e = e2;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, b->graph, 0);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return cuda_status(e, "graph capture of the batched launch");
    }
    find_timing_nodes(b);
  }
  return cuda_status(cudaGraphLaunch(b->exec, s), "graph launch");
}

// Whole-batch time of one candidate (the L2 flushed before each of three timed calls, best
// kept), on the autotuner's operands.
loops_status time_batch(BatchState* b, const std::vector<const void*>& Bs, const std::vector<void*>& Cs,
                        const std::vector<int64_t>& ld, L2Flush& flush, cudaEvent_t e0, cudaEvent_t e1,
                        cudaStream_t s, float* ms_out) {
  loops_status st = LOOPS_OK;
  float ms = INFINITY;
  for (int it = 0; it < 5 && !st; ++it) {
    if (it >= 2) {
      if ((st = cuda_status(flush.run(s), "L2 flush"))) break;
      cudaEventRecord(e0, s);
    }
    st = spmm_batch(b, Bs.data(), ld.data(), Cs.data(), ld.data(), nullptr, s);
    if (it >= 2) {
      cudaEventRecord(e1, s);
      if (!st) st = cuda_status(cudaEventSynchronize(e1), "autotune timing");
      float t = 0.f;
      cudaEventElapsedTime(&t, e0, e1);
      ms = std::min(ms, t);
    }
  }
  *ms_out = ms;
  return st;
}

// Autotuner of a batch. Candidates with one split threshold for every matrix (and, for F32,
// the other tile height) are built and timed as whole batches. With host-resident matrices
// the performance model then proposes one more candidate with a threshold and tile height
// per matrix: Eq. 2 is fitted to the timed candidates' times as a function of their total
// CSR-part and BCSR-part work, and Eq. 3 is applied per matrix (coordinate descent of the
// predicted batch time, over each matrix's candidate splits). That
// candidate reuses the sub-plans built for the timed ones and is timed the same way; the
// fastest candidate is kept.
loops_status autotune_batch(const loops_csr* As, const int64_t* Ns, int32_t count, loops_dtype dtype,
                            const loops_plan_opts& o, int32_t br, const SubBuilder& sub, bool use_model,
                            cudaStream_t s, BatchState** out) {
  *out = nullptr;
  struct Cand {
    double tau;
    int32_t br;
    BatchState* b = nullptr;
    float ms = INFINITY;
  };
  std::vector<Cand> cands;
  for (double t : {(double)INFINITY, 4.0, 2.0, 1.25, 0.0}) cands.push_back({t, br});
  if (dtype == LOOPS_F32 && o.block_rows == 0)
    for (double t : {4.0, 2.0, 1.25}) cands.push_back({t, br == 16 ? 8 : 16});
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  std::vector<void*> bufs;
  std::vector<const void*> Bs((size_t)count);
  std::vector<void*> Cs((size_t)count);
  std::vector<int64_t> ld((size_t)count);
  const int64_t eb = dtype == LOOPS_F32 ? 4 : 2;
  cudaError_t e = cudaSuccess;
  for (int32_t m = 0; m < count && e == cudaSuccess; ++m) {
    void *pb = nullptr, *pc = nullptr;
    e = dev_malloc(&pb, (size_t)std::max<int64_t>(As[m].n_cols * Ns[m] * eb, 16));
    if (e == cudaSuccess) e = dev_malloc(&pc, (size_t)std::max<int64_t>(As[m].n_rows * Ns[m] * 4, 16));
    if (e == cudaSuccess) e = cudaMemsetAsync(pb, 0x3C, (size_t)(As[m].n_cols * Ns[m] * eb), s);
    bufs.push_back(pb);
    bufs.push_back(pc);
    Bs[(size_t)m] = pb;
    Cs[(size_t)m] = pc;
    ld[(size_t)m] = Ns[m];
  }
  loops_status st = cuda_status(e, "autotune buffers");
  L2Flush flush;
  for (Cand& c : cands) {
    if (st) break;
    const std::vector<int32_t> brs((size_t)count, c.br);
    const std::vector<double> taus((size_t)count, c.tau);
    if ((st = build_batch(As, Ns, count, dtype, o, brs, taus, sub, nullptr, &c.b))) break;
    st = time_batch(c.b, Bs, Cs, ld, flush, e0, e1, s, &c.ms);
  }
  double flops = 0.0;
  for (int32_t m = 0; m < count; ++m) flops += 2.0 * (double)As[m].nnz * (double)Ns[m];
  size_t best_c = 0;
  for (size_t c = 1; c < cands.size(); ++c)
    if (cands[c].ms < cands[best_c].ms) best_c = c;
  BatchState* model = nullptr;
  float model_ms = INFINITY;
  double model_pred = NAN;
  if (!st && use_model && count > 0) {
    // per-matrix (x, y) of every candidate, from row-block profiles
    const int32_t kpad = k_pad_for(dtype);
    std::vector<std::vector<SplitWork>> w((size_t)count, std::vector<SplitWork>(cands.size()));
    BlockProfile prof;
    for (int32_t m = 0; m < count; ++m) {
      for (int32_t h : {8, 16}) {
        bool used = false;
        for (const Cand& c : cands) used = used || c.br == h;
        if (!used) continue;
        block_profile(&As[m], h, prof);
        for (size_t c = 0; c < cands.size(); ++c)
          if (cands[c].br == h) w[(size_t)m][c] = split_work(prof, cands[c].tau, kpad, Ns[m]);
      }
    }
    std::vector<double> X(cands.size(), 0.0), Y(cands.size(), 0.0), T(cands.size());
    double tmin = INFINITY;
    for (size_t c = 0; c < cands.size(); ++c) {
      for (int32_t m = 0; m < count; ++m) {
        X[c] += w[(size_t)m][c].x;
        Y[c] += w[(size_t)m][c].y;
      }
      T[c] = (double)cands[c].ms;
      tmin = std::min(tmin, T[c]);
    }
    double a[5];
    if (fit_perf_model(X.data(), Y.data(), T.data(), (int)cands.size(), a)) {
      // Eq. 3 per matrix: coordinate descent of the predicted batch time (the highest
      // predicted throughput) from the best timed candidate, over each matrix's candidate
      // splits; predictions below half the fastest measured time are extrapolations and
      // are not followed
      std::vector<size_t> pick((size_t)count, best_c);
      double x = X[best_c], y = Y[best_c];
      double cur = eval_perf_model(a, x, y);
      for (int pass = 0; pass < 3; ++pass) {
        bool moved = false;
        for (int32_t m = 0; m < count; ++m) {
          const SplitWork& now = w[(size_t)m][pick[(size_t)m]];
          for (size_t c = 0; c < cands.size(); ++c) {
            const SplitWork& alt = w[(size_t)m][c];
            const double nx = x - now.x + alt.x, ny = y - now.y + alt.y;
            const double t = eval_perf_model(a, nx, ny);
            if (t < cur * (1.0 - 1e-9) && t > 0.5 * tmin) {
              cur = t;
              x = nx;
              y = ny;
              pick[(size_t)m] = c;
              moved = true;
              break;
            }
          }
        }
        if (!moved) break;
      }
      bool uniform = true;
      for (int32_t m = 1; m < count; ++m) uniform = uniform && pick[(size_t)m] == pick[0];
      model_pred = flops / (std::max(cur, 1e-6) * 1e-3) / 1e9;
      if (!uniform) {
        std::vector<int32_t> brs((size_t)count);
        std::vector<double> taus((size_t)count);
        std::vector<loops_plan_s*> subs((size_t)count);
        for (int32_t m = 0; m < count; ++m) {
          const Cand& c = cands[pick[(size_t)m]];
          brs[(size_t)m] = c.br;
          taus[(size_t)m] = c.tau;
          subs[(size_t)m] = c.b->subs[(size_t)m];
        }
        if (!(st = build_batch(As, Ns, count, dtype, o, brs, taus, sub, &subs, &model)))
          st = time_batch(model, Bs, Cs, ld, flush, e0, e1, s, &model_ms);
      }
    }
  }
  cudaStreamSynchronize(s);
  for (void* q : bufs)
    if (q) cudaFree(q);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st) {
    if (model) destroy_batch(model);
    for (Cand& c : cands)
      if (c.b) destroy_batch(c.b);
    return st;
  }
  BatchState* best = nullptr;
  const double timed_gflops = flops / (std::max((double)cands[best_c].ms, 1e-6) * 1e-3) / 1e9;
  if (model && model_ms < cands[best_c].ms) {
    // the per-matrix candidate wins: it takes ownership of the sub-plans it borrowed
    for (int32_t m = 0; m < count; ++m) {
      for (Cand& c : cands)
        if (c.b && c.b->subs[(size_t)m] == model->subs[(size_t)m]) c.b->subs[(size_t)m] = nullptr;
      model->owned[(size_t)m] = 1;
    }
    best = model;
    best->tau_source = 2;
    for (Cand& c : cands) destroy_batch(c.b);
  } else {
    if (model) destroy_batch(model);  // borrowed sub-plans stay with their candidates
    best = cands[best_c].b;
    cands[best_c].b = nullptr;
    best->tau_source = 1;
    for (Cand& c : cands)
      if (c.b) destroy_batch(c.b);
  }
  best->model_gflops = model_pred;
  best->model_measured_gflops = model ? flops / (std::max((double)model_ms, 1e-6) * 1e-3) / 1e9 : NAN;
  best->timed_best_gflops = timed_gflops;
  // a plan built during tuning has captured the autotuner's operands: drop its graph state so
  // the first real call uploads the caller's descriptors
  best->copied_once = false;
  *out = best;
  return LOOPS_OK;
}

}  // namespace

}  // namespace loops

using namespace loops;

// loops_plan_batched / loops_plan_batched_device: the matrices' arrays are on the host
// (`device` false) or on the device.
static loops_status plan_batched(const loops_csr* As, const int64_t* Ns, int32_t count, loops_dtype dtype,
                                 const loops_plan_opts* opts, loops_stream_t stream, bool device,
                                 loops_plan_t* out) {
  clear_error();
  NvtxScope nvtx(device ? "loops_plan_batched_device" : "loops_plan_batched");
  if (!out) { set_error("out is NULL"); return LOOPS_ERR_INVALID_ARG; }
  *out = nullptr;
  if (count < 0 || (count > 0 && (!As || !Ns))) { set_error("bad batch arrays"); return LOOPS_ERR_INVALID_ARG; }
  if (dtype != LOOPS_F32 && dtype != LOOPS_F16 && dtype != LOOPS_BF16) {
    set_error("batched SpMM supports F32, F16 and BF16");
    return LOOPS_ERR_UNSUPPORTED;
  }
  loops_plan_opts o;
  loops_plan_opts_default(&o);
  if (opts) o = *opts;
  if (std::isnan(o.tau)) { set_error("tau is NaN"); return LOOPS_ERR_INVALID_ARG; }
  if (o.tile_min > 1) {
    set_error("the tile-level split is not available in batched plans");
    return LOOPS_ERR_UNSUPPORTED;
  }
  o.tile_min = 0;
  o.want_backward = 0;
  o.contiguous_split = 0;
  int32_t br;
  loops_status st = resolve_block_rows(dtype, o, &br);
  if (st) return st;
  cudaStream_t s = (cudaStream_t)stream;
  // per-matrix sub-plan builder: validate and convert on the host, or validate each matrix
  // once on the device (its plan scale kept) and convert on the device
  std::vector<double> vals, scales;
  if (device) {
    scales.assign((size_t)std::max(count, 0), 1.0);
    for (int32_t m = 0; m < count; ++m) {
      if (As[m].vals_dtype != LOOPS_F64 && As[m].vals_dtype != LOOPS_F32) {
        set_error("A values must be LOOPS_F64 or LOOPS_F32 on input (matrix " + std::to_string(m) + ")");
        return LOOPS_ERR_UNSUPPORTED;
      }
      const DevCsrIn d{As[m].n_rows, As[m].n_cols, As[m].nnz, As[m].row_ptr, As[m].col_idx, As[m].vals,
                       As[m].vals_dtype == LOOPS_F32};
      double mx = 0.0;
      if ((st = validate_csr_device(d, dtype, s, &mx))) {
        set_error(std::string(loops_last_error()) + " (matrix " + std::to_string(m) + ")");
        return st;
      }
      scales[(size_t)m] = plan_scale_from_max(mx, dtype);
    }
  }
  const SubBuilder sub = [&](int32_t m, const loops_plan_opts& oc, int32_t brc, double t, loops_plan_s** q) {
    loops_status r;
    if (device) {
      const DevCsrIn d{As[m].n_rows, As[m].n_cols, As[m].nnz, As[m].row_ptr, As[m].col_idx, As[m].vals,
                       As[m].vals_dtype == LOOPS_F32};
      r = make_plan_device(d, nullptr, scales[(size_t)m], Ns[m], dtype, oc, brc, t, false, true, s, q);
      if (!r) r = download_mirrors(*q);
      return r;
    }
    if ((r = validate_csr(&As[m]))) return r;
    read_vals_f64(&As[m], vals);
    return make_plan(&As[m], vals.data(), Ns[m], dtype, oc, brc, t, true, q);
  };
  BatchState* best = nullptr;
  if (o.tau >= 0.0) {
    const std::vector<int32_t> brs((size_t)count, br);
    const std::vector<double> taus((size_t)count, o.tau);
    if ((st = build_batch(As, Ns, count, dtype, o, brs, taus, sub, nullptr, &best))) return st;
  } else {
    if ((st = autotune_batch(As, Ns, count, dtype, o, br, sub, !device, s, &best))) return st;
  }
  loops_plan_s* p = new (std::nothrow) loops_plan_s();
  if (!p) { destroy_batch(best); set_error("host allocation failed"); return LOOPS_ERR_OOM; }
  p->magic = kPlanMagic;
  p->dtype = dtype;
  p->n_rows = best->total_rows;
  p->n_cols = 0;
  p->nnz = best->total_nnz;
  p->N = 0;
  p->br = best->br;
  p->kpad = k_pad_for(dtype);
  p->tau = best->tau;
  p->scale = 1.0;
  p->split_len = 0;
  p->tile_min = 0;
  p->opts = o;
  p->transposed = nullptr;
  p->d_error = nullptr;
  p->side = nullptr;
  p->ev_fork = p->ev_join = nullptr;
  p->stage_B = p->stage_C = nullptr;
  p->stage_B_bytes = p->stage_C_bytes = 0;
  p->pipe = nullptr;
  p->n_subnormal = 0;
  p->nnz_bcsr = 0;
  p->timing = false;
  for (auto& ev : p->tev) ev = nullptr;
  p->batch = best;
  p->other_bytes = best->device_bytes;
  for (auto* sp : best->subs) {
    p->nnz_bcsr += sp->nnz_bcsr;
    p->n_subnormal += sp->n_subnormal;
  }
  p->device_built = device;
  register_plan(p);
  *out = p;
  return LOOPS_OK;
}

extern "C" {

loops_status loops_plan_batched(const loops_csr* As, const int64_t* Ns, int32_t count, loops_dtype dtype,
                                const loops_plan_opts* opts, loops_stream_t stream, loops_plan_t* out) {
  return plan_batched(As, Ns, count, dtype, opts, stream, false, out);
}

loops_status loops_plan_batched_device(const loops_csr* As, const int64_t* Ns, int32_t count, loops_dtype dtype,
                                       const loops_plan_opts* opts, loops_stream_t stream, loops_plan_t* out) {
  return plan_batched(As, Ns, count, dtype, opts, stream, true, out);
}

loops_status loops_spmm_batched(loops_plan_t p, const void* const* Bs, const int64_t* ldbs, void* const* Cs,
                                const int64_t* ldcs, const float* const* col_scales, loops_stream_t stream) {
  clear_error();
  NvtxScope nvtx("loops_spmm_batched");
  loops_status st = check_plan(p);
  if (st) return st;
  if (!p->batch) { set_error("not a batched plan"); return LOOPS_ERR_STATE; }
  BatchState* b = p->batch;
  if (b->count && (!Bs || !Cs || !ldbs || !ldcs)) { set_error("NULL batch array"); return LOOPS_ERR_INVALID_ARG; }
  for (int32_t m = 0; m < b->count; ++m) {
    const loops_plan_s* sp = b->subs[(size_t)m];
    const int64_t N = sp->N;
    const int64_t eb = b->dtype == LOOPS_F32 ? 4 : 2;
    if (ldbs[m] < N || ldcs[m] < N || (!Bs[m] && sp->n_cols > 0) || (!Cs[m] && sp->n_rows > 0)) {
      set_error("bad dense operand of matrix " + std::to_string(m));
      return LOOPS_ERR_INVALID_ARG;
    }
    if (sp->n_cols > 0 && ldbs[m] > (INT32_MAX / sp->n_cols)) {
      set_error("batched SpMM indexes B with 32-bit offsets: n_cols x ldb must stay below 2^31 (matrix " +
                std::to_string(m) + ")");
      return LOOPS_ERR_UNSUPPORTED;
    }
    if (((uintptr_t)Bs[m] % 16) || ((uintptr_t)Cs[m] % 16) || ((ldbs[m] * eb) % 16) || ((ldcs[m] * 4) % 16)) {
      set_error("batched SpMM needs 16-byte aligned rows of B and C (matrix " + std::to_string(m) + ")");
      return LOOPS_ERR_UNSUPPORTED;
    }
    if (col_scales && col_scales[m] && b->dtype == LOOPS_F32) {
      set_error("col_scale is only defined for the 16-bit dtypes");
      return LOOPS_ERR_INVALID_ARG;
    }
  }
  return spmm_batch(b, Bs, ldbs, Cs, ldcs, col_scales, (cudaStream_t)stream);
}

namespace {

// Groups of consecutive matrices for the host call's pipeline, about equal in bytes moved (B
// in, C out). Each group runs its matrices' sub-runs of every class's tasks (the task list is
// in matrix order within a class) with its own task counters, and its own runs of the
// partial-sum lists (in matrix order too).
#ifndef LOOPS_BATCHED_HOST_GROUPS
#define LOOPS_BATCHED_HOST_GROUPS 16
#endif
cudaError_t build_host_groups(BatchState* b) {
  const int64_t eb = b->dtype == LOOPS_F32 ? 4 : 2;
  std::vector<int64_t> bytes((size_t)b->count);
  int64_t total = 0;
  for (int32_t m = 0; m < b->count; ++m) {
    const loops_plan_s* sp = b->subs[(size_t)m];
    bytes[(size_t)m] = sp->n_cols * sp->N * eb + sp->n_rows * sp->N * 4;
    total += bytes[(size_t)m];
  }
  const int ng = std::max(1, std::min<int>(LOOPS_BATCHED_HOST_GROUPS, b->count));
  auto by_m = [](const BatchTask& t, int32_t m) { return t.m < m; };
  auto split_m = [](const int2& x, int32_t m) { return x.x < m; };
  int64_t n_counters = 0, acc = 0;
  int32_t m0 = 0;
  for (int g = 0; g < ng && m0 < b->count; ++g) {
    const int64_t target = total / ng * (g + 1);
    int32_t m1 = m0;
    while (m1 < b->count) {
      if (m1 > m0 && g < ng - 1 && acc + bytes[(size_t)m1] > target) break;
      acc += bytes[(size_t)m1++];
    }
    BatchState::HostGroup hg;
    hg.m0 = m0;
    hg.m1 = m1;
    hg.counter0 = n_counters;
    for (const BatchClass& c : b->classes) {
      auto beg = b->h_tasks.begin() + c.first, end = beg + c.n_tasks;
      auto lo = std::lower_bound(beg, end, m0, by_m);
      auto hi = std::lower_bound(lo, end, m1, by_m);
      if (hi == lo) continue;
      BatchClass gc = c;
      gc.first = (int64_t)(lo - b->h_tasks.begin());
      gc.n_tasks = (int64_t)(hi - lo);
      // one block slot per SM left to the copy kernels, which run beside the class kernels
      gc.grid = batched_class_grid(b->dtype, gc);
      if (gc.grid <= 0) return cudaErrorInvalidValue;
      hg.classes.push_back(gc);
    }
    n_counters += (int64_t)hg.classes.size();
    auto s_lo = std::lower_bound(b->h_splits.begin(), b->h_splits.end(), m0, split_m);
    auto s_hi = std::lower_bound(s_lo, b->h_splits.end(), m1, split_m);
    hg.split0 = (int64_t)(s_lo - b->h_splits.begin());
    hg.n_splits = (int64_t)(s_hi - s_lo);
    auto q_lo = std::lower_bound(b->h_bsplits.begin(), b->h_bsplits.end(), m0, split_m);
    auto q_hi = std::lower_bound(q_lo, b->h_bsplits.end(), m1, split_m);
    hg.bsplit0 = (int64_t)(q_lo - b->h_bsplits.begin());
    hg.n_bsplits = (int64_t)(q_hi - q_lo);
    b->groups.push_back(std::move(hg));
    m0 = m1;
  }
  cudaError_t e = dev_malloc((void**)&b->d_gcounters, sizeof(unsigned long long) * (size_t)std::max<int64_t>(n_counters, 1));
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->copy_in, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->copy_out, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_start, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_fin, cudaEventDisableTiming);
  for (size_t g = 0; g < b->groups.size() && e == cudaSuccess; ++g) {
    cudaEvent_t x = nullptr, y = nullptr;
    e = cudaEventCreateWithFlags(&x, cudaEventDisableTiming);
    if (e == cudaSuccess) b->ev_in.push_back(x);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&y, cudaEventDisableTiming);
    if (e == cudaSuccess) b->ev_out.push_back(y);
  }
  if (e != cudaSuccess) b->groups.clear();  // built again (and the rest freed with the plan)
  return e;
}

// Host <-> device copy of a matrix of `rows` rows of `width` bytes (pitches in bytes): one
// plain copy when both sides are dense.
cudaError_t copy_rows(void* dst, size_t dpitch, const void* src, size_t spitch, size_t width, size_t rows,
                      cudaMemcpyKind kind, cudaStream_t s) {
  if (rows == 0 || width == 0) return cudaSuccess;
  if (dpitch == width && spitch == width) return cudaMemcpyAsync(dst, src, width * rows, kind, s);
  return cudaMemcpy2DAsync(dst, dpitch, src, spitch, width, rows, kind, s);
}

}  // namespace

loops_status loops_spmm_batched_host(loops_plan_t p, const void* const* Bs_host, const int64_t* ldbs,
                                     void* const* Cs_host, const int64_t* ldcs, loops_stream_t stream) {
  clear_error();
  NvtxScope nvtx("loops_spmm_batched_host");
  loops_status st = check_plan(p);
  if (st) return st;
  if (!p->batch) { set_error("not a batched plan"); return LOOPS_ERR_STATE; }
  BatchState* b = p->batch;
  if (b->count && (!Bs_host || !Cs_host || !ldbs || !ldcs)) { set_error("NULL batch array"); return LOOPS_ERR_INVALID_ARG; }
  const int64_t eb = b->dtype == LOOPS_F32 ? 4 : 2;
  for (int32_t m = 0; m < b->count; ++m) {
    const loops_plan_s* sp = b->subs[(size_t)m];
    if (ldbs[m] < sp->N || ldcs[m] < sp->N || (!Bs_host[m] && sp->n_cols > 0) || (!Cs_host[m] && sp->n_rows > 0)) {
      set_error("bad host operand of matrix " + std::to_string(m));
      return LOOPS_ERR_INVALID_ARG;
    }
    if (sp->n_cols > 0 && ldbs[m] > (INT32_MAX / sp->n_cols)) {
      set_error("batched SpMM indexes B with 32-bit offsets: n_cols x ldb must stay below 2^31 (matrix " +
                std::to_string(m) + ")");
      return LOOPS_ERR_UNSUPPORTED;
    }
  }
  if (b->count == 0) return cuda_status(cudaStreamSynchronize((cudaStream_t)stream), "batched host call");
  if (b->groups.empty()) {
    cudaError_t e = build_host_groups(b);
    if (e != cudaSuccess) return cuda_status(e, "batched host pipeline setup");
  }
  // Staging layout: every B, then every C. A matrix with dense host rows whose host operand
  // directly follows the previous matrix's in the same group (one host arena) keeps that
  // offset in the staging area too, so the run moves in one copy that touches no byte outside
  // the operands. Other matrices start on a 256-byte boundary and copy on their own: B with
  // its host pitch when that is a 16-byte multiple (one plain copy of its own storage), else
  // into dense rows; C always into dense rows.
  const int32_t cnt = b->count;
  std::vector<int64_t> boff((size_t)cnt), coff((size_t)cnt), ldB((size_t)cnt), ldC((size_t)cnt);
  std::vector<uint8_t> brun((size_t)cnt), crun((size_t)cnt);  // 1: continues the previous matrix's run
  std::vector<int32_t> grp((size_t)cnt);
  for (size_t g = 0; g < b->groups.size(); ++g)
    for (int32_t m = b->groups[g].m0; m < b->groups[g].m1; ++m) grp[(size_t)m] = (int32_t)g;
  auto host_span = [](const void* p0, int64_t bytes) { return static_cast<const char*>(p0) + bytes; };
  int64_t off = 0;
  for (int32_t m = 0; m < cnt; ++m) {
    const loops_plan_s* sp = b->subs[(size_t)m];
    const loops_plan_s* pp = m > 0 ? b->subs[(size_t)m - 1] : nullptr;
    const bool pitched_ok = (ldbs[m] * eb) % 16 == 0;
    brun[(size_t)m] = m > 0 && grp[(size_t)m] == grp[(size_t)m - 1] && ldbs[m] == sp->N && ldbs[m - 1] == pp->N &&
                      pitched_ok && sp->n_cols > 0 && pp->n_cols > 0 &&
                      Bs_host[m] == host_span(Bs_host[m - 1], pp->n_cols * pp->N * eb);
    if (brun[(size_t)m]) {
      boff[(size_t)m] = boff[(size_t)m - 1] + pp->n_cols * ldbs[m - 1] * eb;
      ldB[(size_t)m] = ldbs[m];
    } else {
      off = (off + 255) / 256 * 256;
      boff[(size_t)m] = off;
      // a run may start here: keep the host pitch when it is a 16-byte multiple
      ldB[(size_t)m] = pitched_ok ? ldbs[m] : sp->N;
    }
    off = boff[(size_t)m] + sp->n_cols * ldB[(size_t)m] * eb;
  }
  for (int32_t m = 0; m < cnt; ++m) {
    const loops_plan_s* sp = b->subs[(size_t)m];
    const loops_plan_s* pp = m > 0 ? b->subs[(size_t)m - 1] : nullptr;
    crun[(size_t)m] = m > 0 && grp[(size_t)m] == grp[(size_t)m - 1] && ldcs[m] == sp->N && ldcs[m - 1] == pp->N &&
                      sp->n_rows > 0 && pp->n_rows > 0 && (sp->N * 4) % 16 == 0 &&
                      Cs_host[m] == host_span(Cs_host[m - 1], pp->n_rows * pp->N * 4);
    if (crun[(size_t)m]) {
      coff[(size_t)m] = coff[(size_t)m - 1] + pp->n_rows * pp->N * 4;
    } else {
      off = (off + 255) / 256 * 256;
      coff[(size_t)m] = off;
    }
    ldC[(size_t)m] = sp->N;
    off = coff[(size_t)m] + sp->n_rows * sp->N * 4;
  }
  off = (off + 255) / 256 * 256;
  if (off > b->stage_bytes) {
    if (b->stage) {
      cudaDeviceSynchronize();
      cudaFree(b->stage);
      b->stage = nullptr;
      b->stage_bytes = 0;
    }
    cudaError_t e = dev_malloc(&b->stage, (size_t)std::max<int64_t>(off, 256));
    if (e != cudaSuccess) return cuda_status(e, "batched staging buffer");
    b->stage_bytes = off;
  }
  cudaStream_t s = (cudaStream_t)stream;
  std::vector<const void*> dB((size_t)cnt);
  std::vector<void*> dC((size_t)cnt);
  char* base = static_cast<char*>(b->stage);
  for (int32_t m = 0; m < cnt; ++m) {
    dB[(size_t)m] = base + boff[(size_t)m];
    dC[(size_t)m] = base + coff[(size_t)m];
  }
  cudaError_t e = refresh_descs(b, dB.data(), ldB.data(), dC.data(), ldC.data(), nullptr, s);
  if (e != cudaSuccess) return cuda_status(e, "descriptor upload");
  // three streams: copies in (every group's B, in order), the kernels on `stream` (group g
  // once its B is in), copies out (group g's C once its kernels are done)
  e = cudaEventRecord(b->ev_start, s);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(b->copy_in, b->ev_start, 0);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(b->copy_out, b->ev_start, 0);
  // copy of B for matrices [m, end of its run): one plain copy of the run's host span, or
  // the matrix alone (pitched into dense staging rows when its host pitch is not kept)
  auto copy_in_from = [&](int32_t m, int32_t m1, int32_t* next) -> cudaError_t {
    const loops_plan_s* sp = b->subs[(size_t)m];
    int32_t k = m + 1;
    int64_t bytes = sp->n_cols * ldB[(size_t)m] * eb;
    if (ldB[(size_t)m] == ldbs[m]) {
      while (k < m1 && brun[(size_t)k]) bytes += b->subs[(size_t)k]->n_cols * ldbs[k] * eb, ++k;
      // a lone pitched matrix: its last row is read only up to its N columns (runs are dense)
      if (sp->n_cols > 0) bytes -= (ldbs[m] - sp->N) * eb;
    }
    *next = k;
    if (sp->n_cols == 0) return cudaSuccess;
    if (ldB[(size_t)m] == ldbs[m])
      return cudaMemcpyAsync(base + boff[(size_t)m], Bs_host[m], (size_t)bytes, cudaMemcpyHostToDevice, b->copy_in);
    return copy_rows(base + boff[(size_t)m], (size_t)(sp->N * eb), Bs_host[m], (size_t)(ldbs[m] * eb),
                     (size_t)(sp->N * eb), (size_t)sp->n_cols, cudaMemcpyHostToDevice, b->copy_in);
  };
  auto copy_out_from = [&](int32_t m, int32_t m1, int32_t* next) -> cudaError_t {
    const loops_plan_s* sp = b->subs[(size_t)m];
    int32_t k = m + 1;
    int64_t bytes = sp->n_rows * sp->N * 4;
    while (k < m1 && crun[(size_t)k]) bytes += b->subs[(size_t)k]->n_rows * b->subs[(size_t)k]->N * 4, ++k;
    *next = k;
    if (k > m + 1)  // a dense run: one plain copy
      return cudaMemcpyAsync(Cs_host[m], base + coff[(size_t)m], (size_t)bytes, cudaMemcpyDeviceToHost, b->copy_out);
    return copy_rows(Cs_host[m], (size_t)(ldcs[m] * 4), base + coff[(size_t)m], (size_t)(sp->N * 4),
                     (size_t)(sp->N * 4), (size_t)sp->n_rows, cudaMemcpyDeviceToHost, b->copy_out);
  };
  for (size_t g = 0; g < b->groups.size() && e == cudaSuccess; ++g) {
    const BatchState::HostGroup& hg = b->groups[g];
    for (int32_t m = hg.m0, nx = 0; m < hg.m1 && e == cudaSuccess; m = nx) e = copy_in_from(m, hg.m1, &nx);
    if (e == cudaSuccess) e = cudaEventRecord(b->ev_in[g], b->copy_in);
  }
  // on a failure, no copy may still be reading or writing the caller's buffers on return
  auto drain = [&](cudaError_t err, const char* what) {
    cudaStreamSynchronize(b->copy_in);
    cudaStreamSynchronize(b->copy_out);
    cudaStreamSynchronize(s);
    return cuda_status(err, what);
  };
  if (e != cudaSuccess) return drain(e, "copy of B to the device");
  for (size_t g = 0; g < b->groups.size() && e == cudaSuccess; ++g) {
    const BatchState::HostGroup& hg = b->groups[g];
    e = cudaStreamWaitEvent(s, b->ev_in[g], 0);
    if (e == cudaSuccess) {
      BatchLaunch L;
      L.descs = b->d_desc;
      L.tasks = b->d_tasks;
      L.classes = hg.classes.data();
      L.n_classes = (int)hg.classes.size();
      L.counters = b->d_gcounters + hg.counter0;
      L.splits = b->d_splits + hg.split0;
      L.n_splits = hg.n_splits;
      L.bsplits = b->d_bsplits + hg.bsplit0;
      L.n_bsplits = hg.n_bsplits;
      L.tev = nullptr;
      L.n_side = (int)b->side.size();
      L.side = b->side.data();
      L.fork = b->ev_fork;
      L.join = b->ev_join.data();
      e = launch_batched(b->dtype, L, s);
    }
    if (e == cudaSuccess) e = cudaEventRecord(b->ev_out[g], s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(b->copy_out, b->ev_out[g], 0);
    for (int32_t m = hg.m0, nx = 0; m < hg.m1 && e == cudaSuccess; m = nx) e = copy_out_from(m, hg.m1, &nx);
  }
  if (e == cudaSuccess) e = cudaEventRecord(b->ev_fin, b->copy_out);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(s, b->ev_fin, 0);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return drain(e, "batched host call");
  return LOOPS_OK;
}

loops_status loops_plan_batched_info(loops_plan_t p, int32_t* count, int64_t* n_tasks, double* tau,
                                     int32_t* block_rows) {
  clear_error();
  loops_status st = check_plan(p);
  if (st) return st;
  if (!p->batch) { set_error("not a batched plan"); return LOOPS_ERR_STATE; }
  if (count) *count = p->batch->count;
  if (n_tasks) *n_tasks = p->batch->n_tasks;
  if (tau) *tau = p->batch->tau;
  if (block_rows) *block_rows = p->batch->br;
  return LOOPS_OK;
}

loops_status loops_plan_batched_stats(loops_plan_t p, loops_batched_info* out) {
  clear_error();
  loops_status st = check_plan(p);
  if (st) return st;
  if (!p->batch) { set_error("not a batched plan"); return LOOPS_ERR_STATE; }
  if (!out) { set_error("out is NULL"); return LOOPS_ERR_INVALID_ARG; }
  std::memset(out, 0, sizeof(*out));
  const BatchState* b = p->batch;
  out->count = b->count;
  out->block_rows = b->br;
  out->tau = b->tau;
  for (const loops_plan_s* sp : b->subs)
    if (!(sp->tau == b->subs[0]->tau)) out->tau = NAN;
  out->n_tasks = b->n_tasks;
  out->n_kernels = batch_kernels_per_call(b);
  out->n_classes = batch_classes(b);
  out->n_split_rows = b->n_splits;
  out->n_split_blocks = b->n_bsplits;
  out->n_rows = b->total_rows;
  out->nnz = b->total_nnz;
  out->nnz_bcsr = p->nnz_bcsr;
  out->device_bytes = b->device_bytes + b->stage_bytes;
  out->tau_source = b->tau_source;
  out->model_gflops = b->model_gflops;
  out->model_measured_gflops = b->model_measured_gflops;
  out->timed_best_gflops = b->timed_best_gflops;
  return LOOPS_OK;
}

loops_status loops_plan_batched_matrix_info(loops_plan_t p, int32_t m, loops_plan_info* out) {
  clear_error();
  loops_status st = check_plan(p);
  if (st) return st;
  if (!p->batch) { set_error("not a batched plan"); return LOOPS_ERR_STATE; }
  if (m < 0 || m >= p->batch->count) { set_error("matrix index out of range"); return LOOPS_ERR_INVALID_ARG; }
  return plan_info_of(p->batch->subs[(size_t)m], out);
}

}  // extern "C"
