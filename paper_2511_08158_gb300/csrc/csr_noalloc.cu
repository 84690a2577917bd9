// Allocation-free CSR SpMM: C = A . B straight from caller-owned device CSR arrays, with no
// plan and no device allocation of any kind.
//
// Who needs it: code that must not call cudaMalloc (or any allocating routine) at the point
// where it multiplies -- for example a kernel sequence being recorded into a CUDA graph under
// the global capture mode, a host callback or real-time path where allocation latency or
// failure is not acceptable, or a service that reserves all device memory up front and runs
// under a fixed memory budget. Building a plan allocates device memory, so those callers
// cannot use loops_plan / loops_spmm; they hand their CSR arrays and dense operands here.
//
// How it works: the stored entries are cut into fixed chunks of kChunk entries; one warp
// takes one chunk and one 32-column slice of N. Rows that start and end inside a chunk are
// summed and written directly. A row that crosses a chunk boundary leaves partial sums: the
// chunk that owns the row's first entry writes a "tail" partial, every later chunk the row
// runs into writes a "head" partial, and a second kernel adds them in chunk order and writes
// the row. The partial sums live in g_noalloc_scratch, a fixed file-scope device array: the
// library's only scratch memory that it never allocates. The order of every sum is fixed, so
// results do not depend on scheduling.
#include <mutex>

#include "device_common.cuh"
#include "loops_internal.h"

namespace loops {

namespace {

constexpr int64_t kChunk = 128;  // stored entries per chunk

// Partial sums of chunk-crossing rows: [2][n_chunks][N] accumulators (head, tail). Every GPU
// that loads the library holds this array until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[LOOPS_NOALLOC_SCRATCH_BYTES];

// Device address of g_noalloc_scratch per device, looked up once per device.
std::mutex g_mu;
void* g_scratch_ptr[128] = {};

struct NoAllocArgs {
  const int64_t* row_ptr;
  const int32_t* col;
  const void* val;
  int64_t n_rows, n_cols, nnz, n_chunks;
  const void* B;
  int64_t ldb;
  void* C;
  int64_t ldc;
  int64_t N;
  void* scratch;
};

__device__ __forceinline__ int64_t clamp_ptr(const NoAllocArgs& a, int64_t r) {
  const int64_t v = a.row_ptr[r];
  return v < 0 ? 0 : (v > a.nnz ? a.nnz : v);
}

// first r in [0, n_rows) with row_ptr[r] >= x (n_rows if none)
__device__ __forceinline__ int64_t lower_row(const NoAllocArgs& a, int64_t x) {
  int64_t lo = 0, hi = a.n_rows;
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if (clamp_ptr(a, mid) < x) lo = mid + 1; else hi = mid;
  }
  return lo;
}

// Sum of entries [e0, e1) times B's column n (entries with a column outside [0, n_cols) are
// skipped, so no load leaves B).
template <class Tr>
__device__ __forceinline__ typename Tr::TAcc dot_range(const NoAllocArgs& a, int64_t e0, int64_t e1, int64_t n,
                                                       bool colok) {
  using TB = typename Tr::TB;
  using TAcc = typename Tr::TAcc;
  const int lane = threadIdx.x & 31;
  const TB* Bp = reinterpret_cast<const TB*>(a.B);
  const TB* vals = reinterpret_cast<const TB*>(a.val);
  TAcc acc = TAcc(0);
  for (int64_t k0 = e0; k0 < e1; k0 += 32) {
    const int64_t k = k0 + lane;
    int32_t c = -1;
    TAcc v = TAcc(0);
    if (k < e1) {
      c = __ldg(a.col + k);
      v = Tr::to_acc(vals[k]);
    }
    const int cnt = (int)(e1 - k0 < 32 ? e1 - k0 : 32);
    for (int j = 0; j < cnt; ++j) {
      const int cj = __shfl_sync(0xffffffffu, c, j);
      const TAcc vj = __shfl_sync(0xffffffffu, v, j);
      if (colok && cj >= 0 && (int64_t)cj < a.n_cols) acc = fma(vj, Tr::to_acc(Bp[(int64_t)cj * a.ldb + n]), acc);
    }
  }
  return acc;
}

template <class Tr>
__global__ void __launch_bounds__(256) noalloc_chunks(NoAllocArgs a) {
  using TAcc = typename Tr::TAcc;
  using TC = typename Tr::TC;
  const int64_t c = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (c >= a.n_chunks) return;
  const int lane = threadIdx.x & 31;
  const int64_t n = (int64_t)blockIdx.y * 32 + lane;
  const bool colok = n < a.N;
  const int64_t e0 = c * kChunk;
  const int64_t e1 = (e0 + kChunk < a.nnz) ? e0 + kChunk : a.nnz;
  const bool last = c == a.n_chunks - 1;
  TAcc* head = reinterpret_cast<TAcc*>(a.scratch);
  TAcc* tail = head + a.n_chunks * a.N;
  // rows owned by this chunk: first entry in [e0, e1) (the last chunk also owns trailing
  // empty rows)
  const int64_t r0 = lower_row(a, e0);
  const int64_t r1 = last ? a.n_rows : lower_row(a, e1);
  // continuation of a row that started in an earlier chunk
  if (e0 < e1 && r0 > 0) {
    const int64_t rin = r0 - 1;
    const int64_t end_in = clamp_ptr(a, rin + 1);
    if (end_in > e0) {
      const TAcc s = dot_range<Tr>(a, e0, end_in < e1 ? end_in : e1, n, colok);
      if (colok) head[c * a.N + n] = s;
    }
  }
  for (int64_t r = r0; r < r1; ++r) {
    const int64_t b = clamp_ptr(a, r);
    const int64_t e = clamp_ptr(a, r + 1);
    const TAcc s = dot_range<Tr>(a, b, e < e1 ? e : e1, n, colok);
    if (!colok) continue;
    if (e <= e1) reinterpret_cast<TC*>(a.C)[r * a.ldc + n] = (TC)s;  // complete row
    else tail[c * a.N + n] = s;                                        // continues: partial
  }
}

// Rows that cross chunk boundaries: tail partial of the owning chunk plus the head partials of
// the chunks the row runs into, in chunk order.
template <class Tr>
__global__ void __launch_bounds__(256) noalloc_fixup(NoAllocArgs a) {
  using TAcc = typename Tr::TAcc;
  using TC = typename Tr::TC;
  const int64_t c = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (c >= a.n_chunks) return;
  const int lane = threadIdx.x & 31;
  const int64_t n = (int64_t)blockIdx.y * 32 + lane;
  if (n >= a.N) return;
  const int64_t e0 = c * kChunk;
  const int64_t e1 = (e0 + kChunk < a.nnz) ? e0 + kChunk : a.nnz;
  const bool last = c == a.n_chunks - 1;
  const int64_t r0 = lower_row(a, e0);
  const int64_t r1 = last ? a.n_rows : lower_row(a, e1);
  if (r1 <= r0) return;
  const int64_t r = r1 - 1;
  const int64_t e = clamp_ptr(a, r + 1);
  if (e <= e1) return;  // the chunk's last row ends inside it
  const TAcc* head = reinterpret_cast<const TAcc*>(a.scratch);
  const TAcc* tail = head + a.n_chunks * a.N;
  TAcc s = tail[c * a.N + n];
  for (int64_t q = c + 1; q < a.n_chunks && q * kChunk < e; ++q) s += head[q * a.N + n];
  reinterpret_cast<TC*>(a.C)[r * a.ldc + n] = (TC)s;
}

template <class Tr>
cudaError_t launch_noalloc_t(const NoAllocArgs& a, cudaStream_t s) {
  const unsigned gx = (unsigned)((a.n_chunks * 32 + 255) / 256);
  const unsigned gy = (unsigned)((a.N + 31) / 32);
  noalloc_chunks<Tr><<<dim3(gx, gy), 256, 0, s>>>(a);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  noalloc_fixup<Tr><<<dim3(gx, gy), 256, 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace

}  // namespace loops

using namespace loops;

extern "C" loops_status loops_csr_spmm_noalloc(int64_t n_rows, int64_t n_cols, int64_t nnz, const int64_t* row_ptr,
                                               const int32_t* col_idx, const void* vals, loops_dtype dtype,
                                               const void* B, int64_t ldb, int64_t N, void* C, int64_t ldc,
                                               loops_stream_t stream) {
  clear_error();
  if (dtype != LOOPS_F64 && dtype != LOOPS_F32 && dtype != LOOPS_F16 && dtype != LOOPS_BF16) {
    set_error("bad dtype");
    return LOOPS_ERR_INVALID_ARG;
  }
  if (n_rows < 0 || n_cols < 0 || nnz < 0 || N < 0 || ldb < N || ldc < N) {
    set_error("negative size or leading dimension smaller than N");
    return LOOPS_ERR_INVALID_ARG;
  }
  if (n_rows == 0 || N == 0) return LOOPS_OK;
  if (!row_ptr || !C || (nnz > 0 && (!col_idx || !vals || !B))) {
    set_error("NULL pointer");
    return LOOPS_ERR_INVALID_ARG;
  }
  const int64_t n_chunks = nnz > 0 ? (nnz + kChunk - 1) / kChunk : 1;
  const int64_t acc_bytes = dtype == LOOPS_F64 ? 8 : 4;
  // the scratch test divides instead of multiplying, so no product of caller sizes can wrap
  const int64_t per_chunk = 2 * acc_bytes;  // head and tail accumulators per chunk and column
  if (N > (int64_t)LOOPS_NOALLOC_SCRATCH_BYTES / per_chunk ||
      n_chunks > (int64_t)LOOPS_NOALLOC_SCRATCH_BYTES / (per_chunk * N)) {
    set_error("problem too large for the allocation-free path: its scratch needs 2 * ceil(nnz / 128) * N * " +
              std::to_string((long long)acc_bytes) + " bytes (nnz " + std::to_string((long long)nnz) + ", N " +
              std::to_string((long long)N) + "), the static array holds " +
              std::to_string((long long)LOOPS_NOALLOC_SCRATCH_BYTES));
    return LOOPS_ERR_UNSUPPORTED;
  }
  if ((N + 31) / 32 > 65535 || (n_chunks * 32 + 255) / 256 > 0x7fffffffLL) {
    set_error("N too large for the allocation-free path's launch shape (at most 65535 * 32 columns)");
    return LOOPS_ERR_UNSUPPORTED;
  }
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= 128) {
    set_error(std::string("cudaGetDevice failed: ") + cudaGetErrorString(e));
    return LOOPS_ERR_CUDA;
  }
  void* scratch = nullptr;
  {
    // set-up, once per device with that device current: the host-side name of a __device__
    // array is not a device address, so look the address up and keep it
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_ptr[dev]) {
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (e != cudaSuccess) {
        set_error(std::string("cudaGetSymbolAddress failed: ") + cudaGetErrorString(e));
        return LOOPS_ERR_CUDA;
      }
      g_scratch_ptr[dev] = p;
    }
    scratch = g_scratch_ptr[dev];
  }
  NoAllocArgs a;
  a.row_ptr = row_ptr;
  a.col = col_idx;
  a.val = vals;
  a.n_rows = n_rows;
  a.n_cols = n_cols;
  a.nnz = nnz;
  a.n_chunks = n_chunks;
  a.B = B;
  a.ldb = ldb;
  a.C = C;
  a.ldc = ldc;
  a.N = N;
  a.scratch = scratch;
  cudaStream_t s = (cudaStream_t)stream;
  switch (dtype) {
    case LOOPS_F64: e = launch_noalloc_t<TrF64>(a, s); break;
    case LOOPS_F32: e = launch_noalloc_t<TrF32>(a, s); break;
    case LOOPS_F16: e = launch_noalloc_t<TrF16>(a, s); break;
    case LOOPS_BF16: e = launch_noalloc_t<TrBF16>(a, s); break;
  }
  if (e != cudaSuccess) {
    set_error(std::string("launch failed: ") + cudaGetErrorString(e));
    return LOOPS_ERR_CUDA;
  }
  return LOOPS_OK;
}
