// Device-side plan build: CSR validation, row-block analysis, the split of Algorithm 1 (with
// the structural reading and the tile-level split) and the packing of both parts, run on the
// GPU from a CSR matrix that is already in device memory. The result is the same plan, bit for
// bit, as the host builder makes from the same matrix (same canonical partition, same work
// items and units, same stored values), so every kernel and every test of the host-built plan
// applies to it. This serves re-planning when the sparsity pattern changes between calls
// (dynamic graphs, Sec. 4.5 amortisation): no host round trip of the matrix.
//
// Steps (one stream, a handful of host reads of totals):
//   1. validate rows / columns and find max|a| (plan scale s_A for 16-bit formats);
//   2. key every entry by (row block, column) and stable-radix-sort it, so entries with the
//      same key stay in input order: runs of equal keys are the B_r x 1 tiles of a block, in
//      ascending column order, and the number of runs in a block is its distinct columns;
//   3. per block: nnz_rb >= tau * distinct columns (or the contiguous boundary) selects BCSR;
//      tiles with fewer than tile_min entries leave for the CSR part;
//   4. BCSR: tile columns, values summed per (tile, row) in input order, rounded once, stored in
//      the MMA fragment order; blocks padded to a multiple of the MMA K; work units cut at
//      kBcsrSplitTiles tiles and ordered by decreasing length (stable);
//   5. CSR: rows (or their moved entries) in row order, long rows cut into segments, items
//      ordered by decreasing length class (stable), values rounded per entry;
//   6. value maps for loops_plan_set_values, and with want_backward the SDDMM items and the
//      plan of A^T (a stable sort of the entries by column).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "device_common.cuh"
#include "loops_internal.h"

namespace loops {

namespace {

constexpr int kThreads = 256;
constexpr int kItems = 8;
constexpr int kTile = kThreads * kItems;  // elements per block in scans and radix passes

// Index checks of the build kernels: an index outside its array is recorded here and the
// access skipped; the host turns a non-zero word into an error status.
__device__ int g_build_err;
#define BUILD_CHECK(cond)                  \
  if (!(cond)) {                            \
    atomicOr(&g_build_err, 1);              \
    continue;                               \
  }

// ------------------------------------------------------------------ temporaries
// Device allocations that live for one build: stream-ordered (the device's memory pool, no
// device-wide synchronisation per allocation), released on the build's stream when the arena
// goes out of scope.
struct Arena {
  std::vector<void*> ptrs;
  cudaStream_t s = nullptr;
  cudaError_t err = cudaSuccess;
  template <class T>
  T* get(int64_t n) {
    if (err != cudaSuccess) return nullptr;
    void* q = nullptr;
    err = dev_malloc_async(&q, (size_t)std::max<int64_t>(n, 1) * sizeof(T), s);
    if (err != cudaSuccess) { cudaGetLastError(); return nullptr; }
    ptrs.push_back(q);
    return (T*)q;
  }
  ~Arena() {
    for (void* q : ptrs) cudaFreeAsync(q, s);
  }
};

// ------------------------------------------------------------------ block scan
// Exclusive prefix sum over a block of kThreads threads; `total` receives the block's sum.
__device__ __forceinline__ int64_t block_excl_scan(int64_t v, int64_t& total) {
  __shared__ int64_t ws[kThreads / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int64_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int64_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) ws[warp] = x;
  __syncthreads();
  if (warp == 0) {
    int64_t w = lane < kThreads / 32 ? ws[lane] : 0;
#pragma unroll
    for (int o = 1; o < kThreads / 32; o <<= 1) {
      const int64_t y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    if (lane < kThreads / 32) ws[lane] = w;
  }
  __syncthreads();
  const int64_t before = warp ? ws[warp - 1] : 0;
  total = ws[kThreads / 32 - 1];
  __syncthreads();
  return before + x - v;
}

// ------------------------------------------------------------------ exclusive scan
// out[i] = sum of in[0 .. i); out[n] = total when `with_total`. `out` may alias `in` (int64).
template <class T>
__global__ void __launch_bounds__(kThreads) scan_reduce_k(const T* in, int64_t n, int64_t* sums) {
  const int64_t base = (int64_t)blockIdx.x * kTile + (int64_t)threadIdx.x * kItems;
  int64_t s = 0;
#pragma unroll
  for (int j = 0; j < kItems; ++j)
    if (base + j < n) s += (int64_t)in[base + j];
  int64_t tot;
  block_excl_scan(s, tot);
  if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(kThreads) scan_sums_k(int64_t* sums, int64_t m) {
  int64_t carry = 0;
  for (int64_t b0 = 0; b0 < m; b0 += kTile) {
    const int64_t base = b0 + (int64_t)threadIdx.x * kItems;
    int64_t v[kItems], s = 0;
#pragma unroll
    for (int j = 0; j < kItems; ++j) {
      v[j] = base + j < m ? sums[base + j] : 0;
      s += v[j];
    }
    int64_t tot;
    int64_t run = carry + block_excl_scan(s, tot);
#pragma unroll
    for (int j = 0; j < kItems; ++j)
      if (base + j < m) {
        sums[base + j] = run;
        run += v[j];
      }
    carry += tot;
  }
  if (threadIdx.x == 0) sums[m] = carry;
}

template <class T>
__global__ void __launch_bounds__(kThreads) scan_down_k(const T* in, int64_t n, const int64_t* sums, int64_t* out,
                                                        int with_total) {
  const int64_t base = (int64_t)blockIdx.x * kTile + (int64_t)threadIdx.x * kItems;
  int64_t v[kItems], s = 0;
#pragma unroll
  for (int j = 0; j < kItems; ++j) {
    v[j] = base + j < n ? (int64_t)in[base + j] : 0;
    s += v[j];
  }
  int64_t tot;
  int64_t run = sums[blockIdx.x] + block_excl_scan(s, tot);
#pragma unroll
  for (int j = 0; j < kItems; ++j)
    if (base + j < n) {
      out[base + j] = run;
      run += v[j];
    }
  if (with_total && blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) out[n] = sums[gridDim.x];
}

template <class T>
cudaError_t excl_scan(const T* in, int64_t* out, int64_t n, bool with_total, Arena& ar, cudaStream_t s) {
  if (n == 0) return with_total ? cudaMemsetAsync(out, 0, sizeof(int64_t), s) : cudaSuccess;
  const int64_t blocks = (n + kTile - 1) / kTile;
  int64_t* sums = ar.get<int64_t>(blocks + 1);
  if (!sums) return ar.err;
  scan_reduce_k<T><<<(unsigned)blocks, kThreads, 0, s>>>(in, n, sums);
  scan_sums_k<<<1, kThreads, 0, s>>>(sums, blocks);
  scan_down_k<T><<<(unsigned)blocks, kThreads, 0, s>>>(in, n, sums, out, with_total ? 1 : 0);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ stable LSD radix sort
// 8-bit digits; per pass a per-block digit histogram (digit-major, so its exclusive scan
// gives every block its output offset per digit) and a stable scatter: an element's rank is
// the count of equal digits before it in the block (earlier rounds, earlier warps, earlier
// lanes), so equal keys keep their input order.
__global__ void __launch_bounds__(kThreads) radix_hist_k(const uint64_t* keys, int64_t n, int shift, uint32_t mask,
                                                         int64_t* hist, int64_t n_blocks) {
  __shared__ int cnt[256];
  cnt[threadIdx.x] = 0;
  __syncthreads();
  const int64_t base = (int64_t)blockIdx.x * kTile;
#pragma unroll
  for (int j = 0; j < kItems; ++j) {
    const int64_t i = base + (int64_t)j * kThreads + threadIdx.x;
    if (i < n) atomicAdd(&cnt[(uint32_t)(keys[i] >> shift) & mask], 1);
  }
  __syncthreads();
  hist[(int64_t)threadIdx.x * n_blocks + blockIdx.x] = cnt[threadIdx.x];
}

template <class V>
__global__ void __launch_bounds__(kThreads) radix_scatter_k(const uint64_t* kin, const V* vin, uint64_t* kout,
                                                            V* vout, int64_t n, int shift, uint32_t mask,
                                                            const int64_t* hist, int64_t n_blocks) {
  __shared__ int64_t base_off[256];
  __shared__ int run[256];
  __shared__ int wcnt[kThreads / 32][256];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  base_off[tid] = hist[(int64_t)tid * n_blocks + blockIdx.x];
  run[tid] = 0;
  const int64_t base = (int64_t)blockIdx.x * kTile;
  for (int j = 0; j < kItems; ++j) {
    const int64_t i = base + (int64_t)j * kThreads + tid;
    const bool valid = i < n;
    const uint64_t k = valid ? kin[i] : 0;
    const uint32_t d = valid ? ((uint32_t)(k >> shift) & mask) : 256u;
#pragma unroll
    for (int w = 0; w < kThreads / 32; ++w) wcnt[w][tid] = 0;
    __syncthreads();
    const unsigned peers = __match_any_sync(0xffffffffu, d);
    const int rank_w = __popc(peers & ((1u << lane) - 1u));
    if (valid && lane == __ffs(peers) - 1) wcnt[warp][d] = __popc(peers);
    __syncthreads();
    {  // thread tid owns digit tid: offsets of each warp's run of that digit in this round
      int acc = run[tid];
#pragma unroll
      for (int w = 0; w < kThreads / 32; ++w) {
        const int c = wcnt[w][tid];
        wcnt[w][tid] = acc;
        acc += c;
      }
      run[tid] = acc;
    }
    __syncthreads();
    if (valid) {
      const int64_t pos = base_off[d] + wcnt[warp][d] + rank_w;
      if (pos >= 0 && pos < n) {
        kout[pos] = k;
        vout[pos] = vin[i];
      } else {
        atomicOr(&g_build_err, 1);
      }
    }
    __syncthreads();
  }
}

// Sorts (keys, vals) by the low `bits` bits of the keys, stably. The sorted arrays end in
// (*keys, *vals); (*kalt, *valt) are scratch of the same size (pointers are swapped).
template <class V>
cudaError_t radix_sort(uint64_t** keys, V** vals, uint64_t** kalt, V** valt, int64_t n, int bits, Arena& ar,
                       cudaStream_t s) {
  if (n <= 1) return cudaSuccess;
  const int64_t blocks = (n + kTile - 1) / kTile;
  int64_t* hist = ar.get<int64_t>(256 * blocks + 1);
  if (!hist) return ar.err;
  for (int shift = 0; shift < bits; shift += 8) {
    const int nb = std::min(8, bits - shift);
    const uint32_t mask = (1u << nb) - 1u;
    radix_hist_k<<<(unsigned)blocks, kThreads, 0, s>>>(*keys, n, shift, mask, hist, blocks);
    cudaError_t e = excl_scan<int64_t>(hist, hist, 256 * blocks, false, ar, s);
    if (e != cudaSuccess) return e;
    radix_scatter_k<V><<<(unsigned)blocks, kThreads, 0, s>>>(*keys, *vals, *kalt, *valt, n, shift, mask, hist,
                                                              blocks);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    std::swap(*keys, *kalt);
    std::swap(*vals, *valt);
  }
  return cudaSuccess;
}

inline int bit_width(uint64_t x) {  // bits needed for x (at least 1)
  int b = 1;
  while (b < 64 && (x >> b)) ++b;
  return b;
}

inline unsigned grid_for(int64_t n) {
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + kThreads - 1) / kThreads, 152 * 16));
}

#define GS_LOOP(i, n) for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < (n); \
                           i += (int64_t)gridDim.x * blockDim.x)

__device__ __forceinline__ double load_val(const void* v, int vf32, int64_t k) {
  return vf32 ? (double)((const float*)v)[k] : ((const double*)v)[k];
}

// ------------------------------------------------------------------ 1. validation
struct ValStat {
  unsigned long long bad_row;     // first row i with row_ptr[i+1] < row_ptr[i]
  unsigned long long bad_entry;   // first entry with a column out of range
  unsigned long long max_bits;    // bits of max |a| over finite values (positive doubles order as integers)
  long long rp0, rpn;
};

__global__ void validate_k(const int64_t* rp, const int32_t* ci, const void* vals, int vf32, int64_t n_rows,
                           int64_t n_cols, int64_t nnz, int want_max, ValStat* st) {
  GS_LOOP(i, n_rows)
    if (rp[i + 1] < rp[i]) atomicMin(&st->bad_row, (unsigned long long)i);
  unsigned long long mx = 0;
  GS_LOOP(k, nnz) {
    const int32_t c = ci[k];
    if (c < 0 || (int64_t)c >= n_cols) atomicMin(&st->bad_entry, (unsigned long long)k);
    if (want_max) {
      const double a = fabs(load_val(vals, vf32, k));
      if (isfinite(a)) {
        const unsigned long long b = (unsigned long long)__double_as_longlong(a);
        mx = b > mx ? b : mx;
      }
    }
  }
  if (want_max && mx) atomicMax(&st->max_bits, mx);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    st->rp0 = rp[0];
    st->rpn = rp[n_rows];
  }
}

// ------------------------------------------------------------------ 2. keys and tiles
// Row of every entry: the last row i with row_ptr[i] <= k (empty rows are skipped over).
__global__ void entry_rows_k(const int64_t* rp, int64_t n_rows, int64_t nnz, int32_t* erow) {
  GS_LOOP(k, nnz) {
    int64_t lo = 0, hi = n_rows;  // rp[lo] <= k < rp[hi]
    while (hi - lo > 1) {
      const int64_t mid = (lo + hi) >> 1;
      if (rp[mid] <= k) lo = mid; else hi = mid;
    }
    erow[k] = (int32_t)lo;
  }
}

__global__ void make_keys_k(const int32_t* ci, const int32_t* erow, int64_t nnz, int32_t br, int cb,
                            uint64_t* key, int64_t* idx) {
  GS_LOOP(k, nnz) {
    key[k] = ((uint64_t)(erow[k] / br) << cb) | (uint64_t)(uint32_t)ci[k];
    idx[k] = k;
  }
}

__global__ void tile_flags_k(const uint64_t* key, int64_t nnz, int32_t* flag) {
  GS_LOOP(p, nnz) flag[p] = (p == 0 || key[p] != key[p - 1]) ? 1 : 0;
}

__global__ void tile_first_k(const int32_t* flag, const int64_t* tpos, int64_t nnz, int64_t* tile_first,
                             int64_t n_t) {
  GS_LOOP(p, nnz) {
    if (!flag[p]) continue;
    BUILD_CHECK(tpos[p] >= 0 && tpos[p] < n_t);
    tile_first[tpos[p]] = p;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) tile_first[n_t] = nnz;
}

// Per tile: its block's distinct-column and kept-tile counts, and the first tile of a block.
__global__ void tile_stats_k(const uint64_t* key, const int64_t* tile_first, int64_t n_t, int cb, int32_t tile_min,
                             int64_t nb, int32_t* u, int32_t* keep, int64_t* blk_first) {
  GS_LOOP(t, n_t) {
    const int64_t b = (int64_t)(key[tile_first[t]] >> cb);
    BUILD_CHECK(b >= 0 && b < nb);
    atomicAdd(&u[b], 1);
    const int64_t cnt = tile_first[t + 1] - tile_first[t];
    if (tile_min <= 1 || cnt >= tile_min) atomicAdd(&keep[b], 1);
    if (t == 0 || (int64_t)(key[tile_first[t - 1]] >> cb) != b) blk_first[b] = t;
  }
}

// ------------------------------------------------------------------ 3. split
__global__ void block_decide_k(const int64_t* rp, int64_t n_rows, int64_t nb, int32_t br, double tau,
                               int contiguous, int64_t rb_first, const int32_t* u, const int32_t* keep,
                               int32_t kpad, uint8_t* is_bcsr, int64_t* isb, int64_t* tpad) {
  GS_LOOP(b, nb) {
    const int64_t i0 = b * br, i1 = min(i0 + (int64_t)br, n_rows);
    const int64_t nnz_rb = rp[i1] - rp[i0];
    bool bcsr;
    if (contiguous) bcsr = b >= rb_first;
    else bcsr = nnz_rb > 0 && (double)nnz_rb >= tau * (double)u[b];  // d_rb >= tau without a division
    bcsr = bcsr && keep[b] > 0;
    is_bcsr[b] = bcsr ? 1 : 0;
    isb[b] = bcsr ? 1 : 0;
    tpad[b] = bcsr ? ((int64_t)keep[b] + kpad - 1) / kpad * kpad : 0;
  }
}

__global__ void block_out_k(const uint8_t* is_bcsr, const int64_t* rb_pos, const int64_t* rb_tile0, int64_t nb,
                            int64_t n_rb, int64_t n_tiles, int32_t* rb_id, int64_t* rb_ptr) {
  GS_LOOP(b, nb) {
    if (!is_bcsr[b]) continue;
    BUILD_CHECK(rb_pos[b] >= 0 && rb_pos[b] < n_rb);
    rb_id[rb_pos[b]] = (int32_t)b;
    rb_ptr[rb_pos[b]] = rb_tile0[b];
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) rb_ptr[n_rb] = n_tiles;
}

__global__ void tile_kept_k(const uint64_t* key, const int64_t* tile_first, int64_t n_t, int cb,
                            const uint8_t* is_bcsr, int32_t tile_min, int64_t nb, int64_t* kept) {
  GS_LOOP(t, n_t) {
    const int64_t b = (int64_t)(key[tile_first[t]] >> cb);
    BUILD_CHECK(b >= 0 && b < nb);
    const int64_t cnt = tile_first[t + 1] - tile_first[t];
    kept[t] = (is_bcsr[b] && (tile_min <= 1 || cnt >= tile_min)) ? 1 : 0;
  }
}

// Entry classes: 0 CSR part (row of a CSR block), 1 moved to the CSR part (sparse tile of a
// BCSR block), 2 BCSR tile. Moved entries are counted per row. `kept` is the exclusive scan
// of the kept-tile flags (tile t is kept when kept[t + 1] > kept[t]).
__global__ void entry_class_k(const uint64_t* key, const int64_t* idx, const int32_t* flag, const int64_t* tpos,
                              const int64_t* kept, const uint8_t* is_bcsr, const int32_t* erow, int64_t nnz, int cb,
                              int64_t n_t, int64_t nb, int64_t n_rows, uint8_t* cls, int32_t* rowlen1) {
  GS_LOOP(p, nnz) {
    const int64_t t = tpos[p] + flag[p] - 1;
    const int64_t b = (int64_t)(key[p] >> cb);
    const int64_t k = idx[p];
    BUILD_CHECK(t >= 0 && t < n_t && b >= 0 && b < nb && k >= 0 && k < nnz && erow[k] >= 0 && erow[k] < n_rows);
    uint8_t c = 0;
    if (is_bcsr[b]) {
      c = kept[t + 1] > kept[t] ? 2 : 1;
      if (c == 1) atomicAdd(&rowlen1[erow[k]], 1);
    }
    cls[k] = c;
  }
}

// ------------------------------------------------------------------ 4. BCSR packing
struct TileArgs {
  const uint64_t* key;
  const int64_t* idx;
  const int64_t* tile_first;
  const int64_t* kept;       // exclusive scan of the kept flags
  const int64_t* blk_first;
  const int64_t* rb_tile0;
  const int32_t* erow;
  const void* vals;
  int vf32;
  int64_t n_t;
  int cb;
  int32_t br;
  loops_dtype dtype;
  double scale;
  double tiny;               // smallest normal of a 16-bit dtype (0 otherwise)
  int32_t* tile_col;
  void* tile_val;
  int64_t* slot_cnt;         // value map: entries per fragment slot
  const int64_t* slot_ptr;   // value map: exclusive scan of slot_cnt (second pass)
  int64_t* slot_src;
  const int64_t* remap;
  unsigned long long* n_sub;
  int64_t n_tiles;           // tiles of the BCSR part (incl. padding)
  int64_t n_src;             // entries of the slot map (second pass)
};

__device__ __forceinline__ bool tile_is_kept(const TileArgs& a, int64_t t) { return a.kept[t + 1] > a.kept[t]; }

__device__ __forceinline__ int64_t tile_out_index(const TileArgs& a, int64_t t, int64_t b) {
  return a.rb_tile0[b] + a.kept[t] - a.kept[a.blk_first[b]];
}

// Tile values: the entries of a tile in input order, summed per row in binary64, then scaled
// and rounded once into the storage type at their fragment position.
template <class TB>
__global__ void tile_values_k(TileArgs a) {
  GS_LOOP(t, a.n_t) {
    if (!tile_is_kept(a, t)) continue;
    const int64_t p0 = a.tile_first[t], p1 = a.tile_first[t + 1];
    const uint64_t key = a.key[p0];
    const int64_t b = (int64_t)(key >> a.cb);
    const int64_t out = tile_out_index(a, t, b);
    BUILD_CHECK(out >= 0 && out < a.n_tiles);
    a.tile_col[out] = (int32_t)(key & ((1ull << a.cb) - 1));
    double acc[16];
    int cnt[16];
#pragma unroll
    for (int r = 0; r < 16; ++r) { acc[r] = 0.0; cnt[r] = 0; }
    for (int64_t p = p0; p < p1; ++p) {
      const int64_t k = a.idx[p];
      const int r = (int)(a.erow[k] - b * a.br);
      if (r < 0 || r >= a.br) { atomicOr(&g_build_err, 1); continue; }
      const double v = load_val(a.vals, a.vf32, k);
#pragma unroll
      for (int q = 0; q < 16; ++q)
        if (q == r) { acc[q] += v; cnt[q]++; }
    }
#pragma unroll
    for (int r = 0; r < 16; ++r) {
      if (r >= a.br) break;
      const int64_t f = frag_index(a.dtype, out, r, a.br);
      const TB x = from_f64<TB>(acc[r] * a.scale);
      reinterpret_cast<TB*>(a.tile_val)[f] = x;
      if (a.slot_cnt) a.slot_cnt[f] = cnt[r];
      if (a.tiny > 0.0) {
        const double y = (double)(float)x;
        if (y != 0.0 && fabs(y) < a.tiny) atomicAdd(a.n_sub, 1ull);
      }
    }
  }
}

// Value map of the fragment slots: input entries of each slot in input order.
__global__ void tile_srcmap_k(TileArgs a) {
  GS_LOOP(t, a.n_t) {
    if (!tile_is_kept(a, t)) continue;
    const int64_t p0 = a.tile_first[t], p1 = a.tile_first[t + 1];
    const int64_t b = (int64_t)(a.key[p0] >> a.cb);
    const int64_t out = tile_out_index(a, t, b);
    BUILD_CHECK(out >= 0 && out < a.n_tiles);
    int fill[16];
#pragma unroll
    for (int r = 0; r < 16; ++r) fill[r] = 0;
    for (int64_t p = p0; p < p1; ++p) {
      const int64_t k = a.idx[p];
      const int r = (int)(a.erow[k] - b * a.br);
      int off = 0;
#pragma unroll
      for (int q = 0; q < 16; ++q)
        if (q == r) off = fill[q]++;
      if (r < 0 || r >= a.br) { atomicOr(&g_build_err, 1); continue; }
      const int64_t f = frag_index(a.dtype, out, r, a.br);
      const int64_t at = a.slot_ptr[f] + off;
      if (at < 0 || at >= a.n_src) { atomicOr(&g_build_err, 1); continue; }
      a.slot_src[at] = a.remap ? a.remap[k] : k;
    }
  }
}

__global__ void pad_tiles_k(const uint8_t* is_bcsr, const int32_t* keep, const int64_t* tpad, const int64_t* rb_tile0,
                            int64_t nb, int64_t n_tiles, int32_t* tile_col) {
  GS_LOOP(b, nb) {
    if (!is_bcsr[b]) continue;
    BUILD_CHECK(rb_tile0[b] >= 0 && rb_tile0[b] + tpad[b] <= n_tiles);
    for (int64_t q = keep[b]; q < tpad[b]; ++q) tile_col[rb_tile0[b] + q] = -1;
  }
}

// Work units of the BCSR blocks: blocks above kBcsrSplitTiles tiles become several units
// (partial-sum slots in block order); pre-order units are keyed by kBcsrSplitTiles - length.
__global__ void unit_count_k(const int64_t* rb_ptr, int64_t n_rb, int64_t* n_units, int64_t* n_slots,
                             int64_t* is_split) {
  GS_LOOP(c, n_rb) {
    const int64_t len = rb_ptr[c + 1] - rb_ptr[c];
    const bool sp = len > kBcsrSplitTiles;
    n_units[c] = sp ? (len + kBcsrSplitTiles - 1) / kBcsrSplitTiles : 1;
    n_slots[c] = sp ? n_units[c] : 0;
    is_split[c] = sp ? 1 : 0;
  }
}

// split_block / split_slot_ptr exist only when some block is cut (n_split > 0).
__global__ void unit_emit_k(const int64_t* rb_ptr, int64_t n_rb, const int64_t* ubase, const int64_t* sbase,
                            const int64_t* spidx, int64_t n_bslots, int64_t n_units, uint64_t* ukey, int64_t* uval,
                            int32_t* pre_b, int64_t* pre_t0, int64_t* pre_t1, int32_t* pre_slot, int32_t* split_block,
                            int32_t* split_slot_ptr, int64_t n_split) {
  GS_LOOP(c, n_rb) {
    const int64_t t0 = rb_ptr[c], t1 = rb_ptr[c + 1];
    const bool sp = t1 - t0 > kBcsrSplitTiles;
    int64_t u = ubase[c], slot = sbase[c];
    BUILD_CHECK(u >= 0 && u + (t1 - t0 + kBcsrSplitTiles - 1) / kBcsrSplitTiles <= n_units);
    if (sp) {
      BUILD_CHECK(split_block && spidx[c] >= 0 && spidx[c] < n_split);
      split_block[spidx[c]] = (int32_t)c;
      split_slot_ptr[spidx[c]] = (int32_t)slot;
    }
    for (int64_t t = t0; t < t1; t += kBcsrSplitTiles) {  // a BCSR block has at least one tile
      const int64_t e = min(t + kBcsrSplitTiles, t1);
      pre_b[u] = (int32_t)c;
      pre_t0[u] = t;
      pre_t1[u] = e;
      pre_slot[u] = sp ? (int32_t)slot++ : -1;
      ukey[u] = (uint64_t)(kBcsrSplitTiles - (e - t));
      uval[u] = u;
      ++u;
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0 && split_slot_ptr) split_slot_ptr[n_split] = (int32_t)n_bslots;
}

__global__ void unit_gather_k(const int64_t* order, int64_t n, const int32_t* pre_b, const int64_t* pre_t0,
                              const int64_t* pre_t1, const int32_t* pre_slot, int32_t* ub, int64_t* u0, int64_t* u1,
                              int32_t* us) {
  GS_LOOP(q, n) {
    const int64_t u = order[q];
    BUILD_CHECK(u >= 0 && u < n);
    ub[q] = pre_b[u];
    u0[q] = pre_t0[u];
    u1[q] = pre_t1[u];
    us[q] = pre_slot[u];
  }
}

// ------------------------------------------------------------------ 5. CSR packing
__global__ void class_flags_k(const uint8_t* cls, int64_t nnz, int32_t* f0, int32_t* f1) {
  GS_LOOP(k, nnz) {
    f0[k] = cls[k] == 0;
    f1[k] = cls[k] == 1;
  }
}

// canonical position -> input entry, for one CSR set
__global__ void canon_src_k(const uint8_t* cls, const int64_t* cpos, int64_t nnz, uint8_t which, int64_t n_src,
                            int64_t* src) {
  GS_LOOP(k, nnz) {
    if (cls[k] != which) continue;
    BUILD_CHECK(cpos[k] >= 0 && cpos[k] < n_src);
    src[cpos[k]] = k;
  }
}

__device__ __forceinline__ int bucket_of_len(int64_t len) {  // floor(log2(len + 1)), at most 62
  const int b = 63 - __clzll((long long)(len + 1));
  return b < 62 ? b : 62;
}

// Rows of one CSR set: set 0 takes every row of a CSR block (empty rows too), set 1 the rows
// of BCSR blocks that have moved entries. Rows longer than L become split rows of
// ceil(len / L) segments.
__global__ void row_count_k(const int64_t* rp, const uint8_t* is_bcsr, const int32_t* rowlen1, int64_t n_rows,
                            int32_t br, int which, int64_t L, int64_t* n_items, int64_t* n_slots, int64_t* is_split) {
  GS_LOOP(i, n_rows) {
    const bool in_b = is_bcsr[i / br] != 0;
    int64_t len = -1;
    if (which == 0 && !in_b) len = rp[i + 1] - rp[i];
    if (which == 1 && in_b && rowlen1[i] > 0) len = rowlen1[i];
    const bool sp = len > L;
    n_items[i] = len < 0 ? 0 : (sp ? (len + L - 1) / L : 1);
    n_slots[i] = sp ? n_items[i] : 0;
    is_split[i] = sp ? 1 : 0;
  }
}

__global__ void row_emit_k(const int64_t* rp, const uint8_t* is_bcsr, const int32_t* rowlen1, const int64_t* cpos,
                           int64_t n_rows, int32_t br, int which, int64_t L, const int64_t* ibase,
                           const int64_t* sbase, const int64_t* spidx, int64_t n_slots, int64_t n_split,
                           int64_t n_items, uint64_t* ikey, int64_t* ival, int32_t* pre_row, int64_t* pre_beg,
                           int64_t* pre_len, int32_t* split_row, int32_t* split_slot_ptr) {
  GS_LOOP(i, n_rows) {
    const bool in_b = is_bcsr[i / br] != 0;
    int64_t len = -1;
    if (which == 0 && !in_b) len = rp[i + 1] - rp[i];
    if (which == 1 && in_b && rowlen1[i] > 0) len = rowlen1[i];
    if (len < 0) continue;
    const int64_t beg = cpos[rp[i]];  // canonical position of the row's first entry in this set
    int64_t it = ibase[i];
    BUILD_CHECK(it >= 0 && it + (len > L ? (len + L - 1) / L : 1) <= n_items);
    if (len > L) {
      int64_t slot = sbase[i];
      BUILD_CHECK(split_row && spidx[i] >= 0 && spidx[i] < n_split);
      split_row[spidx[i]] = (int32_t)i;
      split_slot_ptr[spidx[i]] = (int32_t)slot;
      for (int64_t s0 = 0; s0 < len; s0 += L, ++it, ++slot) {
        pre_row[it] = (int32_t)(-1 - slot);
        pre_beg[it] = beg + s0;
        pre_len[it] = min(L, len - s0);
        ikey[it] = 0;  // bucket 63 first (or row order)
        ival[it] = it;
      }
    } else {
      pre_row[it] = (int32_t)i;
      pre_beg[it] = beg;
      pre_len[it] = len;
      ikey[it] = LOOPS_CSR_ITEMS_BY_LENGTH ? (uint64_t)(63 - bucket_of_len(len)) : 0;
      ival[it] = it;
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0 && split_slot_ptr) split_slot_ptr[n_split] = (int32_t)n_slots;
}

__global__ void item_order_k(const int64_t* order, int64_t n, const int32_t* pre_row, const int64_t* pre_len,
                             int32_t* item_row, int64_t* dlen) {
  GS_LOOP(q, n) {
    const int64_t u = order[q];
    BUILD_CHECK(u >= 0 && u < n);
    item_row[q] = pre_row[u];
    dlen[q] = pre_len[u];
  }
}

// One warp per item: columns and rounded values of its entries, and the value map.
template <class TB>
__global__ void item_gather_k(const int64_t* order, int64_t n, const int64_t* pre_beg, const int64_t* item_ptr,
                              const int64_t* canon_src, int64_t n_canon, int64_t total, const int32_t* ci,
                              const void* vals, int vf32, double scale, double tiny, const int64_t* remap,
                              int32_t* col, TB* val, int64_t* csr_src, unsigned long long* n_sub) {
  const int lane = threadIdx.x & 31;
  for (int64_t q = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; q < n;
       q += ((int64_t)gridDim.x * blockDim.x) >> 5) {
    const int64_t b = pre_beg[order[q]];
    const int64_t d0 = item_ptr[q], len = item_ptr[q + 1] - d0;
    BUILD_CHECK(b >= 0 && b + len <= n_canon && d0 >= 0 && d0 + len <= total);
    unsigned long long sub = 0;
    for (int64_t e = lane; e < len; e += 32) {
      const int64_t k = canon_src[b + e];
      col[d0 + e] = ci[k];
      const TB x = from_f64<TB>(load_val(vals, vf32, k) * scale);
      val[d0 + e] = x;
      if (csr_src) csr_src[d0 + e] = remap ? remap[k] : k;
      if (tiny > 0.0) {
        const double y = (double)(float)x;
        sub += (y != 0.0 && fabs(y) < tiny);
      }
    }
    if (sub) atomicAdd(n_sub, sub);
  }
}

// ------------------------------------------------------------------ 6. backward pieces
__global__ void sddmm_count_k(const int64_t* rp, int64_t n_rows, int64_t L, int64_t* n_items) {
  GS_LOOP(i, n_rows) {
    const int64_t len = rp[i + 1] - rp[i];
    n_items[i] = (len + L - 1) / L;
  }
}

__global__ void sddmm_emit_k(const int64_t* rp, int64_t n_rows, int64_t L, const int64_t* ibase, int64_t n_items,
                             uint64_t* key, int64_t* val, int32_t* pre_row, int64_t* pre_beg, int64_t* pre_end) {
  GS_LOOP(i, n_rows) {
    int64_t it = ibase[i];
    BUILD_CHECK(it >= 0 && it + (rp[i + 1] - rp[i] + L - 1) / L <= n_items);
    for (int64_t b = rp[i]; b < rp[i + 1]; b += L, ++it) {
      const int64_t e = min(b + L, rp[i + 1]);
      pre_row[it] = (int32_t)i;
      pre_beg[it] = b;
      pre_end[it] = e;
      key[it] = (uint64_t)(L - (e - b));
      val[it] = it;
    }
  }
}

__global__ void sddmm_gather_k(const int64_t* order, int64_t n, const int32_t* pre_row, const int64_t* pre_beg,
                               const int64_t* pre_end, int32_t* row, int64_t* beg, int64_t* end) {
  GS_LOOP(q, n) {
    const int64_t u = order[q];
    BUILD_CHECK(u >= 0 && u < n);
    row[q] = pre_row[u];
    beg[q] = pre_beg[u];
    end[q] = pre_end[u];
  }
}

__global__ void col_keys_k(const int32_t* ci, int64_t nnz, uint64_t* key, int64_t* idx, int64_t* col_cnt) {
  GS_LOOP(k, nnz) {
    key[k] = (uint64_t)(uint32_t)ci[k];
    idx[k] = k;
    atomicAdd((unsigned long long*)&col_cnt[ci[k]], 1ull);
  }
}

__global__ void transpose_fill_k(const int64_t* perm, const int32_t* erow, const void* vals, int vf32, int64_t nnz,
                                 int32_t* t_ci, double* t_vals) {
  GS_LOOP(e, nnz) {
    const int64_t k = perm[e];
    t_ci[e] = erow[k];
    t_vals[e] = load_val(vals, vf32, k);
  }
}

// ------------------------------------------------------------------ host helpers
template <class T>
cudaError_t to_host(T* dst, const T* src, cudaStream_t s) {
  cudaError_t e = cudaMemcpyAsync(dst, src, sizeof(T), cudaMemcpyDeviceToHost, s);
  return e == cudaSuccess ? cudaStreamSynchronize(s) : e;
}

// Plan-owned device array (counted in the plan's device bytes).
template <class T>
cudaError_t own(T** dst, int64_t n, int64_t& bytes) {
  *dst = nullptr;
  if (n <= 0) return cudaSuccess;
  cudaError_t e = dev_malloc((void**)dst, (size_t)n * sizeof(T));
  if (e != cudaSuccess) { cudaGetLastError(); *dst = nullptr; return e; }
  bytes += n * (int64_t)sizeof(T);
  return cudaSuccess;
}

template <class TB>
cudaError_t launch_tile_values(const TileArgs& a, cudaStream_t s) {
  tile_values_k<TB><<<grid_for(a.n_t), kThreads, 0, s>>>(a);
  return cudaGetLastError();
}

template <class TB>
cudaError_t launch_item_gather(const int64_t* order, int64_t n, const int64_t* pre_beg, const int64_t* item_ptr,
                               const int64_t* canon_src, int64_t n_canon, int64_t total, const DevCsrIn& A,
                               double scale, double tiny, const int64_t* remap, int32_t* col, void* val,
                               int64_t* csr_src, unsigned long long* n_sub, cudaStream_t s) {
  const unsigned blocks = (unsigned)std::max<int64_t>(1, std::min<int64_t>((n * 32 + kThreads - 1) / kThreads, 152 * 16));
  item_gather_k<TB><<<blocks, kThreads, 0, s>>>(order, n, pre_beg, item_ptr, canon_src, n_canon, total, A.ci,
                                                 A.vals, A.vals_f32, scale, tiny, remap, col, (TB*)val, csr_src,
                                                 n_sub);
  return cudaGetLastError();
}

cudaError_t dispatch_tile_values(loops_dtype d, const TileArgs& a, cudaStream_t s) {
  switch (d) {
    case LOOPS_F64: return launch_tile_values<double>(a, s);
    case LOOPS_F32: return launch_tile_values<float>(a, s);
    case LOOPS_F16: return launch_tile_values<__half>(a, s);
    case LOOPS_BF16: return launch_tile_values<__nv_bfloat16>(a, s);
  }
  return cudaErrorInvalidValue;
}

cudaError_t dispatch_item_gather(loops_dtype d, const int64_t* order, int64_t n, const int64_t* pre_beg,
                                 const int64_t* item_ptr, const int64_t* canon_src, int64_t n_canon, int64_t total,
                                 const DevCsrIn& A, double scale, double tiny, const int64_t* remap, int32_t* col,
                                 void* val, int64_t* csr_src, unsigned long long* n_sub, cudaStream_t s) {
#define LOOPS_GATHER(TB) \
  launch_item_gather<TB>(order, n, pre_beg, item_ptr, canon_src, n_canon, total, A, scale, tiny, remap, col, val, \
                         csr_src, n_sub, s)
  switch (d) {
    case LOOPS_F64: return LOOPS_GATHER(double);
    case LOOPS_F32: return LOOPS_GATHER(float);
    case LOOPS_F16: return LOOPS_GATHER(__half);
    case LOOPS_BF16: return LOOPS_GATHER(__nv_bfloat16);
  }
#undef LOOPS_GATHER
  return cudaErrorInvalidValue;
}

cudaError_t reset_build_err(cudaStream_t s) {
  const int zero = 0;
  return cudaMemcpyToSymbolAsync(g_build_err, &zero, sizeof(int), 0, cudaMemcpyHostToDevice, s);
}

// After a build stage: a recorded index check fails the build (no access was made).
loops_status check_build_err(cudaStream_t s, const char* what) {
  int h = 0;
  cudaError_t e = cudaMemcpyFromSymbolAsync(&h, g_build_err, sizeof(int), 0, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_status(e, what);
  if (h) {
    set_error(std::string(what) + ": an index check failed (access skipped); the plan was not built");
    return LOOPS_ERR_STATE;
  }
  return LOOPS_OK;
}

#define TRY(x) do { cudaError_t e_ = (x); if (e_ != cudaSuccess) return cuda_status(e_, what); } while (0)
#define NEED(ptr) do { if (!(ptr)) return cuda_status(ar.err, what); } while (0)

// One CSR set (0: rows of CSR blocks, 1: moved entries of BCSR blocks) into its work items.
loops_status build_csr_set(loops_plan_s* p, const DevCsrIn& A, const int64_t* remap, int which, const uint8_t* cls,
                           const uint8_t* is_bcsr, const int32_t* rowlen1, const int64_t* cpos, const int64_t* csrc,
                           int64_t n_canon, int64_t N, double tiny, unsigned long long* n_sub, int64_t** csr_src_out, int64_t* n_src,
                           Arena& ar, cudaStream_t s) {
  const char* what = "device plan build (CSR part)";
  CsrDev& cd = which == 0 ? p->dev.csr : p->dev.csr_acc;
  int64_t& bytes = p->dev.device_bytes;
  const int64_t n = A.n_rows, L = std::max<int64_t>(p->split_len, 1);
  int64_t* n_items_r = ar.get<int64_t>(n + 1);
  int64_t* n_slots_r = ar.get<int64_t>(n + 1);
  int64_t* split_r = ar.get<int64_t>(n + 1);
  NEED(split_r);
  if (n) row_count_k<<<grid_for(n), kThreads, 0, s>>>(A.rp, is_bcsr, rowlen1, n, p->br, which, L, n_items_r,
                                                      n_slots_r, split_r);
  TRY(cudaGetLastError());
  TRY(excl_scan<int64_t>(n_items_r, n_items_r, n, true, ar, s));
  TRY(excl_scan<int64_t>(n_slots_r, n_slots_r, n, true, ar, s));
  TRY(excl_scan<int64_t>(split_r, split_r, n, true, ar, s));
  int64_t n_it = 0, n_sl = 0, n_sp = 0;
  TRY(to_host(&n_it, n_items_r + n, s));
  TRY(to_host(&n_sl, n_slots_r + n, s));
  TRY(to_host(&n_sp, split_r + n, s));
  cd.n_items = n_it;
  cd.n_slots = n_sl;
  cd.n_split = n_sp;
  if (n_it == 0) return LOOPS_OK;
  uint64_t* ikey = ar.get<uint64_t>(n_it);
  uint64_t* ikey2 = ar.get<uint64_t>(n_it);
  int64_t* ival = ar.get<int64_t>(n_it);
  int64_t* ival2 = ar.get<int64_t>(n_it);
  int32_t* pre_row = ar.get<int32_t>(n_it);
  int64_t* pre_beg = ar.get<int64_t>(n_it);
  int64_t* pre_len = ar.get<int64_t>(n_it);
  int64_t* dlen = ar.get<int64_t>(n_it + 1);
  NEED(dlen);
  if (n_sp) {
    TRY(own(&cd.split_row, n_sp, bytes));
    TRY(own(&cd.split_slot_ptr, n_sp + 1, bytes));
  }
  row_emit_k<<<grid_for(n), kThreads, 0, s>>>(A.rp, is_bcsr, rowlen1, cpos, n, p->br, which, L, n_items_r, n_slots_r,
                                              split_r, n_sl, n_sp, n_it, ikey, ival, pre_row, pre_beg, pre_len,
                                              cd.split_row, cd.split_slot_ptr);
  TRY(cudaGetLastError());
  TRY(radix_sort<int64_t>(&ikey, &ival, &ikey2, &ival2, n_it, 6, ar, s));
  TRY(own(&cd.item_row, n_it, bytes));
  TRY(own(&cd.item_ptr, n_it + 1, bytes));
  item_order_k<<<grid_for(n_it), kThreads, 0, s>>>(ival, n_it, pre_row, pre_len, cd.item_row, dlen);
  TRY(cudaGetLastError());
  TRY(excl_scan<int64_t>(dlen, cd.item_ptr, n_it, true, ar, s));
  int64_t total = 0;
  TRY(to_host(&total, cd.item_ptr + n_it, s));
  cd.nnz = total;
  const int es = dense_elem_bytes(p->dtype);
  TRY(own(&cd.col, total, bytes));
  TRY(own((uint8_t**)&cd.val, total * es, bytes));
  int64_t* csr_src = nullptr;
  if (csr_src_out) {
    csr_src = ar.get<int64_t>(total);
    NEED(csr_src);
  }
  if (total)
    TRY(dispatch_item_gather(p->dtype, ival, n_it, pre_beg, cd.item_ptr, csrc, n_canon, total, A, p->scale, tiny,
                             remap, cd.col, cd.val, csr_src, n_sub, s));
  if (n_sl) {
    const int acc_bytes = p->dtype == LOOPS_F64 ? 8 : 4;
    TRY(own((uint8_t**)&cd.scratch, n_sl * std::max<int64_t>(N, 1) * acc_bytes, bytes));
  }
  if (csr_src_out) {
    *csr_src_out = csr_src;
    *n_src = total;
  }
  return LOOPS_OK;
}

}  // namespace

loops_status validate_csr_device(const DevCsrIn& A, loops_dtype dtype, cudaStream_t s, double* max_abs) {
  const char* what = "device CSR validation";
  *max_abs = 0.0;
  if (A.n_rows < 0 || A.n_cols < 0 || A.nnz < 0) {
    set_error("negative matrix size");
    return LOOPS_ERR_INVALID_ARG;
  }
  if (A.n_rows >= (int64_t)INT32_MAX || A.n_cols >= (int64_t)INT32_MAX) {
    set_error("n_rows and n_cols must be below 2^31 - 1");
    return LOOPS_ERR_UNSUPPORTED;
  }
  if (!A.rp || (A.nnz > 0 && (!A.ci || !A.vals))) {
    set_error("CSR array pointer is NULL");
    return LOOPS_ERR_INVALID_ARG;
  }
  ValStat h;
  ValStat* d = nullptr;
  TRY(dev_malloc_async(&d, sizeof(ValStat), s));
  h.bad_row = h.bad_entry = ~0ull;
  h.max_bits = 0;
  h.rp0 = h.rpn = 0;
  cudaError_t e = cudaMemcpyAsync(d, &h, sizeof(h), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) {
    validate_k<<<grid_for(std::max(A.n_rows, A.nnz)), kThreads, 0, s>>>(
        A.rp, A.ci, A.vals, A.vals_f32, A.n_rows, A.n_cols, A.nnz, dtype == LOOPS_F16 || dtype == LOOPS_BF16, d);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h, d, sizeof(h), cudaMemcpyDeviceToHost, s);
  cudaFreeAsync(d, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  TRY(e);
  // reported in the order the host validation checks them
  if (h.rp0 != 0) { set_error("row_ptr[0] != 0"); return LOOPS_ERR_INVALID_CSR; }
  if (h.bad_row != ~0ull) {
    set_error("row_ptr is not non-decreasing at row " + std::to_string(h.bad_row));
    return LOOPS_ERR_INVALID_CSR;
  }
  if (h.rpn != A.nnz) { set_error("row_ptr[n_rows] != nnz"); return LOOPS_ERR_INVALID_CSR; }
  if (h.bad_entry != ~0ull) {
    set_error("column index out of range at entry " + std::to_string(h.bad_entry));
    return LOOPS_ERR_INVALID_CSR;
  }
  double mx;
  std::memcpy(&mx, &h.max_bits, 8);
  *max_abs = mx;
  return LOOPS_OK;
}

double plan_scale_from_max(double mx, loops_dtype d) {
  if (d != LOOPS_F16 && d != LOOPS_BF16) return 1.0;
  if (mx == 0.0) return 1.0;
  int e2;
  const double f = std::frexp(mx, &e2);  // mx = f * 2^e2, f in [0.5, 1)
  const int c = (f == 0.5) ? e2 - 1 : e2;
  return std::ldexp(1.0, 14 - c);
}

loops_status build_part_device(loops_plan_s* p, const DevCsrIn& A, const int64_t* remap, int64_t N, double tau,
                               bool contiguous, int64_t r_boundary, bool want_maps, cudaStream_t s) {
  const char* what = "device plan build";
  Arena ar;
  ar.s = s;
  PartDev& d = p->dev;
  d = PartDev();
  int64_t& bytes = d.device_bytes;
  const int64_t n = A.n_rows, nnz = A.nnz;
  const int32_t br = p->br, kpad = p->kpad;
  const int64_t nb = (n + br - 1) / br;
  const int cb = bit_width(A.n_cols > 1 ? (uint64_t)(A.n_cols - 1) : 1);
  const int bb = bit_width(nb > 1 ? (uint64_t)(nb - 1) : 1);
  const int32_t tile_min = p->tile_min;
  const double tiny = p->dtype == LOOPS_F16 ? std::ldexp(1.0, -14) : p->dtype == LOOPS_BF16 ? std::ldexp(1.0, -126) : 0.0;
  unsigned long long* n_sub = ar.get<unsigned long long>(1);
  NEED(n_sub);
  TRY(cudaMemsetAsync(n_sub, 0, sizeof(unsigned long long), s));
  TRY(reset_build_err(s));

  // ---- 2. entries sorted by (row block, column), ties in input order; tiles are the runs
  int32_t* erow = ar.get<int32_t>(nnz);
  uint64_t* key = ar.get<uint64_t>(nnz);
  uint64_t* key2 = ar.get<uint64_t>(nnz);
  int64_t* idx = ar.get<int64_t>(nnz);
  int64_t* idx2 = ar.get<int64_t>(nnz);
  int32_t* flag = ar.get<int32_t>(nnz);
  int64_t* tpos = ar.get<int64_t>(nnz + 1);
  int32_t* u = ar.get<int32_t>(nb);
  int32_t* keep = ar.get<int32_t>(nb);
  int64_t* blk_first = ar.get<int64_t>(nb);
  uint8_t* is_bcsr = ar.get<uint8_t>(nb);
  int64_t* isb = ar.get<int64_t>(nb + 1);
  int64_t* tpad = ar.get<int64_t>(nb + 1);
  int64_t* rb_pos = ar.get<int64_t>(nb + 1);
  int64_t* rb_tile0 = ar.get<int64_t>(nb + 1);
  uint8_t* cls = ar.get<uint8_t>(nnz);
  int32_t* rowlen1 = ar.get<int32_t>(n);
  NEED(rowlen1);
  TRY(cudaMemsetAsync(u, 0, (size_t)std::max<int64_t>(nb, 1) * 4, s));
  TRY(cudaMemsetAsync(keep, 0, (size_t)std::max<int64_t>(nb, 1) * 4, s));
  TRY(cudaMemsetAsync(rowlen1, 0, (size_t)std::max<int64_t>(n, 1) * 4, s));
  int64_t n_t = 0;
  int64_t* tile_first = nullptr;
  if (nnz) {
    entry_rows_k<<<grid_for(nnz), kThreads, 0, s>>>(A.rp, n, nnz, erow);
    make_keys_k<<<grid_for(nnz), kThreads, 0, s>>>(A.ci, erow, nnz, br, cb, key, idx);
    TRY(cudaGetLastError());
    TRY(radix_sort<int64_t>(&key, &idx, &key2, &idx2, nnz, cb + bb, ar, s));
    tile_flags_k<<<grid_for(nnz), kThreads, 0, s>>>(key, nnz, flag);
    TRY(cudaGetLastError());
    TRY(excl_scan<int32_t>(flag, tpos, nnz, true, ar, s));
    TRY(to_host(&n_t, tpos + nnz, s));
    tile_first = ar.get<int64_t>(n_t + 1);
    NEED(tile_first);
    tile_first_k<<<grid_for(nnz), kThreads, 0, s>>>(flag, tpos, nnz, tile_first, n_t);
    tile_stats_k<<<grid_for(n_t), kThreads, 0, s>>>(key, tile_first, n_t, cb, tile_min, nb, u, keep, blk_first);
    TRY(cudaGetLastError());
  }

  // ---- 3. block split
  const int64_t rb_first = contiguous ? (std::max<int64_t>(r_boundary, 0) + br - 1) / br : 0;
  if (nb)
    block_decide_k<<<grid_for(nb), kThreads, 0, s>>>(A.rp, n, nb, br, tau, contiguous ? 1 : 0, rb_first, u, keep,
                                                     kpad, is_bcsr, isb, tpad);
  TRY(cudaGetLastError());
  TRY(excl_scan<int64_t>(isb, rb_pos, nb, true, ar, s));
  TRY(excl_scan<int64_t>(tpad, rb_tile0, nb, true, ar, s));
  int64_t n_rb = 0, n_tiles = 0;
  TRY(to_host(&n_rb, rb_pos + nb, s));
  TRY(to_host(&n_tiles, rb_tile0 + nb, s));
  d.bcsr.n_rb = n_rb;
  d.bcsr.n_tiles = n_tiles;
  p->n_rb = n_rb;
  p->n_tiles = n_tiles;

  int64_t* kept = nullptr;
  if (nnz) {
    kept = ar.get<int64_t>(n_t + 1);
    NEED(kept);
    tile_kept_k<<<grid_for(n_t), kThreads, 0, s>>>(key, tile_first, n_t, cb, is_bcsr, tile_min, nb, kept);
    TRY(cudaGetLastError());
    TRY(excl_scan<int64_t>(kept, kept, n_t, true, ar, s));
    entry_class_k<<<grid_for(nnz), kThreads, 0, s>>>(key, idx, flag, tpos, kept, is_bcsr, erow, nnz, cb, n_t, nb,
                                                     n, cls, rowlen1);
    TRY(cudaGetLastError());
  }

  // ---- 4. BCSR part
  int64_t* slot_ptr = nullptr;
  int64_t* slot_src = nullptr;
  const int64_t n_fslots = n_tiles * br;
  if (n_rb) {
    const int es = dense_elem_bytes(p->dtype);
    TRY(own(&d.bcsr.rb_id, n_rb, bytes));
    TRY(own(&d.bcsr.rb_ptr, n_rb + 1, bytes));
    TRY(own(&d.bcsr.tile_col, n_tiles, bytes));
    TRY(own((uint8_t**)&d.bcsr.tile_val, n_fslots * es, bytes));
    TRY(cudaMemsetAsync(d.bcsr.tile_val, 0, (size_t)(n_fslots * es), s));
    block_out_k<<<grid_for(nb), kThreads, 0, s>>>(is_bcsr, rb_pos, rb_tile0, nb, n_rb, n_tiles, d.bcsr.rb_id,
                                                  d.bcsr.rb_ptr);
    pad_tiles_k<<<grid_for(nb), kThreads, 0, s>>>(is_bcsr, keep, tpad, rb_tile0, nb, n_tiles, d.bcsr.tile_col);
    TRY(cudaGetLastError());
    TileArgs ta;
    ta.key = key;
    ta.idx = idx;
    ta.tile_first = tile_first;
    ta.kept = kept;
    ta.blk_first = blk_first;
    ta.rb_tile0 = rb_tile0;
    ta.erow = erow;
    ta.vals = A.vals;
    ta.vf32 = A.vals_f32;
    ta.n_t = n_t;
    ta.cb = cb;
    ta.br = br;
    ta.dtype = p->dtype;
    ta.scale = p->scale;
    ta.tiny = tiny;
    ta.tile_col = d.bcsr.tile_col;
    ta.tile_val = d.bcsr.tile_val;
    ta.slot_cnt = nullptr;
    ta.slot_ptr = nullptr;
    ta.slot_src = nullptr;
    ta.remap = remap;
    ta.n_sub = n_sub;
    ta.n_tiles = n_tiles;
    ta.n_src = 0;
    int64_t* slot_cnt = nullptr;
    if (want_maps) {
      slot_cnt = ar.get<int64_t>(n_fslots);
      slot_ptr = ar.get<int64_t>(n_fslots + 1);
      NEED(slot_ptr);
      TRY(cudaMemsetAsync(slot_cnt, 0, (size_t)n_fslots * 8, s));  // padding slots stay 0
      ta.slot_cnt = slot_cnt;
    }
    TRY(dispatch_tile_values(p->dtype, ta, s));
    if (want_maps) {
      TRY(excl_scan<int64_t>(slot_cnt, slot_ptr, n_fslots, true, ar, s));
      int64_t n_src = 0;
      TRY(to_host(&n_src, slot_ptr + n_fslots, s));
      slot_src = ar.get<int64_t>(n_src);
      NEED(slot_src);
      ta.slot_ptr = slot_ptr;
      ta.slot_src = slot_src;
      ta.n_src = n_src;
      tile_srcmap_k<<<grid_for(n_t), kThreads, 0, s>>>(ta);
      TRY(cudaGetLastError());
    }
    // work units
    int64_t* nu = ar.get<int64_t>(n_rb + 1);
    int64_t* ns = ar.get<int64_t>(n_rb + 1);
    int64_t* sp = ar.get<int64_t>(n_rb + 1);
    NEED(sp);
    unit_count_k<<<grid_for(n_rb), kThreads, 0, s>>>(d.bcsr.rb_ptr, n_rb, nu, ns, sp);
    TRY(cudaGetLastError());
    TRY(excl_scan<int64_t>(nu, nu, n_rb, true, ar, s));
    TRY(excl_scan<int64_t>(ns, ns, n_rb, true, ar, s));
    TRY(excl_scan<int64_t>(sp, sp, n_rb, true, ar, s));
    int64_t n_units = 0, n_bslots = 0, n_bsplit = 0;
    TRY(to_host(&n_units, nu + n_rb, s));
    TRY(to_host(&n_bslots, ns + n_rb, s));
    TRY(to_host(&n_bsplit, sp + n_rb, s));
    uint64_t* uk = ar.get<uint64_t>(n_units);
    uint64_t* uk2 = ar.get<uint64_t>(n_units);
    int64_t* uv = ar.get<int64_t>(n_units);
    int64_t* uv2 = ar.get<int64_t>(n_units);
    int32_t* pb = ar.get<int32_t>(n_units);
    int64_t* p0 = ar.get<int64_t>(n_units);
    int64_t* p1 = ar.get<int64_t>(n_units);
    int32_t* ps = ar.get<int32_t>(n_units);
    NEED(ps);
    if (n_bsplit) {
      TRY(own(&d.bcsr.split_block, n_bsplit, bytes));
      TRY(own(&d.bcsr.split_slot_ptr, n_bsplit + 1, bytes));
    }
    unit_emit_k<<<grid_for(n_rb), kThreads, 0, s>>>(d.bcsr.rb_ptr, n_rb, nu, ns, sp, n_bslots, n_units, uk, uv, pb,
                                                    p0, p1, ps, d.bcsr.split_block, d.bcsr.split_slot_ptr, n_bsplit);
    TRY(cudaGetLastError());
    TRY(radix_sort<int64_t>(&uk, &uv, &uk2, &uv2, n_units, bit_width((uint64_t)kBcsrSplitTiles - 1), ar, s));
    TRY(own(&d.bcsr.unit_block, n_units, bytes));
    TRY(own(&d.bcsr.unit_t0, n_units, bytes));
    TRY(own(&d.bcsr.unit_t1, n_units, bytes));
    TRY(own(&d.bcsr.unit_slot, n_units, bytes));
    unit_gather_k<<<grid_for(n_units), kThreads, 0, s>>>(uv, n_units, pb, p0, p1, ps, d.bcsr.unit_block,
                                                         d.bcsr.unit_t0, d.bcsr.unit_t1, d.bcsr.unit_slot);
    TRY(cudaGetLastError());
    d.bcsr.n_units = n_units;
    d.bcsr.n_split = n_bsplit;
    d.bcsr.n_slots = n_bslots;
    if (n_bslots) {
      const int acc_bytes = p->dtype == LOOPS_F64 ? 8 : 4;
      TRY(own((uint8_t**)&d.bcsr.scratch, n_bslots * br * std::max<int64_t>(N, 1) * acc_bytes, bytes));
    }
  }

  // ---- 5. CSR part: canonical positions of each set's entries, then the work items
  int32_t* f0 = ar.get<int32_t>(nnz);
  int32_t* f1 = ar.get<int32_t>(nnz);
  int64_t* c0 = ar.get<int64_t>(nnz + 1);
  int64_t* c1 = ar.get<int64_t>(nnz + 1);
  NEED(c1);
  if (nnz) {
    class_flags_k<<<grid_for(nnz), kThreads, 0, s>>>(cls, nnz, f0, f1);
    TRY(cudaGetLastError());
  }
  TRY(excl_scan<int32_t>(f0, c0, nnz, true, ar, s));
  TRY(excl_scan<int32_t>(f1, c1, nnz, true, ar, s));
  int64_t nnz0 = 0, nnz1 = 0;
  TRY(to_host(&nnz0, c0 + nnz, s));
  TRY(to_host(&nnz1, c1 + nnz, s));
  int64_t* src0 = ar.get<int64_t>(nnz0);
  int64_t* src1 = ar.get<int64_t>(nnz1);
  NEED(src1);
  if (nnz) {
    canon_src_k<<<grid_for(nnz), kThreads, 0, s>>>(cls, c0, nnz, 0, nnz0, src0);
    canon_src_k<<<grid_for(nnz), kThreads, 0, s>>>(cls, c1, nnz, 1, nnz1, src1);
    TRY(cudaGetLastError());
  }
  int64_t* csr_src = nullptr;
  int64_t n_csr_src = 0;
  loops_status st;
  if ((st = build_csr_set(p, A, remap, 0, cls, is_bcsr, rowlen1, c0, src0, nnz0, N, tiny, n_sub,
                          want_maps ? &csr_src : nullptr, &n_csr_src, ar, s)))
    return st;
  if ((st = build_csr_set(p, A, remap, 1, cls, is_bcsr, rowlen1, c1, src1, nnz1, N, tiny, n_sub, nullptr, nullptr,
                          ar, s)))
    return st;
  // canonical CSR rows: every row of a CSR block, plus the rows with moved entries. Row blocks
  // hold B_r rows except possibly the last one.
  {
    uint8_t last_in = 0;
    if (n_rb) TRY(to_host(&last_in, is_bcsr + (nb - 1), s));
    const int64_t n_rows_bcsr = n_rb * br - (last_in ? nb * br - n : 0);
    const CsrDev& acc = p->dev.csr_acc;
    const int64_t n_rows1 = acc.n_items - acc.n_slots + acc.n_split;  // unsplit rows + split rows
    p->n_csr_rows = (n - n_rows_bcsr) + n_rows1;
  }
  p->nnz_csr = nnz0 + nnz1;
  p->nnz_bcsr = nnz - nnz0 - nnz1;

  // ---- 6. value maps
  if (want_maps) {
    ValueMapDev& m = p->vmap;
    free_value_maps(m);
    m.n_csr = n_csr_src;
    m.n_slots = n_fslots;
    if (n_csr_src) {
      TRY(own(&m.csr_src, n_csr_src, m.bytes));
      TRY(cudaMemcpyAsync(m.csr_src, csr_src, (size_t)n_csr_src * 8, cudaMemcpyDeviceToDevice, s));
    }
    if (n_fslots) {
      int64_t n_src = 0;
      TRY(to_host(&n_src, slot_ptr + n_fslots, s));
      TRY(own(&m.bcsr_ptr, n_fslots + 1, m.bytes));
      TRY(cudaMemcpyAsync(m.bcsr_ptr, slot_ptr, (size_t)(n_fslots + 1) * 8, cudaMemcpyDeviceToDevice, s));
      if (n_src) {
        TRY(own(&m.bcsr_src, n_src, m.bytes));
        TRY(cudaMemcpyAsync(m.bcsr_src, slot_src, (size_t)n_src * 8, cudaMemcpyDeviceToDevice, s));
      }
    }
    p->has_vmap = true;
  }
  unsigned long long sub = 0;
  TRY(to_host(&sub, n_sub, s));
  p->n_subnormal = (int64_t)sub;
  return check_build_err(s, what);
}

// SDDMM items of A's own pattern (rows cut at L entries, stably ordered by decreasing length)
// and the input-order column array.
loops_status build_sddmm_device(loops_plan_s* p, const DevCsrIn& A, cudaStream_t s) {
  const char* what = "device plan build (SDDMM items)";
  Arena ar;
  ar.s = s;
  const int64_t n = A.n_rows, L = std::max<int64_t>(p->split_len, 1);
  int64_t* ni = ar.get<int64_t>(n + 1);
  NEED(ni);
  TRY(reset_build_err(s));
  if (n) sddmm_count_k<<<grid_for(n), kThreads, 0, s>>>(A.rp, n, L, ni);
  TRY(cudaGetLastError());
  TRY(excl_scan<int64_t>(ni, ni, n, true, ar, s));
  int64_t n_it = 0;
  TRY(to_host(&n_it, ni + n, s));
  p->sddmm.n_items = n_it;
  if (A.nnz) {
    TRY(dev_malloc((void**)&p->sddmm.col, (size_t)A.nnz * 4));
    p->other_bytes += A.nnz * 4;
    TRY(cudaMemcpyAsync(p->sddmm.col, A.ci, (size_t)A.nnz * 4, cudaMemcpyDeviceToDevice, s));
  }
  if (!n_it) return LOOPS_OK;
  uint64_t* k1 = ar.get<uint64_t>(n_it);
  uint64_t* k2 = ar.get<uint64_t>(n_it);
  int64_t* v1 = ar.get<int64_t>(n_it);
  int64_t* v2 = ar.get<int64_t>(n_it);
  int32_t* pr = ar.get<int32_t>(n_it);
  int64_t* pb = ar.get<int64_t>(n_it);
  int64_t* pe = ar.get<int64_t>(n_it);
  NEED(pe);
  sddmm_emit_k<<<grid_for(n), kThreads, 0, s>>>(A.rp, n, L, ni, n_it, k1, v1, pr, pb, pe);
  TRY(cudaGetLastError());
  TRY(radix_sort<int64_t>(&k1, &v1, &k2, &v2, n_it, bit_width((uint64_t)L), ar, s));
  TRY(dev_malloc((void**)&p->sddmm.item_row, (size_t)n_it * 4));
  TRY(dev_malloc((void**)&p->sddmm.item_beg, (size_t)n_it * 8));
  TRY(dev_malloc((void**)&p->sddmm.item_end, (size_t)n_it * 8));
  p->other_bytes += n_it * 20;
  sddmm_gather_k<<<grid_for(n_it), kThreads, 0, s>>>(v1, n_it, pr, pb, pe, p->sddmm.item_row, p->sddmm.item_beg,
                                                     p->sddmm.item_end);
  TRY(cudaGetLastError());
  return check_build_err(s, what);
}

// A^T in CSR on the device: entries stably sorted by column (so each column keeps A's row
// order); perm[e] is the input entry of A^T's entry e. Arrays are allocated here (cudaMalloc)
// and released by the caller.
loops_status transpose_device(const DevCsrIn& A, int64_t** t_rp, int32_t** t_ci, double** t_vals, int64_t** perm,
                              cudaStream_t s) {
  const char* what = "device transpose";
  Arena ar;
  ar.s = s;
  const int64_t nnz = A.nnz, m = A.n_cols;
  *t_rp = nullptr;
  *t_ci = nullptr;
  *t_vals = nullptr;
  *perm = nullptr;
  TRY(dev_malloc((void**)t_rp, (size_t)(m + 1) * 8));
  TRY(dev_malloc((void**)t_ci, (size_t)std::max<int64_t>(nnz, 1) * 4));
  TRY(dev_malloc((void**)t_vals, (size_t)std::max<int64_t>(nnz, 1) * 8));
  int64_t* cnt = ar.get<int64_t>(m + 1);
  int32_t* erow = ar.get<int32_t>(nnz);
  uint64_t* k1 = ar.get<uint64_t>(nnz);
  uint64_t* k2 = ar.get<uint64_t>(nnz);
  int64_t* v1 = ar.get<int64_t>(nnz);
  int64_t* v2 = ar.get<int64_t>(nnz);
  NEED(v2);
  TRY(cudaMemsetAsync(cnt, 0, (size_t)(m + 1) * 8, s));
  TRY(reset_build_err(s));
  if (nnz) {
    entry_rows_k<<<grid_for(nnz), kThreads, 0, s>>>(A.rp, A.n_rows, nnz, erow);
    col_keys_k<<<grid_for(nnz), kThreads, 0, s>>>(A.ci, nnz, k1, v1, cnt);
    TRY(cudaGetLastError());
    TRY(radix_sort<int64_t>(&k1, &v1, &k2, &v2, nnz, bit_width(m > 1 ? (uint64_t)(m - 1) : 1), ar, s));
  }
  TRY(excl_scan<int64_t>(cnt, *t_rp, m, true, ar, s));
  TRY(dev_malloc((void**)perm, (size_t)std::max<int64_t>(nnz, 1) * 8));
  if (nnz) {
    TRY(cudaMemcpyAsync(*perm, v1, (size_t)nnz * 8, cudaMemcpyDeviceToDevice, s));
    transpose_fill_k<<<grid_for(nnz), kThreads, 0, s>>>(v1, erow, A.vals, A.vals_f32, nnz, *t_ci, *t_vals);
    TRY(cudaGetLastError());
  }
  return check_build_err(s, what);
}

loops_status download_mirrors(loops_plan_s* p) {
  const char* what = "device plan build (host mirrors)";
  for (CsrDev* cd : {&p->dev.csr, &p->dev.csr_acc}) {
    cd->h_item_ptr.assign((size_t)(cd->n_items ? cd->n_items + 1 : 0), 0);
    if (cd->n_items)
      TRY(cudaMemcpy(cd->h_item_ptr.data(), cd->item_ptr, (size_t)(cd->n_items + 1) * 8, cudaMemcpyDeviceToHost));
  }
  BcsrDev& bd = p->dev.bcsr;
  bd.h_unit_tiles.assign((size_t)bd.n_units, 0);
  if (bd.n_units) {
    std::vector<int64_t> u0((size_t)bd.n_units), u1((size_t)bd.n_units);
    TRY(cudaMemcpy(u0.data(), bd.unit_t0, (size_t)bd.n_units * 8, cudaMemcpyDeviceToHost));
    TRY(cudaMemcpy(u1.data(), bd.unit_t1, (size_t)bd.n_units * 8, cudaMemcpyDeviceToHost));
    for (size_t i = 0; i < u0.size(); ++i) bd.h_unit_tiles[i] = u1[i] - u0[i];
  }
  return LOOPS_OK;
}

#undef TRY
#undef NEED

}  // namespace loops
