// Batched hybrid SpMM: many sparse matrices of uneven size and N in a few persistent launches.
//
// Each matrix has its own plan (partition and device layout as for a single SpMM). A static
// task list covers every matrix's CSR items (in groups of consecutive items) and BCSR work
// units. Tasks fall into classes by kind and by the lane-group width their N needs; each class
// is a contiguous run of the list, ordered matrix by matrix, and runs as one persistent kernel
// specialised for it (its own register budget, compile-time group width). The warps of a
// class kernel claim its tasks in list order from a counter, so at any time they work on one
// or a few matrices, whose B operands stay in L2 while their rows gather from them. Every
// task writes its own outputs (C rows, or partial-sum slots), so the result does not depend on
// which warp runs which task.
//   CSR class   (kind 0, <G, VPL>): a group of G lanes per item, each lane VPL 16-byte column
//               vectors of the row; 32 / G items at a time per warp.
//   FFMA class  (kind 1, <B_r, G>): F32 BCSR units of one tile height, a group of G lanes per
//               unit (4 columns per lane), register-blocked outer products with several
//               tiles' loads in flight.
//   HMMA class  (kind 2): one F16/BF16 BCSR unit per warp, in 64-column chunks; the 16 B-row
//               pieces of each K-group are copied into the warp's shared-memory ring by
//               cp.async (two groups in flight while one is multiplied) and fed to mma.sync
//               m16n8k16.
// Rows split in segments and blocks cut into units get small follow-up launches that add
// their partial sums in a fixed order.
#include <algorithm>
#include <type_traits>

#include "device_common.cuh"
#include "loops_internal.h"

// Tuning knobs (compile time):
// * resident blocks per SM the class kernels must allow (their register caps): CSR FP32, CSR
//   16-bit, FFMA B_r 8, FFMA B_r 16 (its 64 accumulators per lane spill at 3 blocks);
// * B-row loads in flight per lane in CSR items, FP32 and 16-bit (powers of two);
// * tiles in flight in FFMA units, B_r 8 and B_r 16;
// * cp.async stages of the HMMA units.
#ifndef LOOPS_BATCHED_CSR_MIN_BLOCKS
#define LOOPS_BATCHED_CSR_MIN_BLOCKS 3
#endif
#ifndef LOOPS_BATCHED_CSR16_MIN_BLOCKS
#define LOOPS_BATCHED_CSR16_MIN_BLOCKS 4
#endif
#ifndef LOOPS_BATCHED_CSR_LOADS
#define LOOPS_BATCHED_CSR_LOADS 8
#endif
#ifndef LOOPS_BATCHED_CSR16_LOADS
#define LOOPS_BATCHED_CSR16_LOADS 4
#endif
static_assert(LOOPS_BATCHED_CSR16_LOADS >= 1 && (LOOPS_BATCHED_CSR16_LOADS & (LOOPS_BATCHED_CSR16_LOADS - 1)) == 0,
              "16-bit CSR loads in flight must be a power of two");
static_assert(LOOPS_BATCHED_CSR_LOADS >= 2 && (LOOPS_BATCHED_CSR_LOADS & (LOOPS_BATCHED_CSR_LOADS - 1)) == 0,
              "CSR loads in flight must be a power of two: the load batches tile a chunk exactly");
#ifndef LOOPS_BATCHED_FFMA_TILES
#define LOOPS_BATCHED_FFMA_TILES 4
#endif
#ifndef LOOPS_BATCHED_HMMA_STAGES
#define LOOPS_BATCHED_HMMA_STAGES 3
#endif
#ifndef LOOPS_BATCHED_FFMA_MIN_BLOCKS
#define LOOPS_BATCHED_FFMA_MIN_BLOCKS 3
#endif
#ifndef LOOPS_BATCHED_FFMA16_MIN_BLOCKS
#define LOOPS_BATCHED_FFMA16_MIN_BLOCKS 2
#endif
#ifndef LOOPS_BATCHED_FFMA16_TILES
#define LOOPS_BATCHED_FFMA16_TILES 2
#endif

namespace loops {

namespace {

__device__ __forceinline__ void mma16816_b(float (&d)[4], const uint4& a, uint32_t b0, uint32_t b1, bool bf16) {
  if (bf16)
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a.x), "r"(a.y), "r"(a.z), "r"(a.w), "r"(b0), "r"(b1));
  else
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a.x), "r"(a.y), "r"(a.z), "r"(a.w), "r"(b0), "r"(b1));
}

// 16-byte global -> shared copy that holds no registers while in flight (the asynchronous
// copy, completed by commit groups). src_bytes 0 fills the 16 bytes with zeros and reads
// nothing.
__device__ __forceinline__ void cp_async16(void* dst, const void* src, int src_bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;"
               ::"r"(smem_addr(dst)), "l"(src), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

template <class Tr>
__device__ __forceinline__ float col_mult(const BatchDesc& d, int64_t n) {
  if (!Tr::kScaled) return 1.f;
  return d.col_scale ? d.col_scale[n] * d.inv_scale : d.inv_scale;
}

// Next task of a warp: the next unclaimed one of the class's run of the list (the counter is
// zeroed before the launch).
__device__ __forceinline__ int64_t claim(unsigned long long* counter, int lane) {
  unsigned long long t = 0;
  if (lane == 0) t = atomicAdd(counter, 1ull);
  return (int64_t)__shfl_sync(0xffffffffu, t, 0);
}

// ------------------------------------------------------------------ CSR items
// One CSR item (a row, or a segment of a split row) for a group of G lanes; lane `sub` owns
// the 16-byte column vectors p * G + sub (p < VPL). Entries are read R per lane at a time
// (chunks of G * R entries, broadcast by shuffles), and the next chunk's entries are loaded
// while the current chunk's B rows are in flight.
template <class Tr, int G, int VPL>
__device__ __forceinline__ void csr_item(const BatchDesc& d, int64_t item, int sub, unsigned gmask) {
  using TB = typename Tr::TB;
  using TAcc = typename Tr::TAcc;
  using TC = typename Tr::TC;
  using TV = typename Tr::TV;
  constexpr int VE = Tr::kVE;
  constexpr int R = G >= 8 ? 1 : (G >= 2 ? 8 / G : 4);  // chunks of at least 4-8 entries
  constexpr int CH = G * R;                             // entries per chunk
  // B loads in flight per lane (FP32 and 16-bit rows, each a power of two), half that with two
  // vectors per lane
  constexpr int UMAX = (VE == 8 ? LOOPS_BATCHED_CSR16_LOADS : LOOPS_BATCHED_CSR_LOADS) / VPL;
  constexpr int U = UMAX < CH ? UMAX : CH;
  static_assert(U >= 1 && CH % U == 0, "load batches must tile the chunk");
  // 32-bit indices inside the item and inside B (the batched call keeps every B below 2^31
  // elements), 64-bit pointers only for the bases: fewer registers per lane
  const int64_t beg = d.item_ptr[item];
  const int32_t len = (int32_t)(d.item_ptr[item + 1] - beg);
  const int32_t row = d.item_row[item];
  const int32_t* __restrict__ colp = d.col + beg;
  const TB* __restrict__ valp = reinterpret_cast<const TB*>(d.val) + beg;
  const uint32_t ldb = (uint32_t)d.ldb;
  const int32_t N = (int32_t)d.N;
  const TB* bl[VPL];
  bool colok[VPL];
#pragma unroll
  for (int p = 0; p < VPL; ++p) {
    const int32_t off = (p * G + sub) * VE;
    colok[p] = off < N;
    bl[p] = reinterpret_cast<const TB*>(d.B) + off;
  }
  TAcc acc[VPL][VE];
#pragma unroll
  for (int p = 0; p < VPL; ++p)
#pragma unroll
    for (int e = 0; e < VE; ++e) acc[p][e] = TAcc(0);

  auto fetch = [&](int32_t k0, int32_t (&c)[R], TV (&v)[R]) {
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int32_t k = k0 + r * G + sub;
      c[r] = 0;
      v[r] = TV(0);
      if (k < len) {
        c[r] = __ldg(colp + k);
        v[r] = Tr::load_v(valp + k);
      }
    }
  };
  int32_t c[R];
  TV v[R];
  fetch(0, c, v);
  for (int32_t k0 = 0; k0 < len; k0 += CH) {
    int32_t cn[R];
    TV vn[R];
    fetch(k0 + CH, cn, vn);                             // next chunk's entries, in flight now
    if (k0 + CH <= len) {                               // full chunk: batches of U loads, then FMAs
#pragma unroll
      for (int e0 = 0; e0 < CH; e0 += U) {
        uint4 bv[U][VPL];
        TV av[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int e = e0 + u;
          const uint32_t cj = (uint32_t)__shfl_sync(gmask, c[e / G], e % G, G);
          av[u] = __shfl_sync(gmask, v[e / G], e % G, G);
#pragma unroll
          for (int p = 0; p < VPL; ++p) bv[u][p] = colok[p] ? ldg16(bl[p] + cj * ldb) : make_uint4(0, 0, 0, 0);
        }
#pragma unroll
        for (int u = 0; u < U; ++u)
#pragma unroll
          for (int p = 0; p < VPL; ++p) fma_vec<Tr>(acc[p], bv[u][p], av[u]);
      }
    } else {                                            // the last, partial chunk
      // the same batches under predicates: entries past the row's end load nothing and carry
      // zero values, so they add exact zeros, and the live loads of a batch stay in flight
      // together instead of one entry at a time
      const int cnt = len - k0;
#pragma unroll
      for (int e0 = 0; e0 < CH; e0 += U) {
        if (e0 < cnt) {
          uint4 bv[U][VPL];
          TV av[U];
#pragma unroll
          for (int u = 0; u < U; ++u) {
            const int e = e0 + u;
            const uint32_t cj = (uint32_t)__shfl_sync(gmask, c[e / G], e % G, G);
            av[u] = __shfl_sync(gmask, v[e / G], e % G, G);
#pragma unroll
            for (int p = 0; p < VPL; ++p) bv[u][p] = ldg16_if(colok[p] && e < cnt, bl[p] + cj * ldb);
          }
#pragma unroll
          for (int u = 0; u < U; ++u)
#pragma unroll
            for (int p = 0; p < VPL; ++p) fma_vec<Tr>(acc[p], bv[u][p], av[u]);
        }
      }
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
      c[r] = cn[r];
      v[r] = vn[r];
    }
  }
  if (row >= 0) {
    TC* crow = reinterpret_cast<TC*>(d.C) + (int64_t)row * d.ldc;
#pragma unroll
    for (int p = 0; p < VPL; ++p) {
      if (!colok[p]) continue;
      const int32_t off = (p * G + sub) * VE;
      TC o[VE];
#pragma unroll
      for (int e = 0; e < VE; ++e) o[e] = Tr::kScaled ? (TC)(acc[p][e] * col_mult<Tr>(d, off + e)) : (TC)acc[p][e];
#pragma unroll
      for (int q = 0; q < (int)(VE * sizeof(TC) / 16); ++q)
        *reinterpret_cast<uint4*>(crow + off + q * (16 / sizeof(TC))) =
            *reinterpret_cast<const uint4*>(&o[q * (16 / sizeof(TC))]);
    }
  } else {
    TAcc* srow = reinterpret_cast<TAcc*>(d.scratch) + (int64_t)(-1 - row) * d.N;
#pragma unroll
    for (int p = 0; p < VPL; ++p) {
      if (!colok[p]) continue;
      const int32_t off = (p * G + sub) * VE;
#pragma unroll
      for (int e = 0; e < VE; ++e) srow[off + e] = acc[p][e];
    }
  }
}

template <class Tr>
constexpr int csr_min_blocks() {
  return Tr::kVE == 8 ? LOOPS_BATCHED_CSR16_MIN_BLOCKS : LOOPS_BATCHED_CSR_MIN_BLOCKS;
}

template <class Tr, int G, int VPL>
__global__ void __launch_bounds__(256, csr_min_blocks<Tr>()) batched_csr(const BatchDesc* __restrict__ descs,
                                                      const BatchTask* __restrict__ tasks, int64_t n_tasks,
                                                      unsigned long long* counter) {
  const int lane = threadIdx.x & 31;
  const int grp = lane / G, sub = lane % G;
  const unsigned gmask = G == 32 ? 0xffffffffu : (((1u << G) - 1u) << (grp * G));
  for (int64_t t = claim(counter, lane); t < n_tasks; t = claim(counter, lane)) {
    const BatchTask task = tasks[t];
    const BatchDesc& d = descs[task.m];
    for (int32_t i = grp; i < task.count; i += 32 / G) csr_item<Tr, G, VPL>(d, task.first + i, sub, gmask);
  }
}

// ------------------------------------------------------------------ F32 BCSR units
// One F32 BCSR unit (B_r rows, tile-major values) for a group of G lanes, 4 columns per lane;
// T tiles' B vectors and A values are loaded before their FMAs.
template <int BR, int G>
__device__ __forceinline__ void ffma_unit(const BatchDesc& d, int64_t u, int sub) {
  constexpr int T = BR == 8 ? LOOPS_BATCHED_FFMA_TILES : LOOPS_BATCHED_FFMA16_TILES;
  const int32_t b = d.unit_block[u];
  const int64_t rb = d.rb_id[b];
  const int64_t t0 = d.unit_t0[u], t1 = d.unit_t1[u];
  const int32_t slot = d.unit_slot[u];
  const float* __restrict__ Av = reinterpret_cast<const float*>(d.tile_val);
  const float* __restrict__ Bp = reinterpret_cast<const float*>(d.B);
  const int64_t n = (int64_t)sub * 4;
  const bool colok = n < d.N;
  float acc[BR][4];
#pragma unroll
  for (int r = 0; r < BR; ++r)
#pragma unroll
    for (int e = 0; e < 4; ++e) acc[r][e] = 0.f;
  auto tile_fma = [&](const uint4& v, const uint4 (&w)[BR / 4]) {
    const float bv[4] = {__uint_as_float(v.x), __uint_as_float(v.y), __uint_as_float(v.z), __uint_as_float(v.w)};
#pragma unroll
    for (int r4 = 0; r4 < BR / 4; ++r4) {
      const float a4[4] = {__uint_as_float(w[r4].x), __uint_as_float(w[r4].y), __uint_as_float(w[r4].z),
                           __uint_as_float(w[r4].w)};
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int e = 0; e < 4; ++e) acc[r4 * 4 + i][e] = fmaf(a4[i], bv[e], acc[r4 * 4 + i][e]);
    }
  };
  // tile columns of the next batch are read one batch ahead, so each batch's B and A loads
  // issue together without waiting on their column indices (-1 past the unit's end)
  auto load_cols = [&](int64_t base, int32_t (&cc)[T]) {
#pragma unroll
    for (int q = 0; q < T; ++q) cc[q] = base + q < t1 ? __ldg(d.tile_col + base + q) : -1;
  };
  auto load_tile = [&](bool live, int64_t tt, int32_t c, uint4& v, uint4 (&w)[BR / 4]) {
    v = ldg16_if(live && c >= 0 && colok, Bp + (int64_t)c * d.ldb + n);
#pragma unroll
    for (int r4 = 0; r4 < BR / 4; ++r4) w[r4] = ldg16_if(live, Av + tt * BR + r4 * 4);
  };
  int32_t c[T];
  load_cols(t0, c);
  int64_t tt = t0;
  for (; tt + T <= t1; tt += T) {
    int32_t cn[T];
    load_cols(tt + T, cn);
    uint4 v[T];
    uint4 w[T][BR / 4];
#pragma unroll
    for (int q = 0; q < T; ++q) load_tile(true, tt + q, c[q], v[q], w[q]);
#pragma unroll
    for (int q = 0; q < T; ++q) tile_fma(v[q], w[q]);
#pragma unroll
    for (int q = 0; q < T; ++q) c[q] = cn[q];
  }
  if (tt < t1) {  // the last 1 .. T-1 tiles as one batch under predicates (the rest add zeros)
    uint4 v[T];
    uint4 w[T][BR / 4];
#pragma unroll
    for (int q = 0; q < T; ++q) load_tile(tt + q < t1, tt + q, c[q], v[q], w[q]);
#pragma unroll
    for (int q = 0; q < T; ++q) tile_fma(v[q], w[q]);
  }
  if (!colok) return;
  if (slot >= 0) {  // unit of a split block: partial sums
    float* P = reinterpret_cast<float*>(d.bscratch) + (int64_t)slot * BR * d.N;
#pragma unroll
    for (int r = 0; r < BR; ++r)
      *reinterpret_cast<float4*>(P + r * d.N + n) = make_float4(acc[r][0], acc[r][1], acc[r][2], acc[r][3]);
    return;
  }
  float* C = reinterpret_cast<float*>(d.C);
#pragma unroll
  for (int r = 0; r < BR; ++r) {
    const int64_t row = rb * BR + r;
    if (row >= d.n_rows) break;
    *reinterpret_cast<float4*>(C + row * d.ldc + n) = make_float4(acc[r][0], acc[r][1], acc[r][2], acc[r][3]);
  }
}

template <int BR, int G>
__global__ void __launch_bounds__(256, BR == 8 ? LOOPS_BATCHED_FFMA_MIN_BLOCKS : LOOPS_BATCHED_FFMA16_MIN_BLOCKS)
    batched_ffma(const BatchDesc* __restrict__ descs,
                                                       const BatchTask* __restrict__ tasks, int64_t n_tasks,
                                                       unsigned long long* counter) {
  const int lane = threadIdx.x & 31;
  const int grp = lane / G, sub = lane % G;
  for (int64_t t = claim(counter, lane); t < n_tasks; t = claim(counter, lane)) {
    const BatchTask task = tasks[t];
    const BatchDesc& d = descs[task.m];
    for (int32_t i = grp; i < task.count; i += 32 / G) ffma_unit<BR, G>(d, task.first + i, sub);
  }
}

// ------------------------------------------------------------------ F16/BF16 BCSR units
// One F16/BF16 BCSR unit for the whole warp, in column chunks of up to 64. The 16 gathered
// B-row pieces of each K-group go into the warp's ring of kHStages shared-memory stages by
// cp.async (padding tiles, column -1, are zero-filled without a read); kHStages - 1 groups
// are in flight while the oldest one is multiplied. Row stride 72 elements: conflict-free
// ldmatrix.
constexpr int kHChunk = 64;
constexpr int kHStride = kHChunk + 8;
constexpr int kHStages = LOOPS_BATCHED_HMMA_STAGES;
constexpr int kHStageElems = 16 * kHStride;
constexpr int kHmmaSmemPerWarp = kHStages * kHStageElems * 2;  // bytes

template <class T>
__device__ __forceinline__ void hmma_unit(const BatchDesc& d, int64_t u, T* sB, int lane) {
  constexpr bool kBF16 = std::is_same<T, __nv_bfloat16>::value;
  const int32_t b = d.unit_block[u];
  const int64_t rb = d.rb_id[b];
  const int64_t t0 = d.unit_t0[u];
  const int n_groups = (int)((d.unit_t1[u] - t0) / 16);
  const int32_t slot = d.unit_slot[u];
  const int N = (int)d.N;
  const T* Bp = reinterpret_cast<const T*>(d.B);
  const uint4* Af = reinterpret_cast<const uint4*>(d.tile_val) + (t0 / 16) * 32;
  const int q = lane >> 2, t = lane & 3;
  for (int c0 = 0; c0 < N; c0 += kHChunk) {
    const int NC = min(kHChunk, N - c0);   // columns of this chunk (a multiple of 8)
    const int NF = NC / 8;
    // stage of group g: this lane copies the vectors i = lane, lane + 32, ... of its 16 x NF
    // piece (column -1: zero-filled, nothing read)
    auto issue = [&](int g) {
      T* st = sB + (g % kHStages) * kHStageElems;
      for (int i = lane; i < 16 * NF; i += 32) {
        const int k = i / NF, qv = i - k * NF;
        const int32_t c = __ldg(d.tile_col + t0 + g * 16 + k);
        const T* src = c >= 0 ? Bp + (int64_t)c * d.ldb + c0 + qv * 8 : Bp;
        cp_async16(st + k * kHStride + qv * 8, src, c >= 0 ? 16 : 0);
      }
    };
    float acc[8][4];
#pragma unroll
    for (int f = 0; f < 8; ++f)
#pragma unroll
      for (int i = 0; i < 4; ++i) acc[f][i] = 0.f;
    __syncwarp();                           // every lane is done with the ring's last contents
#pragma unroll
    for (int g = 0; g < kHStages - 1; ++g) {
      if (g < n_groups) issue(g);
      cp_async_commit();
    }
    for (int g = 0; g < n_groups; ++g) {
      if (g + kHStages - 1 < n_groups) issue(g + kHStages - 1);
      cp_async_commit();
      cp_async_wait<kHStages - 1>();        // this lane's copies of group g have landed
      __syncwarp();                         // ... and every lane's
      const uint4 af = __ldg(Af + (int64_t)g * 32 + lane);
      const T* st = sB + (g % kHStages) * kHStageElems;
      const int mi = lane >> 3, r = lane & 7;
#pragma unroll
      for (int f = 0; f < 8; f += 2) {
        if (f >= NF) break;
        if (f + 1 < NF) {
          const uint32_t addr = smem_addr(st + (r + 8 * (mi & 1)) * kHStride + f * 8 + 8 * (mi >> 1));
          uint32_t b0, b1, b2, b3;
          asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];"
                       : "=r"(b0), "=r"(b1), "=r"(b2), "=r"(b3) : "r"(addr));
          mma16816_b(acc[f], af, b0, b1, kBF16);
          mma16816_b(acc[f + 1], af, b2, b3, kBF16);
        } else {
          const uint32_t addr = smem_addr(st + (r + 8 * (mi & 1)) * kHStride + f * 8);
          uint32_t b0, b1;
          asm volatile("ldmatrix.sync.aligned.m8n8.x2.trans.shared.b16 {%0,%1}, [%2];"
                       : "=r"(b0), "=r"(b1) : "r"(addr));
          mma16816_b(acc[f], af, b0, b1, kBF16);
        }
      }
      __syncwarp();                         // stage g % kHStages may be refilled next
    }
    cp_async_wait<0>();
    if (slot >= 0) {  // unit of a split block: unscaled partial sums
      float* P = reinterpret_cast<float*>(d.bscratch) + (int64_t)slot * 16 * d.N;
#pragma unroll
      for (int f = 0; f < 8; ++f) {
        if (f >= NF) break;
        const int64_t n = c0 + f * 8 + 2 * t;
#pragma unroll
        for (int h = 0; h < 2; ++h)
          *reinterpret_cast<float2*>(P + (int64_t)(q + 8 * h) * d.N + n) = make_float2(acc[f][2 * h], acc[f][2 * h + 1]);
      }
      continue;
    }
    float* C = reinterpret_cast<float*>(d.C);
#pragma unroll
    for (int f = 0; f < 8; ++f) {
      if (f >= NF) break;
      const int64_t n = c0 + f * 8 + 2 * t;
      float s0 = d.inv_scale, s1 = d.inv_scale;
      if (d.col_scale) {
        s0 *= d.col_scale[n];
        s1 *= d.col_scale[n + 1];
      }
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int64_t row = rb * 16 + q + 8 * h;
        if (row < d.n_rows)
          *reinterpret_cast<float2*>(C + row * d.ldc + n) = make_float2(acc[f][2 * h] * s0, acc[f][2 * h + 1] * s1);
      }
    }
  }
}

template <class T>
__global__ void __launch_bounds__(256, 3) batched_hmma(const BatchDesc* __restrict__ descs,
                                                       const BatchTask* __restrict__ tasks, int64_t n_tasks,
                                                       unsigned long long* counter) {
  extern __shared__ __align__(128) unsigned char smem[];
  const int lane = threadIdx.x & 31;
  T* sB = reinterpret_cast<T*>(smem + (threadIdx.x >> 5) * kHmmaSmemPerWarp);
  for (int64_t t = claim(counter, lane); t < n_tasks; t = claim(counter, lane)) {
    const BatchTask task = tasks[t];
    hmma_unit<T>(descs[task.m], task.first, sB, lane);
  }
}

// ------------------------------------------------------------------ partial sums
// Sum of split-row partials: one block per (matrix, split row).
template <class Tr>
__global__ void __launch_bounds__(128) batched_split_reduce(const BatchDesc* __restrict__ descs,
                                                            const int2* __restrict__ splits) {
  using TAcc = typename Tr::TAcc;
  using TC = typename Tr::TC;
  const int2 sp = splits[blockIdx.x];
  const BatchDesc& d = descs[sp.x];
  const int32_t row = d.split_row[sp.y];
  const int32_t s0 = d.split_slot_ptr[sp.y], s1 = d.split_slot_ptr[sp.y + 1];
  const TAcc* sc = reinterpret_cast<const TAcc*>(d.scratch);
  for (int64_t n = threadIdx.x; n < d.N; n += blockDim.x) {
    TAcc acc = TAcc(0);
    for (int32_t q = s0; q < s1; ++q) acc += sc[(int64_t)q * d.N + n];
    reinterpret_cast<TC*>(d.C)[(int64_t)row * d.ldc + n] = Tr::kScaled ? (TC)(acc * col_mult<Tr>(d, n)) : (TC)acc;
  }
}

// BCSR blocks cut into units: C rows = scale * sum of the units' partials, in slot order.
template <class Tr>
__global__ void __launch_bounds__(256) batched_bsplit_reduce(const BatchDesc* __restrict__ descs,
                                                             const int2* __restrict__ bsplits) {
  const int2 sp = bsplits[blockIdx.x];
  const BatchDesc& d = descs[sp.x];
  const int32_t b = d.bsplit_block[sp.y];
  const int64_t rb = d.rb_id[b];
  const int32_t s0 = d.bsplit_slot_ptr[sp.y], s1 = d.bsplit_slot_ptr[sp.y + 1];
  const float* P = reinterpret_cast<const float*>(d.bscratch);
  const int64_t total = (int64_t)d.br * d.N;
  for (int64_t i = threadIdx.x; i < total; i += blockDim.x) {
    const int64_t r = i / d.N, n = i - r * d.N;
    const int64_t row = rb * d.br + r;
    if (row >= d.n_rows) continue;
    float acc = 0.f;
    for (int32_t q = s0; q < s1; ++q) acc += P[((int64_t)q * d.br + r) * d.N + n];
    reinterpret_cast<float*>(d.C)[row * d.ldc + n] = Tr::kScaled ? acc * col_mult<Tr>(d, n) : acc;
  }
}

// ------------------------------------------------------------------ class dispatch
using ClassKernel = void (*)(const BatchDesc*, const BatchTask*, int64_t, unsigned long long*);

template <class Tr>
ClassKernel csr_kernel(int G, int VPL) {
  // 16-bit rows (N <= 128) take one vector per lane: at most 16 lanes, never two vectors
  if constexpr (Tr::kVE == 8) {
    switch (VPL == 1 ? G : 0) {
      case 1: return batched_csr<Tr, 1, 1>;
      case 2: return batched_csr<Tr, 2, 1>;
      case 4: return batched_csr<Tr, 4, 1>;
      case 8: return batched_csr<Tr, 8, 1>;
      case 16: return batched_csr<Tr, 16, 1>;
      default: return nullptr;
    }
  } else {
    if (VPL == 2) {
      switch (G) {
        case 8: return batched_csr<Tr, 8, 2>;
        case 16: return batched_csr<Tr, 16, 2>;
        default: return nullptr;
      }
    }
    switch (G) {
      case 1: return batched_csr<Tr, 1, 1>;
      case 2: return batched_csr<Tr, 2, 1>;
      case 4: return batched_csr<Tr, 4, 1>;
      case 8: return batched_csr<Tr, 8, 1>;
      case 16: return batched_csr<Tr, 16, 1>;
      case 32: return batched_csr<Tr, 32, 1>;
      default: return nullptr;
    }
  }
}

template <int BR, int G>
ClassKernel ffma_g(int*, int*) {
  return batched_ffma<BR, G>;
}

template <int BR>
ClassKernel ffma_kernel(int G, int* smem, int* threads) {
  switch (G) {
    case 1: return ffma_g<BR, 1>(smem, threads);
    case 2: return ffma_g<BR, 2>(smem, threads);
    case 4: return ffma_g<BR, 4>(smem, threads);
    case 8: return ffma_g<BR, 8>(smem, threads);
    case 16: return ffma_g<BR, 16>(smem, threads);
    case 32: return ffma_g<BR, 32>(smem, threads);
    default: return nullptr;
  }
}

// The kernel of a class, with its dynamic shared memory and threads per block.
ClassKernel class_kernel(loops_dtype dtype, const BatchClass& c, int* smem, int* threads) {
  *smem = 0;
  *threads = 256;
  if (c.kind == 0) {
    switch (dtype) {
      case LOOPS_F32: return csr_kernel<TrF32>(c.G, c.vpl);
      case LOOPS_F16: return csr_kernel<TrF16>(c.G, c.vpl);
      case LOOPS_BF16: return csr_kernel<TrBF16>(c.G, c.vpl);
      default: return nullptr;
    }
  }
  if (c.kind == 1) {
    if (dtype != LOOPS_F32) return nullptr;
    return c.br == 8 ? ffma_kernel<8>(c.G, smem, threads) : ffma_kernel<16>(c.G, smem, threads);
  }
  *smem = kHmmaSmemPerWarp * 8;
  if (dtype == LOOPS_F16) return batched_hmma<__half>;
  if (dtype == LOOPS_BF16) return batched_hmma<__nv_bfloat16>;
  return nullptr;
}

template <class Tr>
cudaError_t launch_reduces(const BatchLaunch& L, cudaStream_t s) {
  if (L.n_splits > 0) {
    batched_split_reduce<Tr><<<(unsigned)L.n_splits, 128, 0, s>>>(L.descs, L.splits);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  if (L.n_bsplits > 0) {
    batched_bsplit_reduce<Tr><<<(unsigned)L.n_bsplits, 256, 0, s>>>(L.descs, L.bsplits);
    return cudaGetLastError();
  }
  return cudaSuccess;
}

}  // namespace

int batched_class_grid(loops_dtype dtype, const BatchClass& c) {
  int smem = 0, threads = 256;
  ClassKernel k = class_kernel(dtype, c, &smem, &threads);
  if (!k) return 0;
  int dev = 0, sms = 152, per_sm = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (smem > 48 * 1024 && cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, threads, smem) != cudaSuccess || per_sm < 1) {
    cudaGetLastError();
    per_sm = 1;
  }
  // no more blocks than the class has tasks for their warps
  const int64_t need = (c.n_tasks + threads / 32 - 1) / (threads / 32);
  return (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)sms * per_sm, need));
}

cudaError_t launch_batched(loops_dtype dtype, const BatchLaunch& L, cudaStream_t s) {
  // timing events become event nodes of the captured graph (external records)
  auto rec = [&](int i) {
    return L.tev ? cudaEventRecordWithFlags(L.tev[i], s, cudaEventRecordExternal) : cudaSuccess;
  };
  cudaError_t e = rec(0);
  if (e == cudaSuccess && L.n_classes > 0)
    e = cudaMemsetAsync(L.counters, 0, sizeof(unsigned long long) * (size_t)L.n_classes, s);
  // with extra branches, the classes are dealt to n_side + 1 parallel branches of the graph:
  // in two halves of the class list (CSR classes, then BCSR classes, each in N order) for two
  // branches, round-robin for more; the branches join before the partial sums
  const int nb = L.n_side > 0 ? std::min(L.n_side + 1, L.n_classes) : 1;
  if (e == cudaSuccess && nb > 1) {
    e = cudaEventRecord(L.fork, s);
    for (int j = 0; j < nb - 1 && e == cudaSuccess; ++j) e = cudaStreamWaitEvent(L.side[j], L.fork, 0);
  }
  int n_csr = 0;
  for (int i = 0; i < L.n_classes; ++i) n_csr += L.classes[i].kind == 0;
  for (int i = 0; i < L.n_classes && e == cudaSuccess; ++i) {
    const BatchClass& c = L.classes[i];
    int smem = 0, threads = 256;
    ClassKernel k = class_kernel(dtype, c, &smem, &threads);
    if (!k) return cudaErrorInvalidValue;
    if (smem > 48 * 1024) {
      e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
      if (e != cudaSuccess) break;
    }
    int branch = 0;
    if (nb == 2) branch = (n_csr > 0 && n_csr < L.n_classes) ? (c.kind > 0) : (i >= L.n_classes / 2);
    else if (nb > 2) branch = i % nb;
    cudaStream_t st = branch == 0 ? s : L.side[branch - 1];
    k<<<c.grid, threads, smem, st>>>(L.descs, L.tasks + c.first, c.n_tasks, L.counters + i);
    e = cudaGetLastError();
  }
  for (int j = 0; j < nb - 1 && e == cudaSuccess; ++j) {
    e = cudaEventRecord(L.join[j], L.side[j]);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, L.join[j], 0);
  }
  if (e == cudaSuccess) e = rec(1);
  if (e == cudaSuccess) e = rec(2);
  if (e != cudaSuccess) return e;
  switch (dtype) {
    case LOOPS_F32: e = launch_reduces<TrF32>(L, s); break;
    case LOOPS_F16: e = launch_reduces<TrF16>(L, s); break;
    case LOOPS_BF16: e = launch_reduces<TrBF16>(L, s); break;
    default: return cudaErrorInvalidValue;
  }
  if (e != cudaSuccess) return e;
  return rec(3);
}

}  // namespace loops
