// Batched hybrid SpMM: many sparse matrices of uneven size and N in one persistent launch.
//
// Each matrix has its own plan (partition and device layout as for a single SpMM). A static
// task list covers every matrix's CSR items (in groups of consecutive items) and BCSR row
// blocks, sorted by estimated cost; warp w of the persistent grid runs tasks w, w + W, ...
// (no atomics, no inter-block waits, so the launch is deterministic and graph-stable).
//   CSR task   (kind 0): items [first, first + count); a group of G = N / VE lanes per item,
//              32 / G items at a time per warp (VE elements of a 16-byte B vector per lane).
//   BCSR task  (kind 1): F32 units [first, first + count) (a unit is a row block, or a K-aligned
//              range of a block with very many tiles), one group of G lanes per unit,
//              register-blocked outer product.
//   BCSR task  (kind 2): one F16/BF16 unit per warp, in 64-column chunks: the 16 B-row pieces
//              of each K-group are staged in the warp's own shared-memory slice and fed to
//              mma.sync m16n8k16.
// Rows split in segments and blocks cut into units get small follow-up launches that add
// their partial sums in a fixed order.
#include <type_traits>

#include "device_common.cuh"
#include "loops_internal.h"

// Minimum resident blocks per SM for the persistent kernel (register cap; tuning knob).
#ifndef LOOPS_BATCHED_MIN_BLOCKS
#define LOOPS_BATCHED_MIN_BLOCKS 3
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

template <class Tr>
__device__ __forceinline__ float col_mult(const BatchDesc& d, int64_t n) {
  if (!Tr::kScaled) return 1.f;
  return d.col_scale ? d.col_scale[n] * d.inv_scale : d.inv_scale;
}

// One CSR item for a group of G lanes (runtime G): row or segment partial.
template <class Tr>
__device__ __forceinline__ void csr_item(const BatchDesc& d, int64_t item, int G, int sub, unsigned gmask) {
  using TB = typename Tr::TB;
  using TAcc = typename Tr::TAcc;
  using TC = typename Tr::TC;
  constexpr int VE = Tr::kVE;
  constexpr int U = 4;
  const int64_t beg = d.item_ptr[item], end = d.item_ptr[item + 1];
  const int32_t row = d.item_row[item];
  const int64_t coff = (int64_t)sub * VE;
  const TB* Bp = reinterpret_cast<const TB*>(d.B);
  const TB* vals = reinterpret_cast<const TB*>(d.val);
  TAcc acc[VE];
#pragma unroll
  for (int e = 0; e < VE; ++e) acc[e] = TAcc(0);
  for (int64_t k0 = beg; k0 < end; k0 += G) {
    const int64_t k = k0 + sub;
    int32_t c = 0;
    TAcc v = TAcc(0);
    if (k < end) {
      c = __ldg(d.col + k);
      v = Tr::to_acc(vals[k]);
    }
    const int cnt = (int)(end - k0 < (int64_t)G ? end - k0 : (int64_t)G);
    int j0 = 0;
    for (; j0 + U <= cnt; j0 += U) {
      uint4 bv[U];
      TAcc av[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int cj = __shfl_sync(gmask, c, j0 + u, G);
        av[u] = __shfl_sync(gmask, v, j0 + u, G);
        bv[u] = ldg16(Bp + (int64_t)cj * d.ldb + coff);
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        TAcc b[VE];
        unpack16<Tr>(bv[u], b);
#pragma unroll
        for (int e = 0; e < VE; ++e) acc[e] = fma(av[u], b[e], acc[e]);
      }
    }
    for (; j0 < cnt; ++j0) {
      const int cj = __shfl_sync(gmask, c, j0, G);
      const TAcc aj = __shfl_sync(gmask, v, j0, G);
      TAcc b[VE];
      unpack16<Tr>(ldg16(Bp + (int64_t)cj * d.ldb + coff), b);
#pragma unroll
      for (int e = 0; e < VE; ++e) acc[e] = fma(aj, b[e], acc[e]);
    }
  }
  if (row >= 0) {
    TC* crow = reinterpret_cast<TC*>(d.C) + (int64_t)row * d.ldc + coff;
    TC o[VE];
#pragma unroll
    for (int e = 0; e < VE; ++e) o[e] = Tr::kScaled ? (TC)(acc[e] * col_mult<Tr>(d, coff + e)) : (TC)acc[e];
#pragma unroll
    for (int q = 0; q < (int)(VE * sizeof(TC) / 16); ++q)
      *reinterpret_cast<uint4*>(crow + q * (16 / sizeof(TC))) = *reinterpret_cast<const uint4*>(&o[q * (16 / sizeof(TC))]);
  } else {
    TAcc* srow = reinterpret_cast<TAcc*>(d.scratch) + (int64_t)(-1 - row) * d.N + coff;
#pragma unroll
    for (int e = 0; e < VE; ++e) srow[e] = acc[e];
  }
}

// One F32 BCSR unit (B_r rows, tile-major values) for a group of G lanes.
template <int BR>
__device__ __forceinline__ void ffma_block(const BatchDesc& d, int64_t u, int sub) {
  const int32_t b = d.unit_block[u];
  const int64_t rb = d.rb_id[b];
  const int64_t t0 = d.unit_t0[u], t1 = d.unit_t1[u];
  const int32_t slot = d.unit_slot[u];
  const float* Av = reinterpret_cast<const float*>(d.tile_val);
  const float* Bp = reinterpret_cast<const float*>(d.B);
  const int64_t n = (int64_t)sub * 4;
  float acc[BR][4];
#pragma unroll
  for (int r = 0; r < BR; ++r)
#pragma unroll
    for (int e = 0; e < 4; ++e) acc[r][e] = 0.f;
  for (int64_t tt = t0; tt < t1; ++tt) {
    const int32_t c = __ldg(d.tile_col + tt);
    const uint4 v = c >= 0 ? ldg16(Bp + (int64_t)c * d.ldb + n) : make_uint4(0, 0, 0, 0);
    const float bv[4] = {__uint_as_float(v.x), __uint_as_float(v.y), __uint_as_float(v.z), __uint_as_float(v.w)};
#pragma unroll
    for (int r4 = 0; r4 < BR / 4; ++r4) {
      const uint4 w = ldg16(Av + tt * BR + r4 * 4);
      const float a4[4] = {__uint_as_float(w.x), __uint_as_float(w.y), __uint_as_float(w.z), __uint_as_float(w.w)};
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int e = 0; e < 4; ++e) acc[r4 * 4 + i][e] = fmaf(a4[i], bv[e], acc[r4 * 4 + i][e]);
    }
  }
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

// One F16/BF16 BCSR unit for the whole warp, in column chunks of up to 64: sB is the warp's
// shared-memory slice holding the 16 gathered B-row pieces of the current K-group and chunk
// (row stride 72 elements, conflict-free for ldmatrix).
constexpr int kHChunk = 64;
constexpr int kHStride = kHChunk + 8;

template <class T>
__device__ __forceinline__ void hmma_block(const BatchDesc& d, int64_t u, T* sB, int lane) {
  constexpr bool kBF16 = sizeof(T) == 2 && !std::is_same<T, __half>::value;
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
    const int vec_per_row = NC / 8;        // 16-byte vectors per staged row piece
    float acc[8][4];
#pragma unroll
    for (int f = 0; f < 8; ++f)
#pragma unroll
      for (int i = 0; i < 4; ++i) acc[f][i] = 0.f;
    for (int g = 0; g < n_groups; ++g) {
      __syncwarp();
      for (int i = lane; i < 16 * vec_per_row; i += 32) {
        const int k = i / vec_per_row, qv = i % vec_per_row;
        const int32_t c = __ldg(d.tile_col + t0 + g * 16 + k);
        const uint4 v = c >= 0 ? ldg16(Bp + (int64_t)c * d.ldb + c0 + qv * 8) : make_uint4(0, 0, 0, 0);
        *reinterpret_cast<uint4*>(sB + k * kHStride + qv * 8) = v;
      }
      __syncwarp();
      const uint4 af = __ldg(Af + (int64_t)g * 32 + lane);
      const int mi = lane >> 3, r = lane & 7;
#pragma unroll
      for (int f = 0; f < 8; f += 2) {
        if (f >= NF) break;
        if (f + 1 < NF) {
          const uint32_t addr = smem_addr(sB + (r + 8 * (mi & 1)) * kHStride + f * 8 + 8 * (mi >> 1));
          uint32_t b0, b1, b2, b3;
          asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];"
                       : "=r"(b0), "=r"(b1), "=r"(b2), "=r"(b3) : "r"(addr));
          mma16816_b(acc[f], af, b0, b1, kBF16);
          mma16816_b(acc[f + 1], af, b2, b3, kBF16);
        } else {
          const uint32_t addr = smem_addr(sB + (r + 8 * (mi & 1)) * kHStride + f * 8);
          uint32_t b0, b1;
          asm volatile("ldmatrix.sync.aligned.m8n8.x2.trans.shared.b16 {%0,%1}, [%2];"
                       : "=r"(b0), "=r"(b1) : "r"(addr));
          mma16816_b(acc[f], af, b0, b1, kBF16);
        }
      }
    }
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

// Next task of a warp: with `counter` (zeroed before the launch) the warp takes the next
// unclaimed task of the list, so all warps stay within a short window of it (the list is
// ordered matrix by matrix, and the window's B operands stay in L2); without it, warp w takes
// tasks w, w + W, w + 2W, ... Every task writes its own outputs, so either way the result does
// not depend on which warp runs which task.
__device__ __forceinline__ int64_t next_task(unsigned long long* counter, int64_t prev, int64_t W, int lane) {
  if (counter == nullptr) return prev + W;
  unsigned long long t = 0;
  if (lane == 0) t = atomicAdd(counter, 1ull);
  return (int64_t)__shfl_sync(0xffffffffu, t, 0);
}

template <class Tr, int BR>
__global__ void __launch_bounds__(256, LOOPS_BATCHED_MIN_BLOCKS) batched_persistent(const BatchDesc* __restrict__ descs,
                                                          const BatchTask* __restrict__ tasks, int64_t n_tasks,
                                                          int smem_per_warp, unsigned long long* counter) {
  extern __shared__ __align__(128) unsigned char smem[];
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int64_t W = (int64_t)gridDim.x * (blockDim.x >> 5);
  const int64_t first = counter ? next_task(counter, 0, W, lane) : (int64_t)blockIdx.x * (blockDim.x >> 5) + warp;
  for (int64_t t = first; t < n_tasks; t = next_task(counter, t, W, lane)) {
    const BatchTask task = tasks[t];
    const BatchDesc& d = descs[task.m];
    if (task.kind == 2) {
      if constexpr (sizeof(typename Tr::TB) == 2)
        hmma_block<typename Tr::TB>(d, task.first, reinterpret_cast<typename Tr::TB*>(smem + warp * smem_per_warp), lane);
      continue;
    }
    const int G = d.G;
    const int grp = lane / G, sub = lane % G;
    const unsigned gmask = G == 32 ? 0xffffffffu : (((1u << G) - 1u) << (grp * G));
    const int per_round = 32 / G;
    for (int32_t i = grp; i < task.count; i += per_round) {
      if (task.kind == 0) {
        csr_item<Tr>(d, task.first + i, G, sub, gmask);
      } else if constexpr (std::is_same<Tr, TrF32>::value) {
        ffma_block<BR>(d, task.first + i, sub);
      }
    }
  }
}

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

template <class Tr, int BR>
cudaError_t launch_batched_t(const BatchLaunch& L, cudaStream_t s) {
  const int smem = L.smem_per_warp * 8;
  auto kern = batched_persistent<Tr, BR>;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
  }
  // timing events become event nodes of the captured graph (external records)
  auto rec = [&](int i) {
    return L.tev ? cudaEventRecordWithFlags(L.tev[i], s, cudaEventRecordExternal) : cudaSuccess;
  };
  {
    cudaError_t e = rec(0);
    if (e != cudaSuccess) return e;
  }
  if (L.n_tasks > 0) {
    if (L.counter) {
      cudaError_t e = cudaMemsetAsync(L.counter, 0, sizeof(unsigned long long), s);
      if (e != cudaSuccess) return e;
    }
    kern<<<L.grid, 256, smem, s>>>(L.descs, L.tasks, L.n_tasks, L.smem_per_warp, L.counter);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  {
    cudaError_t e = rec(1);
    if (e == cudaSuccess) e = rec(2);
    if (e != cudaSuccess) return e;
  }
  if (L.n_splits > 0) {
    batched_split_reduce<Tr><<<(unsigned)L.n_splits, 128, 0, s>>>(L.descs, L.splits);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  if (L.n_bsplits > 0) {
    batched_bsplit_reduce<Tr><<<(unsigned)L.n_bsplits, 256, 0, s>>>(L.descs, L.bsplits);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return rec(3);
}

}  // namespace

cudaError_t launch_batched(loops_dtype dtype, int32_t br, const BatchLaunch& L, cudaStream_t s) {
  switch (dtype) {
    case LOOPS_F32: return br == 8 ? launch_batched_t<TrF32, 8>(L, s) : launch_batched_t<TrF32, 16>(L, s);
    case LOOPS_F16: return launch_batched_t<TrF16, 16>(L, s);
    case LOOPS_BF16: return launch_batched_t<TrBF16, 16>(L, s);
    default: return cudaErrorInvalidValue;
  }
}

int batched_grid_blocks(loops_dtype dtype, int32_t br, int smem_per_warp) {
  int dev = 0, sms = 152, per_sm = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int smem = smem_per_warp * 8;
  cudaError_t e = cudaSuccess;
  switch (dtype) {
    case LOOPS_F32:
      e = br == 8 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batched_persistent<TrF32, 8>, 256, smem)
                  : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batched_persistent<TrF32, 16>, 256, smem);
      break;
    case LOOPS_F16:
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batched_persistent<TrF16, 16>, 256, smem);
      break;
    default:
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batched_persistent<TrBF16, 16>, 256, smem);
      break;
  }
  if (e != cudaSuccess || per_sm < 1) per_sm = 1;
  return sms * per_sm;
}

}  // namespace loops
