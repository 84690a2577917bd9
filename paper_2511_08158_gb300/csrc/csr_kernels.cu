// CSR-part SpMM (the AXPY row kernel of Sec. 3.3 on CUDA cores), the deterministic sum of
// split-row partials, the SDDMM of the backward pass, and the per-column scaled cast.
//
// A group of G lanes (G divides 32) owns one work item (a CSR row or a segment of a long
// row). Each lane owns VPL 16-byte column vectors of the output row, laid out so that the G
// lanes read consecutive 16-byte pieces of a B row (coalesced 128-bit loads). The group
// reads G (col, val) pairs at once and broadcasts them with shuffles; U B-row loads are kept
// in flight before their FMAs. Accumulation is in f64 for F64 and in f32 otherwise. Every
// output row has one writer; rows split in segments write partials that a second kernel
// sums in segment order, so the result does not depend on scheduling.
#include <type_traits>

#include "device_common.cuh"
#include "loops_internal.h"

// SDDMM: reduce the four in-flight entries' partial dot products with one butterfly (1) or each
// with its own shuffle tree (0).
#ifndef LOOPS_SDDMM_BUTTERFLY
#define LOOPS_SDDMM_BUTTERFLY 1
#endif
// Tuning knobs of the memory-bound (non-FP64) CSR kernel: B-row loads kept in flight per
// lane (per column vector), the minimum resident blocks per SM the register allocation must
// allow, and the 16-byte column vectors each lane owns. Two vectors per lane with two
// entries in flight (four 16-byte loads per lane) measured fastest on GB300 for the R-MAT
// FP16 (N = 128) and GCN FP32 (N = 256) workloads.
#ifndef LOOPS_CSR_UNROLL
#define LOOPS_CSR_UNROLL 2
#endif
#ifndef LOOPS_CSR_MIN_BLOCKS
#define LOOPS_CSR_MIN_BLOCKS 4
#endif
#ifndef LOOPS_CSR_LANE_VECTORS
#define LOOPS_CSR_LANE_VECTORS 2
#endif
// FP64 (bound by the FP64 pipe): entries in flight per lane and resident blocks per SM with
// one vector per lane.
#ifndef LOOPS_CSR_F64_UNROLL
#define LOOPS_CSR_F64_UNROLL 1
#endif
#ifndef LOOPS_CSR_F64_MIN_BLOCKS
#define LOOPS_CSR_F64_MIN_BLOCKS 8
#endif

namespace loops {

namespace {

struct CsrKArgs {
  const int32_t* item_row;
  const int64_t* item_ptr;
  const int32_t* col;
  const void* val;
  int64_t n_items;
  const void* B;
  int64_t ldb;
  void* C;
  int64_t ldc;
  void* scratch;         // n_slots x N accumulators
  const float* col_scale;
  float inv_scale_f;
  double inv_scale_d;
  int64_t N;
  int accumulate;        // add to C (rows a BCSR part wrote first) instead of overwriting it
};

template <class Tr>
__device__ __forceinline__ typename Tr::TAcc out_scale(const CsrKArgs& a, int64_t n);
template <>
__device__ __forceinline__ double out_scale<TrF64>(const CsrKArgs& a, int64_t) { return a.inv_scale_d; }
template <>
__device__ __forceinline__ float out_scale<TrF32>(const CsrKArgs& a, int64_t) { return a.inv_scale_f; }
template <>
__device__ __forceinline__ float out_scale<TrF16>(const CsrKArgs& a, int64_t n) {
  return a.col_scale ? a.col_scale[n] * a.inv_scale_f : a.inv_scale_f;
}
template <>
__device__ __forceinline__ float out_scale<TrBF16>(const CsrKArgs& a, int64_t n) {
  return a.col_scale ? a.col_scale[n] * a.inv_scale_f : a.inv_scale_f;
}

// Vector path: N % VE == 0, B/C/ld aligned for 16-byte B loads and vector C stores.
// FP64: 8 resident blocks (at most 32 registers) keep enough warps in flight to feed the FP64
// pipe with one vector per lane; two vectors (N > 64) need 4 blocks (64 registers) to stay out
// of local memory. The other formats use the tuning knob.
template <class Tr, int VPL>
constexpr int csr_min_blocks() {
  return std::is_same<Tr, TrF64>::value ? (VPL == 1 ? LOOPS_CSR_F64_MIN_BLOCKS : 4) : LOOPS_CSR_MIN_BLOCKS;
}

template <class Tr, int G, int VPL, int U>
__global__ void __launch_bounds__(256, (csr_min_blocks<Tr, VPL>())) csr_spmm_vec(CsrKArgs a) {
  using TB = typename Tr::TB;
  using TAcc = typename Tr::TAcc;
  using TC = typename Tr::TC;
  constexpr int VE = Tr::kVE;
  const int lane = threadIdx.x & 31;
  const int sub = lane & (G - 1);
  const int64_t item = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / G;
  if (item >= a.n_items) return;  // a group leaves as a whole
  const unsigned gmask = (G == 32) ? 0xffffffffu : (((1u << G) - 1u) << (lane & ~(G - 1)));
  const int64_t beg = a.item_ptr[item];
  const int64_t end = a.item_ptr[item + 1];
  const int32_t row = a.item_row[item];
  const int64_t c_base = (int64_t)blockIdx.y * (G * VPL * VE);
  bool colok[VPL];
  int64_t coff[VPL];
#pragma unroll
  for (int p = 0; p < VPL; ++p) {
    coff[p] = c_base + (int64_t)(p * G + sub) * VE;
    colok[p] = coff[p] < a.N;
  }
  TAcc acc[VPL][VE];
#pragma unroll
  for (int p = 0; p < VPL; ++p)
#pragma unroll
    for (int e = 0; e < VE; ++e) acc[p][e] = TAcc(0);

  const TB* __restrict__ Bp = reinterpret_cast<const TB*>(a.B);
  const TB* __restrict__ vals = reinterpret_cast<const TB*>(a.val);
  for (int64_t k0 = beg; k0 < end; k0 += G) {
    const int64_t k = k0 + sub;
    int32_t c = 0;
    TAcc v = TAcc(0);
    if (k < end) {
      c = __ldg(a.col + k);
      v = Tr::to_acc(vals[k]);
    }
    const int cnt = (int)(end - k0 < (int64_t)G ? end - k0 : (int64_t)G);  // uniform in the group
    int j0 = 0;
    for (; j0 + U <= cnt; j0 += U) {  // full batches: U loads in flight, then U FMAs each
      uint4 bv[U][VPL];
      TAcc av[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int cj = __shfl_sync(gmask, c, (j0 + u) & (G - 1), G);
        av[u] = __shfl_sync(gmask, v, (j0 + u) & (G - 1), G);
        const TB* brow = Bp + (int64_t)cj * a.ldb;
#pragma unroll
        for (int p = 0; p < VPL; ++p) bv[u][p] = colok[p] ? ldg16(brow + coff[p]) : make_uint4(0, 0, 0, 0);
      }
#pragma unroll
      for (int u = 0; u < U; ++u)
#pragma unroll
        for (int p = 0; p < VPL; ++p) {
          TAcc b[VE];
          unpack16<Tr>(bv[u][p], b);
#pragma unroll
          for (int e = 0; e < VE; ++e) acc[p][e] = fma(av[u], b[e], acc[p][e]);
        }
    }
    if constexpr (U > 1) {
    if (j0 < cnt) {  // tail of 1 .. U-1 entries: no multiply by padded zeros
      uint4 bv[U - 1][VPL];
      TAcc av[U - 1];
#pragma unroll
      for (int u = 0; u < U - 1; ++u) {
        if (j0 + u < cnt) {
          const int cj = __shfl_sync(gmask, c, (j0 + u) & (G - 1), G);
          av[u] = __shfl_sync(gmask, v, (j0 + u) & (G - 1), G);
          const TB* brow = Bp + (int64_t)cj * a.ldb;
#pragma unroll
          for (int p = 0; p < VPL; ++p) bv[u][p] = colok[p] ? ldg16(brow + coff[p]) : make_uint4(0, 0, 0, 0);
        }
      }
#pragma unroll
      for (int u = 0; u < U - 1; ++u) {
        if (j0 + u < cnt) {
#pragma unroll
          for (int p = 0; p < VPL; ++p) {
            TAcc b[VE];
            unpack16<Tr>(bv[u][p], b);
#pragma unroll
            for (int e = 0; e < VE; ++e) acc[p][e] = fma(av[u], b[e], acc[p][e]);
          }
        }
      }
    }
    }
  }
  if (row >= 0) {
    TC* crow = reinterpret_cast<TC*>(a.C) + (int64_t)row * a.ldc;
#pragma unroll
    for (int p = 0; p < VPL; ++p) {
      if (!colok[p]) continue;
      TC o[VE];
#pragma unroll
      for (int e = 0; e < VE; ++e)
        o[e] = Tr::kScaled ? (TC)(acc[p][e] * out_scale<Tr>(a, coff[p] + e)) : (TC)acc[p][e];
      if (a.accumulate) {
#pragma unroll
        for (int e = 0; e < VE; ++e) o[e] += crow[coff[p] + e];
      }
      // VE outputs are 16 (F64/F32) or 32 (16-bit inputs, f32 outputs) bytes
#pragma unroll
      for (int q = 0; q < (int)(VE * sizeof(TC) / 16); ++q)
        *reinterpret_cast<uint4*>(crow + coff[p] + q * (16 / sizeof(TC))) =
            *reinterpret_cast<const uint4*>(&o[q * (16 / sizeof(TC))]);
    }
  } else {
    TAcc* srow = reinterpret_cast<TAcc*>(a.scratch) + (int64_t)(-1 - row) * a.N;
#pragma unroll
    for (int p = 0; p < VPL; ++p) {
      if (!colok[p]) continue;
#pragma unroll
      for (int e = 0; e < VE; ++e) srow[coff[p] + e] = acc[p][e];
    }
  }
}

// Scalar path for any N and alignment: 32 lanes per item, one column per lane per pass.
template <class Tr, int U>
__global__ void __launch_bounds__(256) csr_spmm_scalar(CsrKArgs a) {
  using TB = typename Tr::TB;
  using TAcc = typename Tr::TAcc;
  using TC = typename Tr::TC;
  const int lane = threadIdx.x & 31;
  const int64_t item = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / 32;
  if (item >= a.n_items) return;
  const int64_t beg = a.item_ptr[item];
  const int64_t end = a.item_ptr[item + 1];
  const int32_t row = a.item_row[item];
  const int64_t n = (int64_t)blockIdx.y * 32 + lane;
  const bool colok = n < a.N;
  const TB* __restrict__ Bp = reinterpret_cast<const TB*>(a.B);
  const TB* __restrict__ vals = reinterpret_cast<const TB*>(a.val);
  TAcc acc = TAcc(0);
  for (int64_t k0 = beg; k0 < end; k0 += 32) {
    const int64_t k = k0 + lane;
    int32_t c = 0;
    TAcc v = TAcc(0);
    if (k < end) {
      c = __ldg(a.col + k);
      v = Tr::to_acc(vals[k]);
    }
    const int cnt = (int)(end - k0 < 32 ? end - k0 : 32);
    for (int j0 = 0; j0 < cnt; j0 += U) {
      TAcc bv[U], av[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int j = j0 + u;
        const int cj = __shfl_sync(0xffffffffu, c, j & 31);
        av[u] = __shfl_sync(0xffffffffu, v, j & 31);
        const bool ok = j < cnt && colok;
        bv[u] = ok ? Tr::to_acc(Bp[(int64_t)cj * a.ldb + n]) : TAcc(0);
        if (j >= cnt) av[u] = TAcc(0);
      }
#pragma unroll
      for (int u = 0; u < U; ++u) acc = fma(av[u], bv[u], acc);
    }
  }
  if (!colok) return;
  if (row >= 0) {
    TC* cp = reinterpret_cast<TC*>(a.C) + (int64_t)row * a.ldc + n;
    const TC v = Tr::kScaled ? (TC)(acc * out_scale<Tr>(a, n)) : (TC)acc;
    *cp = a.accumulate ? *cp + v : v;
  } else {
    reinterpret_cast<TAcc*>(a.scratch)[(int64_t)(-1 - row) * a.N + n] = acc;
  }
}

// C[row, n] = scale_n * sum over the row's segments, in segment order.
template <class Tr>
__global__ void __launch_bounds__(256) split_reduce(const int32_t* __restrict__ split_row,
                                                    const int32_t* __restrict__ slot_ptr,
                                                    int64_t n_split, CsrKArgs a) {
  using TAcc = typename Tr::TAcc;
  using TC = typename Tr::TC;
  const int64_t s = blockIdx.x;
  if (s >= n_split) return;
  const int32_t row = split_row[s];
  const int32_t s0 = slot_ptr[s], s1 = slot_ptr[s + 1];
  const TAcc* sc = reinterpret_cast<const TAcc*>(a.scratch);
  for (int64_t n = (int64_t)blockIdx.y * blockDim.x + threadIdx.x; n < a.N; n += (int64_t)gridDim.y * blockDim.x) {
    TAcc acc = TAcc(0);
    for (int32_t q = s0; q < s1; ++q) acc += sc[(int64_t)q * a.N + n];
    TC* cp = reinterpret_cast<TC*>(a.C) + (int64_t)row * a.ldc + n;
    const TC v = Tr::kScaled ? (TC)(acc * out_scale<Tr>(a, n)) : (TC)acc;
    *cp = a.accumulate ? *cp + v : v;
  }
}

inline int next_pow2(int64_t x) {
  int p = 1;
  while (p < x && p < 32) p <<= 1;
  return p;
}

template <class Tr, int G, int VPL>
cudaError_t launch_vec_g(const CsrKArgs& a, cudaStream_t s) {
  constexpr int VE = Tr::kVE;
  const int64_t per_chunk = (int64_t)G * VPL * VE;
  const int64_t chunks = (a.N + per_chunk - 1) / per_chunk;
  const int64_t threads = a.n_items * G;
  dim3 grid((unsigned)((threads + 255) / 256), (unsigned)chunks);
  // F64 is bound by the FP64 pipe: one entry at a time, so no FMA is ever spent on a padded
  // slot (a predicated-off DFMA still occupies the pipe) and registers stay low for occupancy.
  // The other formats are bound by memory: U x VPL loads in flight per lane (narrow groups with
  // one vector per lane take four entries at a time, the register budget allows it).
  constexpr int U = std::is_same<Tr, TrF64>::value ? LOOPS_CSR_F64_UNROLL
                                                   : ((G >= 8 || VPL > 1) ? LOOPS_CSR_UNROLL : 4);
  csr_spmm_vec<Tr, G, VPL, U><<<grid, 256, 0, s>>>(a);
  return cudaGetLastError();
}

template <class Tr>
cudaError_t launch_csr_t(const loops_plan_s* p, const CsrDev& d, const DenseArgs& da, bool accumulate,
                         cudaStream_t s) {
  CsrKArgs a;
  a.accumulate = accumulate ? 1 : 0;
  a.item_row = d.item_row;
  a.item_ptr = d.item_ptr;
  a.col = d.col;
  a.val = d.val;
  a.n_items = d.n_items;
  a.B = da.B;
  a.ldb = da.ldb;
  a.C = da.C;
  a.ldc = da.ldc;
  a.scratch = d.scratch;
  a.col_scale = da.col_scale;
  a.inv_scale_f = da.inv_scale_f;
  a.inv_scale_d = da.inv_scale_d;
  a.N = da.N;
  using TB = typename Tr::TB;
  using TC = typename Tr::TC;
  constexpr int VE = Tr::kVE;
  const bool vec = (a.N % VE == 0) && ((uintptr_t)a.B % 16 == 0) && ((uintptr_t)a.C % 16 == 0) &&
                   ((a.ldb * (int64_t)sizeof(TB)) % 16 == 0) && ((a.ldc * (int64_t)sizeof(TC)) % 16 == 0);
  cudaError_t e = cudaSuccess;
  if (a.n_items > 0) {
    if (vec) {
      const int64_t nvec = a.N / VE;
      // lanes per item: the 16-byte vectors of a row, LOOPS_CSR_LANE_VECTORS per lane while
      // the group keeps at least 8 lanes (more vectors per lane: fewer shuffles per byte and
      // more loads in flight per lane; narrower groups lose more to the per-row overhead)
      constexpr int LV = LOOPS_CSR_LANE_VECTORS;
      const bool lv = !std::is_same<Tr, TrF64>::value && LV > 1 && nvec >= 8 * LV;
      const int64_t nv = lv ? (nvec + LV - 1) / LV : nvec;
      const int G = next_pow2(nv);
      const bool two = lv || nvec > 32;
      switch (G) {
        case 1: e = two ? launch_vec_g<Tr, 1, 2>(a, s) : launch_vec_g<Tr, 1, 1>(a, s); break;
        case 2: e = two ? launch_vec_g<Tr, 2, 2>(a, s) : launch_vec_g<Tr, 2, 1>(a, s); break;
        case 4: e = two ? launch_vec_g<Tr, 4, 2>(a, s) : launch_vec_g<Tr, 4, 1>(a, s); break;
        case 8: e = two ? launch_vec_g<Tr, 8, 2>(a, s) : launch_vec_g<Tr, 8, 1>(a, s); break;
        case 16: e = two ? launch_vec_g<Tr, 16, 2>(a, s) : launch_vec_g<Tr, 16, 1>(a, s); break;
        default: e = two ? launch_vec_g<Tr, 32, 2>(a, s) : launch_vec_g<Tr, 32, 1>(a, s); break;
      }
    } else {
      dim3 grid((unsigned)((a.n_items * 32 + 255) / 256), (unsigned)((a.N + 31) / 32));
      csr_spmm_scalar<Tr, 8><<<grid, 256, 0, s>>>(a);
      e = cudaGetLastError();
    }
  }
  if (e == cudaSuccess && d.n_split > 0) {
    dim3 grid((unsigned)d.n_split, (unsigned)std::min<int64_t>((a.N + 255) / 256, 64));
    split_reduce<Tr><<<grid, 256, 0, s>>>(d.split_row, d.split_slot_ptr, d.n_split, a);
    e = cudaGetLastError();
  }
  return e;
}

// ------------------------------------------------------------------ SDDMM
// dvals[k] = sum_n dC[i, n] * B[j_k, n] for the entries of an item (row i, range [b, e)).
// G lanes per item hold the dC row slice in registers; each entry's partial dot products are
// reduced across the group with shuffles (a fixed tree, so the result is deterministic).
struct SddmmKArgs {
  const int32_t* item_row;
  const int64_t* item_beg;
  const int64_t* item_end;
  const int32_t* col;
  int64_t n_items;
  const void* dC;
  int64_t lddc;
  const void* B;
  int64_t ldb;
  void* dvals;
  int64_t N;
};

template <class Tr, int G, int VPL>
__global__ void __launch_bounds__(256) sddmm_vec(SddmmKArgs a) {
  using TB = typename Tr::TB;
  using TAcc = typename Tr::TAcc;
  using TC = typename Tr::TC;
  constexpr int VE = Tr::kVE;
  const int lane = threadIdx.x & 31;
  const int sub = lane & (G - 1);
  const int64_t item = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / G;
  if (item >= a.n_items) return;
  const unsigned gmask = (G == 32) ? 0xffffffffu : (((1u << G) - 1u) << (lane & ~(G - 1)));
  const int32_t row = a.item_row[item];
  const int64_t beg = a.item_beg[item], end = a.item_end[item];
  const TB* dcrow = reinterpret_cast<const TB*>(a.dC) + (int64_t)row * a.lddc;
  const TB* Bp = reinterpret_cast<const TB*>(a.B);
  TAcc g[VPL][VE];
  bool colok[VPL];
  int64_t coff[VPL];
#pragma unroll
  for (int p = 0; p < VPL; ++p) {
    coff[p] = (int64_t)(p * G + sub) * VE;
    colok[p] = coff[p] < a.N;
    uint4 v = colok[p] ? ldg16(dcrow + coff[p]) : make_uint4(0, 0, 0, 0);
    unpack16<Tr>(v, g[p]);
  }
  constexpr int U = 4;
  for (int64_t k0 = beg; k0 < end; k0 += U) {
    int32_t cj[U];
    uint4 bv[U][VPL];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const bool ok = k0 + u < end;
      cj[u] = ok ? __ldg(a.col + k0 + u) : 0;
#pragma unroll
      for (int p = 0; p < VPL; ++p)
        bv[u][p] = (ok && colok[p]) ? ldg16(Bp + (int64_t)cj[u] * a.ldb + coff[p]) : make_uint4(0, 0, 0, 0);
    }
    TAcc s[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      s[u] = TAcc(0);
#pragma unroll
      for (int p = 0; p < VPL; ++p) {
        TAcc b[VE];
        unpack16<Tr>(bv[u][p], b);
#pragma unroll
        for (int e = 0; e < VE; ++e) s[u] = fma(g[p][e], b[e], s[u]);
      }
    }
    if constexpr (LOOPS_SDDMM_BUTTERFLY && G >= 4 && U == 4) {
      // the four entries' sums over the group at once (a butterfly that halves the values a
      // lane holds while it halves the lanes it spans): 6 shuffles instead of 4 x log2(G)
      const bool h1 = (sub & (G / 2)) != 0, h2 = (sub & (G / 4)) != 0;
      TAcc k0v = h1 ? s[2] : s[0], k1v = h1 ? s[3] : s[1];
      k0v += __shfl_xor_sync(gmask, h1 ? s[0] : s[2], G / 2, G);
      k1v += __shfl_xor_sync(gmask, h1 ? s[1] : s[3], G / 2, G);
      TAcc v = h2 ? k1v : k0v;
      v += __shfl_xor_sync(gmask, h2 ? k0v : k1v, G / 4, G);
#pragma unroll
      for (int off = G / 8; off > 0; off >>= 1) v += __shfl_xor_sync(gmask, v, off, G);
      const int e = (h1 ? 2 : 0) + (h2 ? 1 : 0);  // the entry this lane's sum belongs to
      if ((sub & (G / 4 - 1)) == 0 && k0 + e < end) reinterpret_cast<TC*>(a.dvals)[k0 + e] = (TC)v;
    } else {
#pragma unroll
      for (int u = 0; u < U; ++u) {
        TAcc t = s[u];
#pragma unroll
        for (int off = G / 2; off > 0; off >>= 1) t += __shfl_xor_sync(gmask, t, off, G);
        if (sub == 0 && k0 + u < end) reinterpret_cast<TC*>(a.dvals)[k0 + u] = (TC)t;
      }
    }
  }
}

template <class Tr>
__global__ void __launch_bounds__(256) sddmm_scalar(SddmmKArgs a) {
  using TB = typename Tr::TB;
  using TAcc = typename Tr::TAcc;
  using TC = typename Tr::TC;
  const int lane = threadIdx.x & 31;
  const int64_t item = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / 32;
  if (item >= a.n_items) return;
  const int32_t row = a.item_row[item];
  const TB* dcrow = reinterpret_cast<const TB*>(a.dC) + (int64_t)row * a.lddc;
  const TB* Bp = reinterpret_cast<const TB*>(a.B);
  for (int64_t k = a.item_beg[item]; k < a.item_end[item]; ++k) {
    const int32_t c = __ldg(a.col + k);
    TAcc s = TAcc(0);
    for (int64_t n = lane; n < a.N; n += 32) s = fma(Tr::to_acc(dcrow[n]), Tr::to_acc(Bp[(int64_t)c * a.ldb + n]), s);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    if (lane == 0) reinterpret_cast<TC*>(a.dvals)[k] = (TC)s;
  }
}

template <class Tr>
cudaError_t launch_sddmm_t(const loops_plan_s* p, const void* dC, int64_t lddc, const void* B, int64_t ldb,
                           void* dvals, cudaStream_t s) {
  SddmmKArgs a;
  a.item_row = p->sddmm.item_row;
  a.item_beg = p->sddmm.item_beg;
  a.item_end = p->sddmm.item_end;
  a.col = p->sddmm.col;
  a.n_items = p->sddmm.n_items;
  a.dC = dC;
  a.lddc = lddc;
  a.B = B;
  a.ldb = ldb;
  a.dvals = dvals;
  a.N = p->N;
  if (a.n_items == 0) return cudaSuccess;
  using TB = typename Tr::TB;
  constexpr int VE = Tr::kVE;
  const bool vec = (a.N % VE == 0) && ((uintptr_t)B % 16 == 0) && ((uintptr_t)dC % 16 == 0) &&
                   ((ldb * (int64_t)sizeof(TB)) % 16 == 0) && ((lddc * (int64_t)sizeof(TB)) % 16 == 0);
  const int64_t nvec = a.N / VE;
  if (vec && nvec <= 64) {
    const int G = next_pow2(nvec);
    const int64_t threads = a.n_items * G;
    dim3 grid((unsigned)((threads + 255) / 256));
    switch (G) {
      case 1: sddmm_vec<Tr, 1, 1><<<grid, 256, 0, s>>>(a); break;
      case 2: sddmm_vec<Tr, 2, 1><<<grid, 256, 0, s>>>(a); break;
      case 4: sddmm_vec<Tr, 4, 1><<<grid, 256, 0, s>>>(a); break;
      case 8: sddmm_vec<Tr, 8, 1><<<grid, 256, 0, s>>>(a); break;
      case 16: sddmm_vec<Tr, 16, 1><<<grid, 256, 0, s>>>(a); break;
      default:
        if (nvec > 32) sddmm_vec<Tr, 32, 2><<<grid, 256, 0, s>>>(a);
        else sddmm_vec<Tr, 32, 1><<<grid, 256, 0, s>>>(a);
        break;
    }
  } else {
    dim3 grid((unsigned)((a.n_items * 32 + 255) / 256));
    sddmm_scalar<Tr><<<grid, 256, 0, s>>>(a);
  }
  return cudaGetLastError();
}

// ------------------------------------------------------------------ per-column scaled cast
__global__ void __launch_bounds__(256) colmax_kernel(const float* __restrict__ X, int64_t rows, int64_t cols,
                                                     int64_t ldx, unsigned int* __restrict__ mx) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= cols) return;
  const int64_t r_per = (rows + gridDim.y - 1) / gridDim.y;
  const int64_t r0 = (int64_t)blockIdx.y * r_per;
  const int64_t r1 = min(rows, r0 + r_per);
  float m = 0.f;
  for (int64_t r = r0; r < r1; ++r) m = fmaxf(m, fabsf(X[r * ldx + c]));
  if (r1 > r0) atomicMax(mx + c, __float_as_uint(m));  // non-negative floats order as integers
}

__global__ void colscale_kernel(float* __restrict__ s, int64_t cols) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= cols) return;
  const float m = s[c];
  float r = 1.f;
  if (m > 0.f) {
    int e;
    const float f = frexpf(m, &e);             // m = f * 2^e, f in [0.5, 1)
    int cexp = (f == 0.5f) ? e - 1 : e;        // ceil(log2 m)
    if (cexp > 127) cexp = 127;                // largest power of two of binary32
    r = ldexpf(1.f, cexp);
  }
  s[c] = r;
}

template <class T>
__device__ __forceinline__ T cvt_rn(float x);
template <>
__device__ __forceinline__ __half cvt_rn<__half>(float x) { return __float2half_rn(x); }
template <>
__device__ __forceinline__ __nv_bfloat16 cvt_rn<__nv_bfloat16>(float x) { return __float2bfloat16_rn(x); }

template <class T>
__global__ void __launch_bounds__(256) scale_cast_kernel(const float* __restrict__ X, int64_t rows, int64_t cols,
                                                         int64_t ldx, const float* __restrict__ s, T* __restrict__ Y,
                                                         int64_t ldy) {
  const int64_t total = rows * cols;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = i / cols, c = i - r * cols;
    // division by a power of two: exact unless the quotient falls below binary32's normal range
    Y[r * ldy + c] = cvt_rn<T>(X[r * ldx + c] / s[c]);
  }
}

// ------------------------------------------------------------------ value refresh from device

// Stored value = round(scale * sum of the slot's input entries in input order), as the host
// packer does: CSR positions have one source each, BCSR fragment slots zero or more.
template <class TB, class TIn>
__global__ void __launch_bounds__(256) set_values_kernel(const TIn* __restrict__ vals, double scale,
                                                         const int64_t* __restrict__ csr_src, int64_t n_csr,
                                                         TB* __restrict__ csr_val,
                                                         const int64_t* __restrict__ bptr,
                                                         const int64_t* __restrict__ bsrc, int64_t n_slots,
                                                         TB* __restrict__ tile_val) {
  const int64_t total = n_csr + n_slots;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    if (i < n_csr) {
      csr_val[i] = from_f64<TB>((double)vals[csr_src[i]] * scale);
    } else {
      const int64_t f = i - n_csr;
      double acc = 0.0;
      for (int64_t q = bptr[f]; q < bptr[f + 1]; ++q) acc += (double)vals[bsrc[q]];
      tile_val[f] = from_f64<TB>(acc * scale);
    }
  }
}

template <class TB>
cudaError_t launch_set_values_t(const loops_plan_s* p, const void* vals, loops_dtype vd, cudaStream_t s) {
  const ValueMapDev& m = p->vmap;
  const int64_t total = m.n_csr + m.n_slots;
  if (total == 0) return cudaSuccess;
  const unsigned blocks = (unsigned)std::min<int64_t>((total + 255) / 256, 152 * 8);
  if (vd == LOOPS_F64)
    set_values_kernel<TB, double><<<blocks, 256, 0, s>>>((const double*)vals, p->scale, m.csr_src, m.n_csr,
                                                          (TB*)p->dev.csr.val, m.bcsr_ptr, m.bcsr_src, m.n_slots,
                                                          (TB*)p->dev.bcsr.tile_val);
  else
    set_values_kernel<TB, float><<<blocks, 256, 0, s>>>((const float*)vals, p->scale, m.csr_src, m.n_csr,
                                                         (TB*)p->dev.csr.val, m.bcsr_ptr, m.bcsr_src, m.n_slots,
                                                         (TB*)p->dev.bcsr.tile_val);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_set_values(const loops_plan_s* p, const void* vals, loops_dtype vd, cudaStream_t s) {
  switch (p->dtype) {
    case LOOPS_F64: return launch_set_values_t<double>(p, vals, vd, s);
    case LOOPS_F32: return launch_set_values_t<float>(p, vals, vd, s);
    case LOOPS_F16: return launch_set_values_t<__half>(p, vals, vd, s);
    case LOOPS_BF16: return launch_set_values_t<__nv_bfloat16>(p, vals, vd, s);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_csr(const loops_plan_s* p, const CsrDev& d, const DenseArgs& a, bool accumulate,
                       cudaStream_t s) {
  switch (p->dtype) {
    case LOOPS_F64: return launch_csr_t<TrF64>(p, d, a, accumulate, s);
    case LOOPS_F32: return launch_csr_t<TrF32>(p, d, a, accumulate, s);
    case LOOPS_F16: return launch_csr_t<TrF16>(p, d, a, accumulate, s);
    case LOOPS_BF16: return launch_csr_t<TrBF16>(p, d, a, accumulate, s);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_sddmm(const loops_plan_s* p, const void* dC, int64_t lddc, const void* B, int64_t ldb,
                         void* dvals, cudaStream_t s) {
  switch (p->dtype) {
    case LOOPS_F64: return launch_sddmm_t<TrF64>(p, dC, lddc, B, ldb, dvals, s);
    case LOOPS_F32: return launch_sddmm_t<TrF32>(p, dC, lddc, B, ldb, dvals, s);
    case LOOPS_F16: return launch_sddmm_t<TrF16>(p, dC, lddc, B, ldb, dvals, s);
    case LOOPS_BF16: return launch_sddmm_t<TrBF16>(p, dC, lddc, B, ldb, dvals, s);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_cast_scaled(const float* X, int64_t rows, int64_t cols, int64_t ldx, loops_dtype yd, void* Y,
                               int64_t ldy, float* col_scale, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(col_scale, 0, (size_t)cols * sizeof(float), s);
  if (e != cudaSuccess) return e;
  if (rows > 0) {
    const int64_t ychunks = std::min<int64_t>(std::max<int64_t>(rows / 256, 1), 1024);
    dim3 g1((unsigned)((cols + 255) / 256), (unsigned)ychunks);
    colmax_kernel<<<g1, 256, 0, s>>>(X, rows, cols, ldx, reinterpret_cast<unsigned int*>(col_scale));
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  colscale_kernel<<<(unsigned)((cols + 255) / 256), 256, 0, s>>>(col_scale, cols);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if (rows == 0) return cudaSuccess;
  const int64_t total = rows * cols;
  const unsigned blocks = (unsigned)std::min<int64_t>((total + 255) / 256, 152 * 16);
  if (yd == LOOPS_F16)
    scale_cast_kernel<__half><<<blocks, 256, 0, s>>>(X, rows, cols, ldx, col_scale, (__half*)Y, ldy);
  else
    scale_cast_kernel<__nv_bfloat16><<<blocks, 256, 0, s>>>(X, rows, cols, ldx, col_scale, (__nv_bfloat16*)Y, ldy);
  return cudaGetLastError();
}

}  // namespace loops
