// CSR-part SpMM (the AXPY row kernel of Sec. 3.3 on CUDA cores) and the deterministic sum of
// split-row partials.
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
  using TV = typename Tr::TV;
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
  // FP32 loads the next chunk's G entries before the current chunk's B rows, so their
  // latency overlaps (measured: GCN layer 0.572 -> 0.547 ms); the 16-bit formats, whose
  // unpacking needs the registers, and FP64, bound by its FMA pipe, load them in turn
  constexpr bool kPrefetch = std::is_same<Tr, TrF32>::value;
  int32_t c_next = 0;
  TV v_next = TV(0);
  if (kPrefetch && beg + sub < end) {
    c_next = __ldg(a.col + beg + sub);
    v_next = Tr::load_v(vals + beg + sub);
  }
  for (int64_t k0 = beg; k0 < end; k0 += G) {
    int32_t c = c_next;
    TV v = v_next;
    const int64_t kn = kPrefetch ? k0 + G + sub : k0 + sub;
    if (kn < end) {
      c_next = __ldg(a.col + kn);
      v_next = Tr::load_v(vals + kn);
    }
    if constexpr (!kPrefetch) {
      c = kn < end ? c_next : 0;
      v = kn < end ? v_next : TV(0);
    }
    const int cnt = (int)(end - k0 < (int64_t)G ? end - k0 : (int64_t)G);  // uniform in the group
    int j0 = 0;
    for (; j0 + U <= cnt; j0 += U) {  // full batches: U loads in flight, then U FMAs each
      uint4 bv[U][VPL];
      TV av[U];
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
        for (int p = 0; p < VPL; ++p) fma_vec<Tr>(acc[p], bv[u][p], av[u]);
    }
    if constexpr (U > 1) {
    if (j0 < cnt) {  // tail of 1 .. U-1 entries: one batch under predicates
      // entries past the tail load nothing and take a zero value, so they add exact zeros;
      // the live loads issue together instead of one per round trip
      uint4 bv[U - 1][VPL];
      TV av[U - 1];
#pragma unroll
      for (int u = 0; u < U - 1; ++u) {
        const bool live = j0 + u < cnt;
        const int cj = __shfl_sync(gmask, c, (j0 + u) & (G - 1), G);
        const TV vj = __shfl_sync(gmask, v, (j0 + u) & (G - 1), G);
        av[u] = live ? vj : TV(0);
        const TB* brow = Bp + (int64_t)cj * a.ldb;
#pragma unroll
        for (int p = 0; p < VPL; ++p) bv[u][p] = ldg16_if(live && colok[p], brow + coff[p]);
      }
#pragma unroll
      for (int u = 0; u < U - 1; ++u)
#pragma unroll
        for (int p = 0; p < VPL; ++p) fma_vec<Tr>(acc[p], bv[u][p], av[u]);
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
      // (the plan's csr_vpl, when the autotuner set it, overrides this heuristic)
      constexpr int LV = LOOPS_CSR_LANE_VECTORS;
      const bool lv = p->csr_vpl == 2 ? nvec >= 2
                    : p->csr_vpl == 1 ? false
                    : (!std::is_same<Tr, TrF64>::value && LV > 1 && nvec >= 8 * LV);
      const int64_t nv = lv ? (nvec + 1) / 2 : nvec;
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

}  // namespace

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

}  // namespace loops
