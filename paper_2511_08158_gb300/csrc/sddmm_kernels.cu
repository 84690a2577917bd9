// The kernels around the SpMM: the SDDMM of the backward pass (dvals on A's pattern), the
// refresh of a plan's stored values from a device array, and the per-column scaled cast of a
// dense FP32 operand into FP16/BF16.
#include <algorithm>
#include <type_traits>

#include "device_common.cuh"
#include "loops_internal.h"

// SDDMM: reduce the four in-flight entries' partial dot products with one butterfly (1) or each
// with its own shuffle tree (0).
#ifndef LOOPS_SDDMM_BUTTERFLY
#define LOOPS_SDDMM_BUTTERFLY 1
#endif
// SDDMM: batches that lie inside the segment run without per-entry bounds predicates (1), or
// every batch is predicated (0).
#ifndef LOOPS_SDDMM_FULL_BATCHES
#define LOOPS_SDDMM_FULL_BATCHES 1
#endif
namespace loops {

namespace {

inline int next_pow2(int64_t x) {
  int p = 1;
  while (p < x && p < 32) p <<= 1;
  return p;
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
  const float* dc_scale;   // optional per-column scales of dC and of B (16-bit dtypes): the
  const float* b_scale;    // sum runs over dC[i, n] * B[j, n] * dc_scale[n] * b_scale[n]
};

// Per-column weight of the dot product (product of the two optional scales; exact for powers
// of two).
__device__ __forceinline__ float col_weight(const SddmmKArgs& a, int64_t n) {
  return (a.dc_scale ? a.dc_scale[n] : 1.f) * (a.b_scale ? a.b_scale[n] : 1.f);
}

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
    if constexpr (Tr::kScaled) {
      if (colok[p] && (a.dc_scale || a.b_scale)) {
#pragma unroll
        for (int e = 0; e < VE; ++e) g[p][e] *= col_weight(a, coff[p] + e);
      }
    }
  }
  constexpr int U = 4;
  // one batch of U entries from k0; TAIL: the batch may run past the segment's end (bounds
  // predicates on the loads and stores), otherwise all U entries exist
  auto batch = [&](int64_t k0, auto tail_tag) {
    constexpr bool TAIL = decltype(tail_tag)::value;
    int32_t cj[U];
    uint4 bv[U][VPL];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const bool ok = !TAIL || k0 + u < end;
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
      if ((sub & (G / 4 - 1)) == 0 && (!TAIL || k0 + e < end)) reinterpret_cast<TC*>(a.dvals)[k0 + e] = (TC)v;
    } else {
#pragma unroll
      for (int u = 0; u < U; ++u) {
        TAcc t = s[u];
#pragma unroll
        for (int off = G / 2; off > 0; off >>= 1) t += __shfl_xor_sync(gmask, t, off, G);
        if (sub == 0 && (!TAIL || k0 + u < end)) reinterpret_cast<TC*>(a.dvals)[k0 + u] = (TC)t;
      }
    }
  };
  int64_t k0 = beg;
  if (LOOPS_SDDMM_FULL_BATCHES)
    for (; k0 + U <= end; k0 += U) batch(k0, std::false_type());
  for (; k0 < end; k0 += U) batch(k0, std::true_type());
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
    for (int64_t n = lane; n < a.N; n += 32) {
      TAcc g = Tr::to_acc(dcrow[n]);
      if constexpr (Tr::kScaled) g *= col_weight(a, n);
      s = fma(g, Tr::to_acc(Bp[(int64_t)c * a.ldb + n]), s);
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    if (lane == 0) reinterpret_cast<TC*>(a.dvals)[k] = (TC)s;
  }
}

template <class Tr>
cudaError_t launch_sddmm_t(const loops_plan_s* p, const void* dC, int64_t lddc, const void* B, int64_t ldb,
                           void* dvals, const float* dc_scale, const float* b_scale, cudaStream_t s) {
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
  a.dc_scale = dc_scale;
  a.b_scale = b_scale;
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

cudaError_t launch_sddmm(const loops_plan_s* p, const void* dC, int64_t lddc, const void* B, int64_t ldb,
                         void* dvals, const float* dc_scale, const float* b_scale, cudaStream_t s) {
  switch (p->dtype) {
    case LOOPS_F64: return launch_sddmm_t<TrF64>(p, dC, lddc, B, ldb, dvals, dc_scale, b_scale, s);
    case LOOPS_F32: return launch_sddmm_t<TrF32>(p, dC, lddc, B, ldb, dvals, dc_scale, b_scale, s);
    case LOOPS_F16: return launch_sddmm_t<TrF16>(p, dC, lddc, B, ldb, dvals, dc_scale, b_scale, s);
    case LOOPS_BF16: return launch_sddmm_t<TrBF16>(p, dC, lddc, B, ldb, dvals, dc_scale, b_scale, s);
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
