// Device helpers shared by the kernels: element traits, vector loads, inline PTX wrappers.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace loops {

// Element traits per plan dtype: storage type of A values and B (TB), accumulator (TAcc),
// output (TC), and conversion of a stored element to the accumulator type.
// TV is the register form of an A value in the SpMM inner loops (load_v reads one): the
// accumulator type, or for the 16-bit formats the raw 16 bits, which the mixed-precision FMA
// (fma_vec below) takes as they are.
struct TrF64 {
  using TB = double; using TAcc = double; using TC = double; using TV = double;
  static constexpr bool kScaled = false;  // outputs carry 1/s_A and column scales
  static constexpr int kVE = 2;  // elements per 16-byte vector
  __device__ static __forceinline__ TAcc to_acc(TB x) { return x; }
  __device__ static __forceinline__ TV load_v(const TB* p) { return *p; }
};
struct TrF32 {
  using TB = float; using TAcc = float; using TC = float; using TV = float;
  static constexpr bool kScaled = false;  // outputs carry 1/s_A and column scales
  static constexpr int kVE = 4;
  __device__ static __forceinline__ TAcc to_acc(TB x) { return x; }
  __device__ static __forceinline__ TV load_v(const TB* p) { return *p; }
};
struct TrF16 {
  using TB = __half; using TAcc = float; using TC = float; using TV = uint32_t;
  static constexpr bool kScaled = true;  // outputs carry 1/s_A and column scales
  static constexpr int kVE = 8;
  __device__ static __forceinline__ TAcc to_acc(TB x) { return __half2float(x); }
  __device__ static __forceinline__ TV load_v(const TB* p) {
    return *reinterpret_cast<const unsigned short*>(p);
  }
};
struct TrBF16 {
  using TB = __nv_bfloat16; using TAcc = float; using TC = float; using TV = uint32_t;
  static constexpr bool kScaled = true;  // outputs carry 1/s_A and column scales
  static constexpr int kVE = 8;
  __device__ static __forceinline__ TAcc to_acc(TB x) { return __bfloat162float(x); }
  __device__ static __forceinline__ TV load_v(const TB* p) {
    return *reinterpret_cast<const unsigned short*>(p);
  }
};

// binary64 -> storage type, round to nearest even (the stored-value rounding of a plan).
template <class T>
__device__ __forceinline__ T from_f64(double x);
template <>
__device__ __forceinline__ double from_f64<double>(double x) { return x; }
template <>
__device__ __forceinline__ float from_f64<float>(double x) { return __double2float_rn(x); }
template <>
__device__ __forceinline__ __half from_f64<__half>(double x) { return __double2half(x); }
template <>
__device__ __forceinline__ __nv_bfloat16 from_f64<__nv_bfloat16>(double x) { return __double2bfloat16(x); }

// 16-byte vector of B elements, unpacked to accumulator values.
template <class Tr>
__device__ __forceinline__ void unpack16(const uint4& v, typename Tr::TAcc (&out)[Tr::kVE]);

template <>
__device__ __forceinline__ void unpack16<TrF64>(const uint4& v, double (&out)[2]) {
  out[0] = __hiloint2double((int)v.y, (int)v.x);
  out[1] = __hiloint2double((int)v.w, (int)v.z);
}
template <>
__device__ __forceinline__ void unpack16<TrF32>(const uint4& v, float (&out)[4]) {
  out[0] = __uint_as_float(v.x); out[1] = __uint_as_float(v.y);
  out[2] = __uint_as_float(v.z); out[3] = __uint_as_float(v.w);
}
template <>
__device__ __forceinline__ void unpack16<TrF16>(const uint4& v, float (&out)[8]) {
  const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    __half2 h = *reinterpret_cast<const __half2*>(&w[i]);
    float2 f = __half22float2(h);
    out[2 * i] = f.x; out[2 * i + 1] = f.y;
  }
}
template <>
__device__ __forceinline__ void unpack16<TrBF16>(const uint4& v, float (&out)[8]) {
  const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    // bfloat16 -> float is exact: the 16 bits become the high half of the binary32 pattern
    out[2 * i] = __uint_as_float(w[i] << 16);
    out[2 * i + 1] = __uint_as_float(w[i] & 0xffff0000u);
  }
}

// acc[e] += a * (element e of the 16-byte vector v), one rounding per element. The 16-bit
// formats use the mixed-precision FMA (16-bit operands, binary32 addend and result): the
// product of two 16-bit values is exact in binary32, so this equals converting both operands
// and one binary32 FMA, without the conversions.
template <class Tr>
__device__ __forceinline__ void fma_vec(typename Tr::TAcc (&acc)[Tr::kVE], const uint4& v, typename Tr::TV a) {
  typename Tr::TAcc b[Tr::kVE];
  unpack16<Tr>(v, b);
#pragma unroll
  for (int e = 0; e < Tr::kVE; ++e) acc[e] = fma(a, b[e], acc[e]);
}
template <>
__device__ __forceinline__ void fma_vec<TrF16>(float (&acc)[8], const uint4& v, uint32_t a) {
  const unsigned short a16 = (unsigned short)a;
  const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
  for (int i = 0; i < 4; ++i)
    asm("{\n\t.reg .f16 lo, hi;\n\tmov.b32 {lo, hi}, %2;\n\t"
        "fma.rn.f32.f16 %0, lo, %3, %0;\n\tfma.rn.f32.f16 %1, hi, %3, %1;\n\t}"
        : "+f"(acc[2 * i]), "+f"(acc[2 * i + 1])
        : "r"(w[i]), "h"(a16));
}
template <>
__device__ __forceinline__ void fma_vec<TrBF16>(float (&acc)[8], const uint4& v, uint32_t a) {
  const unsigned short a16 = (unsigned short)a;
  const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
  for (int i = 0; i < 4; ++i)
    asm("{\n\t.reg .b16 lo, hi;\n\tmov.b32 {lo, hi}, %2;\n\t"
        "fma.rn.f32.bf16 %0, lo, %3, %0;\n\tfma.rn.f32.bf16 %1, hi, %3, %1;\n\t}"
        : "+f"(acc[2 * i]), "+f"(acc[2 * i + 1])
        : "r"(w[i]), "h"(a16));
}

__device__ __forceinline__ uint4 ldg16(const void* p) {
  uint4 r;
  asm volatile("ld.global.nc.v4.u32 {%0,%1,%2,%3}, [%4];"
               : "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w) : "l"(p));
  return r;
}

// 16-byte load under a predicate, zeros when it is off: no branch, so a batch of them issues
// back to back like unpredicated loads
__device__ __forceinline__ uint4 ldg16_if(bool on, const void* p) {
  uint4 r = make_uint4(0, 0, 0, 0);
  asm volatile(
      "{\n\t.reg .pred q;\n\tsetp.ne.b32 q, %4, 0;\n\t"
      "@q ld.global.nc.v4.u32 {%0,%1,%2,%3}, [%5];\n\t}"
      : "+r"(r.x), "+r"(r.y), "+r"(r.z), "+r"(r.w)
      : "r"((int)on), "l"(p));
  return r;
}

// ------------------------------------------------------------------ mbarrier / bulk copy
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count));
}

__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;"
               ::"r"(smem_addr(bar)), "r"(bytes) : "memory");
}

// One bulk copy global -> shared (the TMA engine), completing on `bar` with `bytes`.
// dst, src 16-byte aligned; bytes a multiple of 16.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
      ::"r"(smem_addr(dst)), "l"(src), "r"(bytes), "r"(smem_addr(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok) : "r"(smem_addr(bar)), "r"(parity) : "memory");
  return ok != 0;
}

// Bounded wait: returns false after `max_polls` unsuccessful polls.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, long long max_polls) {
  for (long long i = 0; i < max_polls; ++i) {
    if (mbar_try_wait(bar, parity)) return true;
    if (i > 64) __nanosleep(64);
  }
  return false;
}

}  // namespace loops
