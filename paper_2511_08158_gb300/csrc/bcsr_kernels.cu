// BCSR-part SpMM: the outer-product tile kernel of Algorithms 2 and 3, on tensor cores.
//
// A row block of B_r rows holds tiles (B_r x 1 columns of A, one per distinct column) padded
// to a multiple of the MMA K. Kernels run over work units (a block, or a K-aligned range of a
// block with very many tiles, whose partial sums a last kernel adds in a fixed order). One K-group of tiles against the matching K gathered rows of B
// is one MMA: the paper's sum of rank-1 updates (fmopa) of a B_r x 1 tile with a 1 x N row
// of B becomes a B_r x K by K x 8 product. Accumulators stay in registers for the whole row
// block and are stored once (C = A.B overwrites C).
//
//   F16/BF16  mma.sync m16n8k16, f32 accumulate (the 2-way widening fmopa of Algorithm 3).
//             The 16 B rows of a group are staged in shared memory by bulk copies of the
//             TMA engine (cp.async.bulk + mbarrier, a ring of stages) and transposed into B
//             fragments with ldmatrix.trans; padded tiles (col -1) are zero rows.
//   F64       mma.sync m8n8k4 (DMMA). A lane's B fragment is one element, so B is read
//             straight from global memory with 16-byte loads, two N-fragments per load.
//   F32       CUDA-core register-blocked outer product (TF32 MMA would not meet FP32
//             accuracy): a group of lanes owns B_r x 4*G outputs and updates them per tile.
#include "device_common.cuh"
#include "loops_internal.h"

namespace loops {

namespace {

struct BcsrKArgs {
  const int32_t* rb_id;
  const int64_t* rb_ptr;
  const int32_t* tile_col;
  const void* tile_val;
  const int32_t* unit_block;
  const int64_t* unit_t0;
  const int64_t* unit_t1;
  const int32_t* unit_slot;
  int64_t n_units;
  void* scratch;           // partial sums of units of split blocks: [slot][B_r][N]
  const void* B;
  int64_t ldb;
  void* C;
  int64_t ldc;
  const float* col_scale;
  float inv_scale_f;
  double inv_scale_d;
  int64_t N;
  int64_t n_rows;
  int32_t* err;
  long long max_polls;     // bound of each mbarrier wait (kMaxWaitPolls unless a test lowers it)
};

// ------------------------------------------------------------------ F16 / BF16: m16n8k16
template <class T>
__device__ __forceinline__ void mma16816(float (&d)[4], const uint4& a, uint32_t b0, uint32_t b1);

template <>
__device__ __forceinline__ void mma16816<__half>(float (&d)[4], const uint4& a, uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a.x), "r"(a.y), "r"(a.z), "r"(a.w), "r"(b0), "r"(b1));
}
template <>
__device__ __forceinline__ void mma16816<__nv_bfloat16>(float (&d)[4], const uint4& a, uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a.x), "r"(a.y), "r"(a.z), "r"(a.w), "r"(b0), "r"(b1));
}

__device__ __forceinline__ void ldsm_x4_trans(uint32_t addr, uint32_t& r0, uint32_t& r1, uint32_t& r2, uint32_t& r3) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];"
               : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3) : "r"(addr));
}
__device__ __forceinline__ void ldsm_x2_trans(uint32_t addr, uint32_t& r0, uint32_t& r1) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x2.trans.shared.b16 {%0,%1}, [%2];"
               : "=r"(r0), "=r"(r1) : "r"(addr));
}

constexpr int kStages = 4;

// WARPS warps, each owning NF n8-fragments: the CTA covers CT = WARPS * 8 * NF columns of one
// row block. BULK: B rows are fetched with cp.async.bulk (needs 16-byte aligned rows and a
// multiple-of-8 N); otherwise the threads copy them element-wise.
template <class T, int WARPS, int NF, bool BULK>
__global__ void __launch_bounds__(WARPS * 32) bcsr_hmma(BcsrKArgs a) {
  constexpr int CT = WARPS * 8 * NF;
  constexpr int RS = CT + 8;  // smem row stride in elements (+16 B: conflict-free ldmatrix)
  __shared__ __align__(128) T sB[kStages][16][RS];
  __shared__ __align__(8) uint64_t bar[kStages];
  const int tid = threadIdx.x;
  const int warp = tid >> 5, lane = tid & 31;
  const int64_t u = blockIdx.x;
  const int32_t b = a.unit_block[u];
  const int64_t rb = a.rb_id[b];
  const int64_t t0 = a.unit_t0[u];
  const int n_groups = (int)((a.unit_t1[u] - t0) / 16);
  const int32_t slot = a.unit_slot[u];
  const int64_t n0 = (int64_t)blockIdx.y * CT;
  const int width = (int)(a.N - n0 < (int64_t)CT ? a.N - n0 : (int64_t)CT);  // valid columns in this tile
  const T* Bp = reinterpret_cast<const T*>(a.B);
  const uint4* Af = reinterpret_cast<const uint4*>(a.tile_val) + (t0 / 16) * 32;
  const int32_t* cols = a.tile_col + t0;

  if (BULK && tid == 0) {
    for (int s = 0; s < kStages; ++s) mbar_init(&bar[s], 1);
    fence_mbar_init();
  }
  __syncthreads();

  // stage g: B rows of tiles g*16 .. g*16+15 into sB[g % kStages]. With bulk copies, lane k
  // of warp 0 (k < 16) fetches row k: a padding tile's row (column -1) is zero-filled by its
  // lane first, then lane 0 announces the stage's total bytes on its barrier (its arrival
  // releases the zero rows to the waiting threads), then the lanes issue their copies at once.
  auto issue = [&](int g) {
    const int s = g % kStages;
    if (BULK) {
      if (warp == 0) {
        const uint32_t row_bytes = (uint32_t)width * sizeof(T);
        const int32_t c = lane < 16 ? cols[g * 16 + lane] : -1;
        if (lane < 16 && c < 0) {
          uint4* z = reinterpret_cast<uint4*>(&sB[s][lane][0]);
          for (int q = 0; q < CT * (int)sizeof(T) / 16; ++q) z[q] = make_uint4(0, 0, 0, 0);
        }
        const uint32_t bytes = __reduce_add_sync(0xffffffffu, (lane < 16 && c >= 0) ? row_bytes : 0u);
        __syncwarp();
        if (lane == 0) mbar_arrive_expect_tx(&bar[s], bytes);
        __syncwarp();
        if (lane < 16 && c >= 0) {
          fence_proxy_async_smem();
          bulk_g2s(&sB[s][lane][0], Bp + (int64_t)c * a.ldb + n0, row_bytes, &bar[s]);
        }
      }
    } else {
      for (int i = tid; i < 16 * CT; i += WARPS * 32) {
        const int k = i / CT, n = i % CT;
        const int32_t c = cols[g * 16 + k];
        sB[s][k][n] = (c >= 0 && n < width) ? Bp[(int64_t)c * a.ldb + n0 + n] : T(0.f);
      }
    }
  };

  float acc[NF][4];
#pragma unroll
  for (int f = 0; f < NF; ++f)
#pragma unroll
    for (int i = 0; i < 4; ++i) acc[f][i] = 0.f;

  bool failed = false;
  int fail_g = -1;
  const int pre = min(n_groups, kStages - 1);
  for (int g = 0; g < pre; ++g) issue(g);
  for (int g = 0; g < n_groups; ++g) {
    // every warp is done with stage (g - 1) % kStages; a failed wait anywhere stops the CTA
    if (__syncthreads_or(failed)) { fail_g = g - 1; break; }
    if (g + kStages - 1 < n_groups) issue(g + kStages - 1);
    if (!BULK) __syncthreads();
    const int s = g % kStages;
    if (BULK && !mbar_wait_bounded(&bar[s], (uint32_t)((g / kStages) & 1), a.max_polls)) {
      failed = true;
      atomicOr(a.err, kErrWaitTimeout);
      continue;
    }
    const uint4 af = __ldg(Af + (int64_t)g * 32 + lane);
    // lanes 0-7 / 8-15 / 16-23 / 24-31 address rows k of the four 8x8 matrices:
    // (k 0-7, frag f), (k 8-15, frag f), (k 0-7, frag f+1), (k 8-15, frag f+1)
    const int mi = lane >> 3, r = lane & 7;
#pragma unroll
    for (int f = 0; f < NF; f += 2) {
      const int ncol = (warp * NF + f) * 8;
      if (f + 1 < NF) {
        const uint32_t addr = smem_addr(&sB[s][r + 8 * (mi & 1)][ncol + 8 * (mi >> 1)]);
        uint32_t b0, b1, b2, b3;
        ldsm_x4_trans(addr, b0, b1, b2, b3);
        mma16816<T>(acc[f], af, b0, b1);
        mma16816<T>(acc[f + 1], af, b2, b3);
      } else {
        const uint32_t addr = smem_addr(&sB[s][r + 8 * (mi & 1)][ncol]);
        uint32_t b0, b1;
        ldsm_x2_trans(addr, b0, b1);
        mma16816<T>(acc[f], af, b0, b1);
      }
    }
  }
  if (__syncthreads_or(failed) && fail_g < 0) fail_g = n_groups - 1;
  if (BULK && fail_g >= 0) {
    // a wait gave up: before leaving, let every copy that may still be in flight into this
    // CTA's shared memory land (bounded), then skip the store
    if (tid == 0) {
      const int last = min(n_groups - 1, fail_g + kStages - 1);
      for (int g = fail_g; g <= last; ++g) mbar_wait_bounded(&bar[g % kStages], (uint32_t)((g / kStages) & 1), 1 << 20);
    }
    __syncthreads();
    return;
  }
  // epilogue: acc[f] = C rows (q, q + 8) x columns (2t, 2t + 1) of fragment f
  const int q = lane >> 2, t = lane & 3;
  float* C = reinterpret_cast<float*>(a.C);
  const bool vec2 = ((a.ldc & 1) == 0) && (((uintptr_t)a.C & 7) == 0);
  if (slot >= 0) {  // one unit of a split block: unscaled partial sums
    float* P = reinterpret_cast<float*>(a.scratch) + (int64_t)slot * 16 * a.N;
#pragma unroll
    for (int f = 0; f < NF; ++f) {
      const int64_t n = n0 + (warp * NF + f) * 8 + 2 * t;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        float* pp = P + (int64_t)(q + 8 * h) * a.N + n;
        if (n < a.N) pp[0] = acc[f][2 * h];
        if (n + 1 < a.N) pp[1] = acc[f][2 * h + 1];
      }
    }
    return;
  }
#pragma unroll
  for (int f = 0; f < NF; ++f) {
    const int64_t n = n0 + (warp * NF + f) * 8 + 2 * t;
    float s0 = a.inv_scale_f, s1 = a.inv_scale_f;
    if (a.col_scale) {
      if (n < a.N) s0 *= a.col_scale[n];
      if (n + 1 < a.N) s1 *= a.col_scale[n + 1];
    }
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int64_t row = rb * 16 + q + 8 * h;
      if (row >= a.n_rows) continue;
      float* cp = C + row * a.ldc + n;
      const float v0 = acc[f][2 * h] * s0, v1 = acc[f][2 * h + 1] * s1;
      if (vec2 && n + 1 < a.N) {
        *reinterpret_cast<float2*>(cp) = make_float2(v0, v1);
      } else {
        if (n < a.N) cp[0] = v0;
        if (n + 1 < a.N) cp[1] = v1;
      }
    }
  }
}

template <class T, int WARPS, int NF>
cudaError_t launch_hmma_cfg(const BcsrKArgs& a, bool bulk, cudaStream_t s) {
  constexpr int CT = WARPS * 8 * NF;
  dim3 grid((unsigned)a.n_units, (unsigned)((a.N + CT - 1) / CT));
  if (bulk) bcsr_hmma<T, WARPS, NF, true><<<grid, WARPS * 32, 0, s>>>(a);
  else bcsr_hmma<T, WARPS, NF, false><<<grid, WARPS * 32, 0, s>>>(a);
  return cudaGetLastError();
}

// Column tile of a CTA: the plan's bcsr_ntile when the autotuner set it (32, 64 or 128), else
// the smallest of 8 .. 128 that covers N.
template <class T>
cudaError_t launch_hmma(const BcsrKArgs& a, int ntile, cudaStream_t s) {
  const bool bulk = (a.N % 8 == 0) && ((uintptr_t)a.B % 16 == 0) && ((a.ldb * 2) % 16 == 0);
  const int64_t ct = ntile > 0 ? ntile : (a.N <= 8 ? 8 : a.N <= 16 ? 16 : a.N <= 32 ? 32 : a.N <= 64 ? 64 : 128);
  if (ct <= 8) return launch_hmma_cfg<T, 1, 1>(a, bulk, s);
  if (ct <= 16) return launch_hmma_cfg<T, 1, 2>(a, bulk, s);
  if (ct <= 32) return launch_hmma_cfg<T, 2, 2>(a, bulk, s);
  if (ct <= 64) return launch_hmma_cfg<T, 4, 2>(a, bulk, s);
  return launch_hmma_cfg<T, 4, 4>(a, bulk, s);
}

// ------------------------------------------------------------------ F64: m8n8k4 DMMA
__device__ __forceinline__ void dmma884(double (&d)[2], double a, double b) {
  asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};"
               : "+d"(d[0]), "+d"(d[1]) : "d"(a), "d"(b));
}

// One warp per (row block, 16*NP columns). Lane (q, t) = (lane / 4, lane % 4) holds A[q][t] of
// the group and loads B[col_t][n0 + 16p + 2q .. +1]: the "even" fragment takes column
// 16p + 2q as its n = q, the "odd" one 16p + 2q + 1. The outputs of lane (q, t) are then the
// four consecutive columns 16p + 4t .. 16p + 4t + 3 of row q.
template <int NP>
__global__ void __launch_bounds__(128) bcsr_dmma(BcsrKArgs a) {
  const int lane = threadIdx.x & 31;
  const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t n_ct = (a.N + 16 * NP - 1) / (16 * NP);
  if (wid >= a.n_units * n_ct) return;
  const int64_t u = wid / n_ct;
  const int64_t n0 = (wid % n_ct) * (16 * NP);
  const int32_t b = a.unit_block[u];
  const int64_t rb = a.rb_id[b];
  const int64_t t0 = a.unit_t0[u];
  const int n_groups = (int)((a.unit_t1[u] - t0) / 4);
  const int32_t slot = a.unit_slot[u];
  const int q = lane >> 2, t = lane & 3;
  const double* Av = reinterpret_cast<const double*>(a.tile_val) + t0 * 8;
  const double* Bp = reinterpret_cast<const double*>(a.B);
  const bool vec = ((a.ldb & 1) == 0) && (((uintptr_t)a.B & 15) == 0);
  double acc[NP][2][2];
#pragma unroll
  for (int p = 0; p < NP; ++p)
#pragma unroll
    for (int h = 0; h < 2; ++h) acc[p][h][0] = acc[p][h][1] = 0.0;
  for (int g = 0; g < n_groups; ++g) {
    const double av = __ldg(Av + g * 32 + lane);
    const int32_t c = __ldg(a.tile_col + t0 + g * 4 + t);
    const double* brow = Bp + (int64_t)(c >= 0 ? c : 0) * a.ldb;
#pragma unroll
    for (int p = 0; p < NP; ++p) {
      const int64_t n = n0 + 16 * p + 2 * q;
      double b0 = 0.0, b1 = 0.0;
      if (c >= 0) {
        if (vec && n + 1 < a.N) {
          const uint4 v = ldg16(brow + n);
          b0 = __hiloint2double((int)v.y, (int)v.x);
          b1 = __hiloint2double((int)v.w, (int)v.z);
        } else {
          if (n < a.N) b0 = __ldg(brow + n);
          if (n + 1 < a.N) b1 = __ldg(brow + n + 1);
        }
      }
      dmma884(acc[p][0], av, b0);
      dmma884(acc[p][1], av, b1);
    }
  }
  if (slot >= 0) {  // one unit of a split block: partial sums of its 8 rows
    double* prow = reinterpret_cast<double*>(a.scratch) + ((int64_t)slot * 8 + q) * a.N;
#pragma unroll
    for (int p = 0; p < NP; ++p) {
      const int64_t n = n0 + 16 * p + 4 * t;
      const double o[4] = {acc[p][0][0], acc[p][1][0], acc[p][0][1], acc[p][1][1]};
#pragma unroll
      for (int i = 0; i < 4; ++i)
        if (n + i < a.N) prow[n + i] = o[i];
    }
    return;
  }
  const int64_t row = rb * 8 + q;
  if (row >= a.n_rows) return;
  double* crow = reinterpret_cast<double*>(a.C) + row * a.ldc;
  const bool cvec = ((a.ldc & 1) == 0) && (((uintptr_t)a.C & 15) == 0);
#pragma unroll
  for (int p = 0; p < NP; ++p) {
    const int64_t n = n0 + 16 * p + 4 * t;
    const double o[4] = {acc[p][0][0] * a.inv_scale_d, acc[p][1][0] * a.inv_scale_d,
                         acc[p][0][1] * a.inv_scale_d, acc[p][1][1] * a.inv_scale_d};
    if (cvec && n + 3 < a.N) {
      *reinterpret_cast<double2*>(crow + n) = make_double2(o[0], o[1]);
      *reinterpret_cast<double2*>(crow + n + 2) = make_double2(o[2], o[3]);
    } else {
#pragma unroll
      for (int i = 0; i < 4; ++i)
        if (n + i < a.N) crow[n + i] = o[i];
    }
  }
}

cudaError_t launch_dmma(const BcsrKArgs& a, cudaStream_t s) {
  auto go = [&](auto np_tag) {
    constexpr int NP = decltype(np_tag)::value;
    const int64_t n_ct = (a.N + 16 * NP - 1) / (16 * NP);
    const int64_t warps = a.n_units * n_ct;
    bcsr_dmma<NP><<<(unsigned)((warps + 3) / 4), 128, 0, s>>>(a);
    return cudaGetLastError();
  };
  if (a.N <= 16) return go(std::integral_constant<int, 1>());
  if (a.N <= 32) return go(std::integral_constant<int, 2>());
  return go(std::integral_constant<int, 4>());
}

// ------------------------------------------------------------------ F32: CUDA-core outer product
// A group of G lanes owns one work unit (tiles of a row block) and VE*G columns (a float4 per
// lane, or one float). The group reads G tile columns at once and broadcasts them with
// shuffles; LOOPS_FFMA_BATCH tiles' B loads are kept in flight before their FMAs. Per tile a
// lane loads the B_r tile values (the same 64 bytes for the whole group: an L1 broadcast) and
// does B_r * VE FMAs.
#ifndef LOOPS_FFMA_BATCH
#define LOOPS_FFMA_BATCH 4
#endif
template <int BR, int G, bool VEC>
__global__ void __launch_bounds__(256) bcsr_ffma(BcsrKArgs a) {
  constexpr int VE = VEC ? 4 : 1;
  constexpr int U = LOOPS_FFMA_BATCH;
  const int lane = threadIdx.x & 31;
  const int sub = lane & (G - 1);
  const unsigned gmask = (G == 32) ? 0xffffffffu : (((1u << G) - 1u) << (lane & ~(G - 1)));
  const int64_t gid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / G;
  const int64_t n_ct = (a.N + G * VE - 1) / (G * VE);
  if (gid >= a.n_units * n_ct) return;  // a group leaves as a whole
  const int64_t u = gid / n_ct;
  const int64_t n = (gid % n_ct) * (G * VE) + (int64_t)sub * VE;
  const int32_t b = a.unit_block[u];
  const int64_t rb = a.rb_id[b];
  const int64_t t0 = a.unit_t0[u], t1 = a.unit_t1[u];
  const int32_t slot = a.unit_slot[u];
  const float* Av = reinterpret_cast<const float*>(a.tile_val);
  const float* Bp = reinterpret_cast<const float*>(a.B);
  float acc[BR][VE];
#pragma unroll
  for (int r = 0; r < BR; ++r)
#pragma unroll
    for (int e = 0; e < VE; ++e) acc[r][e] = 0.f;
  const bool colok = n < a.N;
  for (int64_t k0 = t0; k0 < t1; k0 += G) {
    const int32_t cmine = k0 + sub < t1 ? __ldg(a.tile_col + k0 + sub) : -1;
    const int cnt = (int)(t1 - k0 < (int64_t)G ? t1 - k0 : (int64_t)G);  // uniform in the group
    for (int j0 = 0; j0 < cnt; j0 += U) {
      float bv[U][VE];
#pragma unroll
      for (int q = 0; q < U; ++q) {
        const int32_t c = __shfl_sync(gmask, cmine, (j0 + q) & (G - 1), G);
        const bool ok = colok && j0 + q < cnt && c >= 0;
        if (VEC) {
          const uint4 v = ok ? ldg16(Bp + (int64_t)c * a.ldb + n) : make_uint4(0, 0, 0, 0);
          bv[q][0] = __uint_as_float(v.x);
          if (VE > 1) {
            bv[q][1 % VE] = __uint_as_float(v.y);
            bv[q][2 % VE] = __uint_as_float(v.z);
            bv[q][3 % VE] = __uint_as_float(v.w);
          }
        } else {
          bv[q][0] = ok ? __ldg(Bp + (int64_t)c * a.ldb + n) : 0.f;
        }
      }
#pragma unroll
      for (int q = 0; q < U; ++q) {
        if (j0 + q >= cnt) break;  // uniform in the group: no FMA on a slot past the unit
        const int64_t tt = k0 + j0 + q;
        float av[BR];
#pragma unroll
        for (int r4 = 0; r4 < BR / 4; ++r4) {
          const uint4 v = ldg16(Av + tt * BR + r4 * 4);
          av[r4 * 4 + 0] = __uint_as_float(v.x);
          av[r4 * 4 + 1] = __uint_as_float(v.y);
          av[r4 * 4 + 2] = __uint_as_float(v.z);
          av[r4 * 4 + 3] = __uint_as_float(v.w);
        }
#pragma unroll
        for (int r = 0; r < BR; ++r)
#pragma unroll
          for (int e = 0; e < VE; ++e) acc[r][e] = fmaf(av[r], bv[q][e], acc[r][e]);
      }
    }
  }
  if (!colok) return;
  if (slot >= 0) {  // one unit of a split block: partial sums of its BR rows
    float* P = reinterpret_cast<float*>(a.scratch) + (int64_t)slot * BR * a.N;
#pragma unroll
    for (int r = 0; r < BR; ++r)
#pragma unroll
      for (int e = 0; e < VE; ++e) P[(int64_t)r * a.N + n + e] = acc[r][e];
    return;
  }
  float* C = reinterpret_cast<float*>(a.C);
#pragma unroll
  for (int r = 0; r < BR; ++r) {
    const int64_t row = rb * BR + r;
    if (row >= a.n_rows) break;
    float* cp = C + row * a.ldc + n;
    if (VEC) {
      *reinterpret_cast<float4*>(cp) = make_float4(acc[r][0], acc[r][1 % VE], acc[r][2 % VE], acc[r][3 % VE]);
    } else {
      cp[0] = acc[r][0];
    }
  }
}

template <int BR>
cudaError_t launch_ffma_br(const BcsrKArgs& a, cudaStream_t s) {
  const bool vec = (a.N % 4 == 0) && ((uintptr_t)a.B % 16 == 0) && ((uintptr_t)a.C % 16 == 0) &&
                   (a.ldb % 4 == 0) && (a.ldc % 4 == 0);
  auto go = [&](auto g_tag, auto v_tag) {
    constexpr int G = decltype(g_tag)::value;
    constexpr bool V = decltype(v_tag)::value;
    constexpr int VE = V ? 4 : 1;
    const int64_t n_ct = (a.N + G * VE - 1) / (G * VE);
    const int64_t threads = a.n_units * n_ct * G;
    bcsr_ffma<BR, G, V><<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(a);
    return cudaGetLastError();
  };
  if (!vec) return go(std::integral_constant<int, 32>(), std::false_type());
  const int64_t nvec = a.N / 4;
  if (nvec <= 1) return go(std::integral_constant<int, 1>(), std::true_type());
  if (nvec <= 2) return go(std::integral_constant<int, 2>(), std::true_type());
  if (nvec <= 4) return go(std::integral_constant<int, 4>(), std::true_type());
  if (nvec <= 8) return go(std::integral_constant<int, 8>(), std::true_type());
  if (nvec <= 16) return go(std::integral_constant<int, 16>(), std::true_type());
  return go(std::integral_constant<int, 32>(), std::true_type());
}

// Blocks cut into several units: C rows = scale * sum of the units' partials, in slot order.
template <class TAcc, class TC, bool SCALED>
__global__ void __launch_bounds__(256) bcsr_split_reduce(const int32_t* __restrict__ split_block,
                                                         const int32_t* __restrict__ slot_ptr, int32_t br,
                                                         BcsrKArgs a) {
  const int64_t sidx = blockIdx.x;
  const int32_t b = split_block[sidx];
  const int64_t rb = a.rb_id[b];
  const int32_t s0 = slot_ptr[sidx], s1 = slot_ptr[sidx + 1];
  const TAcc* P = reinterpret_cast<const TAcc*>(a.scratch);
  const int64_t total = (int64_t)br * a.N;
  for (int64_t i = (int64_t)blockIdx.y * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.y * blockDim.x) {
    const int64_t r = i / a.N, n = i - r * a.N;
    const int64_t row = rb * br + r;
    if (row >= a.n_rows) continue;
    TAcc acc = TAcc(0);
    for (int32_t q = s0; q < s1; ++q) acc += P[((int64_t)q * br + r) * a.N + n];
    if (SCALED) {
      const float sc = a.col_scale ? a.col_scale[n] * a.inv_scale_f : a.inv_scale_f;
      reinterpret_cast<TC*>(a.C)[row * a.ldc + n] = (TC)(acc * sc);
    } else {
      reinterpret_cast<TC*>(a.C)[row * a.ldc + n] = (TC)acc;
    }
  }
}

}  // namespace

cudaError_t launch_bcsr(const loops_plan_s* p, const BcsrDev& d, const DenseArgs& da, cudaStream_t s) {
  if (d.n_rb == 0) return cudaSuccess;
  BcsrKArgs a;
  a.rb_id = d.rb_id;
  a.rb_ptr = d.rb_ptr;
  a.tile_col = d.tile_col;
  a.tile_val = d.tile_val;
  a.unit_block = d.unit_block;
  a.unit_t0 = d.unit_t0;
  a.unit_t1 = d.unit_t1;
  a.unit_slot = d.unit_slot;
  a.n_units = d.n_units;
  a.scratch = d.scratch;
  a.B = da.B;
  a.ldb = da.ldb;
  a.C = da.C;
  a.ldc = da.ldc;
  a.col_scale = da.col_scale;
  a.inv_scale_f = da.inv_scale_f;
  a.inv_scale_d = da.inv_scale_d;
  a.N = da.N;
  a.n_rows = da.n_rows;
  a.err = p->d_error;
  a.max_polls = wait_poll_limit();
  cudaError_t e = cudaErrorInvalidValue;
  switch (p->dtype) {
    case LOOPS_F64: e = launch_dmma(a, s); break;
    case LOOPS_F32: e = p->br == 8 ? launch_ffma_br<8>(a, s) : launch_ffma_br<16>(a, s); break;
    case LOOPS_F16: e = launch_hmma<__half>(a, p->bcsr_ntile, s); break;
    case LOOPS_BF16: e = launch_hmma<__nv_bfloat16>(a, p->bcsr_ntile, s); break;
  }
  if (e != cudaSuccess || d.n_split == 0) return e;
  dim3 grid((unsigned)d.n_split, (unsigned)std::min<int64_t>((p->br * a.N + 255) / 256, 64));
  switch (p->dtype) {
    case LOOPS_F64:
      bcsr_split_reduce<double, double, false><<<grid, 256, 0, s>>>(d.split_block, d.split_slot_ptr, p->br, a);
      break;
    case LOOPS_F32:
      bcsr_split_reduce<float, float, false><<<grid, 256, 0, s>>>(d.split_block, d.split_slot_ptr, p->br, a);
      break;
    default:
      bcsr_split_reduce<float, float, true><<<grid, 256, 0, s>>>(d.split_block, d.split_slot_ptr, p->br, a);
      break;
  }
  return cudaGetLastError();
}

}  // namespace loops
