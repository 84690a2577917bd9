// Host side of the plan: CSR validation, number-format rounding, Algorithm 1 with the
// structural split (canonical partition), and the device layout of both parts.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <thread>

#include "loops_internal.h"

namespace loops {

// ------------------------------------------------------------------ number formats
// Round a binary64 value into a binary format with `mant` stored significand bits, minimum
// normal exponent `emin` and exponent bias `bias` (round to nearest, ties to even), returning
// the target's bit pattern (sign | exponent | fraction). Written from IEEE 754's definition:
// the quantum of the result is 2^(max(E, emin) - mant) for the input's exponent E.
static uint32_t round_binary(double x, int mant, int emin, int bias, int exp_bits) {
  uint64_t b;
  std::memcpy(&b, &x, 8);
  const uint32_t sign = (uint32_t)(b >> 63) << (mant + exp_bits);
  const int e = (int)((b >> 52) & 0x7FF);
  const uint64_t m = b & ((1ull << 52) - 1);
  const uint32_t inf_bits = ((1u << exp_bits) - 1) << mant;
  if (e == 0x7FF) return sign | inf_bits | (m ? (1u << (mant - 1)) : 0u);
  if (e == 0 && m == 0) return sign;
  const int E = e ? e - 1023 : -1022;                 // unbiased exponent of 1.m (or 0.m)
  const uint64_t sig = e ? (m | (1ull << 52)) : m;    // value = sig * 2^(E - 52)
  const int qexp = (E < emin ? emin : E) - mant;      // quantum exponent
  const int shift = qexp - (E - 52);                  // bits of sig below the quantum
  uint64_t q;
  if (shift >= 64) {
    q = 0;                                            // below half a quantum
  } else if (shift <= 0) {
    q = sig << (-shift);
  } else {
    q = sig >> shift;
    const uint64_t rem = sig & ((1ull << shift) - 1);
    const uint64_t half = 1ull << (shift - 1);
    if (rem > half || (rem == half && (q & 1))) ++q;
  }
  // q * 2^qexp. Subnormal range (E < emin): the pattern is q itself (q = 2^mant carries into
  // the smallest normal). Normal range: biased exponent field plus the fraction; a carry to
  // 2^(mant+1) moves into the next exponent seamlessly.
  uint64_t bits;
  if (E < emin) {
    bits = q;
  } else {
    bits = ((uint64_t)(E + bias) << mant) + (q - (1ull << mant));
  }
  if (bits >= inf_bits) bits = inf_bits;              // overflow rounds to infinity
  return sign | (uint32_t)bits;
}

uint16_t f64_to_f16_bits(double x) { return (uint16_t)round_binary(x, 10, -14, 15, 5); }
uint16_t f64_to_bf16_bits(double x) { return (uint16_t)round_binary(x, 7, -126, 127, 8); }

static double decode_binary(uint32_t h, int mant, int bias, int exp_bits) {
  const bool neg = (h >> (mant + exp_bits)) & 1;
  const int e = (int)((h >> mant) & ((1u << exp_bits) - 1));
  const uint32_t f = h & ((1u << mant) - 1);
  double v;
  if (e == (1 << exp_bits) - 1) {
    v = f ? NAN : INFINITY;
  } else if (e == 0) {
    v = std::ldexp((double)f, 1 - bias - mant);
  } else {
    v = std::ldexp((double)(f | (1u << mant)), e - bias - mant);
  }
  return neg ? -v : v;
}

double f16_bits_to_f64(uint16_t h) { return decode_binary(h, 10, 15, 5); }
double bf16_bits_to_f64(uint16_t h) { return decode_binary(h, 7, 127, 8); }

double round_store(double v, double scale, loops_dtype d) {
  const double x = v * scale;
  switch (d) {
    case LOOPS_F64: return x;
    case LOOPS_F32: return (double)(float)x;
    case LOOPS_F16: return f16_bits_to_f64(f64_to_f16_bits(x));
    case LOOPS_BF16: return bf16_bits_to_f64(f64_to_bf16_bits(x));
  }
  return x;
}

double plan_scale_for(const double* vals, int64_t nnz, loops_dtype d) {
  if (d != LOOPS_F16 && d != LOOPS_BF16) return 1.0;
  double mx = 0.0;
  for (int64_t k = 0; k < nnz; ++k) {
    const double a = std::fabs(vals[k]);
    if (std::isfinite(a) && a > mx) mx = a;
  }
  if (mx == 0.0) return 1.0;
  int e2;
  const double f = std::frexp(mx, &e2);               // mx = f * 2^e2, f in [0.5, 1)
  const int c = (f == 0.5) ? e2 - 1 : e2;             // ceil(log2 mx)
  return std::ldexp(1.0, 14 - c);
}

// ------------------------------------------------------------------ validation
loops_status validate_csr(const loops_csr* A) {
  if (!A) { set_error("A is NULL"); return LOOPS_ERR_INVALID_ARG; }
  if (A->n_rows < 0 || A->n_cols < 0 || A->nnz < 0) {
    set_error("negative matrix size");
    return LOOPS_ERR_INVALID_ARG;
  }
  if (A->n_rows >= (int64_t)INT32_MAX || A->n_cols >= (int64_t)INT32_MAX) {
    set_error("n_rows and n_cols must be below 2^31 - 1");
    return LOOPS_ERR_UNSUPPORTED;
  }
  if (!A->row_ptr || (A->nnz > 0 && (!A->col_idx || !A->vals))) {
    set_error("CSR array pointer is NULL");
    return LOOPS_ERR_INVALID_ARG;
  }
  if (A->vals_dtype != LOOPS_F64 && A->vals_dtype != LOOPS_F32) {
    set_error("A values must be LOOPS_F64 or LOOPS_F32 on input");
    return LOOPS_ERR_UNSUPPORTED;
  }
  if (A->row_ptr[0] != 0) { set_error("row_ptr[0] != 0"); return LOOPS_ERR_INVALID_CSR; }
  for (int64_t i = 0; i < A->n_rows; ++i) {
    if (A->row_ptr[i + 1] < A->row_ptr[i]) {
      set_error("row_ptr is not non-decreasing at row " + std::to_string(i));
      return LOOPS_ERR_INVALID_CSR;
    }
  }
  if (A->row_ptr[A->n_rows] != A->nnz) {
    set_error("row_ptr[n_rows] != nnz");
    return LOOPS_ERR_INVALID_CSR;
  }
  for (int64_t k = 0; k < A->nnz; ++k) {
    const int32_t c = A->col_idx[k];
    if (c < 0 || (int64_t)c >= A->n_cols) {
      set_error("column index out of range at entry " + std::to_string(k));
      return LOOPS_ERR_INVALID_CSR;
    }
  }
  return LOOPS_OK;
}

void read_vals_f64(const loops_csr* A, std::vector<double>& out) {
  out.resize((size_t)A->nnz);
  if (A->vals_dtype == LOOPS_F64) {
    if (A->nnz) std::memcpy(out.data(), A->vals, (size_t)A->nnz * 8);
  } else {
    const float* v = (const float*)A->vals;
    for (int64_t k = 0; k < A->nnz; ++k) out[(size_t)k] = (double)v[k];
  }
}

// ------------------------------------------------------------------ Algorithm 1
namespace {

struct Ent {
  int32_t col;
  int32_t r;
  int64_t k;
};

struct Chunk {  // partition of a contiguous range of row blocks
  std::vector<int32_t> csr_rows;
  std::vector<int64_t> csr_len;
  std::vector<int32_t> csr_col;
  std::vector<double> csr_val;
  std::vector<int64_t> csr_src;   // input entry of each CSR slot
  std::vector<int32_t> rb_ids;
  std::vector<int64_t> rb_len;
  std::vector<int32_t> tile_col;
  std::vector<double> tile_val;
  std::vector<int64_t> bcsr_src;  // (input entry, local slot) pairs
  std::vector<int64_t> bcsr_slot;
};

void partition_blocks(const loops_csr* A, const double* vals, loops_dtype dtype, int32_t br,
                      int32_t kpad, double scale, double tau, bool contiguous, int64_t rb_first,
                      int32_t tile_min, int64_t b0, int64_t b1, Chunk& out) {
  const int64_t* rp = A->row_ptr;
  const int32_t* ci = A->col_idx;
  std::vector<Ent> ents;
  std::vector<uint8_t> moved;
  auto csr_row = [&](int64_t i, bool only_moved, int64_t i0) {
    int64_t len = 0;
    for (int64_t k = rp[i]; k < rp[i + 1]; ++k) {
      if (only_moved && !moved[(size_t)(k - rp[i0])]) continue;
      out.csr_col.push_back(ci[k]);
      out.csr_val.push_back(round_store(vals[k], scale, dtype));
      out.csr_src.push_back(k);
      ++len;
    }
    if (!only_moved || len > 0) {
      out.csr_rows.push_back((int32_t)i);
      out.csr_len.push_back(len);
    }
  };
  for (int64_t b = b0; b < b1; ++b) {
    const int64_t i0 = b * br;
    const int64_t i1 = std::min<int64_t>(i0 + br, A->n_rows);
    const int64_t nnz_rb = rp[i1] - rp[i0];
    bool bcsr;
    ents.clear();
    if (contiguous) {
      bcsr = b >= rb_first;
      if (bcsr) {
        for (int64_t i = i0; i < i1; ++i)
          for (int64_t k = rp[i]; k < rp[i + 1]; ++k) ents.push_back({ci[k], (int32_t)(i - i0), k});
        std::sort(ents.begin(), ents.end(), [](const Ent& x, const Ent& y) {
          return x.col != y.col ? x.col < y.col : x.k < y.k;
        });
      }
    } else if (nnz_rb == 0) {
      bcsr = false;
    } else {
      for (int64_t i = i0; i < i1; ++i)
        for (int64_t k = rp[i]; k < rp[i + 1]; ++k) ents.push_back({ci[k], (int32_t)(i - i0), k});
      std::sort(ents.begin(), ents.end(), [](const Ent& x, const Ent& y) {
        return x.col != y.col ? x.col < y.col : x.k < y.k;
      });
      int64_t u = 0;
      for (size_t x = 0; x < ents.size(); ++x)
        if (x == 0 || ents[x].col != ents[x - 1].col) ++u;
      // block density nnz_rb / u compared with tau, without a division
      bcsr = (double)nnz_rb >= tau * (double)u;
    }
    // tile-level split: tiles with fewer than tile_min stored entries leave the block
    moved.assign((size_t)std::max<int64_t>(nnz_rb, 1), 0);
    int64_t n_keep = 0;
    if (bcsr) {
      for (size_t y = 0; y < ents.size();) {
        size_t z = y;
        while (z < ents.size() && ents[z].col == ents[y].col) ++z;
        if (tile_min > 1 && (int64_t)(z - y) < tile_min) {
          for (size_t w = y; w < z; ++w) moved[(size_t)(ents[w].k - rp[i0])] = 1;
        } else {
          ++n_keep;
        }
        y = z;
      }
    }
    if (!bcsr || n_keep == 0) {
      for (int64_t i = i0; i < i1; ++i) csr_row(i, false, i0);
      continue;
    }
    if (tile_min > 1)
      for (int64_t i = i0; i < i1; ++i) csr_row(i, true, i0);  // the moved entries, input order
    // kept tiles keyed by column, ascending; duplicates of (row, col) summed in input order
    const int64_t t_begin = (int64_t)out.tile_col.size();
    int32_t last_col = 0;
    for (size_t x = 0; x < ents.size(); ++x) {
      if (moved[(size_t)(ents[x].k - rp[i0])]) continue;
      if ((int64_t)out.tile_col.size() == t_begin || ents[x].col != last_col) {
        last_col = ents[x].col;
        out.tile_col.push_back(ents[x].col);
        out.tile_val.resize(out.tile_val.size() + br, 0.0);
      }
      const int64_t t = (int64_t)out.tile_col.size() - 1;
      out.tile_val[(size_t)(t * br + ents[x].r)] += vals[ents[x].k];
      out.bcsr_src.push_back(ents[x].k);
      out.bcsr_slot.push_back(t * br + ents[x].r);
    }
    const int64_t t_real = (int64_t)out.tile_col.size() - t_begin;
    for (int64_t t = t_begin; t < t_begin + t_real; ++t)
      for (int32_t r = 0; r < br; ++r) {
        double& v = out.tile_val[(size_t)(t * br + r)];
        v = round_store(v, scale, dtype);
      }
    const int64_t t_pad = (t_real + kpad - 1) / kpad * kpad;
    for (int64_t p = t_real; p < t_pad; ++p) {
      out.tile_col.push_back(-1);
      out.tile_val.resize(out.tile_val.size() + br, 0.0);
    }
    out.rb_ids.push_back((int32_t)b);
    out.rb_len.push_back(t_pad);
  }
}

}  // namespace

loops_status build_canon(const loops_csr* A, const double* vals, loops_dtype dtype, int32_t br,
                         double tau, bool contiguous, int64_t r_boundary, int32_t tile_min, Canon& out) {
  out = Canon();
  out.n_rows = A->n_rows;
  out.n_cols = A->n_cols;
  out.br = br;
  out.kpad = k_pad_for(dtype);
  out.scale = plan_scale_for(vals, A->nnz, dtype);
  const int64_t n_blocks = (A->n_rows + br - 1) / br;
  const int64_t rb_first = contiguous ? (std::max<int64_t>(r_boundary, 0) + br - 1) / br : 0;

  unsigned hw = std::thread::hardware_concurrency();
  int n_thr = (int)std::max(1u, std::min(hw ? hw : 1u, 32u));
  if (A->nnz < (1 << 16)) n_thr = 1;
  const int64_t per = (n_blocks + n_thr - 1) / std::max(n_thr, 1);
  std::vector<Chunk> chunks((size_t)n_thr);
  std::vector<std::thread> thr;
  for (int t = 0; t < n_thr; ++t) {
    const int64_t b0 = std::min<int64_t>(n_blocks, t * per);
    const int64_t b1 = std::min<int64_t>(n_blocks, b0 + per);
    auto job = [&, t, b0, b1]() {
      partition_blocks(A, vals, dtype, br, out.kpad, out.scale, tau, contiguous, rb_first, tile_min, b0, b1,
                       chunks[(size_t)t]);
    };
    if (n_thr == 1) job(); else thr.emplace_back(job);
  }
  for (auto& th : thr) th.join();

  // concatenate the chunks in block order
  size_t n_csr = 0, nnz_csr = 0, n_rb = 0, n_t = 0;
  for (auto& c : chunks) {
    n_csr += c.csr_rows.size();
    nnz_csr += c.csr_col.size();
    n_rb += c.rb_ids.size();
    n_t += c.tile_col.size();
  }
  out.csr_rows.reserve(n_csr);
  out.csr_ptr.reserve(n_csr + 1);
  out.csr_col.reserve(nnz_csr);
  out.csr_val.reserve(nnz_csr);
  out.rb_ids.reserve(n_rb);
  out.rb_ptr.reserve(n_rb + 1);
  out.tile_col.reserve(n_t);
  out.tile_val.reserve(n_t * br);
  out.src_slot.assign((size_t)A->nnz, -1);
  out.src_kind.assign((size_t)A->nnz, 0);
  out.csr_ptr.push_back(0);
  out.rb_ptr.push_back(0);
  for (auto& c : chunks) {
    const int64_t csr_base = (int64_t)out.csr_col.size();
    const int64_t tile_base = (int64_t)out.tile_col.size();
    for (size_t x = 0; x < c.csr_rows.size(); ++x) {
      out.csr_rows.push_back(c.csr_rows[x]);
      out.csr_ptr.push_back(out.csr_ptr.back() + c.csr_len[x]);
    }
    out.csr_col.insert(out.csr_col.end(), c.csr_col.begin(), c.csr_col.end());
    out.csr_val.insert(out.csr_val.end(), c.csr_val.begin(), c.csr_val.end());
    for (size_t x = 0; x < c.csr_src.size(); ++x) {
      out.src_slot[(size_t)c.csr_src[x]] = csr_base + (int64_t)x;
      out.src_kind[(size_t)c.csr_src[x]] = 0;
    }
    for (size_t x = 0; x < c.rb_ids.size(); ++x) {
      out.rb_ids.push_back(c.rb_ids[x]);
      out.rb_ptr.push_back(out.rb_ptr.back() + c.rb_len[x]);
    }
    out.tile_col.insert(out.tile_col.end(), c.tile_col.begin(), c.tile_col.end());
    out.tile_val.insert(out.tile_val.end(), c.tile_val.begin(), c.tile_val.end());
    for (size_t x = 0; x < c.bcsr_src.size(); ++x) {
      out.src_slot[(size_t)c.bcsr_src[x]] = tile_base * br + c.bcsr_slot[x];
      out.src_kind[(size_t)c.bcsr_src[x]] = 1;
    }
    c = Chunk();  // release the chunk's memory early
  }
  return LOOPS_OK;
}

}  // namespace loops
