// Device layout of a plan's two parts, and its inverse (export back to canonical order).
//
// CSR part: rows become work items processed in storage order; rows longer than split_len
// are cut into segments whose partial sums go to scratch slots and are summed afterwards in
// slot order (deterministic). Items are ordered by decreasing length class, so the longest
// work starts first; within a class the row order is kept.
//
// BCSR part: tile values are stored in the register-fragment order of the dtype's MMA, so a
// lane loads its whole A fragment of a K-group with one vector load:
//   F64  (m8n8k4, K = 4 tiles, B_r = 8):  group g, lane l = 4*row + t -> A[row][t]
//   F16/BF16 (m16n8k16, K = 16, B_r = 16): group g, lane l = 4*q + t, j = 0..7 ->
//        row = q + 8*(j>>1 & 1), tile = 2t + (j & 1) + 8*(j >> 2)
//   F32  (CUDA-core outer product): tile-major, B_r values of a tile contiguous.
#include <algorithm>
#include <cstring>

#include "loops_internal.h"

namespace loops {

namespace {

template <typename T>
loops_status dev_upload(T** dst, const T* src, size_t n, int64_t& bytes) {
  *dst = nullptr;
  if (n == 0) return LOOPS_OK;
  cudaError_t e = dev_malloc((void**)dst, n * sizeof(T));
  if (e != cudaSuccess) {
    cudaGetLastError();
    *dst = nullptr;
    set_error(std::string("cudaMalloc failed: ") + cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? LOOPS_ERR_OOM : LOOPS_ERR_CUDA;
  }
  bytes += (int64_t)(n * sizeof(T));
  if (src) {
    e = cudaMemcpy(*dst, src, n * sizeof(T), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
      set_error(std::string("cudaMemcpy failed: ") + cudaGetErrorString(e));
      return LOOPS_ERR_CUDA;
    }
  }
  return LOOPS_OK;
}

template <typename T>
loops_status dev_download(std::vector<T>& dst, const T* src, size_t n) {
  dst.resize(n);
  if (n == 0) return LOOPS_OK;
  cudaError_t e = cudaMemcpy(dst.data(), src, n * sizeof(T), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) {
    set_error(std::string("cudaMemcpy failed: ") + cudaGetErrorString(e));
    return LOOPS_ERR_CUDA;
  }
  return LOOPS_OK;
}

// f64 values that are already representable in the dtype -> storage bytes.
void encode_values(const double* v, size_t n, loops_dtype d, std::vector<uint8_t>& out) {
  const int es = d == LOOPS_F64 ? 8 : d == LOOPS_F32 ? 4 : 2;
  out.resize(n * es);
  for (size_t i = 0; i < n; ++i) {
    switch (d) {
      case LOOPS_F64: std::memcpy(&out[i * 8], &v[i], 8); break;
      case LOOPS_F32: { float f = (float)v[i]; std::memcpy(&out[i * 4], &f, 4); break; }
      case LOOPS_F16: { uint16_t h = f64_to_f16_bits(v[i]); std::memcpy(&out[i * 2], &h, 2); break; }
      case LOOPS_BF16: { uint16_t h = f64_to_bf16_bits(v[i]); std::memcpy(&out[i * 2], &h, 2); break; }
    }
  }
}

double decode_value(const uint8_t* p, loops_dtype d) {
  switch (d) {
    case LOOPS_F64: { double x; std::memcpy(&x, p, 8); return x; }
    case LOOPS_F32: { float x; std::memcpy(&x, p, 4); return (double)x; }
    case LOOPS_F16: { uint16_t h; std::memcpy(&h, p, 2); return f16_bits_to_f64(h); }
    case LOOPS_BF16: { uint16_t h; std::memcpy(&h, p, 2); return bf16_bits_to_f64(h); }
  }
  return 0.0;
}

int bucket_of(int64_t len) {
  int b = 0;
  while ((1ll << (b + 1)) <= len + 1 && b < 62) ++b;
  return b;  // floor(log2(len + 1))
}

}  // namespace

loops_status upload_part(loops_plan_s* p, int64_t N) {
  const Canon& c = p->canon;
  PartDev& d = p->dev;
  d = PartDev();
  loops_status st;
  const int acc_bytes = p->dtype == LOOPS_F64 ? 8 : 4;

  // ---- CSR work items: rows inside BCSR blocks (tile-level split) go to csr_acc
  std::vector<uint8_t> in_bcsr;
  if (!c.rb_ids.empty()) {
    in_bcsr.assign((size_t)std::max<int64_t>(p->n_rows, 1), 0);
    for (int32_t b : c.rb_ids)
      for (int64_t i = (int64_t)b * c.br; i < std::min<int64_t>((int64_t)b * c.br + c.br, p->n_rows); ++i)
        in_bcsr[(size_t)i] = 1;
  }
  int64_t& bytes = d.device_bytes;
  std::vector<uint8_t> enc;
  for (int which = 0; which < 2; ++which) {
    CsrDev& cd = which == 0 ? d.csr : d.csr_acc;
    struct It { int32_t row; int64_t beg, end; int bucket; };
    std::vector<It> items;
    const int64_t n_csr = (int64_t)c.csr_rows.size();
    const int64_t L = std::max<int64_t>(p->split_len, 1);
    int64_t n_slots = 0;
    for (int64_t x = 0; x < n_csr; ++x) {
      const int32_t row = c.csr_rows[(size_t)x];
      const int mixed = in_bcsr.empty() ? 0 : in_bcsr[(size_t)row];
      if (mixed != which) continue;
      const int64_t b = c.csr_ptr[(size_t)x], e = c.csr_ptr[(size_t)x + 1];
      const int64_t len = e - b;
      if (len > L) {
        cd.h_split_row.push_back(row);
        cd.h_split_slot_ptr.push_back((int32_t)n_slots);
        for (int64_t s0 = b; s0 < e; s0 += L) {
          items.push_back({(int32_t)(-1 - n_slots), s0, std::min(s0 + L, e), 63});
          ++n_slots;
        }
      } else {
        items.push_back({row, b, e, bucket_of(len)});
      }
    }
    cd.h_split_slot_ptr.push_back((int32_t)n_slots);
    if (LOOPS_CSR_ITEMS_BY_LENGTH)
      std::stable_sort(items.begin(), items.end(), [](const It& a, const It& b) { return a.bucket > b.bucket; });
    cd.n_items = (int64_t)items.size();
    cd.n_split = (int64_t)cd.h_split_row.size();
    cd.n_slots = n_slots;
    cd.h_item_row.resize(items.size());
    cd.h_item_ptr.resize(items.size() + 1);
    int64_t total = 0;
    for (auto& it : items) total += it.end - it.beg;
    cd.nnz = total;
    std::vector<int32_t> col((size_t)total);
    std::vector<double> val((size_t)total);
    int64_t pos = 0;
    cd.h_item_ptr[0] = 0;
    for (size_t i = 0; i < items.size(); ++i) {
      cd.h_item_row[i] = items[i].row;
      for (int64_t k = items[i].beg; k < items[i].end; ++k) {
        col[(size_t)pos] = c.csr_col[(size_t)k];
        val[(size_t)pos] = c.csr_val[(size_t)k];
        ++pos;
      }
      cd.h_item_ptr[i + 1] = pos;
    }
    if (items.empty()) continue;
    encode_values(val.data(), val.size(), p->dtype, enc);
    if ((st = dev_upload(&cd.item_row, cd.h_item_row.data(), items.size(), bytes))) return st;
    if ((st = dev_upload(&cd.item_ptr, cd.h_item_ptr.data(), items.size() + 1, bytes))) return st;
    if ((st = dev_upload(&cd.col, col.data(), col.size(), bytes))) return st;
    if ((st = dev_upload((uint8_t**)&cd.val, enc.data(), enc.size(), bytes))) return st;
    if (cd.n_split) {
      if ((st = dev_upload(&cd.split_row, cd.h_split_row.data(), cd.h_split_row.size(), bytes))) return st;
      if ((st = dev_upload(&cd.split_slot_ptr, cd.h_split_slot_ptr.data(), cd.h_split_slot_ptr.size(), bytes))) return st;
      if ((st = dev_upload((uint8_t**)&cd.scratch, (const uint8_t*)nullptr,
                           (size_t)(n_slots * std::max<int64_t>(N, 1) * acc_bytes), bytes))) return st;
    }
  }

  // ---- BCSR part
  const int64_t n_rb = (int64_t)c.rb_ids.size();
  const int64_t n_t = (int64_t)c.tile_col.size();
  d.bcsr.n_rb = n_rb;
  d.bcsr.n_tiles = n_t;
  if (n_rb) {
    std::vector<double> fv((size_t)(n_t * c.br), 0.0);
    for (int64_t t = 0; t < n_t; ++t)
      for (int32_t r = 0; r < c.br; ++r)
        fv[(size_t)frag_index(p->dtype, t, r, c.br)] = c.tile_val[(size_t)(t * c.br + r)];
    encode_values(fv.data(), fv.size(), p->dtype, enc);
    // work units: blocks with more than kBcsrSplitTiles tiles are cut (a multiple of the K)
    struct Unit { int32_t b; int64_t t0, t1; int32_t slot; };
    std::vector<Unit> units;
    std::vector<int32_t> split_block, split_slot_ptr;
    int64_t n_bslots = 0;
    for (int64_t b = 0; b < n_rb; ++b) {
      const int64_t t0 = c.rb_ptr[(size_t)b], t1 = c.rb_ptr[(size_t)b + 1];
      if (t1 - t0 > kBcsrSplitTiles) {
        split_block.push_back((int32_t)b);
        split_slot_ptr.push_back((int32_t)n_bslots);
        for (int64_t t = t0; t < t1; t += kBcsrSplitTiles)
          units.push_back({(int32_t)b, t, std::min(t + kBcsrSplitTiles, t1), (int32_t)n_bslots++});
      } else {
        units.push_back({(int32_t)b, t0, t1, -1});
      }
    }
    split_slot_ptr.push_back((int32_t)n_bslots);
    std::stable_sort(units.begin(), units.end(), [](const Unit& x, const Unit& y) { return x.t1 - x.t0 > y.t1 - y.t0; });
    std::vector<int32_t> ub(units.size()), us(units.size());
    std::vector<int64_t> u0(units.size()), u1(units.size());
    d.bcsr.h_unit_tiles.resize(units.size());
    for (size_t i = 0; i < units.size(); ++i) {
      ub[i] = units[i].b;
      u0[i] = units[i].t0;
      u1[i] = units[i].t1;
      us[i] = units[i].slot;
      d.bcsr.h_unit_tiles[i] = units[i].t1 - units[i].t0;
    }
    d.bcsr.n_units = (int64_t)units.size();
    d.bcsr.n_split = (int64_t)split_block.size();
    d.bcsr.n_slots = n_bslots;
    if ((st = dev_upload(&d.bcsr.rb_id, c.rb_ids.data(), (size_t)n_rb, bytes))) return st;
    if ((st = dev_upload(&d.bcsr.rb_ptr, c.rb_ptr.data(), (size_t)n_rb + 1, bytes))) return st;
    if ((st = dev_upload(&d.bcsr.tile_col, c.tile_col.data(), (size_t)n_t, bytes))) return st;
    if ((st = dev_upload((uint8_t**)&d.bcsr.tile_val, enc.data(), enc.size(), bytes))) return st;
    if ((st = dev_upload(&d.bcsr.unit_block, ub.data(), ub.size(), bytes))) return st;
    if ((st = dev_upload(&d.bcsr.unit_t0, u0.data(), u0.size(), bytes))) return st;
    if ((st = dev_upload(&d.bcsr.unit_t1, u1.data(), u1.size(), bytes))) return st;
    if ((st = dev_upload(&d.bcsr.unit_slot, us.data(), us.size(), bytes))) return st;
    if (n_bslots) {
      if ((st = dev_upload(&d.bcsr.split_block, split_block.data(), split_block.size(), bytes))) return st;
      if ((st = dev_upload(&d.bcsr.split_slot_ptr, split_slot_ptr.data(), split_slot_ptr.size(), bytes))) return st;
      if ((st = dev_upload((uint8_t**)&d.bcsr.scratch, (const uint8_t*)nullptr,
                           (size_t)(n_bslots * c.br * std::max<int64_t>(N, 1) * acc_bytes), bytes))) return st;
    }
  }
  return LOOPS_OK;
}

void free_part(PartDev& d) {
  void* ptrs[] = {d.csr.item_row, d.csr.item_ptr, d.csr.col, d.csr.val, d.csr.split_row,
                  d.csr.split_slot_ptr, d.csr.scratch, d.csr_acc.item_row, d.csr_acc.item_ptr,
                  d.csr_acc.col, d.csr_acc.val, d.csr_acc.split_row, d.csr_acc.split_slot_ptr,
                  d.csr_acc.scratch, d.bcsr.rb_id, d.bcsr.rb_ptr,
                  d.bcsr.tile_col, d.bcsr.tile_val, d.bcsr.unit_block, d.bcsr.unit_t0,
                  d.bcsr.unit_t1, d.bcsr.unit_slot, d.bcsr.split_block, d.bcsr.split_slot_ptr,
                  d.bcsr.scratch};
  for (void* q : ptrs)
    if (q) cudaFree(q);
  d = PartDev();
}

loops_status upload_value_maps(loops_plan_s* p, const std::vector<int64_t>* remap) {
  const Canon& c = p->canon;
  const CsrDev& d = p->dev.csr;
  ValueMapDev& m = p->vmap;
  free_value_maps(m);
  const int64_t nnz = (int64_t)c.src_slot.size();
  // canonical CSR slot -> input entry, then device position -> input entry
  std::vector<int64_t> canon_src(c.csr_col.size(), -1);
  for (int64_t k = 0; k < nnz; ++k)
    if (c.src_kind[(size_t)k] == 0) canon_src[(size_t)c.src_slot[(size_t)k]] = remap ? (*remap)[(size_t)k] : k;
  // device order of the CSR entries: items in storage order, each a canonical range
  std::vector<int64_t> csr_src;
  csr_src.reserve(c.csr_col.size());
  {
    // rebuild the canonical start of each item: items cover canonical rows (or segments of
    // them) and were laid out in item order; recover the canonical range from the row id and
    // the segment offset
    std::vector<int64_t> row_pos(c.csr_rows.size());
    std::vector<int64_t> canon_row_of((size_t)std::max<int64_t>(p->n_rows, 1), -1);
    for (size_t x = 0; x < c.csr_rows.size(); ++x) canon_row_of[(size_t)c.csr_rows[x]] = (int64_t)x;
    std::vector<int64_t> seg_cursor(c.csr_rows.size(), 0);
    // slot -> split row
    std::vector<int32_t> slot_row((size_t)d.n_slots, -1);
    for (int64_t sidx = 0; sidx < d.n_split; ++sidx)
      for (int32_t q = d.h_split_slot_ptr[(size_t)sidx]; q < d.h_split_slot_ptr[(size_t)sidx + 1]; ++q)
        slot_row[(size_t)q] = d.h_split_row[(size_t)sidx];
    for (int64_t i = 0; i < d.n_items; ++i) {
      const int32_t r = d.h_item_row[(size_t)i];
      const int32_t row = r >= 0 ? r : slot_row[(size_t)(-1 - r)];
      const int64_t x = canon_row_of[(size_t)row];
      const int64_t len = d.h_item_ptr[(size_t)i + 1] - d.h_item_ptr[(size_t)i];
      const int64_t b = c.csr_ptr[(size_t)x] + seg_cursor[(size_t)x];
      for (int64_t e = 0; e < len; ++e) csr_src.push_back(canon_src[(size_t)(b + e)]);
      seg_cursor[(size_t)x] += len;
    }
  }
  // BCSR fragment slots -> input entries (ascending input order within a slot)
  const int64_t n_slots = (int64_t)c.tile_col.size() * c.br;
  std::vector<int64_t> cnt((size_t)n_slots + 1, 0);
  for (int64_t k = 0; k < nnz; ++k)
    if (c.src_kind[(size_t)k] == 1) {
      const int64_t sl = c.src_slot[(size_t)k];
      cnt[(size_t)frag_index(p->dtype, sl / c.br, (int32_t)(sl % c.br), c.br) + 1]++;
    }
  for (int64_t f = 0; f < n_slots; ++f) cnt[(size_t)f + 1] += cnt[(size_t)f];
  std::vector<int64_t> pos(cnt.begin(), cnt.end() - 1), bsrc((size_t)cnt[(size_t)n_slots]);
  // input order: for the transposed plan the entries' input order is given by remap
  std::vector<std::pair<int64_t, int64_t>> order;  // (input index, entry)
  for (int64_t k = 0; k < nnz; ++k)
    if (c.src_kind[(size_t)k] == 1) order.push_back({remap ? (*remap)[(size_t)k] : k, k});
  std::sort(order.begin(), order.end());
  for (auto& ok : order) {
    const int64_t sl = c.src_slot[(size_t)ok.second];
    const int64_t f = frag_index(p->dtype, sl / c.br, (int32_t)(sl % c.br), c.br);
    bsrc[(size_t)pos[(size_t)f]++] = ok.first;
  }
  m.n_csr = (int64_t)csr_src.size();
  m.n_slots = n_slots;
  loops_status st;
  if ((st = dev_upload(&m.csr_src, csr_src.data(), csr_src.size(), m.bytes))) return st;
  if (n_slots) {
    if ((st = dev_upload(&m.bcsr_ptr, cnt.data(), cnt.size(), m.bytes))) return st;
    if ((st = dev_upload(&m.bcsr_src, bsrc.data(), bsrc.size(), m.bytes))) return st;
  }
  return LOOPS_OK;
}

void free_value_maps(ValueMapDev& m) {
  void* ptrs[] = {m.csr_src, m.bcsr_ptr, m.bcsr_src};
  for (void* q : ptrs)
    if (q) cudaFree(q);
  m = ValueMapDev();
}

// Download the device arrays of a plan and rebuild the canonical partition from them.
loops_status export_part(const loops_plan_s* p, loops_partition* out) {
  const PartDev& d = p->dev;
  const int es = p->dtype == LOOPS_F64 ? 8 : p->dtype == LOOPS_F32 ? 4 : 2;
  loops_status st;
  // rows of both CSR item sets, each with its entries (column, value) in segment order
  struct Row { int32_t row; std::vector<std::pair<int32_t, double>> ents; };
  std::vector<Row> rows;
  int64_t nnz_csr = 0;
  for (const CsrDev* cd : {&d.csr, &d.csr_acc}) {
    std::vector<int32_t> item_row, col, split_row, split_slot;
    std::vector<int64_t> item_ptr;
    std::vector<uint8_t> val;
    if ((st = dev_download(item_row, cd->item_row, (size_t)cd->n_items))) return st;
    if ((st = dev_download(item_ptr, cd->item_ptr, (size_t)(cd->n_items ? cd->n_items + 1 : 0)))) return st;
    if ((st = dev_download(col, cd->col, (size_t)cd->nnz))) return st;
    if ((st = dev_download(val, (const uint8_t*)cd->val, (size_t)(cd->nnz * es)))) return st;
    if ((st = dev_download(split_row, cd->split_row, (size_t)cd->n_split))) return st;
    if ((st = dev_download(split_slot, cd->split_slot_ptr, (size_t)(cd->n_split ? cd->n_split + 1 : 0)))) return st;
    nnz_csr += cd->nnz;
    // slot -> split row index
    std::vector<int32_t> slot_owner((size_t)cd->n_slots, -1);
    for (int64_t sidx = 0; sidx < cd->n_split; ++sidx)
      for (int32_t q = split_slot[(size_t)sidx]; q < split_slot[(size_t)sidx + 1]; ++q)
        slot_owner[(size_t)q] = (int32_t)sidx;
    std::vector<std::vector<std::pair<int64_t, int64_t>>> split_segs((size_t)cd->n_split);  // (slot, item)
    auto add_item = [&](Row& r, int64_t i) {
      for (int64_t e = item_ptr[(size_t)i]; e < item_ptr[(size_t)i + 1]; ++e)
        r.ents.push_back({col[(size_t)e], decode_value(&val[(size_t)(e * es)], p->dtype)});
    };
    for (int64_t i = 0; i < cd->n_items; ++i) {
      const int32_t r = item_row[(size_t)i];
      if (r >= 0) {
        rows.push_back({r, {}});
        add_item(rows.back(), i);
      } else {
        const int32_t slot = -1 - r;
        split_segs[(size_t)slot_owner[(size_t)slot]].push_back({slot, i});
      }
    }
    for (int64_t sidx = 0; sidx < cd->n_split; ++sidx) {
      auto segs = split_segs[(size_t)sidx];
      std::sort(segs.begin(), segs.end());
      rows.push_back({split_row[(size_t)sidx], {}});
      for (auto& sg : segs) add_item(rows.back(), sg.second);
    }
  }
  std::sort(rows.begin(), rows.end(), [](const Row& a, const Row& b) { return a.row < b.row; });
  out->n_rows = p->n_rows;
  out->n_cols = p->n_cols;
  out->block_rows = p->br;
  out->k_pad = p->kpad;
  out->scale = p->scale;
  out->n_csr_rows = (int64_t)rows.size();
  out->nnz_csr = nnz_csr;
  out->csr_rows = (int32_t*)std::malloc(sizeof(int32_t) * (rows.size() + 1));
  out->csr_ptr = (int64_t*)std::malloc(sizeof(int64_t) * (rows.size() + 1));
  out->csr_col = (int32_t*)std::malloc(sizeof(int32_t) * (size_t)(nnz_csr + 1));
  out->csr_val = (double*)std::malloc(sizeof(double) * (size_t)(nnz_csr + 1));
  int64_t k = 0;
  out->csr_ptr[0] = 0;
  for (size_t x = 0; x < rows.size(); ++x) {
    out->csr_rows[x] = rows[x].row;
    for (auto& en : rows[x].ents) {
      out->csr_col[k] = en.first;
      out->csr_val[k] = en.second;
      ++k;
    }
    out->csr_ptr[x + 1] = k;
  }
  // BCSR
  std::vector<int32_t> rb_id, tcol;
  std::vector<int64_t> rb_ptr;
  std::vector<uint8_t> tval;
  const int64_t n_rb = d.bcsr.n_rb, n_t = d.bcsr.n_tiles;
  if ((st = dev_download(rb_id, d.bcsr.rb_id, (size_t)n_rb))) return st;
  if ((st = dev_download(rb_ptr, d.bcsr.rb_ptr, (size_t)(n_rb ? n_rb + 1 : 0)))) return st;
  if ((st = dev_download(tcol, d.bcsr.tile_col, (size_t)n_t))) return st;
  if ((st = dev_download(tval, (const uint8_t*)d.bcsr.tile_val, (size_t)(n_t * p->br * es)))) return st;
  out->n_row_blocks = n_rb;
  out->n_tiles = n_t;
  out->rb_ids = (int32_t*)std::malloc(sizeof(int32_t) * (size_t)(n_rb + 1));
  out->rb_ptr = (int64_t*)std::malloc(sizeof(int64_t) * (size_t)(n_rb + 1));
  out->tile_col = (int32_t*)std::malloc(sizeof(int32_t) * (size_t)(n_t + 1));
  out->tile_val = (double*)std::malloc(sizeof(double) * (size_t)(n_t * p->br + 1));
  out->rb_ptr[0] = 0;
  for (int64_t b = 0; b < n_rb; ++b) {
    out->rb_ids[b] = rb_id[(size_t)b];
    out->rb_ptr[b + 1] = rb_ptr[(size_t)b + 1];
  }
  for (int64_t t = 0; t < n_t; ++t) {
    out->tile_col[t] = tcol[(size_t)t];
    for (int32_t r = 0; r < p->br; ++r)
      out->tile_val[t * p->br + r] =
          decode_value(&tval[(size_t)(frag_index(p->dtype, t, r, p->br) * es)], p->dtype);
  }
  return LOOPS_OK;
}

}  // namespace loops
