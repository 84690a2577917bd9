/*
 * Plain, slow CPU oracle for the LOOPS hybrid SpMM (arxiv 2511.08158).
 *
 * TEST INFRASTRUCTURE ONLY. Only tests, the smoke check and the bench's CPU-baseline
 * leg may load this file's library. It shares no code with the CUDA library.
 *
 * Every routine computes in IEEE binary64 with plain loops, in the order the paper
 * states, so a reader can check it against the paper by eye:
 *   oracle_spmm           C = A.B by the inner-product definition c_ij = sum_k a_ik b_kj
 *                         (Sec. 2.1), row by row with a dense accumulator of length N.
 *   oracle_spmm_rows      the same for a chosen subset of rows (sampled parity at full size).
 *   oracle_spmm_t         dB = A^T.dC by scattering each row of A (chain rule of Sec. 2.1;
 *                         no transpose is built, so it is independent of a transposed plan).
 *   oracle_sddmm          dvals[k] = sum_n dC[i_k, n] * B[j_k, n] on A's pattern.
 *   oracle_gemm_dense     brute-force dense triple loop (pins oracle_spmm on tiny inputs).
 *   oracle_partition_*    Algorithm 1 (CSR -> LOOPS conversion) with the structural split
 *                         reading: row blocks of B_r rows aligned at row 0; a block is BCSR
 *                         when nnz_rb >= tau * (distinct columns of the block); otherwise
 *                         (and for empty blocks) its rows are CSR-part rows. Paper mode
 *                         instead takes rows [0, r_b) as CSR with r_b rounded up to B_r
 *                         (Eq. 1 boundary, Algorithm 1 step 1/step 2).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

/* Sec. 2.1 inner-product SpMM: for each row i, acc[:] = 0; acc[:] += a_ik * B[k, :]; C[i, :] = acc. */
void oracle_spmm(int64_t n_rows, int64_t N, const int64_t* row_ptr, const int32_t* col_idx,
                 const double* vals, const double* B, int64_t ldb, double* C, int64_t ldc) {
  double* acc = (double*)malloc((size_t)(N > 0 ? N : 1) * sizeof(double));
  for (int64_t i = 0; i < n_rows; ++i) {
    for (int64_t n = 0; n < N; ++n) acc[n] = 0.0;
    for (int64_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k) {
      const double a = vals[k];
      const double* b = B + (int64_t)col_idx[k] * ldb;
      for (int64_t n = 0; n < N; ++n) acc[n] += a * b[n];
    }
    for (int64_t n = 0; n < N; ++n) C[i * ldc + n] = acc[n];
  }
  free(acc);
}

/* Same definition, restricted to rows[0..n_sel); C_sel is n_sel x N, row-major. */
void oracle_spmm_rows(const int64_t* row_ptr, const int32_t* col_idx, const double* vals,
                      const double* B, int64_t ldb, int64_t N, const int64_t* rows, int64_t n_sel,
                      double* C_sel) {
  for (int64_t s = 0; s < n_sel; ++s) {
    const int64_t i = rows[s];
    double* c = C_sel + s * N;
    for (int64_t n = 0; n < N; ++n) c[n] = 0.0;
    for (int64_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k) {
      const double a = vals[k];
      const double* b = B + (int64_t)col_idx[k] * ldb;
      for (int64_t n = 0; n < N; ++n) c[n] += a * b[n];
    }
  }
}

/* dB = A^T . dC, by scattering: for each stored a_ij, dB[j, :] += a_ij * dC[i, :]. */
void oracle_spmm_t(int64_t n_rows, int64_t n_cols, int64_t N, const int64_t* row_ptr,
                   const int32_t* col_idx, const double* vals, const double* dC, int64_t lddc,
                   double* dB, int64_t lddb) {
  for (int64_t j = 0; j < n_cols; ++j)
    for (int64_t n = 0; n < N; ++n) dB[j * lddb + n] = 0.0;
  for (int64_t i = 0; i < n_rows; ++i) {
    for (int64_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k) {
      const double a = vals[k];
      double* d = dB + (int64_t)col_idx[k] * lddb;
      const double* g = dC + i * lddc;
      for (int64_t n = 0; n < N; ++n) d[n] += a * g[n];
    }
  }
}

/* dvals[k] = <dC[i_k, :], B[j_k, :]> for every stored entry k of A, in A's storage order. */
void oracle_sddmm(int64_t n_rows, int64_t N, const int64_t* row_ptr, const int32_t* col_idx,
                  const double* dC, int64_t lddc, const double* B, int64_t ldb, double* dvals) {
  for (int64_t i = 0; i < n_rows; ++i) {
    for (int64_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k) {
      const double* g = dC + i * lddc;
      const double* b = B + (int64_t)col_idx[k] * ldb;
      double s = 0.0;
      for (int64_t n = 0; n < N; ++n) s += g[n] * b[n];
      dvals[k] = s;
    }
  }
}

/* Brute force: C (M x N) = A (M x K, dense row-major) . B (K x N). */
void oracle_gemm_dense(int64_t M, int64_t K, int64_t N, const double* A, const double* B, double* C) {
  for (int64_t i = 0; i < M; ++i)
    for (int64_t n = 0; n < N; ++n) {
      double s = 0.0;
      for (int64_t k = 0; k < K; ++k) s += A[i * K + k] * B[k * N + n];
      C[i * N + n] = s;
    }
}

/* ------------------------------------------------------------------------------------------ */
/* Algorithm 1 (CSR -> LOOPS), restated with these readings:                                  */
/*  - tile shape B_r x 1 (B_c = 1, Sec. 3.2.1); tile_r = i div B_r, tile_c = j, offset i mod B_r */
/*  - row blocks are aligned at row 0; the split unit is the row block;                         */
/*  - duplicate (i, j) entries are summed in storage order (the tile map accumulates);          */
/*  - tiles of a block are ordered by column ascending (the map's order is unspecified);        */
/*  - each block's tile list is padded to a multiple of k_pad with padding tiles (col = -1,     */
/*    values 0), the zero register that the paper pairs with a remaining tile (Algorithm 3);    */
/*  - CSR-part rows keep their entries in storage order; empty rows are CSR rows (written 0).   */
/* ------------------------------------------------------------------------------------------ */

typedef struct { int32_t col; int32_t r; int64_t k; } oracle_entry;

static int oracle_entry_cmp(const void* pa, const void* pb) {
  const oracle_entry* a = (const oracle_entry*)pa;
  const oracle_entry* b = (const oracle_entry*)pb;
  if (a->col != b->col) return a->col < b->col ? -1 : 1;
  if (a->k != b->k) return a->k < b->k ? -1 : 1; /* keep storage order among duplicates */
  return 0;
}

static int oracle_int_cmp(const void* pa, const void* pb) {
  const int32_t a = *(const int32_t*)pa, b = *(const int32_t*)pb;
  return (a > b) - (a < b);
}

/* Decide per row block whether it is BCSR (1) or CSR (0). Returns the number of row blocks. */
static int64_t oracle_block_kinds(int64_t n_rows, const int64_t* row_ptr, const int32_t* col_idx,
                                  int64_t block_rows, double tau, int contiguous, int64_t r_boundary,
                                  unsigned char* kind) {
  const int64_t n_blocks = (n_rows + block_rows - 1) / block_rows;
  int64_t rb_first_bcsr = 0;
  if (contiguous) {
    /* Eq. 1 boundary r_b, rounded up to a multiple of B_r so no block straddles it. */
    int64_t rb = r_boundary < 0 ? 0 : r_boundary;
    rb_first_bcsr = (rb + block_rows - 1) / block_rows;
  }
  for (int64_t b = 0; b < n_blocks; ++b) {
    const int64_t i0 = b * block_rows;
    const int64_t i1 = (i0 + block_rows < n_rows) ? i0 + block_rows : n_rows;
    const int64_t nnz_rb = row_ptr[i1] - row_ptr[i0];
    if (contiguous) { kind[b] = (b >= rb_first_bcsr) ? 1 : 0; continue; }
    if (nnz_rb == 0) { kind[b] = 0; continue; }
    /* distinct columns of the block: sort a copy of its column indices */
    int32_t* cols = (int32_t*)malloc((size_t)nnz_rb * sizeof(int32_t));
    int64_t m = 0;
    for (int64_t k = row_ptr[i0]; k < row_ptr[i1]; ++k) cols[m++] = col_idx[k];
    qsort(cols, (size_t)m, sizeof(int32_t), oracle_int_cmp);
    int64_t u_rb = 0;
    for (int64_t x = 0; x < m; ++x) if (x == 0 || cols[x] != cols[x - 1]) ++u_rb;
    free(cols);
    /* block density d_rb = nnz_rb / u_rb compared with tau without a division */
    kind[b] = ((double)nnz_rb >= tau * (double)u_rb) ? 1 : 0;
  }
  return n_blocks;
}

/* One pass of Algorithm 1 over the row blocks. With out_sizes it only counts; otherwise it
 * fills the arrays. tile_min > 1 keeps in a BCSR block only the tiles holding at least
 * tile_min stored entries; the entries of the other tiles become CSR-part entries of their
 * rows (in input order), and a block left with no tile is entirely CSR. */
static int oracle_partition_run(int64_t n_rows, const int64_t* row_ptr, const int32_t* col_idx,
                                const double* vals, int64_t block_rows, int64_t k_pad, double tau,
                                int contiguous, int64_t r_boundary, int64_t tile_min, int64_t* out_sizes,
                                int32_t* csr_rows, int64_t* csr_ptr, int32_t* csr_col, double* csr_val,
                                int32_t* rb_ids, int64_t* rb_ptr, int32_t* tile_col, double* tile_val) {
  const int fill = out_sizes == NULL;
  const int64_t n_blocks = (n_rows + block_rows - 1) / block_rows;
  unsigned char* kind = (unsigned char*)malloc((size_t)(n_blocks > 0 ? n_blocks : 1));
  oracle_block_kinds(n_rows, row_ptr, col_idx, block_rows, tau, contiguous, r_boundary, kind);
  int64_t rc = 0, kc = 0, rbc = 0, tc = 0;
  if (fill) { csr_ptr[0] = 0; rb_ptr[0] = 0; }
  for (int64_t b = 0; b < n_blocks; ++b) {
    const int64_t i0 = b * block_rows;
    const int64_t i1 = (i0 + block_rows < n_rows) ? i0 + block_rows : n_rows;
    const int64_t m = row_ptr[i1] - row_ptr[i0];
    unsigned char* moved = (unsigned char*)calloc((size_t)(m > 0 ? m : 1), 1);
    int64_t n_keep = 0;
    oracle_entry* e = NULL;
    if (kind[b]) {
      /* Step 2: group the block's entries into B_r x 1 tiles keyed by column */
      e = (oracle_entry*)malloc((size_t)(m > 0 ? m : 1) * sizeof(oracle_entry));
      int64_t x = 0;
      for (int64_t i = i0; i < i1; ++i)
        for (int64_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k) { e[x].col = col_idx[k]; e[x].r = (int32_t)(i - i0); e[x].k = k; ++x; }
      qsort(e, (size_t)m, sizeof(oracle_entry), oracle_entry_cmp);
      for (int64_t y = 0; y < m;) {
        int64_t z = y;
        while (z < m && e[z].col == e[y].col) ++z;
        if (tile_min > 1 && z - y < tile_min) {
          for (int64_t w = y; w < z; ++w) moved[e[w].k - row_ptr[i0]] = 1;
        } else {
          ++n_keep;
        }
        y = z;
      }
      if (n_keep == 0) {            /* nothing left for BCSR: the whole block is CSR */
        for (int64_t w = 0; w < m; ++w) moved[w] = 0;
      }
    }
    if (!kind[b] || n_keep == 0) {
      /* Step 1: copy the rows into the CSR part, preserving their structure */
      for (int64_t i = i0; i < i1; ++i) {
        for (int64_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k) {
          if (fill) { csr_col[kc] = col_idx[k]; csr_val[kc] = vals[k]; }
          ++kc;
        }
        if (fill) { csr_rows[rc] = (int32_t)i; csr_ptr[rc + 1] = kc; }
        ++rc;
      }
    } else {
      /* entries of dropped tiles: CSR-part rows, entries in input order */
      for (int64_t i = i0; i < i1; ++i) {
        int64_t any = 0;
        for (int64_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k) {
          if (!moved[k - row_ptr[i0]]) continue;
          if (fill) { csr_col[kc] = col_idx[k]; csr_val[kc] = vals[k]; }
          ++kc;
          any = 1;
        }
        if (any) {
          if (fill) { csr_rows[rc] = (int32_t)i; csr_ptr[rc + 1] = kc; }
          ++rc;
        }
      }
      /* kept tiles, ascending by column, duplicates summed in input order, then padding */
      const int64_t t_begin = tc;
      int32_t last_col = 0;
      for (int64_t y = 0; y < m; ++y) {
        if (moved[e[y].k - row_ptr[i0]]) continue;
        if (tc == t_begin || e[y].col != last_col) {
          last_col = e[y].col;
          if (fill) {
            tile_col[tc] = e[y].col;
            for (int64_t r = 0; r < block_rows; ++r) tile_val[tc * block_rows + r] = 0.0;
          }
          ++tc;
        }
        if (fill) tile_val[(tc - 1) * block_rows + e[y].r] += vals[e[y].k];
      }
      const int64_t t_real = tc - t_begin;
      const int64_t t_pad = (t_real + k_pad - 1) / k_pad * k_pad;
      for (int64_t p = t_real; p < t_pad; ++p) {
        if (fill) {
          tile_col[tc] = -1;
          for (int64_t r = 0; r < block_rows; ++r) tile_val[tc * block_rows + r] = 0.0;
        }
        ++tc;
      }
      if (fill) { rb_ids[rbc] = (int32_t)b; rb_ptr[rbc + 1] = tc; }
      ++rbc;
    }
    free(e);
    free(moved);
  }
  free(kind);
  if (!fill) { out_sizes[0] = rc; out_sizes[1] = kc; out_sizes[2] = rbc; out_sizes[3] = tc; }
  return 0;
}

/* out[0] = CSR-part rows, out[1] = CSR-part nnz, out[2] = BCSR row blocks, out[3] = BCSR tiles
 * (padding included). Returns 0. */
int oracle_partition_sizes(int64_t n_rows, const int64_t* row_ptr, const int32_t* col_idx,
                           int64_t block_rows, int64_t k_pad, double tau, int contiguous,
                           int64_t r_boundary, int64_t tile_min, int64_t* out) {
  return oracle_partition_run(n_rows, row_ptr, col_idx, NULL, block_rows, k_pad, tau, contiguous, r_boundary,
                              tile_min, out, NULL, NULL, NULL, NULL, NULL, NULL, NULL, NULL);
}

/* Fill the canonical partition. Arrays sized by oracle_partition_sizes:
 *   csr_rows[n_csr], csr_ptr[n_csr + 1], csr_col[nnz_csr], csr_val[nnz_csr]
 *   rb_ids[n_rb], rb_ptr[n_rb + 1], tile_col[n_tiles], tile_val[n_tiles * block_rows]
 * tile_val[t * B_r + r] holds the value of row (rb_id * B_r + r) in tile t (Algorithm 1 offset
 * (i mod B_r) * B_c + (j mod B_c) with B_c = 1). Values are the f64 sums of the input values.
 * With tile_min > 1 a CSR-part row may also lie in a BCSR block (its remaining entries). */
int oracle_partition_fill(int64_t n_rows, const int64_t* row_ptr, const int32_t* col_idx,
                          const double* vals, int64_t block_rows, int64_t k_pad, double tau,
                          int contiguous, int64_t r_boundary, int64_t tile_min, int32_t* csr_rows,
                          int64_t* csr_ptr, int32_t* csr_col, double* csr_val, int32_t* rb_ids,
                          int64_t* rb_ptr, int32_t* tile_col, double* tile_val) {
  return oracle_partition_run(n_rows, row_ptr, col_idx, vals, block_rows, k_pad, tau, contiguous, r_boundary,
                              tile_min, NULL, csr_rows, csr_ptr, csr_col, csr_val, rb_ids, rb_ptr, tile_col,
                              tile_val);
}
