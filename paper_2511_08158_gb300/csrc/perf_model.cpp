// The performance model of Sec. 3.5 (Eq. 2 and Eq. 3), restated for one GPU.
//
// On the M4 Pro, the model predicts a performance score from the numbers of threads given to
// the two parts: x NEON threads run the CSR part, y SME threads the BCSR part. Eq. 2 is
// perf(x, y) = a0 + a1 x + a2 y + a3 x^2 + a4 y^2. It has no cross term because the two parts
// run on their own pipelines. The coefficients are fitted by least squares over warm-up runs
// of candidate configurations, and Eq. 3 takes the configuration of highest predicted
// performance.
//
// On the GPU both parts run on every SM, so a configuration decides how much work each part
// gets rather than how many units:
//   x = CSR-part work   = stored entries of the CSR part x N (the B elements it gathers),
//   y = BCSR-part work  = tiles of the BCSR part x B_r x N (padding tiles included).
// A configuration is a split threshold (per matrix, in a batch). Its (x, y) follows from a
// profile of the row blocks (stored entries and distinct columns of each block), so every
// threshold can be predicted without building its plan. The quadratic is fitted to the
// measured time of the warm-up runs, and the performance score of Eq. 3 is the throughput
// flops / predicted time: on the GPU both parts' work adds to one time, which grows about
// linearly with the work, so a fit of the time extrapolates between and beyond the warm-up
// splits far better than a fit of the throughput.
#include <algorithm>
#include <cmath>
#include <thread>

#include "loops_internal.h"

namespace loops {

void block_profile(const loops_csr* A, int32_t br, BlockProfile& out) {
  const int64_t n_blocks = (A->n_rows + br - 1) / br;
  out.br = br;
  out.nnz.assign((size_t)n_blocks, 0);
  out.ucols.assign((size_t)n_blocks, 0);
  const int64_t* rp = A->row_ptr;
  const int32_t* ci = A->col_idx;
  unsigned hw = std::thread::hardware_concurrency();
  int n_thr = (int)std::max(1u, std::min(hw ? hw : 1u, 32u));
  if (A->nnz < (1 << 16)) n_thr = 1;
  const int64_t per = (n_blocks + n_thr - 1) / std::max(n_thr, 1);
  auto job = [&](int64_t b0, int64_t b1) {
    std::vector<int32_t> cols;
    for (int64_t b = b0; b < b1; ++b) {
      const int64_t k0 = rp[b * br], k1 = rp[std::min<int64_t>((b + 1) * br, A->n_rows)];
      cols.assign(ci + k0, ci + k1);
      std::sort(cols.begin(), cols.end());
      out.nnz[(size_t)b] = k1 - k0;
      out.ucols[(size_t)b] = (int64_t)(std::unique(cols.begin(), cols.end()) - cols.begin());
    }
  };
  std::vector<std::thread> thr;
  for (int t = 0; t < n_thr; ++t) {
    const int64_t b0 = std::min<int64_t>(n_blocks, t * per), b1 = std::min<int64_t>(n_blocks, b0 + per);
    if (n_thr == 1) job(b0, b1); else thr.emplace_back(job, b0, b1);
  }
  for (auto& th : thr) th.join();
}

// (x, y) of the split at threshold tau: the same rule as the partitioner (a non-empty block
// with nnz >= tau * distinct columns is BCSR; its tiles are padded to a multiple of kpad).
SplitWork split_work(const BlockProfile& p, double tau, int32_t kpad, int64_t N) {
  SplitWork w{0.0, 0.0};
  for (size_t b = 0; b < p.nnz.size(); ++b) {
    const int64_t nz = p.nnz[b], u = p.ucols[b];
    if (nz > 0 && (double)nz >= tau * (double)u)
      w.y += (double)((u + kpad - 1) / kpad * kpad) * p.br * (double)N;
    else
      w.x += (double)nz * (double)N;
  }
  return w;
}

std::vector<double> tau_grid(const BlockProfile& p, size_t max_cands) {
  std::vector<double> d;
  for (size_t b = 0; b < p.nnz.size(); ++b)
    if (p.nnz[b] > 0) d.push_back((double)p.nnz[b] / (double)p.ucols[b]);
  std::sort(d.begin(), d.end());
  d.erase(std::unique(d.begin(), d.end()), d.end());
  std::vector<double> g;
  g.push_back((double)INFINITY);
  if (d.size() <= max_cands) {
    g.insert(g.end(), d.begin(), d.end());
  } else {  // quantiles of the distinct block densities
    for (size_t i = 0; i < max_cands; ++i) g.push_back(d[i * (d.size() - 1) / (max_cands - 1)]);
  }
  g.push_back(0.0);
  return g;
}

// Least squares for the five coefficients of Eq. 2: the normal equations of the features
// (1, x, y, x^2, y^2), with x and y scaled to [0, 1] first (conditioning), solved by Gaussian
// elimination with partial pivoting in binary64. When the samples do not determine all five
// coefficients (samples on a line: one matrix, whose x and y move together), a pivot
// vanishes; the system is then solved again with a ridge of 1e-10 times its largest diagonal
// entry, which picks a solution that still fits the samples.
namespace {
bool solve5(double M[5][6], double ridge, double c[5]) {
  double A[5][6];
  double dmax = 0.0;
  for (int r = 0; r < 5; ++r) {
    for (int k = 0; k < 6; ++k) A[r][k] = M[r][k];
    dmax = std::max(dmax, A[r][r]);
  }
  if (dmax <= 0.0) return false;
  for (int r = 0; r < 5; ++r) A[r][r] += ridge * dmax;
  for (int col = 0; col < 5; ++col) {
    int piv = col;
    for (int r = col + 1; r < 5; ++r)
      if (std::fabs(A[r][col]) > std::fabs(A[piv][col])) piv = r;
    if (std::fabs(A[piv][col]) <= 1e-12 * dmax) return false;
    if (piv != col)
      for (int k = 0; k < 6; ++k) std::swap(A[col][k], A[piv][k]);
    for (int r = 0; r < 5; ++r) {
      if (r == col) continue;
      const double f = A[r][col] / A[col][col];
      for (int k = col; k < 6; ++k) A[r][k] -= f * A[col][k];
    }
  }
  for (int r = 0; r < 5; ++r) c[r] = A[r][5] / A[r][r];
  return true;
}
}  // namespace

bool fit_perf_model(const double* x, const double* y, const double* perf, int n, double a[5]) {
  for (int i = 0; i < 5; ++i) a[i] = 0.0;
  if (n <= 0) return false;
  double sx = 0.0, sy = 0.0;
  for (int i = 0; i < n; ++i) {
    sx = std::max(sx, std::fabs(x[i]));
    sy = std::max(sy, std::fabs(y[i]));
  }
  if (sx == 0.0) sx = 1.0;
  if (sy == 0.0) sy = 1.0;
  double M[5][6] = {};
  for (int i = 0; i < n; ++i) {
    const double u = x[i] / sx, v = y[i] / sy;
    const double f[5] = {1.0, u, v, u * u, v * v};
    for (int r = 0; r < 5; ++r) {
      for (int c = 0; c < 5; ++c) M[r][c] += f[r] * f[c];
      M[r][5] += f[r] * perf[i];
    }
  }
  double c[5];
  if (!solve5(M, 0.0, c) && !solve5(M, 1e-10, c)) return false;
  a[0] = c[0];
  a[1] = c[1] / sx;
  a[2] = c[2] / sy;
  a[3] = c[3] / (sx * sx);
  a[4] = c[4] / (sy * sy);
  for (int i = 0; i < 5; ++i)
    if (!std::isfinite(a[i])) return false;
  return true;
}

double eval_perf_model(const double a[5], double x, double y) {
  return a[0] + a[1] * x + a[2] * y + a[3] * x * x + a[4] * y * y;
}

}  // namespace loops

using namespace loops;

extern "C" {

loops_status loops_perf_model_fit(const double* x, const double* y, const double* perf, int32_t n, double* coef) {
  clear_error();
  if (!coef || n < 0 || (n > 0 && (!x || !y || !perf))) { set_error("bad arguments"); return LOOPS_ERR_INVALID_ARG; }
  if (!fit_perf_model(x, y, perf, n, coef)) { set_error("no least-squares solution"); return LOOPS_ERR_STATE; }
  return LOOPS_OK;
}

loops_status loops_perf_model_argmax(const double* coef, const double* x, const double* y, int32_t n,
                                     int32_t* best, double* best_perf) {
  clear_error();
  if (!coef || !best || n <= 0 || !x || !y) { set_error("bad arguments"); return LOOPS_ERR_INVALID_ARG; }
  int32_t b = 0;
  double bp = eval_perf_model(coef, x[0], y[0]);
  for (int32_t i = 1; i < n; ++i) {
    const double p = eval_perf_model(coef, x[i], y[i]);
    if (p > bp) { bp = p; b = i; }
  }
  *best = b;
  if (best_perf) *best_perf = bp;
  return LOOPS_OK;
}

}  // extern "C"
