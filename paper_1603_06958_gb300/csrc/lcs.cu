// Launch planning for the LCS kernels: split a row list (sorted by width)
// into segments of one kernel width and launch thread-per-pair or
// warp-per-pair kernels over the family's length-sorted column groups.
#include <atomic>

#include "lcs_kernels.cuh"

namespace famsa {

cudaError_t launch_tpp_a(int W, int R, const KParams &p, dim3 grid, cudaStream_t st);
cudaError_t launch_tpp_b(int W, int R, const KParams &p, dim3 grid, cudaStream_t st);
cudaError_t launch_tpp_c(int W, int R, const KParams &p, dim3 grid, cudaStream_t st);
cudaError_t launch_tpp_d(int W, int R, const KParams &p, dim3 grid, cudaStream_t st);

cudaError_t launch_tpp(int W, int R, const KParams &p, dim3 grid, cudaStream_t st) {
  if (W < 1 || W > kTppMaxW || !tpp_rows_allowed(W, R)) return cudaErrorInvalidValue;
  if (W <= 8) return launch_tpp_a(W, R, p, grid, st);
  if (W <= 16) return launch_tpp_b(W, R, p, grid, st);
  if (W <= 24) return launch_tpp_c(W, R, p, grid, st);
  return launch_tpp_d(W, R, p, grid, st);
}

// rows per tile for each width (0 = the default); the batch autotuner writes it
static std::atomic<int> g_tpp_rows[kTppMaxW + 1];

int tpp_rows(int W) {
  const int r = (W >= 1 && W <= kTppMaxW) ? g_tpp_rows[W].load() : 0;
  return r ? r : tpp_default_rows(W);
}

void set_tpp_rows(int W, int R) {
  if (W >= 1 && W <= kTppMaxW && (R == 0 || tpp_rows_allowed(W, R))) g_tpp_rows[W].store(R);
}

// Rows of 24..28 words take the step in parts (tpp_use_parts); tests and timing turn it off.
static std::atomic<int> g_tpp_parts{1};
bool tpp_parts_enabled() { return g_tpp_parts.load() != 0; }

// Rows wider than this use warp-per-pair (tests lower it to exercise that path).
static std::atomic<int> g_tpp_max_w{kTppMaxW};

static int wpp_nw(int W) {
  int nw = 1;
  while (32 * nw < W) nw *= 2;
  return nw;
}

cudaError_t launch_lcs(const LcsBatch &b, cudaStream_t st, int64_t *launches) {
  if (b.n_rows <= 0 || b.n_cols <= 0) return cudaSuccess;
  const int tmax = g_tpp_max_w.load();
  KParams p;
  p.peq = b.peq;
  p.row_peq_off = b.row_peq_off;
  p.row_len = b.row_len;
  p.row_id = b.row_id;
  p.row_orig = b.row_orig;
  p.colres = b.colres;
  p.group_off = b.group_off;
  p.group_chunks = b.group_chunks;
  p.col_perm = b.col_perm;
  p.col_len = b.col_len;
  p.n_cols = b.n_cols;
  p.n_groups = (b.n_cols + kGroup - 1) / kGroup;
  p.mode = b.mode;
  p.out = b.out;
  p.ld = b.ld;
  p.row0 = b.row0;
  p.k = b.k;
  p.triangle = b.triangle ? 1 : 0;
  p.items = nullptr;
  p.row_base = b.row_base;
  int32_t e0 = 0;
  while (e0 < b.n_rows) {
    const int w0 = b.h_row_w[e0];
    const bool wpp = w0 > tmax;
    const int kw = wpp ? wpp_nw(w0) : w0;
    int32_t e1 = e0 + 1;
    while (e1 < b.n_rows) {
      const int w = b.h_row_w[e1];
      const bool wp = w > tmax;
      if (wp != wpp || (wp ? wpp_nw(w) : w) != kw) break;
      ++e1;
    }
    p.e0 = e0;
    p.e1 = e1;
    // columns needed: triangle mode stops at the largest row id of the segment
    int64_t col_bound = b.triangle ? b.h_row_id[e1 - 1] : b.n_cols;
    if (col_bound > 0) {
      cudaError_t err;
      if (!wpp) {
        int R = tpp_rows(kw);
        dim3 grid((unsigned)((e1 - e0 + R - 1) / R), (unsigned)((col_bound + kTppThreads - 1) / kTppThreads));
        err = launch_tpp(kw, R, p, grid, st);
      } else {
        dim3 grid((unsigned)(e1 - e0), (unsigned)((col_bound + kWppCols - 1) / kWppCols));
        err = launch_wpp(kw, p, grid, st);
      }
      if (err != cudaSuccess) return err;
      if (launches) ++*launches;
    }
    e0 = e1;
  }
  return cudaSuccess;
}

}  // namespace famsa

extern "C" int famsa_debug_set_tpp_max_w(int w) {
  if (w < 0 || w > famsa::kTppMaxW) return FAMSA_EINVAL;
  famsa::g_tpp_max_w.store(w);
  return FAMSA_OK;
}

extern "C" int famsa_debug_set_tpp_parts(int on) {
  famsa::g_tpp_parts.store(on ? 1 : 0);
  return FAMSA_OK;
}

extern "C" int famsa_debug_set_tpp_rows(int w, int r) {
  if (w < 1 || w > famsa::kTppMaxW || (r != 0 && !famsa::tpp_rows_allowed(w, r))) return FAMSA_EINVAL;
  famsa::set_tpp_rows(w, r);
  return FAMSA_OK;
}

extern "C" int famsa_debug_tpp_rows(int w) {
  if (w < 1 || w > famsa::kTppMaxW) return -1;
  return famsa::tpp_rows(w);
}
