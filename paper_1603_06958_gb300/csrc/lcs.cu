// Launch planning for the LCS kernels: split a row list (sorted by width)
// into segments of one kernel choice and launch thread-per-pair, sliced or
// warp-per-pair kernels over the family's length-sorted column groups.
#include <algorithm>
#include <atomic>

#include "lcs_kernels.cuh"

namespace famsa {

cudaError_t launch_tpp_a(int W, int R, const KParams &p, dim3 grid, cudaStream_t st);
cudaError_t launch_tpp_b(int W, int R, const KParams &p, dim3 grid, cudaStream_t st);
cudaError_t launch_tpp_c(int W, int R, const KParams &p, dim3 grid, cudaStream_t st);
cudaError_t launch_tpp_d(int W, int R, const KParams &p, dim3 grid, cudaStream_t st);

cudaError_t launch_slice_a(int WL, int G, const KParams &p, dim3 grid, cudaStream_t st);
cudaError_t launch_slice_b(int WL, int G, const KParams &p, dim3 grid, cudaStream_t st);

cudaError_t launch_slice(int WL, int G, const KParams &p, dim3 grid, cudaStream_t st) {
  if (WL < 1 || WL > kSliceWords || G < 1 || G > kSliceMaxG) return cudaErrorInvalidValue;
  return WL <= 8 ? launch_slice_a(WL, G, p, grid, st) : launch_slice_b(WL, G, p, grid, st);
}

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

// Rows wider than this do not use thread-per-pair (tests lower it to exercise the other kernels).
static std::atomic<int> g_tpp_max_w{kTppMaxW};
// Rows of at least this many words use the sliced kernel (0: never), in
// slices of at most g_slice_words words.  Thread-per-pair keeps a row's whole
// vector in one thread's registers; from 24 words on that costs it
// resident warps, and two or more slices of 12..16 words run faster.
static std::atomic<int> g_slice_min_w{kSliceMinW};
static std::atomic<int> g_slice_words{kSliceWords};

static int wpp_nw(int W) {
  int nw = 1;
  while (32 * nw < W) nw *= 2;
  return nw;
}

LcsChoice lcs_choice(int W) {
  const int smin = g_slice_min_w.load(), tmax = g_tpp_max_w.load();
  const bool slice = smin > 0 && W >= smin && W <= kSliceMaxW;
  if (W <= tmax && !slice) return LcsChoice{kLcsTpp, W, 1};
  if (slice) {
    // a power of two of slices (CTAs of 3, 5, 6, 7 warps measured 15-25 % slower
    // than 2 or 4), each as even as whole words allow
    const int wl0 = std::max(g_slice_words.load(), (W + kSliceMaxG - 1) / kSliceMaxG);
    int g = 1;
    while (g * wl0 < W) g *= 2;
    return LcsChoice{kLcsSlice, (W + g - 1) / g, g};
  }
  return LcsChoice{kLcsWpp, wpp_nw(W), 1};
}

cudaError_t launch_lcs(const LcsBatch &b, cudaStream_t st, int64_t *launches) {
  if (b.n_rows <= 0 || b.n_cols <= 0) return cudaSuccess;
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
    const LcsChoice c = lcs_choice(b.h_row_w[e0]);
    int32_t e1 = e0 + 1;
    while (e1 < b.n_rows && lcs_choice(b.h_row_w[e1]) == c) ++e1;
    p.e0 = e0;
    p.e1 = e1;
    // columns needed: triangle mode stops at the largest row id of the segment
    int64_t col_bound = b.triangle ? b.h_row_id[e1 - 1] : b.n_cols;
    if (col_bound > 0) {
      cudaError_t err;
      if (c.kind == kLcsTpp) {
        int R = tpp_rows(c.kw);
        dim3 grid((unsigned)((e1 - e0 + R - 1) / R), (unsigned)((col_bound + kTppThreads - 1) / kTppThreads));
        err = launch_tpp(c.kw, R, p, grid, st);
      } else if (c.kind == kLcsSlice) {
        dim3 grid((unsigned)(e1 - e0), (unsigned)((col_bound + kGroup - 1) / kGroup));
        err = launch_slice(c.kw, c.g, p, grid, st);
      } else {
        dim3 grid((unsigned)(e1 - e0), (unsigned)((col_bound + kWppCols - 1) / kWppCols));
        err = launch_wpp(c.kw, p, grid, st);
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

extern "C" int famsa_debug_set_slices(int min_w, int words) {
  if (min_w < 0 || words < 0 || words > famsa::kSliceWords) return FAMSA_EINVAL;
  famsa::g_slice_min_w.store(min_w);
  famsa::g_slice_words.store(words ? words : famsa::kSliceWords);
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
