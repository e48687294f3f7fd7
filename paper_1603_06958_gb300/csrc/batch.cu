// Batched families: many independent families packed side by side and built
// into guide trees by one CUDA graph.
//
// FAMSA Methods, "Pairwise similarities calculation" and "Determination of
// the guide tree", applied to every family of a batch at once.  The families
// share one length-sorted layout in which each family's block of sorted
// positions is padded to a multiple of 32, so no 32-sequence column group
// mixes families.  The LCS kernels then run over explicit work lists, one
// launch per kernel width, covering the lower triangle of every family:
// small families no longer leave the GPU idle between launches.  The 16-bit
// rows of each family stay in HBM, and the row update runs one cluster per
// family (state in that cluster's shared memory), all families of one
// cluster size in one launch.  The finalisation gives each family's pointer
// representation and merge list in that family's own labels.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <mutex>
#include <numeric>
#include <vector>

#include "lcs_kernels.cuh"
#include "slink_common.cuh"

namespace famsa {

// packing kernels shared with the single-family path (pack.cu)
__global__ void k_lengths(const int64_t *off, int32_t k, int64_t base, int32_t *len, int64_t *off0,
                          int *status, int *max_len);
__global__ void k_codes(const uint8_t *res, int64_t n, int *status);
__global__ void k_merge_pass(const uint64_t *in, uint64_t *out, int32_t n, int32_t width);
__global__ void k_scan_excl(const int64_t *in, int64_t *out, int64_t n, int64_t *total);
__global__ void k_pack_peq(const uint8_t *res, const int64_t *off, const int32_t *map,
                           const int64_t *peq_off, int32_t n, uint32_t *peq);
__global__ void k_col_layout(const uint8_t *res, const int64_t *off, const int32_t *perm,
                             const int32_t *slen, int32_t k, const int64_t *group_off,
                             const int32_t *group_chunks, uint8_t *colres);

// sort key (family, length, index): 16 + 16 + 32 bits
__global__ void k_batch_keys(const int32_t *len, const int64_t *fam_off, int32_t F, int32_t N,
                             uint64_t *keys) {
  const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  int32_t lo = 0, hi = F - 1;  // the family holding sequence i
  while (lo < hi) {
    const int32_t mid = (lo + hi + 1) >> 1;
    if (fam_off[mid] <= i) lo = mid; else hi = mid - 1;
  }
  keys[i] = ((uint64_t)lo << 48) | ((uint64_t)(uint32_t)len[i] << 32) | (uint32_t)i;
}

// sorted rank s -> padded position S[f] + (s - fam_off[f]); pads keep perm -1, length 0
__global__ void k_batch_fields(const uint64_t *keys, int32_t N, const int64_t *fam_off,
                               const int64_t *S, int32_t *perm, int32_t *perm_local,
                               int32_t *slen, int64_t *words) {
  const int32_t s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= N) return;
  const uint64_t key = keys[s];
  const int32_t f = (int32_t)(key >> 48);
  const int32_t l = (int32_t)((key >> 32) & 0xffffu);
  const int32_t idx = (int32_t)(key & 0xffffffffu);
  const int64_t P = S[f] + (s - fam_off[f]);
  perm[P] = idx;
  perm_local[P] = (int32_t)(idx - fam_off[f]);
  slen[P] = l;
  words[P] = (l + 63) / 64;
}

__global__ void k_batch_group_sizes(const int32_t *slen, int32_t n_groups, int32_t *chunks,
                                    int64_t *bytes) {
  const int32_t g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= n_groups) return;
  int32_t mx = 0;
  for (int j = 0; j < kGroup; ++j) mx = max(mx, slen[(int64_t)g * kGroup + j]);
  const int32_t c = (mx + kChunk - 1) / kChunk;
  chunks[g] = c;
  bytes[g] = (int64_t)c * kGroup * kChunk;
}

// the layout of one point (point 0) in buffer 1 of every family's state, and
// the outputs of single-point families
struct BatchInit {
  int32_t *ord1, *olen1, *pi1;
  uint64_t *lam1;
  uint64_t inf;          // +inf in the key packing of the family's row-update kernel
  int32_t len0;
  int32_t single;        // 1: the family is one point
  int64_t out_at;        // its output position
};
__global__ void k_batch_init(const BatchInit *d, int32_t n, int32_t *pi_out, uint64_t *lnum_out,
                             uint32_t *lden_out) {
  const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const BatchInit b = d[i];
  if (b.single) {
    pi_out[b.out_at] = 0;
    lnum_out[b.out_at] = 1;
    lden_out[b.out_at] = 0;
    return;
  }
  b.ord1[0] = 0;
  b.olen1[0] = b.len0;
  b.lam1[0] = b.inf;
  b.pi1[0] = 0;
}

struct Batch {
  int device = 0;
  int32_t F = 0, N = 0;
  int64_t Kpad = 0;
  int32_t max_len = 0;
  std::vector<int64_t> fam_off, S;  // F+1 each
  std::vector<int32_t> h_slen;      // Kpad
  uint8_t *d_res = nullptr;
  int64_t *d_off = nullptr, *d_fam_off = nullptr, *d_S = nullptr;
  int32_t *d_len = nullptr, *d_perm = nullptr, *d_perm_local = nullptr, *d_slen = nullptr;
  int64_t *d_peq_off = nullptr;
  uint32_t *d_peq = nullptr;
  int32_t n_groups = 0;
  int64_t *d_group_off = nullptr;
  int32_t *d_group_chunks = nullptr;
  uint8_t *d_colres = nullptr;
  // execution plan (built by the first tree call)
  bool planned = false;
  std::vector<void *> plan_mem;
  cudaStream_t cap = nullptr;
  std::vector<cudaStream_t> side;
  std::vector<cudaEvent_t> ev, ev_stage;
  cudaGraphExec_t exec = nullptr;
  int32_t *d_pi = nullptr, *d_merges = nullptr, *d_sizes = nullptr;
  uint64_t *d_lnum = nullptr, *d_hnum = nullptr;
  uint32_t *d_lden = nullptr, *d_hden = nullptr;
  // graph start, LCS, update, end: recorded by event-record nodes of the graph
  cudaEvent_t tev[4] = {nullptr, nullptr, nullptr, nullptr};
  bool launched = false;
  int64_t stats[16] = {0};
  std::mutex mu;
};

static void batch_free_plan(Batch *b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  b->exec = nullptr;
  for (auto e : b->ev) cudaEventDestroy(e);
  b->ev.clear();
  for (auto e : b->ev_stage) cudaEventDestroy(e);
  b->ev_stage.clear();
  for (auto &e : b->tev) {
    if (e) cudaEventDestroy(e);
    e = nullptr;
  }
  b->launched = false;
  for (auto s : b->side) cudaStreamDestroy(s);
  b->side.clear();
  if (b->cap) cudaStreamDestroy(b->cap);
  b->cap = nullptr;
  for (void *p : b->plan_mem) dev_free(p);
  b->plan_mem.clear();
  b->planned = false;
}

static void batch_free(Batch *b) {
  if (!b) return;
  batch_free_plan(b);
  dev_free(b->d_res); dev_free(b->d_off); dev_free(b->d_fam_off); dev_free(b->d_S);
  dev_free(b->d_len); dev_free(b->d_perm); dev_free(b->d_perm_local); dev_free(b->d_slen);
  dev_free(b->d_peq_off); dev_free(b->d_peq); dev_free(b->d_group_off);
  dev_free(b->d_group_chunks); dev_free(b->d_colres);
  delete b;
}

static unsigned nblk(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

#define BCK(x)                                          \
  do {                                                  \
    cudaError_t e_ = (x);                               \
    if (e_ != cudaSuccess) { err = e_; goto fail; }     \
  } while (0)

static int batch_pack(const uint8_t *residues, const int64_t *offsets, int64_t n_seqs,
                      const int64_t *fam_off, int32_t F, bool on_device, cudaStream_t st,
                      Batch **out) {
  *out = nullptr;
  if (n_seqs < 1 || n_seqs >= (1ll << 31) || F < 1 || F > 65535 || !fam_off) return FAMSA_EINVAL;
  if (fam_off[0] != 0 || fam_off[F] != n_seqs) return FAMSA_EINVAL;
  for (int32_t f = 0; f < F; ++f)
    if (fam_off[f + 1] <= fam_off[f]) return FAMSA_EINVAL;
  const int32_t N = (int32_t)n_seqs;
  AllocStream alloc_on(st);
  Batch *b = new Batch();
  cudaError_t err = cudaSuccess;
  cudaGetDevice(&b->device);
  b->F = F;
  b->N = N;
  b->fam_off.assign(fam_off, fam_off + F + 1);
  b->S.resize(F + 1);
  b->S[0] = 0;
  for (int32_t f = 0; f < F; ++f)
    b->S[f + 1] = b->S[f] + ((fam_off[f + 1] - fam_off[f] + kGroup - 1) / kGroup) * kGroup;
  b->Kpad = b->S[F];
  b->n_groups = (int32_t)(b->Kpad / kGroup);
  const int T = 256;
  int64_t base = 0, total = 0;
  int64_t *d_off_in = nullptr, *words = nullptr, *gbytes = nullptr, *d_tot = nullptr;
  uint64_t *keys = nullptr, *keys2 = nullptr;
  int *d_status = nullptr;
  int h_status[2] = {0, 0};
  int64_t h_tot[2] = {0, 0};
  if (on_device) {
    int64_t ends[2];
    BCK(cudaMemcpyAsync(&ends[0], offsets, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    BCK(cudaMemcpyAsync(&ends[1], offsets + N, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    BCK(cudaStreamSynchronize(st));
    base = ends[0];
    total = ends[1] - ends[0];
    d_off_in = const_cast<int64_t *>(offsets);
  } else {
    for (int32_t i = 0; i < N; ++i)
      if (offsets[i + 1] <= offsets[i]) { batch_free(b); return FAMSA_EINVAL; }
    for (int32_t i = 0; i < N; ++i)
      if (offsets[i + 1] - offsets[i] > kMaxLen) { batch_free(b); return FAMSA_ERANGE; }
    base = offsets[0];
    total = offsets[N] - offsets[0];
  }
  if (base < 0 || total < N) { batch_free(b); return FAMSA_EINVAL; }
  BCK(dev_alloc((void **)&b->d_off, sizeof(int64_t) * (N + 1)));
  BCK(dev_alloc((void **)&b->d_res, (size_t)total));
  BCK(dev_alloc((void **)&b->d_len, sizeof(int32_t) * N));
  BCK(dev_alloc((void **)&d_status, sizeof(int) * 2));
  BCK(cudaMemsetAsync(d_status, 0, sizeof(int) * 2, st));
  if (on_device) {
    BCK(cudaMemcpyAsync(b->d_res, residues + base, (size_t)total, cudaMemcpyDeviceToDevice, st));
  } else {
    BCK(dev_alloc((void **)&d_off_in, sizeof(int64_t) * (N + 1)));
    BCK(cudaMemcpyAsync(d_off_in, offsets, sizeof(int64_t) * (N + 1), cudaMemcpyHostToDevice, st));
    BCK(cudaMemcpyAsync(b->d_res, residues + base, (size_t)total, cudaMemcpyHostToDevice, st));
  }
  k_lengths<<<nblk(N + 1, T), T, 0, st>>>(d_off_in, N, base, b->d_len, b->d_off, d_status,
                                          d_status + 1);
  k_codes<<<std::min<int64_t>(nblk(total, T), 4096), T, 0, st>>>(b->d_res, total, d_status);
  BCK(cudaGetLastError());
  BCK(cudaMemcpyAsync(h_status, d_status, sizeof(int) * 2, cudaMemcpyDeviceToHost, st));
  BCK(cudaStreamSynchronize(st));
  if (!on_device) { dev_free(d_off_in); d_off_in = nullptr; }
  if (h_status[0]) {
    dev_free(d_status);
    batch_free(b);
    return (h_status[0] & kTooLong) ? FAMSA_ERANGE : FAMSA_EINVAL;
  }
  b->max_len = h_status[1];

  // sort by (family, length, index), then the padded sorted layout
  BCK(dev_alloc((void **)&b->d_fam_off, sizeof(int64_t) * (F + 1)));
  BCK(dev_alloc((void **)&b->d_S, sizeof(int64_t) * (F + 1)));
  BCK(cudaMemcpyAsync(b->d_fam_off, fam_off, sizeof(int64_t) * (F + 1), cudaMemcpyHostToDevice, st));
  BCK(cudaMemcpyAsync(b->d_S, b->S.data(), sizeof(int64_t) * (F + 1), cudaMemcpyHostToDevice, st));
  BCK(dev_alloc((void **)&keys, sizeof(uint64_t) * N));
  BCK(dev_alloc((void **)&keys2, sizeof(uint64_t) * N));
  k_batch_keys<<<nblk(N, T), T, 0, st>>>(b->d_len, b->d_fam_off, F, N, keys);
  for (int64_t width = 1; width < N; width *= 2) {
    k_merge_pass<<<nblk(N, T), T, 0, st>>>(keys, keys2, N, (int32_t)width);
    std::swap(keys, keys2);
  }
  BCK(dev_alloc((void **)&b->d_perm, sizeof(int32_t) * b->Kpad));
  BCK(dev_alloc((void **)&b->d_perm_local, sizeof(int32_t) * b->Kpad));
  BCK(dev_alloc((void **)&b->d_slen, sizeof(int32_t) * b->Kpad));
  BCK(dev_alloc((void **)&b->d_peq_off, sizeof(int64_t) * (b->Kpad + 1)));
  BCK(dev_alloc((void **)&words, sizeof(int64_t) * (b->Kpad + 1)));
  BCK(dev_alloc((void **)&d_tot, sizeof(int64_t) * 2));
  BCK(cudaMemsetAsync(b->d_perm, 0xff, sizeof(int32_t) * b->Kpad, st));
  BCK(cudaMemsetAsync(b->d_perm_local, 0xff, sizeof(int32_t) * b->Kpad, st));
  BCK(cudaMemsetAsync(b->d_slen, 0, sizeof(int32_t) * b->Kpad, st));
  BCK(cudaMemsetAsync(words, 0, sizeof(int64_t) * (b->Kpad + 1), st));
  k_batch_fields<<<nblk(N, T), T, 0, st>>>(keys, N, b->d_fam_off, b->d_S, b->d_perm,
                                           b->d_perm_local, b->d_slen, words);
  k_scan_excl<<<1, 1024, 0, st>>>(words, b->d_peq_off, b->Kpad, d_tot);
  BCK(cudaGetLastError());
  BCK(dev_alloc((void **)&b->d_group_chunks, sizeof(int32_t) * b->n_groups));
  BCK(dev_alloc((void **)&b->d_group_off, sizeof(int64_t) * (b->n_groups + 1)));
  BCK(dev_alloc((void **)&gbytes, sizeof(int64_t) * b->n_groups));
  k_batch_group_sizes<<<nblk(b->n_groups, T), T, 0, st>>>(b->d_slen, b->n_groups, b->d_group_chunks,
                                                          gbytes);
  k_scan_excl<<<1, 1024, 0, st>>>(gbytes, b->d_group_off, b->n_groups, d_tot + 1);
  BCK(cudaGetLastError());
  BCK(cudaMemcpyAsync(h_tot, d_tot, sizeof(int64_t) * 2, cudaMemcpyDeviceToHost, st));
  b->h_slen.resize(b->Kpad);
  BCK(cudaMemcpyAsync(b->h_slen.data(), b->d_slen, sizeof(int32_t) * b->Kpad, cudaMemcpyDeviceToHost, st));
  BCK(cudaStreamSynchronize(st));
  BCK(cudaMemcpyAsync(b->d_peq_off + b->Kpad, &d_tot[0], sizeof(int64_t), cudaMemcpyDeviceToDevice, st));
  BCK(cudaMemcpyAsync(b->d_group_off + b->n_groups, &d_tot[1], sizeof(int64_t),
                      cudaMemcpyDeviceToDevice, st));
  BCK(dev_alloc((void **)&b->d_peq, sizeof(uint32_t) * kPeqWordU32 * (size_t)std::max<int64_t>(h_tot[0], 1)));
  BCK(dev_alloc((void **)&b->d_colres, (size_t)std::max<int64_t>(h_tot[1], 16)));
  k_pack_peq<<<nblk(b->Kpad * 32, T), T, 0, st>>>(b->d_res, b->d_off, b->d_perm, b->d_peq_off,
                                                  (int32_t)b->Kpad, b->d_peq);
  k_col_layout<<<b->n_groups, 256, 0, st>>>(b->d_res, b->d_off, b->d_perm, b->d_slen,
                                            (int32_t)b->Kpad, b->d_group_off, b->d_group_chunks,
                                            b->d_colres);
  BCK(cudaGetLastError());
  BCK(cudaStreamSynchronize(st));
  dev_free(keys); dev_free(keys2); dev_free(words); dev_free(gbytes); dev_free(d_tot);
  dev_free(d_status);
  *out = b;
  return FAMSA_OK;

fail:
  cudaStreamSynchronize(st);
  if (!on_device) dev_free(d_off_in);
  dev_free(keys); dev_free(keys2); dev_free(words); dev_free(gbytes); dev_free(d_tot);
  dev_free(d_status);
  batch_free(b);
  return status_from_cuda(err);
}

// ---------------------------------------------------------------- the plan
struct Arena {
  std::vector<void *> *mem;
  cudaError_t err = cudaSuccess;
  template <typename T>
  T *get(size_t n) {
    void *p = nullptr;
    if (err != cudaSuccess) return nullptr;
    err = dev_alloc(&p, std::max<size_t>(n, 1) * sizeof(T));
    if (err != cudaSuccess) return nullptr;
    mem->push_back(p);
    return static_cast<T *>(p);
  }
};

template <typename T>
static cudaError_t upload_vec(Arena &A, const std::vector<T> &v, T **d, cudaStream_t st) {
  *d = A.get<T>(v.size());
  if (A.err != cudaSuccess) return A.err;
  if (v.empty()) return cudaSuccess;
  return cudaMemcpyAsync(*d, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice, st);
}

struct Bucket {
  LcsChoice c;  // the LCS kernel of its rows (lcs_choice of their width)
  int R = 1;    // rows per tile
  // one descriptor per row tile: (first row entry, rows, first column group,
  // group step); its work items take the column groups gstart + j * gstep
  std::vector<int4> tiles;
  std::vector<int32_t> tile_items;
};

struct BRow {
  int32_t rid;
  int32_t f;
};

// Row entries (Peq offset, length, sorted id, output base) and work items of
// a list of rows, tiles of at most R rows of one family.
struct RowArrays {
  std::vector<int64_t> peq, base;
  std::vector<int32_t> len, id;
};

// columns per work item: thread-per-pair 4 groups, sliced 1 group, warp-per-pair kWppCols
static int item_cols(const LcsChoice &c) {
  return c.kind == kLcsTpp ? 4 * kGroup : (c.kind == kLcsSlice ? kGroup : kWppCols);
}

static void append_rows(const Batch *b, const std::vector<BRow> &rows, size_t count, int cols, int R,
                        const std::vector<int64_t> &h_peq_off, const std::vector<int64_t> &rb_off,
                        const std::vector<int64_t> &ld, RowArrays &ra, std::vector<int4> &tiles,
                        std::vector<int32_t> &tile_items) {
  size_t i = 0;
  while (i < count) {
    const int32_t f = rows[i].f;
    size_t j = i + 1;
    while (j < count && j - i < (size_t)R && rows[j].f == f) ++j;
    const int32_t e0 = (int32_t)ra.id.size();
    for (size_t q = i; q < j; ++q) {
      const int32_t rid = rows[q].rid;
      ra.peq.push_back(h_peq_off[rid]);
      ra.len.push_back(b->h_slen[rid]);
      ra.id.push_back(rid);
      ra.base.push_back(rb_off[f] + (int64_t)(rid - b->S[f] - 1) * ld[f] - b->S[f]);
    }
    // the tile meets the columns [S[f], rid_last), `cols` of them per item
    const int32_t rid_last = rows[j - 1].rid;
    const int32_t g0 = (int32_t)(b->S[f] / kGroup);  // S[f] is a multiple of kGroup
    const int32_t span = rid_last - g0 * kGroup;
    tiles.push_back(make_int4(e0, (int)(j - i), g0, cols / kGroup));
    tile_items.push_back(span > 0 ? (span + cols - 1) / cols : 0);
    i = j;
  }
}

// Work items from tile descriptors, one warp per tile: item j of tile t is
// (e0, rows, gstart + j * gstep, 0), written at items[tstart[t] + j].
__global__ void k_expand_items(const int4 *tiles, const int64_t *tstart, int64_t n_tiles, int4 *items) {
  const int64_t t = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (t >= n_tiles) return;
  const int4 d = tiles[t];
  const int64_t o = tstart[t], n = tstart[t + 1] - o;
  for (int64_t j = threadIdx.x & 31; j < n; j += 32) items[o + j] = make_int4(d.x, d.y, d.z + (int)j * d.w, 0);
}

static void expand_on_host(const std::vector<int4> &tiles, const std::vector<int32_t> &tile_items,
                           std::vector<int4> &items) {
  for (size_t t = 0; t < tiles.size(); ++t)
    for (int32_t j = 0; j < tile_items[t]; ++j)
      items.push_back(make_int4(tiles[t].x, tiles[t].y, tiles[t].z + j * tiles[t].w, 0));
}

static KParams batch_params(const Batch *b, uint16_t *rowbuf) {
  KParams p = {};
  p.peq = b->d_peq;
  p.colres = b->d_colres;
  p.group_off = b->d_group_off;
  p.group_chunks = b->d_group_chunks;
  p.col_perm = b->d_perm;
  p.col_len = b->d_slen;
  p.n_cols = (int32_t)b->Kpad;
  p.n_groups = b->n_groups;
  p.mode = kOutBatch;
  p.out = rowbuf;
  p.triangle = 1;
  return p;
}

// ---- the autotuner: rows per thread-per-pair tile, per kernel width.  The
// first batch with enough rows of a width times each allowed R on the same
// sample of its rows (identical work) and keeps the fastest for the process
// (the single-family launch planner uses it too).  The sample is sized by
// work, about 4e9 word steps (1.5 ms at the kernel's rate), so that every R
// fills the GPU many times over: a sample of a few hundred CTAs favours the
// smallest R only because it makes more of them.  Another R replaces the
// default only when it is at least 2% faster.
// Groups of LCS widths after which row updates may start.  Four groups
// (updates of the narrow families beside the LCS of the wide buckets) were
// measured no faster on 512 families: a row-update cluster holds whole SMs
// while it waits at its barriers, so what it saves at the end it costs the
// LCS.  One group: every update after the last LCS launch.
constexpr int kStageGroups = 1;

static std::mutex g_tune_mu;
static bool g_tuned[kTppMaxW + 1] = {false};
static std::atomic<int> g_autotune{1};
constexpr size_t kTuneMinRows = 64;
constexpr double kTuneWordSteps = 4e9, kTuneMargin = 0.98;

static cudaError_t time_rows(const Batch *b, uint16_t *rowbuf, const std::vector<BRow> &rows, size_t count,
                             int W, int R, const std::vector<int64_t> &h_peq_off,
                             const std::vector<int64_t> &rb_off, const std::vector<int64_t> &ld,
                             cudaStream_t st, float *ms) {
  RowArrays ra;
  std::vector<int4> tiles, items;
  std::vector<int32_t> tile_items;
  append_rows(b, rows, count, 4 * kGroup, R, h_peq_off, rb_off, ld, ra, tiles, tile_items);
  expand_on_host(tiles, tile_items, items);
  int64_t *d_peq = nullptr, *d_base = nullptr;
  int32_t *d_len = nullptr, *d_id = nullptr;
  int4 *d_items = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t err = dev_alloc((void **)&d_peq, sizeof(int64_t) * ra.peq.size());
  if (err == cudaSuccess) err = dev_alloc((void **)&d_base, sizeof(int64_t) * ra.base.size());
  if (err == cudaSuccess) err = dev_alloc((void **)&d_len, sizeof(int32_t) * ra.len.size());
  if (err == cudaSuccess) err = dev_alloc((void **)&d_id, sizeof(int32_t) * ra.id.size());
  if (err == cudaSuccess) err = dev_alloc((void **)&d_items, sizeof(int4) * items.size());
  if (err == cudaSuccess) err = cudaMemcpyAsync(d_peq, ra.peq.data(), sizeof(int64_t) * ra.peq.size(), cudaMemcpyHostToDevice, st);
  if (err == cudaSuccess) err = cudaMemcpyAsync(d_base, ra.base.data(), sizeof(int64_t) * ra.base.size(), cudaMemcpyHostToDevice, st);
  if (err == cudaSuccess) err = cudaMemcpyAsync(d_len, ra.len.data(), sizeof(int32_t) * ra.len.size(), cudaMemcpyHostToDevice, st);
  if (err == cudaSuccess) err = cudaMemcpyAsync(d_id, ra.id.data(), sizeof(int32_t) * ra.id.size(), cudaMemcpyHostToDevice, st);
  if (err == cudaSuccess) err = cudaMemcpyAsync(d_items, items.data(), sizeof(int4) * items.size(), cudaMemcpyHostToDevice, st);
  if (err == cudaSuccess) err = cudaEventCreate(&e0);
  if (err == cudaSuccess) err = cudaEventCreate(&e1);
  if (err == cudaSuccess) {
    KParams p = batch_params(b, rowbuf);
    p.row_peq_off = d_peq;
    p.row_len = d_len;
    p.row_id = d_id;
    p.row_base = d_base;
    p.items = d_items;
    p.e0 = 0;
    p.e1 = (int32_t)ra.id.size();
    const dim3 grid((unsigned)items.size());
    err = launch_tpp(W, R, p, grid, st);  // warm-up
    if (err == cudaSuccess) err = cudaEventRecord(e0, st);
    for (int i = 0; i < 2 && err == cudaSuccess; ++i) err = launch_tpp(W, R, p, grid, st);
    if (err == cudaSuccess) err = cudaEventRecord(e1, st);
    if (err == cudaSuccess) err = cudaEventSynchronize(e1);
    if (err == cudaSuccess) err = cudaEventElapsedTime(ms, e0, e1);
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  dev_free(d_peq); dev_free(d_base); dev_free(d_len); dev_free(d_id); dev_free(d_items);
  return err;
}

// autotune rows per tile for the widths of this batch not tuned yet in this process
static cudaError_t autotune_rows(Batch *b, uint16_t *rowbuf, const std::vector<Bucket> &buckets,
                                 const std::vector<std::vector<BRow>> &rows_by_bucket,
                                 const std::vector<int64_t> &h_peq_off, const std::vector<int64_t> &rb_off,
                                 const std::vector<int64_t> &ld, cudaStream_t st) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  const auto t0 = std::chrono::steady_clock::now();
  std::vector<int64_t> len_pre(b->Kpad + 1, 0);  // residues before each sorted position
  for (int64_t s = 0; s < b->Kpad; ++s) len_pre[s + 1] = len_pre[s] + b->h_slen[s];
  for (size_t bk = 0; bk < buckets.size(); ++bk) {
    const Bucket &B = buckets[bk];
    const auto &rows = rows_by_bucket[bk];
    if (B.c.kind != kLcsTpp || g_tuned[B.c.kw] || rows.size() < kTuneMinRows) continue;
    // rows in bucket order until the sample holds kTuneWordSteps (a row of W
    // words takes W word steps per residue of the columns before it)
    size_t count = 0;
    double steps = 0.0;
    while (count < rows.size() && steps < kTuneWordSteps) {
      const BRow &r = rows[count];
      steps += (double)B.c.kw * (double)(len_pre[r.rid] - len_pre[b->S[r.f]]);
      ++count;
    }
    const int W = B.c.kw;
    const int R0 = tpp_default_rows(W);
    int best_R = R0;
    float best_ms = 0.f;
    cudaError_t e = time_rows(b, rowbuf, rows, count, W, R0, h_peq_off, rb_off, ld, st, &best_ms);
    if (e != cudaSuccess) return e;
    const float bar = best_ms * (float)kTuneMargin;
    for (int R : {1, 2, 4}) {
      if (R == R0 || !tpp_rows_allowed(W, R)) continue;
      float ms = 0.f;
      e = time_rows(b, rowbuf, rows, count, W, R, h_peq_off, rb_off, ld, st, &ms);
      if (e != cudaSuccess) return e;
      if (ms < bar && ms < best_ms) { best_ms = ms; best_R = R; }
    }
    set_tpp_rows(W, best_R);
    g_tuned[W] = true;
    b->stats[10] += 1;
  }
  b->stats[11] = std::chrono::duration_cast<std::chrono::nanoseconds>(std::chrono::steady_clock::now() - t0).count();
  return cudaSuccess;
}

static int batch_plan(Batch *b, cudaStream_t st) {
  AllocStream alloc_on(st);
  const auto t_plan0 = std::chrono::steady_clock::now();
  auto ns_since = [](std::chrono::steady_clock::time_point t) {
    return (int64_t)std::chrono::duration_cast<std::chrono::nanoseconds>(std::chrono::steady_clock::now() - t).count();
  };
  const int32_t F = b->F;
  RowArrays ra;  // row entries of every bucket, concatenated
  Arena A{&b->plan_mem};
  cudaError_t err = cudaSuccess;
  const int T = 256;
  // per-family sizes and row blocks (rows 1..k-1 of each family, its own leading dimension)
  std::vector<int64_t> rb_off(F + 1, 0), ld(F);
  for (int32_t f = 0; f < F; ++f) {
    const int64_t k = b->fam_off[f + 1] - b->fam_off[f];
    ld[f] = (k + 1) & ~1ll;
    rb_off[f + 1] = rb_off[f] + (k - 1) * ld[f];
  }
  // row entries, grouped by kernel width; within a width, family by family
  std::vector<Bucket> buckets;
  std::vector<int> bucket_of(kMaxLen / 64 + 2, -1);  // per row width
  auto bucket_for = [&](int W) -> int {
    if (bucket_of[W] < 0) {
      const LcsChoice c = lcs_choice(W);
      for (size_t i = 0; i < buckets.size() && bucket_of[W] < 0; ++i)
        if (buckets[i].c == c) bucket_of[W] = (int)i;
      if (bucket_of[W] < 0) {
        bucket_of[W] = (int)buckets.size();
        buckets.push_back(Bucket{c});
      }
    }
    return bucket_of[W];
  };
  std::vector<std::vector<int64_t>> e_peq(1), e_base(1);
  std::vector<std::vector<int32_t>> e_len(1), e_id(1);
  // first pass: which rows go to which bucket, in order
  std::vector<std::vector<BRow>> rows_by_bucket;
  int64_t cells = 0, words = 0, pairs = 0;
  std::vector<int64_t> h_peq_off(b->Kpad + 1, 0);
  for (int64_t s = 0; s < b->Kpad; ++s) h_peq_off[s + 1] = h_peq_off[s] + (b->h_slen[s] + 63) / 64;
  for (int32_t f = 0; f < F; ++f) {
    const int32_t k = (int32_t)(b->fam_off[f + 1] - b->fam_off[f]);
    int64_t colsum = 0;
    pairs += (int64_t)k * (k - 1) / 2;
    for (int32_t n = 0; n < k; ++n) {
      const int32_t rid = (int32_t)(b->S[f] + n);
      const int32_t l = b->h_slen[rid];
      const int W = (l + 63) / 64;
      words += (int64_t)W * colsum;
      cells += (int64_t)l * colsum;
      colsum += l;
      if (n == 0) continue;
      const int bk = bucket_for(W);
      if ((int)rows_by_bucket.size() <= bk) rows_by_bucket.resize(bk + 1);
      rows_by_bucket[bk].push_back(BRow{rid, f});
    }
  }
  // buckets in increasing width, and the families in kStageGroups groups by
  // the last bucket that holds one of their rows: a family's row update can
  // start as soon as its group's LCS launches are done, beside the LCS of the
  // wider buckets (groups cut the LCS work into about equal parts)
  {
    std::vector<int> order(buckets.size());
    std::iota(order.begin(), order.end(), 0);
    std::sort(order.begin(), order.end(), [&](int x, int y) {
      const LcsChoice &a = buckets[x].c, &c = buckets[y].c;
      return a.kind != c.kind ? a.kind < c.kind : a.kw * a.g < c.kw * c.g;
    });
    std::vector<Bucket> nb;
    std::vector<std::vector<BRow>> nr;
    for (int i : order) {
      nb.push_back(std::move(buckets[i]));
      nr.push_back(std::move(rows_by_bucket[i]));
    }
    buckets.swap(nb);
    rows_by_bucket.swap(nr);
  }
  std::vector<int> bucket_group(buckets.size(), 0), fam_group(F, 0);
  {
    std::vector<int64_t> len_pre(b->Kpad + 1, 0);
    for (int64_t s = 0; s < b->Kpad; ++s) len_pre[s + 1] = len_pre[s] + b->h_slen[s];
    std::vector<double> work(buckets.size(), 0.0);
    std::vector<int> fam_last(F, -1);
    double total = 0.0;
    for (size_t bk = 0; bk < buckets.size(); ++bk) {
      for (const BRow &r : rows_by_bucket[bk]) {
        const int W = (b->h_slen[r.rid] + 63) / 64;
        work[bk] += (double)W * (double)(len_pre[r.rid] - len_pre[b->S[r.f]]);
        fam_last[r.f] = std::max(fam_last[r.f], (int)bk);
      }
      total += work[bk];
    }
    double before = 0.0;
    for (size_t bk = 0; bk < buckets.size(); ++bk) {
      bucket_group[bk] = total > 0 ? std::min(kStageGroups - 1, (int)(kStageGroups * before / total)) : 0;
      before += work[bk];
    }
    for (int32_t f = 0; f < F; ++f) fam_group[f] = fam_last[f] < 0 ? 0 : bucket_group[fam_last[f]];
  }
  // the row blocks (the autotuner's trial launches write into them too)
  cudaError_t pre_err = cudaSuccess;
  uint16_t *rowbuf = A.get<uint16_t>((size_t)rb_off[F]);
  if (A.err != cudaSuccess) pre_err = A.err;
  if (pre_err == cudaSuccess && g_autotune.load())
    pre_err = autotune_rows(b, rowbuf, buckets, rows_by_bucket, h_peq_off, rb_off, ld, st);
  // second pass: row arrays and work items
  for (size_t bk = 0; bk < buckets.size(); ++bk) {
    Bucket &B = buckets[bk];
    B.R = B.c.kind == kLcsTpp ? tpp_rows(B.c.kw) : 1;
    append_rows(b, rows_by_bucket[bk], rows_by_bucket[bk].size(), item_cols(B.c), B.R, h_peq_off, rb_off, ld,
                ra, B.tiles, B.tile_items);
  }
  // item offsets per bucket and per tile (the items themselves are expanded on the device)
  std::vector<int64_t> item_off(buckets.size() + 1, 0);
  std::vector<int4> all_tiles;
  std::vector<int64_t> tstart(1, 0);
  for (size_t bk = 0; bk < buckets.size(); ++bk) {
    const Bucket &B = buckets[bk];
    all_tiles.insert(all_tiles.end(), B.tiles.begin(), B.tiles.end());
    for (int32_t c : B.tile_items) tstart.push_back(tstart.back() + c);
    item_off[bk + 1] = tstart.back();
  }
  const int64_t n_items = tstart.back();
  b->stats[0] = cells;
  b->stats[1] = words;
  b->stats[2] = pairs;
  b->stats[3] = n_items;

  // device copies of the row arrays and items
  int64_t *d_rpeq = nullptr, *d_rbase = nullptr, *d_tstart = nullptr;
  int32_t *d_rlen = nullptr, *d_rid = nullptr;
  int4 *d_items = nullptr, *d_tiles = nullptr;
  std::vector<SmemArgs> smem_args[5][kStageGroups];  // cluster sizes 1, 2, 4, 8, 16 by group
  size_t smem_dyn[5] = {0, 0, 0, 0, 0};
  struct GlobalFam { SlinkState S; int64_t off, ld; int32_t k; int group; };
  std::vector<GlobalFam> global_fams;
  std::vector<BatchInit> inits;
  struct FinJob { int32_t f, k; bool widen; const int32_t *ord; uint64_t *gap; FinBufs FB; };
  std::vector<FinJob> fins;
  const bool narrow = b->max_len <= 32767;
  const uint64_t inf_narrow = KeysNarrow::kInf, inf_wide = KeysWide::kInf;
  uint64_t *ctl_all = nullptr;
  int64_t n_ctl = 0;
  BatchInit *d_init = nullptr;
  SmemArgs *d_sargs[5][kStageGroups] = {};
  const int max_cl = max_cluster_global();

  BCK(pre_err);
  BCK(upload_vec(A, ra.peq, &d_rpeq, st));
  BCK(upload_vec(A, ra.base, &d_rbase, st));
  BCK(upload_vec(A, ra.len, &d_rlen, st));
  BCK(upload_vec(A, ra.id, &d_rid, st));
  BCK(upload_vec(A, all_tiles, &d_tiles, st));
  BCK(upload_vec(A, tstart, &d_tstart, st));
  d_items = A.get<int4>((size_t)std::max<int64_t>(n_items, 1));
  if (A.err != cudaSuccess) { err = A.err; goto fail; }
  if (!all_tiles.empty()) {
    const int64_t nt = (int64_t)all_tiles.size();
    k_expand_items<<<(unsigned)((nt + 7) / 8), 256, 0, st>>>(d_tiles, d_tstart, nt, d_items);
    BCK(cudaGetLastError());
  }
  // outputs (whole batch)
  b->d_pi = A.get<int32_t>(b->N);
  b->d_lnum = A.get<uint64_t>(b->N);
  b->d_lden = A.get<uint32_t>(b->N);
  b->d_merges = A.get<int32_t>(2 * (size_t)(b->N - F));
  b->d_hnum = A.get<uint64_t>(b->N - F);
  b->d_hden = A.get<uint32_t>(b->N - F);
  b->d_sizes = A.get<int32_t>(b->N - F);
  for (int32_t f = 0; f < F; ++f) n_ctl += kCtlWords;
  ctl_all = A.get<uint64_t>((size_t)n_ctl);
  if (A.err != cudaSuccess) { err = A.err; goto fail; }

  // per-family row-update state and finalisation buffers
  for (int32_t f = 0; f < F; ++f) {
    const int32_t k = (int32_t)(b->fam_off[f + 1] - b->fam_off[f]);
    BatchInit in = {};
    in.out_at = b->fam_off[f];
    if (k == 1) {
      in.single = 1;
      inits.push_back(in);
      continue;
    }
    SlinkState S = {};
    const size_t kp = (size_t)k + 1;
    for (int i = 0; i < 2; ++i) {
      S.ord[i] = A.get<int32_t>(kp);
      S.olen[i] = A.get<int32_t>(kp);
      S.gap[i] = A.get<uint64_t>(kp);
      S.lam[i] = A.get<uint64_t>(kp);
      S.pi[i] = A.get<int32_t>(kp);
      S.mD[i] = A.get<uint64_t>(kp);
      S.mOrd[i] = A.get<int32_t>(kp);
      S.mLen[i] = A.get<int32_t>(kp);
      S.mOld[i] = A.get<int32_t>(kp);
      S.mLam[i] = A.get<uint64_t>(kp);
      S.mPi[i] = A.get<int32_t>(kp);
      S.mRaw[i] = A.get<int32_t>(kp);
    }
    S.D = A.get<uint64_t>(kp);
    S.mGap = A.get<uint64_t>(kp);
    S.runsA = A.get<int32_t>(kp);
    S.runsB = A.get<int32_t>(kp);
    S.ctl = ctl_all + (size_t)f * kCtlWords;
    S.slen = b->d_slen + b->S[f];
    const int cl = smem_cluster_for(k, 0);
    const bool smem = cl > 0 && cl <= max_cl;
    in.ord1 = S.ord[1];
    in.olen1 = S.olen[1];
    in.pi1 = S.pi[1];
    in.lam1 = S.lam[1];
    in.len0 = b->h_slen[b->S[f]];
    in.inf = narrow ? inf_narrow : inf_wide;
    inits.push_back(in);
    if (smem) {
      const int ci = __builtin_ctz(cl);
      SmemArgs a = {};
      a.s = S;
      a.rowbuf = rowbuf + rb_off[f];
      a.ld = ld[f];
      a.r0 = 1;
      a.r1 = k;
      a.P = (k + cl - 1) / cl;
      a.sshift = smem_sample_shift(a.P, a.P * cl);
      a.batch = nullptr;
      a.dyn_bytes = 0;
      smem_args[ci][fam_group[f]].push_back(a);
      smem_dyn[ci] = std::max(smem_dyn[ci], smem_dyn_bytes(a.P, a.P * cl, a.sshift));
    } else {
      global_fams.push_back(GlobalFam{S, rb_off[f], ld[f], k, fam_group[f]});
    }
    const size_t lv = fin_levels(k);
    FinBufs FB = {};
    FB.idx = A.get<int32_t>(k); FB.posof = A.get<int32_t>(k);
    FB.it = A.get<int32_t>(lv * k); FB.rt = A.get<int32_t>(lv * k);
    FB.gt = A.get<uint64_t>(lv * k);
    FB.sub_lo = A.get<int32_t>(k); FB.sub_hi = A.get<int32_t>(k);
    FB.ordA = A.get<int32_t>(k); FB.ordB = A.get<int32_t>(k); FB.rank = A.get<int32_t>(k);
    FB.sorder = A.get<int32_t>(k);
    FB.lam = A.get<uint64_t>(k); FB.hkey = A.get<uint64_t>(k);
    FB.sz = A.get<int64_t>(k); FB.szpre = A.get<int64_t>(k); FB.tot = A.get<int64_t>(2);
    const int64_t o = b->fam_off[f], om = b->fam_off[f] - f;
    FB.pi = b->d_pi + o;
    FB.lnum = b->d_lnum + o;
    FB.lden = b->d_lden + o;
    FB.merges = b->d_merges + 2 * om;
    FB.hnum = b->d_hnum + om;
    FB.hden = b->d_hden + om;
    FB.sizes = b->d_sizes + om;
    const int bk = k & 1;
    fins.push_back(FinJob{f, k, narrow, S.ord[bk], S.gap[bk], FB});
  }
  if (A.err != cudaSuccess) { err = A.err; goto fail; }
  BCK(upload_vec(A, inits, &d_init, st));
  for (int ci = 0; ci < 5; ++ci)
    for (int g = 0; g < kStageGroups; ++g)
      if (!smem_args[ci][g].empty()) BCK(upload_vec(A, smem_args[ci][g], &d_sargs[ci][g], st));
  BCK(cudaStreamSynchronize(st));

  // ---- capture the whole pipeline once
  BCK(cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking));
  {
    // side branches at the highest priority: a row-update cluster takes SMs
    // as they free up rather than after the whole LCS grid
    int prio_lo = 0, prio_hi = 0;
    BCK(cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi));
    b->side.resize(6 * kStageGroups);
    for (auto &s : b->side) BCK(cudaStreamCreateWithPriority(&s, cudaStreamNonBlocking, prio_hi));
  }
  b->ev.resize(1 + b->side.size());
  for (auto &e : b->ev) BCK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  b->ev_stage.resize(kStageGroups + 6 * kStageGroups);
  for (auto &e : b->ev_stage) BCK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  for (auto &e : b->tev) BCK(cudaEventCreate(&e));
  {
    cudaGraph_t graph = nullptr;
    int64_t launches = 0;
    b->stats[12] = ns_since(t_plan0);
    const auto t_cap0 = std::chrono::steady_clock::now();
    BCK(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal));
    {
      cudaError_t e = cudaEventRecordWithFlags(b->tev[0], b->cap, cudaEventRecordExternal);
      // the row-update state of every family first (it needs no LCS)
      if (e == cudaSuccess) e = cudaMemsetAsync(ctl_all, 0, sizeof(uint64_t) * n_ctl, b->cap);
      if (e == cudaSuccess && !inits.empty()) {
        k_batch_init<<<nblk((int64_t)inits.size(), T), T, 0, b->cap>>>(
            d_init, (int32_t)inits.size(), b->d_pi, b->d_lnum, b->d_lden);
        e = cudaGetLastError();
        ++launches;
      }
      // stage I: every family's triangle, one launch per kernel width in
      // increasing width; after each group of widths, the row updates of the
      // families whose rows are all done start on side branches (one per
      // cluster size, and one for the global-memory families), beside the
      // LCS of the wider buckets
      KParams p = batch_params(b, rowbuf);
      p.row_peq_off = d_rpeq;
      p.row_len = d_rlen;
      p.row_id = d_rid;
      p.row_base = d_rbase;
      int joins = 0;
      size_t bk = 0;
      for (int g = 0; g < kStageGroups && e == cudaSuccess; ++g) {
        for (; bk < buckets.size() && bucket_group[bk] == g && e == cudaSuccess; ++bk) {
          const int64_t n = item_off[bk + 1] - item_off[bk];
          if (n == 0) continue;
          p.items = d_items + item_off[bk];
          p.e0 = 0;
          p.e1 = (int32_t)ra.id.size();
          const LcsChoice &c = buckets[bk].c;
          e = c.kind == kLcsTpp ? launch_tpp(c.kw, buckets[bk].R, p, dim3((unsigned)n), b->cap)
              : c.kind == kLcsSlice ? launch_slice(c.kw, c.g, p, dim3((unsigned)n), b->cap)
                                    : launch_wpp(c.kw, p, dim3((unsigned)n), b->cap);
          ++launches;
        }
        if (e == cudaSuccess) e = cudaEventRecord(b->ev_stage[g], b->cap);
        for (int ci = 0; ci < 6 && e == cudaSuccess; ++ci) {
          bool any = false;
          if (ci < 5) any = !smem_args[ci][g].empty();
          for (size_t gi = 0; ci == 5 && gi < global_fams.size(); ++gi) any = any || global_fams[gi].group == g;
          if (!any) continue;
          cudaStream_t s = b->side[6 * g + ci];
          e = cudaStreamWaitEvent(s, b->ev_stage[g], 0);
          if (e == cudaSuccess && ci < 5) {
            e = launch_slink_smem_batch(d_sargs[ci][g], (int32_t)smem_args[ci][g].size(), 1 << ci, smem_dyn[ci],
                                        narrow, s);
            ++launches;
          }
          for (size_t gi = 0; ci == 5 && gi < global_fams.size() && e == cudaSuccess; ++gi) {
            const GlobalFam &gf = global_fams[gi];
            if (gf.group != g) continue;
            e = launch_slink_global(gf.S, rowbuf + gf.off, gf.ld, 1, gf.k, max_cl, narrow, s);
            ++launches;
          }
          if (e == cudaSuccess) e = cudaEventRecord(b->ev_stage[kStageGroups + joins++], s);
        }
      }
      // stage II ends when every branch has joined
      if (e == cudaSuccess) e = cudaEventRecordWithFlags(b->tev[1], b->cap, cudaEventRecordExternal);
      for (int j = 0; j < joins && e == cudaSuccess; ++j)
        e = cudaStreamWaitEvent(b->cap, b->ev_stage[kStageGroups + j], 0);
      // finalisation, spread over side streams
      if (e == cudaSuccess) e = cudaEventRecordWithFlags(b->tev[2], b->cap, cudaEventRecordExternal);
      if (e == cudaSuccess) e = cudaEventRecord(b->ev[0], b->cap);
      for (auto &s : b->side)
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s, b->ev[0], 0);
      for (size_t j = 0; j < fins.size() && e == cudaSuccess; ++j) {
        FinJob &J = fins[j];
        cudaStream_t s = b->side[j % b->side.size()];
        e = launch_finalize(J.ord, J.gap, b->d_perm_local + b->S[J.f], J.k, J.FB, s, &launches, J.widen);
      }
      for (size_t i = 0; i < b->side.size() && e == cudaSuccess; ++i) {
        e = cudaEventRecord(b->ev[1 + i], b->side[i]);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(b->cap, b->ev[1 + i], 0);
      }
      if (e == cudaSuccess) e = cudaEventRecordWithFlags(b->tev[3], b->cap, cudaEventRecordExternal);
      cudaError_t e2 = cudaStreamEndCapture(b->cap, &graph);
      if (e == cudaSuccess) e = e2;
      if (e != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        err = e;
        goto fail;
      }
    }
    b->stats[13] = ns_since(t_cap0);
    {
      size_t nodes = 0;
      if (cudaGraphGetNodes(graph, nullptr, &nodes) == cudaSuccess) b->stats[15] = (int64_t)nodes;
    }
    const auto t_inst0 = std::chrono::steady_clock::now();
    err = cudaGraphInstantiateWithFlags(&b->exec, graph, cudaGraphInstantiateFlagUseNodePriority);
    b->stats[14] = ns_since(t_inst0);
    cudaGraphDestroy(graph);
    if (err != cudaSuccess) goto fail;
    b->stats[4] = launches;
    b->stats[5] = (int64_t)buckets.size();
    b->stats[6] = (int64_t)global_fams.size();
  }
  b->planned = true;
  return FAMSA_OK;

fail:
  cudaStreamSynchronize(st);
  batch_free_plan(b);
  return status_from_cuda(err);
}

}  // namespace famsa

using namespace famsa;

extern "C" {

int famsa_batch_pack(const uint8_t *residues, const int64_t *offsets, int64_t n_seqs,
                     const int64_t *family_offsets, int32_t n_families, int residues_on_device,
                     void *cuda_stream, famsa_batch **out) {
  if (!out) return FAMSA_EINVAL;
  *out = nullptr;
  if (!residues || !offsets || !family_offsets) return FAMSA_EINVAL;
  TraceRange trace("famsa_batch_pack");
  Batch *b = nullptr;
  int rc = batch_pack(residues, offsets, n_seqs, family_offsets, n_families, residues_on_device != 0,
                      (cudaStream_t)cuda_stream, &b);
  if (rc != FAMSA_OK) return rc;
  *out = reinterpret_cast<famsa_batch *>(b);
  return FAMSA_OK;
}

int famsa_batch_tree(famsa_batch *bh, int32_t *pi, uint64_t *lambda_num, uint32_t *lambda_den,
                     int32_t *merges, uint64_t *h_num, uint32_t *h_den, int32_t *sizes,
                     int out_on_device, void *cuda_stream) {
  if (!bh) return FAMSA_EINVAL;
  Batch *b = reinterpret_cast<Batch *>(bh);
  std::lock_guard<std::mutex> lk(b->mu);
  cudaStream_t st = (cudaStream_t)cuda_stream;
  TraceRange trace("famsa_batch_tree");
  if (!b->planned) {
    TraceRange trace_plan("batch plan and graph capture");
    int rc = batch_plan(b, st);
    if (rc != FAMSA_OK) return rc;
  }
  cudaError_t err = cudaGraphLaunch(b->exec, st);
  if (err == cudaSuccess) b->launched = true;
  const cudaMemcpyKind kind = out_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  const size_t N = (size_t)b->N, M = (size_t)(b->N - b->F);
  if (err == cudaSuccess && pi) err = cudaMemcpyAsync(pi, b->d_pi, sizeof(int32_t) * N, kind, st);
  if (err == cudaSuccess && lambda_num)
    err = cudaMemcpyAsync(lambda_num, b->d_lnum, sizeof(uint64_t) * N, kind, st);
  if (err == cudaSuccess && lambda_den)
    err = cudaMemcpyAsync(lambda_den, b->d_lden, sizeof(uint32_t) * N, kind, st);
  if (M > 0) {
    if (err == cudaSuccess && merges)
      err = cudaMemcpyAsync(merges, b->d_merges, sizeof(int32_t) * 2 * M, kind, st);
    if (err == cudaSuccess && h_num) err = cudaMemcpyAsync(h_num, b->d_hnum, sizeof(uint64_t) * M, kind, st);
    if (err == cudaSuccess && h_den) err = cudaMemcpyAsync(h_den, b->d_hden, sizeof(uint32_t) * M, kind, st);
    if (err == cudaSuccess && sizes) err = cudaMemcpyAsync(sizes, b->d_sizes, sizeof(int32_t) * M, kind, st);
  }
  if (err == cudaSuccess && !out_on_device) err = cudaStreamSynchronize(st);
  return status_from_cuda(err);
}

int famsa_batch_stats(const famsa_batch *bh, int64_t *stats) {
  if (!bh || !stats) return FAMSA_EINVAL;
  Batch *b = const_cast<Batch *>(reinterpret_cast<const Batch *>(bh));
  std::lock_guard<std::mutex> lk(b->mu);
  if (b->launched) {
    // device time of the stages of the last graph launch (waits for it)
    float ms[3] = {0.f, 0.f, 0.f};
    cudaError_t err = cudaEventSynchronize(b->tev[3]);
    for (int i = 0; i < 3 && err == cudaSuccess; ++i) err = cudaEventElapsedTime(&ms[i], b->tev[i], b->tev[i + 1]);
    if (err != cudaSuccess) return status_from_cuda(err);
    for (int i = 0; i < 3; ++i) b->stats[7 + i] = (int64_t)(ms[i] * 1e6);
  }
  for (int i = 0; i < 16; ++i) stats[i] = b->stats[i];
  return FAMSA_OK;
}

void famsa_batch_free(famsa_batch *bh) {
  if (!bh) return;
  Batch *b = reinterpret_cast<Batch *>(bh);
  {
    std::lock_guard<std::mutex> lk(b->mu);
    cudaDeviceSynchronize();
  }
  batch_free(b);
}

}  // extern "C"

extern "C" int famsa_debug_set_autotune(int on) {
  famsa::g_autotune.store(on ? 1 : 0);
  if (!on) {
    std::lock_guard<std::mutex> lk(famsa::g_tune_mu);
    for (int w = 1; w <= famsa::kTppMaxW; ++w) famsa::g_tuned[w] = false;
  }
  return FAMSA_OK;
}
