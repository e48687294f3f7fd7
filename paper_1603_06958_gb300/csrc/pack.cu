// Family packing: validation, length sort, Peq match-bitmask tables, column layout.
//
// FAMSA Methods, "Pairwise similarities calculation": the LCS length is
// computed bit-parallel with w = 64 DP cells per machine word, which needs,
// for each sequence A and symbol c, the bitmask Peq_A[c] of the positions of
// A that hold c.  This file builds those tables on the device, plus the
// length-sorted, interleaved column layout the LCS kernels stream.
#include <algorithm>
#include <atomic>
#include <cstring>
#include <vector>

#include "famsa_internal.cuh"

namespace famsa {

static std::atomic<int> g_alloc_fail_after{-1};
static thread_local cudaStream_t tl_alloc_stream = nullptr;

AllocStream::AllocStream(cudaStream_t st) : prev(tl_alloc_stream) { tl_alloc_stream = st; }
AllocStream::~AllocStream() { tl_alloc_stream = prev; }

// every device allocation of the library, counted process-wide
static std::atomic<int64_t> g_alloc_count{0};
cudaError_t lib_malloc_async(void **p, size_t bytes, cudaStream_t st) {
  g_alloc_count.fetch_add(1);
  return cudaMallocAsync(p, bytes, st);
}

cudaError_t dev_alloc(void **p, size_t bytes) {
  int n = g_alloc_fail_after.load();
  if (n >= 0) {
    if (n == 0) { *p = nullptr; return cudaErrorMemoryAllocation; }
    g_alloc_fail_after.store(n - 1);
  }
  if (bytes == 0) bytes = 16;
  return lib_malloc_async(p, bytes, tl_alloc_stream);
}
void dev_free(void *p) {
  if (p) cudaFreeAsync(p, tl_alloc_stream);
}

int status_from_cuda(cudaError_t e) {
  if (e == cudaSuccess) return FAMSA_OK;
  if (e == cudaErrorMemoryAllocation) return FAMSA_ENOMEM;
  return FAMSA_ECUDA;
}

// one reader per translation unit of the checked build (none in the normal one)
static std::vector<CheckReader> &check_readers() {
  static std::vector<CheckReader> r;
  return r;
}

int register_check_reader(CheckReader r) {
  check_readers().push_back(r);
  return 1;
}

void read_checks(unsigned long long *count, unsigned long long *first_line) {
  *count = 0;
  *first_line = 0;
  for (CheckReader r : check_readers()) {
    unsigned long long v[2] = {0, 0};
    r(v);
    *count += v[0];
    if (!*first_line && v[1]) *first_line = v[1];
  }
}

// ----------------------------------------------------------------- kernels

__global__ void k_lengths(const int64_t *off, int32_t k, int64_t base, int32_t *len,
                          int64_t *off0, int *status, int *max_len) {
  int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i > k) return;
  off0[i] = off[i] - base;
  if (i == k) return;
  int64_t l = off[i + 1] - off[i];
  int bad = 0;
  if (l < 1) bad |= kBadArg;
  if (l > kMaxLen) bad |= kTooLong;
  if (bad) atomicOr(status, bad);
  int32_t li = (int32_t)(l < 0 ? 0 : (l > kMaxLen ? kMaxLen : l));
  len[i] = li;
  atomicMax(max_len, li);
}

__global__ void k_codes(const uint8_t *res, int64_t n, int *status) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int64_t stride = (int64_t)gridDim.x * blockDim.x;
  int bad = 0;
  for (; i < n; i += stride) bad |= res[i] >= kCodes;
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(status, kBadArg);
}

// keys (len << 32 | idx), unique
__global__ void k_sort_keys(const int32_t *len, int32_t n, uint64_t *keys) {
  int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) keys[i] = ((uint64_t)(uint32_t)len[i] << 32) | (uint32_t)i;
}

// One bottom-up merge pass over sorted runs of `width`: each element finds
// its place in the merged run by a binary search in the partner run.
__global__ void k_merge_pass(const uint64_t *in, uint64_t *out, int32_t n, int32_t width) {
  int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int64_t run = i / width;
  int64_t start = run * width;
  int64_t pair_start = (run & ~1LL) * width;
  int64_t pstart = (run ^ 1) * width;
  uint64_t key = in[i];
  if (pstart >= n) { out[i] = key; return; }
  int64_t pend = pstart + width < n ? pstart + width : n;
  // count partner elements < key (keys are unique)
  int64_t lo = pstart, hi = pend;
  while (lo < hi) {
    int64_t mid = (lo + hi) >> 1;
    if (in[mid] < key) lo = mid + 1; else hi = mid;
  }
  int64_t pos = pair_start + (i - start) + (lo - pstart);
  out[pos] = key;
}

__global__ void k_sorted_fields(const uint64_t *keys, int32_t n, int32_t *perm, int32_t *rank,
                                int32_t *slen, int64_t *words) {
  int32_t s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n) return;
  uint64_t key = keys[s];
  int32_t idx = (int32_t)(key & 0xffffffffu);
  int32_t l = (int32_t)(key >> 32);
  perm[s] = idx;
  rank[idx] = s;
  slen[s] = l;
  words[s] = (l + 63) / 64;
}

// single-CTA exclusive scan of n int64 (in place allowed), writes the total to *total
__global__ void k_scan_excl(const int64_t *in, int64_t *out, int64_t n, int64_t *total) {
  __shared__ int64_t warp_sums[32];
  __shared__ int64_t carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int64_t base = 0; base < n; base += blockDim.x) {
    int64_t i = base + threadIdx.x;
    int64_t v = i < n ? in[i] : 0;
    int64_t x = v;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      int64_t y = __shfl_up_sync(0xffffffffu, x, d);
      if (lane >= d) x += y;
    }
    if (lane == 31) warp_sums[warp] = x;
    __syncthreads();
    if (warp == 0) {
      int nw = blockDim.x >> 5;
      int64_t w = lane < nw ? warp_sums[lane] : 0;
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        int64_t y = __shfl_up_sync(0xffffffffu, w, d);
        if (lane >= d) w += y;
      }
      if (lane < nw) warp_sums[lane] = w;
    }
    __syncthreads();
    int64_t pre = carry + (warp > 0 ? warp_sums[warp - 1] : 0) + x - v;
    if (i < n) out[i] = pre;
    __syncthreads();
    if (threadIdx.x == blockDim.x - 1) carry = pre + v;
    __syncthreads();
  }
  if (threadIdx.x == 0 && total) *total = carry;
}

__global__ void k_group_sizes(const int32_t *slen, int32_t k, int32_t n_groups, int32_t *chunks,
                              int64_t *bytes) {
  int32_t g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= n_groups) return;
  int32_t last = min(g * kGroup + kGroup - 1, k - 1);
  int32_t c = (slen[last] + kChunk - 1) / kChunk;
  chunks[g] = c;
  bytes[g] = (int64_t)c * kGroup * kChunk;
}

// One warp per sequence: Peq words via ballots, 32 positions per ballot.
// Row sequence s (any order) with residues res[off[idx]..] where idx = map[s]
// (or s itself when map is null).
__global__ void k_pack_peq(const uint8_t *res, const int64_t *off, const int32_t *map,
                           const int64_t *peq_off, int32_t n, uint32_t *peq) {
  int32_t s = (int32_t)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  int lane = threadIdx.x & 31;
  if (s >= n) return;
  int32_t idx = map ? map[s] : s;
  if (idx < 0) return;  // a pad slot of a batched family: no sequence, no Peq words
  const uint8_t *a = res + off[idx];
  int32_t len = (int32_t)(off[idx + 1] - off[idx]);
  int32_t W = (len + 63) / 64;
  // the sequence's words are exactly its slot's share of the table
  if (!FAMSA_EXPECT(len >= 1 && peq_off[s + 1] - peq_off[s] == W)) return;
  uint32_t *dst = peq + peq_off[s] * kPeqWordU32;
  for (int32_t w = 0; w < W; ++w) {
    int32_t p0 = w * 64 + lane, p1 = p0 + 32;
    int c0 = p0 < len ? a[p0] : 255;
    int c1 = p1 < len ? a[p1] : 255;
    uint32_t mylo = 0, myhi = 0;
#pragma unroll
    for (int c = 0; c < kCodes; ++c) {
      uint32_t lo = __ballot_sync(0xffffffffu, c0 == c);
      uint32_t hi = __ballot_sync(0xffffffffu, c1 == c);
      if (lane == c) { mylo = lo; myhi = hi; }
    }
    dst[w * kPeqWordU32 + lane] = mylo;
    dst[w * kPeqWordU32 + 32 + lane] = myhi;
  }
}

// One CTA per column group: interleaved 16-residue chunks, codes stored as 4*code.
__global__ void k_col_layout(const uint8_t *res, const int64_t *off, const int32_t *perm,
                             const int32_t *slen, int32_t k, const int64_t *group_off,
                             const int32_t *group_chunks, uint8_t *colres) {
  int32_t g = blockIdx.x;
  int32_t nch = group_chunks[g];
  uint8_t *dst = colres + group_off[g];
  for (int32_t t = threadIdx.x; t < nch * kGroup; t += blockDim.x) {
    int32_t q = t / kGroup, lane = t % kGroup;
    int32_t s = g * kGroup + lane;
    uint32_t w[4];
    int32_t len = s < k ? slen[s] : 0;
    // a slot's residues fit its group's chunks, and its label is a sequence
    if (len > 0 && !FAMSA_EXPECT(len <= nch * kChunk && perm[s] >= 0)) len = 0;
    const uint8_t *a = len > 0 ? res + off[perm[s]] : res;  // pad slots have length 0
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      uint32_t v = 0;
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        int32_t p = q * kChunk + j * 4 + b;
        uint32_t code = p < len ? a[p] : kPadCode;
        v |= (code * 4u) << (8 * b);
      }
      w[j] = v;
    }
    reinterpret_cast<uint4 *>(dst)[t] = make_uint4(w[0], w[1], w[2], w[3]);
  }
}

// ----------------------------------------------------------------- host side
static unsigned blocks_for(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

#define CK(x)                                  \
  do {                                         \
    cudaError_t e_ = (x);                      \
    if (e_ != cudaSuccess) { err = e_; goto fail; } \
  } while (0)

void free_family(Family *f) {
  if (!f) return;
  dev_free(f->d_off); dev_free(f->d_res); dev_free(f->d_len); dev_free(f->d_perm);
  dev_free(f->d_rank); dev_free(f->d_slen); dev_free(f->d_peq_off); dev_free(f->d_peq);
  dev_free(f->d_group_off); dev_free(f->d_group_chunks); dev_free(f->d_colres);
  for (auto &b : f->scratch) dev_free(b.ptr);
  delete f;
}

int pack_family(const uint8_t *residues, const int64_t *offsets, int32_t k, bool on_device,
                cudaStream_t st, Family **out) {
  *out = nullptr;
  cudaError_t err = cudaSuccess;
  AllocStream alloc_on(st);
  Family *f = new Family();
  f->k = k;
  cudaGetDevice(&f->device);
  int64_t base = 0, total = 0;
  int64_t *d_off_in = nullptr;   // caller offsets on device (or staged copy)
  int *d_status = nullptr;        // [0] status, [1] max_len
  uint64_t *keys = nullptr, *keys2 = nullptr;
  int64_t *words = nullptr, *gbytes = nullptr, *d_tot = nullptr;
  int h_status[2] = {0, 0};
  int64_t h_tot[2] = {0, 0};
  const int T = 256;

  // offsets: validate monotonicity of the endpoints on the host side first
  if (on_device) {
    int64_t ends[2];
    CK(cudaMemcpyAsync(&ends[0], offsets, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(&ends[1], offsets + k, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    base = ends[0];
    total = ends[1] - ends[0];
    d_off_in = const_cast<int64_t *>(offsets);
  } else {
    base = offsets[0];
    total = offsets[k] - offsets[0];
  }
  if (base < 0 || total < k) { free_family(f); return FAMSA_EINVAL; }
  f->total = total;
  CK(dev_alloc((void **)&f->d_off, sizeof(int64_t) * (k + 1)));
  CK(dev_alloc((void **)&f->d_res, (size_t)total));
  CK(dev_alloc((void **)&f->d_len, sizeof(int32_t) * k));
  CK(dev_alloc((void **)&d_status, sizeof(int) * 2));
  CK(cudaMemsetAsync(d_status, 0, sizeof(int) * 2, st));
  if (on_device) {
    CK(cudaMemcpyAsync(f->d_res, residues + base, (size_t)total, cudaMemcpyDeviceToDevice, st));
  } else {
    CK(dev_alloc((void **)&d_off_in, sizeof(int64_t) * (k + 1)));
    CK(cudaMemcpyAsync(d_off_in, offsets, sizeof(int64_t) * (k + 1), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(f->d_res, residues + base, (size_t)total, cudaMemcpyHostToDevice, st));
  }
  k_lengths<<<blocks_for(k + 1, T), T, 0, st>>>(d_off_in, k, base, f->d_len, f->d_off, d_status,
                                                d_status + 1);
  k_codes<<<std::min<int64_t>(blocks_for(total, T), 4096), T, 0, st>>>(f->d_res, total, d_status);
  CK(cudaGetLastError());
  CK(cudaMemcpyAsync(h_status, d_status, sizeof(int) * 2, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  if (!on_device) { dev_free(d_off_in); d_off_in = nullptr; }
  if (h_status[0] & kBadArg) { dev_free(d_status); free_family(f); return FAMSA_EINVAL; }
  if (h_status[0] & kTooLong) { dev_free(d_status); free_family(f); return FAMSA_ERANGE; }
  f->max_len = h_status[1];
  f->max_w = (f->max_len + 63) / 64;

  // sort by (length, index)
  CK(dev_alloc((void **)&keys, sizeof(uint64_t) * k));
  CK(dev_alloc((void **)&keys2, sizeof(uint64_t) * k));
  k_sort_keys<<<blocks_for(k, T), T, 0, st>>>(f->d_len, k, keys);
  for (int64_t width = 1; width < k; width *= 2) {
    k_merge_pass<<<blocks_for(k, T), T, 0, st>>>(keys, keys2, k, (int32_t)width);
    std::swap(keys, keys2);
  }
  CK(dev_alloc((void **)&f->d_perm, sizeof(int32_t) * k));
  CK(dev_alloc((void **)&f->d_rank, sizeof(int32_t) * k));
  CK(dev_alloc((void **)&f->d_slen, sizeof(int32_t) * k));
  CK(dev_alloc((void **)&f->d_peq_off, sizeof(int64_t) * (k + 1)));
  CK(dev_alloc((void **)&words, sizeof(int64_t) * (k + 1)));
  CK(dev_alloc((void **)&d_tot, sizeof(int64_t) * 2));
  k_sorted_fields<<<blocks_for(k, T), T, 0, st>>>(keys, k, f->d_perm, f->d_rank, f->d_slen, words);
  k_scan_excl<<<1, 1024, 0, st>>>(words, f->d_peq_off, k, d_tot);
  CK(cudaGetLastError());

  // column groups
  f->n_groups = (k + kGroup - 1) / kGroup;
  CK(dev_alloc((void **)&f->d_group_chunks, sizeof(int32_t) * f->n_groups));
  CK(dev_alloc((void **)&f->d_group_off, sizeof(int64_t) * (f->n_groups + 1)));
  CK(dev_alloc((void **)&gbytes, sizeof(int64_t) * f->n_groups));
  k_group_sizes<<<blocks_for(f->n_groups, T), T, 0, st>>>(f->d_slen, k, f->n_groups,
                                                          f->d_group_chunks, gbytes);
  k_scan_excl<<<1, 1024, 0, st>>>(gbytes, f->d_group_off, f->n_groups, d_tot + 1);
  CK(cudaGetLastError());
  CK(cudaMemcpyAsync(h_tot, d_tot, sizeof(int64_t) * 2, cudaMemcpyDeviceToHost, st));
  f->h_slen.resize(k);
  f->h_perm.resize(k);
  CK(cudaMemcpyAsync(f->h_slen.data(), f->d_slen, sizeof(int32_t) * k, cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(f->h_perm.data(), f->d_perm, sizeof(int32_t) * k, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  f->peq_words = h_tot[0];
  f->colres_bytes = h_tot[1];
  CK(cudaMemcpyAsync(f->d_peq_off + k, &d_tot[0], sizeof(int64_t), cudaMemcpyDeviceToDevice, st));
  CK(cudaMemcpyAsync(f->d_group_off + f->n_groups, &d_tot[1], sizeof(int64_t),
                     cudaMemcpyDeviceToDevice, st));

  // Peq tables (sorted order) and column layout
  CK(dev_alloc((void **)&f->d_peq, sizeof(uint32_t) * kPeqWordU32 * (size_t)f->peq_words));
  CK(dev_alloc((void **)&f->d_colres, (size_t)f->colres_bytes));
  k_pack_peq<<<blocks_for((int64_t)k * 32, T), T, 0, st>>>(f->d_res, f->d_off, f->d_perm,
                                                          f->d_peq_off, k, f->d_peq);
  k_col_layout<<<f->n_groups, 256, 0, st>>>(f->d_res, f->d_off, f->d_perm, f->d_slen, k,
                                            f->d_group_off, f->d_group_chunks, f->d_colres);
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(st));
  dev_free(keys); dev_free(keys2); dev_free(words); dev_free(gbytes); dev_free(d_tot);
  dev_free(d_status);
  {
    int64_t passes = 0;
    for (int64_t width = 1; width < k; width *= 2) ++passes;
    // k_lengths, k_codes, k_sort_keys, merge passes, k_sorted_fields, 2 scans,
    // k_group_sizes, k_pack_peq, k_col_layout
    f->pack_launches = 9 + passes;
  }
  *out = f;
  return FAMSA_OK;

fail:
  cudaStreamSynchronize(st);
  if (!on_device) dev_free(d_off_in);
  dev_free(keys); dev_free(keys2); dev_free(words); dev_free(gbytes); dev_free(d_tot);
  dev_free(d_status);
  free_family(f);
  return status_from_cuda(err);
}

static void release_rows(cudaStream_t st, int *d_status, int64_t *rebased, int32_t **d_len,
                         int64_t **d_peq_off, uint32_t **d_peq) {
  if (d_status) cudaFreeAsync(d_status, st);
  if (rebased) cudaFreeAsync(rebased, st);
  if (*d_len) cudaFreeAsync(*d_len, st);
  if (*d_peq_off) cudaFreeAsync(*d_peq_off, st);
  if (*d_peq) cudaFreeAsync(*d_peq, st);
  *d_len = nullptr; *d_peq_off = nullptr; *d_peq = nullptr;
  cudaStreamSynchronize(st);
}

// Peq for an arbitrary list of n sequences (query rows), input on the device.
int pack_rows(const uint8_t *d_res, const int64_t *d_off, int32_t n, cudaStream_t st,
              uint32_t **d_peq, int64_t **d_peq_off, int32_t **d_len, std::vector<int32_t> &h_len) {
  cudaError_t err = cudaSuccess;
  *d_peq = nullptr; *d_peq_off = nullptr; *d_len = nullptr;
  int *d_status = nullptr;
  int64_t *rebased = nullptr;
  std::vector<int64_t> h_off(n + 1);
  int h_status[2] = {0, 0};
  const int T = 256;
  CK(lib_malloc_async((void **)&d_status, sizeof(int) * 2, st));
  CK(lib_malloc_async((void **)d_len, sizeof(int32_t) * n, st));
  CK(lib_malloc_async((void **)&rebased, sizeof(int64_t) * (n + 1), st));
  CK(cudaMemsetAsync(d_status, 0, sizeof(int) * 2, st));
  k_lengths<<<blocks_for(n + 1, T), T, 0, st>>>(d_off, n, 0, *d_len, rebased, d_status,
                                                d_status + 1);
  CK(cudaGetLastError());
  CK(cudaMemcpyAsync(h_status, d_status, sizeof(int) * 2, cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(h_off.data(), d_off, sizeof(int64_t) * (n + 1), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  if (h_status[0] & kBadArg) { err = cudaErrorInvalidValue; goto bad; }
  if (h_status[0] & kTooLong) { err = cudaErrorInvalidValue; goto toolong; }
  {
    int64_t totalres = h_off[n] - h_off[0];
    k_codes<<<std::min<int64_t>(blocks_for(totalres, T), 4096), T, 0, st>>>(d_res + h_off[0],
                                                                           totalres, d_status);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(h_status, d_status, sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (h_status[0] & kBadArg) goto bad;
    h_len.resize(n);
    std::vector<int64_t> h_po(n + 1);
    h_po[0] = 0;
    for (int32_t i = 0; i < n; ++i) {
      h_len[i] = (int32_t)(h_off[i + 1] - h_off[i]);
      h_po[i + 1] = h_po[i] + (h_len[i] + 63) / 64;
    }
    CK(lib_malloc_async((void **)d_peq_off, sizeof(int64_t) * (n + 1), st));
    CK(lib_malloc_async((void **)d_peq, sizeof(uint32_t) * kPeqWordU32 * (size_t)std::max<int64_t>(h_po[n], 1), st));
    CK(cudaMemcpyAsync(*d_peq_off, h_po.data(), sizeof(int64_t) * (n + 1), cudaMemcpyHostToDevice, st));
    k_pack_peq<<<blocks_for((int64_t)n * 32, T), T, 0, st>>>(d_res, d_off, nullptr, *d_peq_off, n,
                                                            *d_peq);
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(st));
  }
  cudaFreeAsync(d_status, st); cudaFreeAsync(rebased, st);
  return FAMSA_OK;
bad:
  release_rows(st, d_status, rebased, d_len, d_peq_off, d_peq);
  return FAMSA_EINVAL;
toolong:
  release_rows(st, d_status, rebased, d_len, d_peq_off, d_peq);
  return FAMSA_ERANGE;
fail:
  release_rows(st, d_status, rebased, d_len, d_peq_off, d_peq);
  return status_from_cuda(err);
}

}  // namespace famsa

extern "C" int famsa_debug_fail_alloc_after(int n) {
  famsa::g_alloc_fail_after.store(n);
  return 0;
}

extern "C" int64_t famsa_debug_alloc_count(void) { return famsa::g_alloc_count.load(); }

// one check that fails on purpose and guards nothing: the checker's own test
__global__ void k_check_selftest() { (void)FAMSA_EXPECT(threadIdx.x != 0); }

extern "C" int famsa_debug_check_selftest(void) {
#ifdef FAMSA_CHECKED
  k_check_selftest<<<1, 1>>>();
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  return famsa::status_from_cuda(e);
#else
  return -1;
#endif
}

extern "C" int64_t famsa_debug_check_count(int64_t *first_line) {
#ifdef FAMSA_CHECKED
  unsigned long long n = 0, line = 0;
  famsa::read_checks(&n, &line);
  if (first_line) *first_line = (int64_t)line;
  return (int64_t)n;
#else
  if (first_line) *first_line = 0;
  return -1;
#endif
}

// The packed match-bitmask tables of a family, for tests: peq (words x 64
// u32, host) in the family's (length, index) order, the first word of each
// sequence (k + 1 host int64, the last entry the total), and the caller's
// label of each sorted sequence (k host int32).  Any output may be NULL; with
// peq NULL, *n_words still receives the total.
extern "C" int famsa_debug_peq(const famsa_family *fh, uint32_t *peq, int64_t *word_off, int32_t *perm,
                               int64_t *n_words) {
  if (!fh) return FAMSA_EINVAL;
  const famsa::Family *f = reinterpret_cast<const famsa::Family *>(fh);
  if (n_words) *n_words = f->peq_words;
  cudaError_t e = cudaSuccess;
  if (peq)
    e = cudaMemcpy(peq, f->d_peq, sizeof(uint32_t) * famsa::kPeqWordU32 * (size_t)f->peq_words,
                   cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && word_off)
    e = cudaMemcpy(word_off, f->d_peq_off, sizeof(int64_t) * ((size_t)f->k + 1), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && perm)
    e = cudaMemcpy(perm, f->d_perm, sizeof(int32_t) * (size_t)f->k, cudaMemcpyDeviceToHost);
  return famsa::status_from_cuda(e);
}
