// Shared device helpers of the single-linkage row update: exact distance keys,
// clamp-function scans, the row-update state and small sorts.
//
// FAMSA Methods, "Determination of the guide tree": single linkage by SLINK
// (Sibson 1973), computed from the similarity rows one new point at a time.
// Pairs are ordered by the exact rational distance indel^2 / LCS (the
// paper's similarity LCS / indel^2 reversed; "Pairwise similarities
// calculation"), indel = |A| + |B| - 2 LCS.
#pragma once

#include <cooperative_groups.h>

#include "famsa_internal.cuh"

namespace cg = cooperative_groups;

namespace famsa {

// ----------------------------------------------------------------- keys
// Packed exact distance: (indel^2 << 16) | LCS, indel^2 < 2^34, LCS <= 65535.
// LCS = 0 gives +inf, encoded (1 << 16) (num 1, den 0); 0 has num 0.
// a < b by cross multiplication (products < 2^50, no overflow).
constexpr uint64_t kKeyInf = 1ull << 16;
constexpr uint64_t kKeyZero = 1ull;

__host__ __device__ __forceinline__ bool klt(uint64_t a, uint64_t b) {
  return (a >> 16) * (b & 0xffffu) < (b >> 16) * (a & 0xffffu);
}
__host__ __device__ __forceinline__ uint64_t kmin(uint64_t a, uint64_t b) { return klt(b, a) ? b : a; }
__host__ __device__ __forceinline__ uint64_t kmax(uint64_t a, uint64_t b) { return klt(a, b) ? b : a; }
__device__ __forceinline__ uint64_t make_key(uint32_t L, uint32_t la, uint32_t lb) {
  if (L == 0) return kKeyInf;
  uint64_t indel = (uint64_t)(la + lb - 2 * L);
  return ((indel * indel) << 16) | L;
}

// Exact order codes.  For a distance num / den with num < 2^32 and
// 1 <= den <= 32767, code = floor(num * 2^30 / den) is strictly increasing in
// the value: two different values differ by at least 1 / (den_a * den_b) >
// 2^-30 (32767^2 < 2^30), so their scaled floors differ, and equal values get
// equal codes.  Comparing codes is one 64-bit integer compare instead of two
// multiplies.  The quotient is taken in three 15-bit digits after the integer
// part, each a 32-bit division.
__host__ __device__ __forceinline__ uint64_t order_code(uint32_t num, uint32_t den) {
  const uint32_t q0 = num / den, r0 = num - q0 * den;
  const uint32_t t1 = r0 << 15, q1 = t1 / den, r1 = t1 - q1 * den;
  const uint32_t q2 = (r1 << 15) / den;
  return ((uint64_t)q0 << 30) | ((uint64_t)q1 << 15) | q2;
}

// The distance an order code came from, as a reduced fraction p / q.  At most
// one fraction with a denominator <= 32767 lies in [code, code + 1) / 2^30
// (interval shorter than their spacing), so it is the fraction of smallest
// denominator there: the continued-fraction descent of the Stern-Brocot tree
// finds it.  y is tracked as x = (P1 y + P0) / (Q1 y + Q0) over intervals
// [lo, hi) of y, each step peeling off the integer part and inverting.
__host__ __device__ inline void code_fraction(uint64_t code, uint64_t *p, uint32_t *q) {
  const uint64_t whole = code >> 30;
  const uint32_t a = (uint32_t)(code & ((1u << 30) - 1));
  if (a == 0) {
    *p = whole;
    *q = 1;
    return;
  }
  // y in [ln/ld, hn/hd) with closedness flags; hd == 0 means +infinity
  uint32_t ln = a, ld = 1u << 30, hn = a + 1, hd = 1u << 30;
  bool lc = true, hc = false;
  uint64_t P1 = 1, P0 = 0, Q1 = 0, Q0 = 1, y = 0;
  for (int it = 0; it < 64; ++it) {
    const uint32_t f = ln / ld, rem = ln - f * ld;
    if (rem == 0 && lc) { y = f; break; }
    const uint64_t g = (uint64_t)f + 1;  // the smallest integer above lo
    if (hd == 0 || g * hd < hn || (g * hd == hn && hc)) { y = g; break; }
    // no integer inside: y = f + 1/z, z in (1/(hi - f), 1/(lo - f)) with the ends swapped
    const uint32_t nln = hd, nld = hn - f * hd;
    const bool nlc = hc;
    uint32_t nhn = 1, nhd = 0;
    bool nhc = false;
    if (rem != 0) { nhn = ld; nhd = rem; nhc = lc; }
    uint64_t t = P1 * f + P0; P0 = P1; P1 = t;
    t = Q1 * f + Q0; Q0 = Q1; Q1 = t;
    ln = nln; ld = nld; lc = nlc; hn = nhn; hd = nhd; hc = nhc;
  }
  const uint64_t r = P1 * y + P0, s = Q1 * y + Q0;
  *p = whole * s + r;
  *q = (uint32_t)s;
}

// Two packings of the same exact key.  Wide: (num << 16) | den, any length
// up to 65535, compared by cross multiplication.  Narrow: the order code
// above, when every length is <= 32767 so that num = indel^2 < 2^32 and
// den = LCS <= 32767; +inf (LCS 0) is all ones.
struct KeysWide {
  static constexpr uint64_t kInf = 1ull << 16;
  static constexpr uint64_t kZero = 1ull;
  __device__ __forceinline__ static bool lt(uint64_t a, uint64_t b) { return klt(a, b); }
  __device__ __forceinline__ static uint64_t make(uint32_t L, uint32_t la, uint32_t lb) {
    return make_key(L, la, lb);
  }
  __device__ __forceinline__ static uint64_t wide(uint64_t k) { return k; }
};
struct KeysNarrow {
  static constexpr uint64_t kInf = ~0ull;
  static constexpr uint64_t kZero = 0ull;
  __device__ __forceinline__ static bool lt(uint64_t a, uint64_t b) { return a < b; }
  __device__ __forceinline__ static uint64_t make(uint32_t L, uint32_t la, uint32_t lb) {
    if (L == 0) return kInf;
    const uint32_t indel = la + lb - 2 * L;
    return order_code(indel * indel, L);
  }
  // the same distance as a wide key, reduced (finalisation reduces every
  // fraction it reports, so reduced and unreduced keys give the same output)
  __host__ __device__ static uint64_t wide(uint64_t k) {
    if (k == kInf) return KeysWide::kInf;
    uint64_t p;
    uint32_t q;
    code_fraction(k, &p, &q);
    return (p << 16) | q;
  }
};

// ----------------------------------------------------------------- clamps
// The minimax distance from a new point n along a dendrogram leaf order
// (u(x_p, x_q) = max gap between p and q) satisfies
//   Lf[q] = min(d[q], max(Lf[q-1], gap[q-1])),  Rf[q] = min(d[q], max(Rf[q+1], gap[q])),
//   D[q]  = min(Lf[q], Rf[q]).
// Each step is the clamp x -> min(hi, max(x, lo)); clamps compose into
// clamps, so the recurrences run as parallel scans.
struct Clamp {
  uint64_t lo, hi;
};
template <class K>
__device__ __forceinline__ uint64_t kmin_t(uint64_t a, uint64_t b) { return K::lt(b, a) ? b : a; }
template <class K>
__device__ __forceinline__ uint64_t kmax_t(uint64_t a, uint64_t b) { return K::lt(a, b) ? b : a; }
template <class K = KeysWide>
__device__ __forceinline__ Clamp identity_clamp() { return Clamp{K::kZero, K::kInf}; }
// a, then b
template <class K = KeysWide>
__device__ __forceinline__ Clamp compose(const Clamp &a, const Clamp &b) {
  return Clamp{kmax_t<K>(a.lo, b.lo), kmin_t<K>(b.hi, kmax_t<K>(a.hi, b.lo))};
}
__device__ __forceinline__ Clamp shfl_clamp_up(const Clamp &c, int d) {
  return Clamp{__shfl_up_sync(0xffffffffu, c.lo, d), __shfl_up_sync(0xffffffffu, c.hi, d)};
}
__device__ __forceinline__ Clamp shfl_clamp_down(const Clamp &c, int d) {
  return Clamp{__shfl_down_sync(0xffffffffu, c.lo, d), __shfl_down_sync(0xffffffffu, c.hi, d)};
}
__device__ __forceinline__ Clamp shfl_clamp_idx(const Clamp &c, int src) {
  return Clamp{__shfl_sync(0xffffffffu, c.lo, src), __shfl_sync(0xffffffffu, c.hi, src)};
}

// The first shuffle distance of a tree reduction over the first n lanes (the
// others hold the identity): the largest power of two below n, 0 for n <= 1.
__device__ __forceinline__ int red_top(int n) { return n <= 1 ? 0 : 1 << (31 - __clz(n - 1)); }

// Block-level exclusive scans of clamps, forward (thread order) and backward
// (reverse thread order) at once.  sw needs 4*32+2 entries.  Returns the
// thread's exclusive prefixes and the block totals.
template <class K = KeysWide>
__device__ __forceinline__ void block_scan2(Clamp vf, Clamp vb, Clamp *pf, Clamp *pb, Clamp *tf,
                                            Clamp *tb, Clamp *sw) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  Clamp incf = vf, incb = vb;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    Clamp yf = shfl_clamp_up(incf, d);
    Clamp yb = shfl_clamp_down(incb, d);
    if (lane >= d) incf = compose<K>(yf, incf);
    if (lane + d < 32) incb = compose<K>(yb, incb);
  }
  Clamp excf = shfl_clamp_up(incf, 1);
  Clamp excb = shfl_clamp_down(incb, 1);
  if (lane == 0) excf = identity_clamp<K>();
  if (lane == 31) excb = identity_clamp<K>();
  if (lane == 31) sw[warp] = incf;
  if (lane == 0) sw[32 + warp] = incb;
  __syncthreads();
  if (warp == 0) {
    Clamp wf = lane < nw ? sw[lane] : identity_clamp<K>();
    Clamp wb = lane < nw ? sw[32 + lane] : identity_clamp<K>();
    for (int d = 1; d < nw; d <<= 1) {  // lanes >= nw hold the identity
      Clamp yf = shfl_clamp_up(wf, d);
      Clamp yb = shfl_clamp_down(wb, d);
      if (lane >= d) wf = compose<K>(yf, wf);
      if (lane + d < 32) wb = compose<K>(yb, wb);
    }
    Clamp ef = shfl_clamp_up(wf, 1);
    Clamp eb = shfl_clamp_down(wb, 1);
    if (lane == 0) ef = identity_clamp<K>();
    if (lane >= nw - 1) eb = identity_clamp<K>();
    if (lane < nw) { sw[64 + lane] = ef; sw[96 + lane] = eb; }
    if (lane == nw - 1) sw[128] = wf;
    if (lane == 0) sw[129] = wb;
  }
  __syncthreads();
  *pf = compose<K>(sw[64 + warp], excf);
  *pb = compose<K>(sw[96 + warp], excb);
  *tf = sw[128];
  *tb = sw[129];
  // no trailing barrier: the next call writes sw[0..64) before its first
  // barrier and the result slots sw[64..130) only after it
}

// ----------------------------------------------------------------- state
// Row-update state, one entry per position of the current dendrogram leaf
// order.  Buffers alternate with the number of points: the layout of m
// points is in buffer m & 1.  lam/pi are Sibson's pointer representation of
// the point at that position (insertion labels); they move with the point.
struct SlinkState {
  int32_t *ord[2];   // point (insertion label)
  int32_t *olen[2];  // its length
  uint64_t *gap[2];  // gap[p] = minimax distance between positions p and p+1
  uint64_t *lam[2];
  int32_t *pi[2];
  uint64_t *D;       // minimax distances to the new point (global kernel)
  // run-merge buffers (positions), ping-pong
  uint64_t *mD[2];
  int32_t *mOrd[2], *mLen[2], *mOld[2], *mPi[2], *mRaw[2];
  uint64_t *mLam[2];
  uint64_t *mGap;    // old gaps (cluster shared-memory kernel's merge path)
  int32_t *runsA, *runsB;  // run starts, unsorted
  uint64_t *ctl;
  const int32_t *slen;     // lengths in insertion order
};

constexpr int kMaxClusterCtas = 16;
constexpr int kRunsSmem = 2048;  // natural-run merges keep up to this many run starts per side

// ctl layout (uint64 words)
constexpr int kCtlAggL = 0;                               // 2 words per CTA
constexpr int kCtlAggR = kCtlAggL + 2 * kMaxClusterCtas;
constexpr int kCtlArg = kCtlAggR + 2 * kMaxClusterCtas;   // 2 words per CTA
constexpr int kCtlCnt = kCtlArg + 2 * kMaxClusterCtas;    // 6 words: run counts A,B, 3 slots
constexpr int kCtlStats = kCtlCnt + 6;                    // merges, rounds, phase cycles A..D, fast merges, sub-phase cycles
constexpr int kCtlWords = kCtlStats + 24;

__device__ __forceinline__ void chunk_of(int32_t m, int32_t tid, int32_t nthreads, int32_t *b,
                                         int32_t *e) {
  int32_t c = (m + nthreads - 1) / nthreads;
  int64_t bb = (int64_t)tid * c;
  *b = (int32_t)(bb < m ? bb : (int64_t)m);
  *e = (int32_t)(bb + c < m ? bb + c : (int64_t)m);
}

// index of the last run start <= i (starts sorted ascending, starts[0] <= i)
__device__ __forceinline__ int32_t run_of(const int32_t *starts, int32_t nruns, int32_t i) {
  int32_t lo = 0, hi = nruns - 1;
  while (lo < hi) {
    int32_t mid = (lo + hi + 1) >> 1;
    if (starts[mid] <= i) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// in-place bitonic sort of n ints in shared memory (cap: power of two >= n)
__device__ __forceinline__ void smem_sort(int32_t *a, int32_t n, int32_t cap) {
  for (int32_t i = n + threadIdx.x; i < cap; i += blockDim.x) a[i] = INT32_MAX;
  __syncthreads();
  for (int32_t size = 2; size <= cap; size <<= 1) {
    for (int32_t stride = size >> 1; stride > 0; stride >>= 1) {
      for (int32_t i = threadIdx.x; i < cap; i += blockDim.x) {
        int32_t j = i ^ stride;
        if (j > i) {
          bool up = (i & size) == 0;
          int32_t x = a[i], y = a[j];
          if ((x > y) == up) { a[i] = y; a[j] = x; }
        }
      }
      __syncthreads();
    }
  }
}

// Stable pairwise merge of sorted runs on one side of the re-layout.  The
// left side (positions < x0) sorts by D descending, the right side ascending;
// an element of the left run of a pair counts partner elements strictly
// before it, an element of the right run counts partner elements before or
// equal.  Returns the number of partner elements that precede value v.
template <class K = KeysWide>
__device__ __forceinline__ int32_t merge_count(const uint64_t *key, int32_t sbase, int32_t ps,
                                               int32_t pe, uint64_t v, bool left_side,
                                               bool in_left_run) {
  int32_t lo = ps, hi = pe;
  while (lo < hi) {
    int32_t mid = (lo + hi) >> 1;
    uint64_t w = key[sbase + mid];
    bool before;
    if (left_side) before = in_left_run ? K::lt(v, w) : !K::lt(w, v);
    else before = in_left_run ? K::lt(w, v) : !K::lt(v, w);
    if (before) lo = mid + 1; else hi = mid;
  }
  return lo - ps;
}

// one element of a bottom-up merge pass on an index array under a strict total order
template <class Cmp>
__device__ __forceinline__ void msort_at(int32_t i, const int32_t *in, int32_t *out, int32_t n, int32_t width,
                                         Cmp cmp) {
  int64_t run = i / width;
  int64_t start = run * width;
  int64_t pair_start = (run & ~1LL) * width;
  int64_t pstart = (run ^ 1) * width;
  int32_t x = in[i];
  if (pstart >= n) { out[i] = x; return; }
  int64_t pend = pstart + width < n ? pstart + width : (int64_t)n;
  int64_t lo = pstart, hi = pend;
  while (lo < hi) {
    int64_t mid = (lo + hi) >> 1;
    if (cmp(in[mid], x)) lo = mid + 1; else hi = mid;
  }
  out[pair_start + (i - start) + (lo - pstart)] = x;
}

// Buffers for the finalisation (all device, caller-owned)
// Arguments of the cluster shared-memory row update: insert points r0..r1-1,
// whose similarity rows are rowbuf[(n - r0) * ld ..].
struct SmemArgs {
  SlinkState s;
  const uint16_t *rowbuf;
  int64_t ld;  // even, so every row starts on a 4-byte boundary
  int32_t r0, r1;
  int32_t P;   // positions per CTA
  int32_t sshift;  // every 2^sshift-th D is sampled for the run-merge searches
  // batched families: cluster c takes batch[c] (its own state, rows and sizes)
  const SmemArgs *batch;
  size_t dyn_bytes;  // batched launch: dynamic shared memory of every cluster
};
cudaError_t launch_slink_smem_batch(const SmemArgs *d_args, int32_t n_clusters, int cl, size_t dyn_bytes,
                                    bool narrow, cudaStream_t st);
size_t smem_dyn_bytes(int32_t P, int32_t k, int shift);
int smem_sample_shift(int32_t P, int32_t k);

struct FinBufs {
  int32_t *idx, *posof, *it, *rt, *pi, *sub_lo, *sub_hi, *ordA, *ordB, *rank, *sorder, *merges,
      *sizes;
  uint64_t *gt, *lam, *hkey, *lnum, *hnum;
  uint32_t *lden, *hden;
  int64_t *sz, *szpre, *tot;
};

size_t fin_levels(int32_t k);

// Stream-ordered scratch of one call: every get() allocates on st (through
// lib_malloc_async); release() frees all of it on st.  The first failure is
// kept in err and later gets return nullptr.
struct Scratch {
  std::vector<void *> ptrs;
  cudaStream_t st = nullptr;
  cudaError_t err = cudaSuccess;
  template <typename T>
  T *get(size_t n) {
    void *p = nullptr;
    if (err != cudaSuccess) return nullptr;
    err = lib_malloc_async(&p, (n > 0 ? n : 1) * sizeof(T), st);
    if (err != cudaSuccess) return nullptr;
    ptrs.push_back(p);
    return static_cast<T *>(p);
  }
  void release() {
    for (void *p : ptrs) cudaFreeAsync(p, st);
    ptrs.clear();
  }
};

// the finalisation's buffers for k points
inline FinBufs alloc_fin_bufs(Scratch &sc, int32_t k) {
  const size_t lv = fin_levels(k);
  FinBufs FB;
  FB.idx = sc.get<int32_t>(k); FB.posof = sc.get<int32_t>(k);
  FB.it = sc.get<int32_t>(lv * k); FB.rt = sc.get<int32_t>(lv * k);
  FB.gt = sc.get<uint64_t>(lv * k);
  FB.pi = sc.get<int32_t>(k); FB.sub_lo = sc.get<int32_t>(k); FB.sub_hi = sc.get<int32_t>(k);
  FB.ordA = sc.get<int32_t>(k); FB.ordB = sc.get<int32_t>(k); FB.rank = sc.get<int32_t>(k);
  FB.sorder = sc.get<int32_t>(k); FB.merges = sc.get<int32_t>(2 * (size_t)k);
  FB.sizes = sc.get<int32_t>(k);
  FB.lam = sc.get<uint64_t>(k); FB.hkey = sc.get<uint64_t>(k);
  FB.lnum = sc.get<uint64_t>(k); FB.hnum = sc.get<uint64_t>(k);
  FB.lden = sc.get<uint32_t>(k); FB.hden = sc.get<uint32_t>(k);
  FB.sz = sc.get<int64_t>(k); FB.szpre = sc.get<int64_t>(k); FB.tot = sc.get<int64_t>(2);
  return FB;
}
cudaError_t launch_finalize(const int32_t *ord, uint64_t *gap, const int32_t *perm, int32_t k,
                            FinBufs &B, cudaStream_t st, int64_t *launches, bool widen);
cudaError_t launch_slink_global(const SlinkState &S, const uint16_t *rowbuf, int64_t ld, int32_t r0,
                                int32_t r1, int cl, bool narrow, cudaStream_t st);
int max_cluster_global();
int smem_cluster_for(int32_t k, int force);
int smem_cluster_latency(int32_t k);
cudaError_t launch_slink_smem(const SlinkState &S, const uint16_t *rowbuf, int64_t ld, int32_t r0,
                              int32_t r1, int cl, int32_t k, bool narrow, cudaStream_t st);
cudaError_t widen_keys(uint64_t *key, int32_t n, cudaStream_t st);

}  // namespace famsa
