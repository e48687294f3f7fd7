// Finalisation: the canonical pointer representation and the merge list in
// the caller's labels, computed in parallel from the final dendrogram leaf
// order (positions -> points) and its gap array.
//
// In a leaf order with gaps g, the single-link distance is
// u(x_p, x_q) = max g[p..q-1].  For point j at position p:
//   lambda(j) = min over l > j of u(j, l): the nearest positions left and
//     right of p holding a larger label give the two candidates (further
//     ones only see larger maxima);
//   pi(j) = the largest label in the maximal interval around p whose gaps are
//     <= lambda(j) (j's cluster at height lambda(j)).
// The merge list takes j in (lambda(j), j) order.  At that point j's cluster
// is its pointer subtree -- the maximal interval around p with gaps
// < lambda(j) -- whose id is k + the largest merge rank inside it (or j
// alone), and pi(j)'s cluster is pi(j) plus the subtrees of its children
// merged earlier (children = points c with pi(c) = pi(j), ordered by
// (lambda(c), c)).  All queries use sparse tables of range maxima.
#include <algorithm>
#include <vector>

#include "slink_common.cuh"

namespace famsa {

__global__ void k_scan_excl(const int64_t *in, int64_t *out, int64_t n, int64_t *total);

// ---- per-element steps, shared by the multi-kernel path (one launch per
// step) and the single-CTA path (every step in one launch)

__device__ __forceinline__ void fin_idx_at(int32_t p, const int32_t *ord, const int32_t *perm, int32_t *idx) {
  idx[p] = perm[ord[p]];
}

// level j of the range-max tables: T[j][p] = max over [p, p + 2^j)
__device__ __forceinline__ void fin_level_at(int32_t p, uint64_t *gt, int32_t *it, int32_t k, int32_t j) {
  const int32_t h = 1 << (j - 1);
  const int64_t K = k;
  if (p + 2 * h <= k - 1) gt[j * K + p] = kmax(gt[(j - 1) * K + p], gt[(j - 1) * K + p + h]);
  if (p + 2 * h <= k) it[j * K + p] = max(it[(j - 1) * K + p], it[(j - 1) * K + p + h]);
}

__device__ __forceinline__ void fin_level_int_at(int32_t p, int32_t *rt, int32_t k, int32_t j) {
  const int32_t h = 1 << (j - 1);
  const int64_t K = k;
  if (p + 2 * h <= k) rt[j * K + p] = max(rt[(j - 1) * K + p], rt[(j - 1) * K + p + h]);
}

__device__ __forceinline__ int ilog2(int32_t x) { return 31 - __clz(x); }

__device__ __forceinline__ uint64_t gap_max(const uint64_t *gt, int64_t K, int32_t a, int32_t b) {
  // max over gaps a..b inclusive (a <= b)
  int j = ilog2(b - a + 1);
  return kmax(gt[j * K + a], gt[j * K + b - (1 << j) + 1]);
}
__device__ __forceinline__ int32_t int_max(const int32_t *t, int64_t K, int32_t a, int32_t b) {
  int j = ilog2(b - a + 1);
  return max(t[j * K + a], t[j * K + b - (1 << j) + 1]);
}

// lambda, pi and the pointer-subtree interval of the point at position p
__device__ __forceinline__ void fin_lambda_at(int32_t p, const uint64_t *gt, const int32_t *it,
                                              const int32_t *idx, int32_t k, int levels, uint64_t *lam,
                                              int32_t *pi, int32_t *sub_lo, int32_t *sub_hi) {
  const int64_t K = k;
  const int32_t j = idx[p];
  uint64_t L = kKeyInf;
  if (j == k - 1) {
    lam[j] = kKeyInf;
    pi[j] = k - 1;
  } else {
    // nearest position to the left holding a larger label
    int32_t pos = p;
    for (int s = levels - 1; s >= 0; --s)
      if (pos - (1 << s) >= 0 && it[s * K + pos - (1 << s)] < j) pos -= 1 << s;
    uint64_t cand = kKeyInf;
    if (pos > 0) cand = gap_max(gt, K, pos - 1, p - 1);
    L = cand;
    pos = p;
    for (int s = levels - 1; s >= 0; --s)
      if (pos + (1 << s) <= k - 1 && it[s * K + pos + 1] < j) pos += 1 << s;
    if (pos + 1 < k) L = kmin(L, gap_max(gt, K, p, pos));
    // cluster at height lambda: gaps <= lambda around p
    int32_t a = p, b = p;
    for (int s = levels - 1; s >= 0; --s) {
      if (a - (1 << s) >= 0 && !klt(L, gt[s * K + a - (1 << s)])) a -= 1 << s;
      if (b + (1 << s) <= k - 1 && !klt(L, gt[s * K + b])) b += 1 << s;
    }
    lam[j] = L;
    pi[j] = int_max(it, K, a, b);
  }
  // pointer subtree: gaps < lambda around p
  int32_t a = p, b = p;
  for (int s = levels - 1; s >= 0; --s) {
    if (a - (1 << s) >= 0 && klt(gt[s * K + a - (1 << s)], L)) a -= 1 << s;
    if (b + (1 << s) <= k - 1 && klt(gt[s * K + b], L)) b += 1 << s;
  }
  sub_lo[j] = a;
  sub_hi[j] = b;
}

struct ByLambda {
  const uint64_t *lam;
  __device__ bool operator()(int32_t x, int32_t y) const {
    uint64_t a = lam[x], b = lam[y];
    if (klt(a, b)) return true;
    if (klt(b, a)) return false;
    return x < y;
  }
};
struct ByParent {
  const int32_t *pi;
  const uint64_t *lam;
  __device__ bool operator()(int32_t x, int32_t y) const {
    if (pi[x] != pi[y]) return pi[x] < pi[y];
    uint64_t a = lam[x], b = lam[y];
    if (klt(a, b)) return true;
    if (klt(b, a)) return false;
    return x < y;
  }
};

__device__ __forceinline__ void fin_merges_at(int32_t s, const int32_t *sorder, const int32_t *pi,
                                              const uint64_t *lam, const int32_t *rank,
                                              const int32_t *sub_lo, const int32_t *sub_hi,
                                              const int32_t *posof, const int32_t *rt, const int64_t *szpre,
                                              int32_t k, int32_t *merges, uint64_t *hkey, int32_t *sizes) {
  const int64_t K = k;
  const int32_t j = sorder[s];
  const int32_t par = pi[j];
  // first sibling of j in the (parent, lambda, label) order
  int32_t lo = 0, hi = s;
  while (lo < hi) {
    int32_t mid = (lo + hi) >> 1;
    if (pi[sorder[mid]] < par) lo = mid + 1; else hi = mid;
  }
  const int32_t head = lo;
  const int32_t a = sub_lo[j], b = sub_hi[j];
  const int32_t sz_j = b - a + 1;
  // j's cluster just before its merge: its pointer subtree [a, b], last formed
  // by the merge of largest rank inside it other than j's own
  int32_t id_j = j;
  if (sz_j > 1) {
    const int32_t pj = posof[j];
    int32_t best = -1;
    if (pj > a) best = max(best, int_max(rt, K, a, pj - 1));
    if (pj < b) best = max(best, int_max(rt, K, pj + 1, b));
    id_j = k + best;
  }
  // pi(j)'s cluster: pi(j) plus the subtrees of its earlier children
  int32_t id_p = par;
  int64_t before = 0;
  if (s > head) {
    id_p = k + rank[sorder[s - 1]];
    before = szpre[s] - szpre[head];
  }
  const int32_t t = rank[j];
  merges[2 * t] = min(id_j, id_p);
  merges[2 * t + 1] = max(id_j, id_p);
  hkey[t] = lam[j];
  sizes[t] = (int32_t)(sz_j + 1 + before);
}

__device__ uint64_t gcd_u64(uint64_t a, uint64_t b) {
  while (b) { uint64_t t = a % b; a = b; b = t; }
  return a;
}

// packed key -> reduced (num, den)
__device__ __forceinline__ void fin_reduce_at(int32_t i, const uint64_t *key, uint64_t *num, uint32_t *den) {
  uint64_t kk = key[i];
  uint64_t nu = kk >> 16;
  uint32_t de = (uint32_t)(kk & 0xffffu);
  if (de == 0) nu = 1;
  else if (nu == 0) de = 1;
  else {
    uint64_t g = gcd_u64(nu, de);
    nu /= g;
    de = (uint32_t)(de / g);
  }
  num[i] = nu;
  den[i] = de;
}

// ---- the multi-kernel path: one launch per step
#define FIN_ELEMENTWISE(name, n_expr)                         \
  const int32_t name = blockIdx.x * blockDim.x + threadIdx.x; \
  if (name >= (n_expr)) return;

__global__ void k_fin_widen(uint64_t *key, int32_t n) {
  FIN_ELEMENTWISE(i, n)
  key[i] = KeysNarrow::wide(key[i]);
}
__global__ void k_fin_idx(const int32_t *ord, const int32_t *perm, int32_t k, int32_t *idx) {
  FIN_ELEMENTWISE(p, k)
  fin_idx_at(p, ord, perm, idx);
}
__global__ void k_fin_level(uint64_t *gt, int32_t *it, int32_t k, int32_t j) {
  FIN_ELEMENTWISE(p, k)
  fin_level_at(p, gt, it, k, j);
}
__global__ void k_fin_level_int(int32_t *rt, int32_t k, int32_t j) {
  FIN_ELEMENTWISE(p, k)
  fin_level_int_at(p, rt, k, j);
}
__global__ void k_fin_lambda(const uint64_t *gt, const int32_t *it, const int32_t *idx, int32_t k,
                             int levels, uint64_t *lam, int32_t *pi, int32_t *sub_lo,
                             int32_t *sub_hi) {
  FIN_ELEMENTWISE(p, k)
  fin_lambda_at(p, gt, it, idx, k, levels, lam, pi, sub_lo, sub_hi);
}
template <class Cmp>
__global__ void k_msort(const int32_t *in, int32_t *out, int32_t n, int32_t width, Cmp cmp) {
  FIN_ELEMENTWISE(i, n)
  msort_at(i, in, out, n, width, cmp);
}
__global__ void k_fin_iota(int32_t *a, int32_t n) {
  FIN_ELEMENTWISE(i, n)
  a[i] = i;
}
__global__ void k_fin_rank(const int32_t *order, int32_t n, int32_t *rank) {
  FIN_ELEMENTWISE(t, n)
  rank[order[t]] = t;
}
__global__ void k_fin_rankpos(const int32_t *idx, const int32_t *rank, int32_t k, int32_t *rt0) {
  FIN_ELEMENTWISE(p, k)
  rt0[p] = idx[p] == k - 1 ? -1 : rank[idx[p]];
}
__global__ void k_fin_sizes(const int32_t *sorder, const int32_t *sub_lo, const int32_t *sub_hi,
                            int32_t n, int64_t *sz) {
  FIN_ELEMENTWISE(s, n)
  const int32_t j = sorder[s];
  sz[s] = sub_hi[j] - sub_lo[j] + 1;
}
__global__ void k_fin_merges(const int32_t *sorder, const int32_t *pi, const uint64_t *lam,
                             const int32_t *rank, const int32_t *sub_lo, const int32_t *sub_hi,
                             const int32_t *posof, const int32_t *rt, const int64_t *szpre,
                             int32_t n, int32_t k, int32_t *merges, uint64_t *hkey,
                             int32_t *sizes) {
  FIN_ELEMENTWISE(s, n)
  fin_merges_at(s, sorder, pi, lam, rank, sub_lo, sub_hi, posof, rt, szpre, k, merges, hkey, sizes);
}
__global__ void k_fin_posof(const int32_t *idx, int32_t k, int32_t *posof) {
  FIN_ELEMENTWISE(p, k)
  posof[idx[p]] = p;
}
__global__ void k_fin_reduce(const uint64_t *key, int32_t n, uint64_t *num, uint32_t *den) {
  FIN_ELEMENTWISE(i, n)
  fin_reduce_at(i, key, num, den);
}
#undef FIN_ELEMENTWISE

// ---- the single-CTA path: every step of one family in one launch, the
// steps separated by block barriers (families up to kFinSmall points)
constexpr int kFinSmall = 4096;
constexpr int kFinThreads = 1024;
static int g_fin_small = kFinSmall;  // test hook: 0 sends every family to the multi-kernel path

#define FIN_FOR(v, n) for (int32_t v = (int32_t)threadIdx.x; v < (n); v += kFinThreads)

// exclusive prefix sums of in[0, n) into out, total into *total (one block)
__device__ void fin_block_scan(const int64_t *in, int64_t *out, int32_t n, int64_t *total, int64_t *warp_sums) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  // each thread takes a contiguous chunk, then the chunk sums are scanned
  const int32_t chunk = (n + kFinThreads - 1) / kFinThreads;
  const int32_t b = min(n, (int32_t)threadIdx.x * chunk), e = min(n, b + chunk);
  int64_t sum = 0;
  for (int32_t i = b; i < e; ++i) sum += in[i];
  int64_t x = sum;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const int64_t y = __shfl_up_sync(0xffffffffu, x, d);
    if (lane >= d) x += y;
  }
  if (lane == 31) warp_sums[warp] = x;
  __syncthreads();
  if (warp == 0) {
    int64_t w = warp_sums[lane];  // kFinThreads / 32 == 32 warps
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const int64_t y = __shfl_up_sync(0xffffffffu, w, d);
      if (lane >= d) w += y;
    }
    warp_sums[lane] = w;
  }
  __syncthreads();
  int64_t run = x - sum + (warp > 0 ? warp_sums[warp - 1] : 0);
  for (int32_t i = b; i < e; ++i) {
    out[i] = run;
    run += in[i];
  }
  if (threadIdx.x == kFinThreads - 1) *total = run;
}

__global__ void __launch_bounds__(kFinThreads, 1) k_fin_small(const int32_t *ord, uint64_t *gap, const int32_t *perm,
                                                           int32_t k, int widen, FinBufs B) {
  __shared__ int64_t warp_sums[32];
  const int levels = ilog2(k) + 1;  // the number of levels fin_levels gives
  const int64_t K = k;
  const int32_t n = k - 1;
  if (widen) {
    FIN_FOR(i, n) gap[i] = KeysNarrow::wide(gap[i]);
    __syncthreads();
  }
  FIN_FOR(p, k) fin_idx_at(p, ord, perm, B.idx);
  __syncthreads();
  FIN_FOR(p, k) {
    B.posof[B.idx[p]] = p;
    B.it[p] = B.idx[p];
    if (p < n) B.gt[p] = gap[p];
  }
  __syncthreads();
  for (int j = 1; j < levels; ++j) {
    FIN_FOR(p, k) fin_level_at(p, B.gt, B.it, k, j);
    __syncthreads();
  }
  FIN_FOR(p, k) fin_lambda_at(p, B.gt, B.it, B.idx, k, levels, B.lam, B.pi, B.sub_lo, B.sub_hi);
  FIN_FOR(i, n) {
    B.ordA[i] = i;
    B.sorder[i] = i;
  }
  __syncthreads();
  // merge order (lambda, j), then sibling order (pi, lambda, j)
  int32_t *a = B.ordA, *b = B.ordB;
  for (int32_t w = 1; w < n; w *= 2) {
    FIN_FOR(i, n) msort_at(i, a, b, n, w, ByLambda{B.lam});
    __syncthreads();
    int32_t *t = a; a = b; b = t;
  }
  FIN_FOR(t, n) B.rank[a[t]] = t;
  __syncthreads();
  FIN_FOR(p, k) B.rt[p] = B.idx[p] == k - 1 ? -1 : B.rank[B.idx[p]];
  __syncthreads();
  for (int j = 1; j < levels; ++j) {
    FIN_FOR(p, k) fin_level_int_at(p, B.rt, k, j);
    __syncthreads();
  }
  int32_t *c = B.sorder, *d = b;  // b: the free one of ordA / ordB
  for (int32_t w = 1; w < n; w *= 2) {
    FIN_FOR(i, n) msort_at(i, c, d, n, w, ByParent{B.pi, B.lam});
    __syncthreads();
    int32_t *t = c; c = d; d = t;
  }
  FIN_FOR(s, n) {
    const int32_t j = c[s];
    B.sz[s] = B.sub_hi[j] - B.sub_lo[j] + 1;
  }
  __syncthreads();
  fin_block_scan(B.sz, B.szpre, n, B.tot, warp_sums);
  __syncthreads();
  FIN_FOR(s, n)
    fin_merges_at(s, c, B.pi, B.lam, B.rank, B.sub_lo, B.sub_hi, B.posof, B.rt, B.szpre, k, B.merges, B.hkey,
                  B.sizes);
  FIN_FOR(i, k) fin_reduce_at(i, B.lam, B.lnum, B.lden);
  __syncthreads();
  FIN_FOR(i, n) fin_reduce_at(i, B.hkey, B.hnum, B.hden);
  (void)K;
}
#undef FIN_FOR

size_t fin_levels(int32_t k) {
  int l = 1;
  while ((1 << l) <= k) ++l;
  return (size_t)l;
}

// Enqueue the finalisation for a layout of k >= 2 points; returns launches via
// *launches.  With widen, the gaps are order codes and are first turned into
// wide keys in place.  Up to kFinSmall points one CTA runs every step in one
// launch (the same per-element steps, separated by block barriers).
cudaError_t launch_finalize(const int32_t *ord, uint64_t *gap, const int32_t *perm, int32_t k,
                            FinBufs &B, cudaStream_t st, int64_t *launches, bool widen) {
  if (k <= g_fin_small) {
    k_fin_small<<<1, kFinThreads, 0, st>>>(ord, gap, perm, k, widen ? 1 : 0, B);
    if (launches) *launches += 1;
    return cudaGetLastError();
  }
  const int T = 256;
  const unsigned nb = (unsigned)((k + T - 1) / T);
  const int levels = (int)fin_levels(k);
  const int64_t K = k;
  int64_t L = 0;
  if (widen) {
    k_fin_widen<<<(unsigned)((k - 1 + T - 1) / T), T, 0, st>>>(gap, k - 1);
    ++L;
  }
  k_fin_idx<<<nb, T, 0, st>>>(ord, perm, k, B.idx);
  k_fin_posof<<<nb, T, 0, st>>>(B.idx, k, B.posof);
  cudaMemcpyAsync(B.gt, gap, sizeof(uint64_t) * (k - 1), cudaMemcpyDeviceToDevice, st);
  cudaMemcpyAsync(B.it, B.idx, sizeof(int32_t) * k, cudaMemcpyDeviceToDevice, st);
  L += 2;
  for (int j = 1; j < levels; ++j) {
    k_fin_level<<<nb, T, 0, st>>>(B.gt, B.it, k, j);
    ++L;
  }
  k_fin_lambda<<<nb, T, 0, st>>>(B.gt, B.it, B.idx, k, levels, B.lam, B.pi, B.sub_lo, B.sub_hi);
  ++L;
  // merge order: (lambda, j) over j < k-1
  const int32_t n = k - 1;
  const unsigned nbn = (unsigned)((n + T - 1) / T);
  k_fin_iota<<<nbn, T, 0, st>>>(B.ordA, n);
  ++L;
  int32_t *a = B.ordA, *b = B.ordB;
  for (int64_t w = 1; w < n; w *= 2) {
    k_msort<<<nbn, T, 0, st>>>(a, b, n, (int32_t)w, ByLambda{B.lam});
    std::swap(a, b);
    ++L;
  }
  k_fin_rank<<<nbn, T, 0, st>>>(a, n, B.rank);
  k_fin_rankpos<<<nb, T, 0, st>>>(B.idx, B.rank, k, B.rt);
  L += 2;
  for (int j = 1; j < levels; ++j) {
    k_fin_level_int<<<nb, T, 0, st>>>(B.rt, k, j);
    ++L;
  }
  // sibling order: (pi, lambda, j)
  k_fin_iota<<<nbn, T, 0, st>>>(B.sorder, n);
  ++L;
  int32_t *c = B.sorder, *d = a == B.ordA ? B.ordB : B.ordA;
  for (int64_t w = 1; w < n; w *= 2) {
    k_msort<<<nbn, T, 0, st>>>(c, d, n, (int32_t)w, ByParent{B.pi, B.lam});
    std::swap(c, d);
    ++L;
  }
  k_fin_sizes<<<nbn, T, 0, st>>>(c, B.sub_lo, B.sub_hi, n, B.sz);
  k_scan_excl<<<1, 1024, 0, st>>>(B.sz, B.szpre, n, B.tot);
  k_fin_merges<<<nbn, T, 0, st>>>(c, B.pi, B.lam, B.rank, B.sub_lo, B.sub_hi, B.posof, B.rt,
                                  B.szpre, n, k, B.merges, B.hkey, B.sizes);
  k_fin_reduce<<<nb, T, 0, st>>>(B.lam, k, B.lnum, B.lden);
  k_fin_reduce<<<nbn, T, 0, st>>>(B.hkey, n, B.hnum, B.hden);
  L += 5;
  (void)K;
  if (launches) *launches += L;
  return cudaGetLastError();
}

}  // namespace famsa

extern "C" int famsa_debug_set_fin_small(int on) {
  famsa::g_fin_small = on ? famsa::kFinSmall : 0;
  return FAMSA_OK;
}

namespace famsa {
// similarity = LCS / indel^2 = den / num of a height num / den (distance indel^2 / LCS)
__global__ void k_merge_similarity(const uint64_t *num, const uint32_t *den, int64_t n, double *out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint64_t a = num[i];
  const uint32_t b = den[i];
  out[i] = b == 0 ? 0.0 : (a == 0 ? __longlong_as_double(0x7ff0000000000000LL) : (double)b / (double)a);
}
}  // namespace famsa

extern "C" int famsa_merge_similarity(const uint64_t *h_num, const uint32_t *h_den, int64_t n,
                                      double *similarity, void *cuda_stream) {
  if (n < 0 || (n > 0 && (!h_num || !h_den || !similarity))) return FAMSA_EINVAL;
  if (n == 0) return FAMSA_OK;
  const int T = 256;
  famsa::k_merge_similarity<<<(unsigned)((n + T - 1) / T), T, 0, (cudaStream_t)cuda_stream>>>(
      h_num, h_den, n, similarity);
  return famsa::status_from_cuda(cudaGetLastError());
}
