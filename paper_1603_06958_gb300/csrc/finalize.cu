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

__global__ void k_fin_idx(const int32_t *ord, const int32_t *perm, int32_t k, int32_t *idx) {
  int32_t p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < k) idx[p] = perm[ord[p]];
}

// level j of the range-max tables: T[j][p] = max over [p, p + 2^j)
__global__ void k_fin_level(uint64_t *gt, int32_t *it, int32_t k, int32_t j) {
  int32_t p = blockIdx.x * blockDim.x + threadIdx.x;
  const int32_t h = 1 << (j - 1);
  const int64_t K = k;
  if (p + 2 * h <= k - 1) gt[j * K + p] = kmax(gt[(j - 1) * K + p], gt[(j - 1) * K + p + h]);
  if (p + 2 * h <= k) it[j * K + p] = max(it[(j - 1) * K + p], it[(j - 1) * K + p + h]);
}

__global__ void k_fin_level_int(int32_t *rt, int32_t k, int32_t j) {
  int32_t p = blockIdx.x * blockDim.x + threadIdx.x;
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

// lambda, pi and the pointer-subtree interval of each point
__global__ void k_fin_lambda(const uint64_t *gt, const int32_t *it, const int32_t *idx, int32_t k,
                             int levels, uint64_t *lam, int32_t *pi, int32_t *sub_lo,
                             int32_t *sub_hi) {
  int32_t p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= k) return;
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

// bottom-up merge pass on an index array under a strict total order
template <class Cmp>
__global__ void k_msort(const int32_t *in, int32_t *out, int32_t n, int32_t width, Cmp cmp) {
  int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
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

__global__ void k_fin_iota(int32_t *a, int32_t n) {
  int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) a[i] = i;
}

__global__ void k_fin_rank(const int32_t *order, int32_t n, int32_t *rank) {
  int32_t t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) rank[order[t]] = t;
}

__global__ void k_fin_rankpos(const int32_t *idx, const int32_t *rank, int32_t k, int32_t *rt0) {
  int32_t p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < k) rt0[p] = idx[p] == k - 1 ? -1 : rank[idx[p]];
}

__global__ void k_fin_sizes(const int32_t *sorder, const int32_t *sub_lo, const int32_t *sub_hi,
                            int32_t n, int64_t *sz) {
  int32_t s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s < n) {
    int32_t j = sorder[s];
    sz[s] = sub_hi[j] - sub_lo[j] + 1;
  }
}

__global__ void k_fin_merges(const int32_t *sorder, const int32_t *pi, const uint64_t *lam,
                             const int32_t *rank, const int32_t *sub_lo, const int32_t *sub_hi,
                             const int32_t *posof, const int32_t *rt, const int64_t *szpre,
                             int32_t n, int32_t k, int32_t *merges, uint64_t *hkey,
                             int32_t *sizes) {
  int32_t s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n) return;
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

__global__ void k_fin_posof(const int32_t *idx, int32_t k, int32_t *posof) {
  int32_t p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < k) posof[idx[p]] = p;
}

__device__ uint64_t gcd_u64(uint64_t a, uint64_t b) {
  while (b) { uint64_t t = a % b; a = b; b = t; }
  return a;
}

// packed key -> reduced (num, den)
__global__ void k_fin_reduce(const uint64_t *key, int32_t n, uint64_t *num, uint32_t *den) {
  int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
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

size_t fin_levels(int32_t k) {
  int l = 1;
  while ((1 << l) <= k) ++l;
  return (size_t)l;
}

// Enqueue the finalisation for a layout of k >= 2 points; returns launches via *launches.
cudaError_t launch_finalize(const int32_t *ord, const uint64_t *gap, const int32_t *perm, int32_t k,
                            FinBufs &B, cudaStream_t st, int64_t *launches) {
  const int T = 256;
  const unsigned nb = (unsigned)((k + T - 1) / T);
  const int levels = (int)fin_levels(k);
  const int64_t K = k;
  int64_t L = 0;
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
