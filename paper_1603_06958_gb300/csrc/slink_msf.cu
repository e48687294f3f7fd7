// Row update by minimum spanning tree: the default for families whose
// lengths are all <= 32767 (exact order-code keys).
//
// FAMSA Methods, "Determination of the guide tree": the guide tree is single
// linkage over the similarity rows, built while the rows stream, without the
// k x k matrix.  Single linkage is fixed by a minimum spanning tree of the
// complete distance graph -- its merges are the tree's edges taken in
// increasing order (Gower & Ross 1969) -- so the tree can be kept as that
// spanning tree instead of Sibson's pointer representation.
//
// Per row block (rows r0..r1-1, each with its edges to every earlier point):
// the minimum spanning tree of points 0..r1-1 is rebuilt from the previous
// tree's edges plus the block's edges.  An edge that was left out of the
// previous tree is the heaviest on a cycle of earlier edges and stays out,
// so nothing else is needed.  The rebuild is Boruvka's algorithm: in every
// round each component takes its lightest edge to another component; under a
// strict total order on edges (exact distance, then the smaller endpoint,
// then the larger) all of those are tree edges and every round at least
// halves the number of components.  Each round is data-parallel over all
// points and all block edges, so the whole GPU works on it -- unlike one
// SLINK insertion at a time, a dependent chain over the whole state per
// point.
//
// After the last block the tree's k-1 edges are sorted and joined in that
// order by a union-find whose components carry their leaf lists:
// concatenating the two lists at each join gives a dendrogram leaf order in
// which the gap between neighbours is the height at which they first join.
// The parallel finalisation reads that order and turns it into Sibson's
// canonical pointer representation and the merge list.
#include <algorithm>
#include <vector>

#include "slink_msf.cuh"

namespace famsa {

namespace {

__device__ __forceinline__ uint64_t msf_key(uint32_t L, uint32_t la, uint32_t lb) {
  if (L == 0) return kMsfInf;
  const uint32_t indel = la + lb - 2 * L;
  return order_code(indel * indel, L);
}

// (key, ab) lexicographic: the strict total order on edges
__device__ __forceinline__ bool edge_lt(uint64_t ka, uint64_t aa, uint64_t kb, uint64_t ab) {
  return ka < kb || (ka == kb && aa < ab);
}

__device__ __forceinline__ uint64_t pack_ab(int32_t a, int32_t b) {
  return ((uint64_t)(uint32_t)a << 32) | (uint32_t)b;
}

// minimum of (key, other) over a block; other breaks ties (lower first)
template <int NT>
__device__ __forceinline__ void block_min_pair(uint64_t &key, int32_t &oth, uint64_t *sk, int32_t *so) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) {
    const uint64_t k2 = __shfl_down_sync(0xffffffffu, key, d);
    const int32_t o2 = __shfl_down_sync(0xffffffffu, oth, d);
    if (k2 < key || (k2 == key && o2 < oth)) { key = k2; oth = o2; }
  }
  if (lane == 0) { sk[warp] = key; so[warp] = oth; }
  __syncthreads();
  if (warp == 0) {
    key = lane < NT / 32 ? sk[lane] : kMsfNone;
    oth = lane < NT / 32 ? so[lane] : INT32_MAX;
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
      const uint64_t k2 = __shfl_down_sync(0xffffffffu, key, d);
      const int32_t o2 = __shfl_down_sync(0xffffffffu, oth, d);
      if (k2 < key || (k2 == key && o2 < oth)) { key = k2; oth = o2; }
    }
  }
}

// 64-bit minimum over the lanes of a group (a mask from __match_any_sync)
__device__ __forceinline__ uint64_t group_min64(unsigned mask, uint64_t v) {
  const unsigned hi = (unsigned)(v >> 32);
  const unsigned mh = __reduce_min_sync(mask, hi);
  const unsigned lo = hi == mh ? (unsigned)v : 0xffffffffu;
  const unsigned ml = __reduce_min_sync(mask, lo);
  return ((uint64_t)mh << 32) | ml;
}

constexpr int kRowThreads = 256;

// Row minimum: block row q's lightest edge (q, t), t < q, to another
// component.  The first round also turns the 16-bit LCS values into keys.
template <bool kFirst>
__global__ void __launch_bounds__(kRowThreads) k_msf_rowmin(MsfState S, const uint16_t *rowbuf, int64_t ld,
                                                            int32_t r0, int32_t r1) {
  if (S.ctl[kMsfDone]) return;
  __shared__ uint64_t sk[kRowThreads / 32];
  __shared__ int32_t so[kRowThreads / 32];
  const int32_t q = r0 + (int32_t)blockIdx.x;
  const int32_t cq = S.comp[q];
  const int64_t base = (int64_t)(q - r0) * ld;
  uint64_t bk = kMsfNone;
  int32_t bo = INT32_MAX;
  const uint32_t lq = kFirst ? (uint32_t)S.slen[q] : 0;
#pragma unroll 4
  if (threadIdx.x == 0) (void)FAMSA_EXPECT(q < r1 && q <= ld && cq >= 0 && cq < r1);
  for (int32_t t = threadIdx.x; t < q; t += kRowThreads) {
    uint64_t key;
    if (kFirst) {
      key = msf_key(rowbuf[base + t], lq, (uint32_t)S.slen[t]);
      S.keys[base + t] = key;
    }
    if (S.comp[t] != cq) {
      if (!kFirst) key = S.keys[base + t];
      if (key < bk) { bk = key; bo = t; }  // t ascends per thread: the first minimum is kept
    }
  }
  block_min_pair<kRowThreads>(bk, bo, sk, so);
  if (threadIdx.x == 0) {
    S.rkey[q - r0] = bk;
    S.roth[q - r0] = bo;
  }
}

// Column minimum: point t's lightest edge (t, q) to a block row q > t in
// another component.  32 columns per CTA, 8 row slices, coalesced by column.
constexpr int kColX = 32, kColY = 8;
__global__ void __launch_bounds__(kColX * kColY) k_msf_colmin(MsfState S, int64_t ld, int32_t r0, int32_t r1) {
  if (S.ctl[kMsfDone]) return;
  __shared__ uint64_t sk[kColY][kColX];
  __shared__ int32_t so[kColY][kColX];
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int32_t t = (int32_t)blockIdx.x * kColX + tx;
  uint64_t bk = kMsfNone;
  int32_t bo = INT32_MAX;
  if (t < r1 - 1) {
    const int32_t ct = S.comp[t];
    const int32_t qb = max(r0, t + 1);
#pragma unroll 4
    for (int32_t q = qb + ty; q < r1; q += kColY) {
      if (FAMSA_EXPECT(t < ld) && S.comp[q] != ct) {
        const uint64_t key = S.keys[(int64_t)(q - r0) * ld + t];
        if (key < bk) { bk = key; bo = q; }  // q ascends per thread
      }
    }
  }
  sk[ty][tx] = bk;
  so[ty][tx] = bo;
  __syncthreads();
  if (ty == 0 && t < r1) {
    for (int y = 1; y < kColY; ++y) {
      const uint64_t k2 = sk[y][tx];
      const int32_t o2 = so[y][tx];
      if (k2 < bk || (k2 == bk && o2 < bo)) { bk = k2; bo = o2; }
    }
    S.ckey[t] = bk;
    S.coth[t] = bo;
  }
}

// Phases A and B of the per-component minimum.  Threads [0, r1) take the
// points (their lightest candidate edge), threads [r1, r1 + m) the previous
// tree's edges.  Phase A takes the lightest key per component, phase B the
// lightest endpoint pair among the edges with that key.
template <bool kPhaseB>
__global__ void k_msf_cmin(MsfState S, int32_t r0, int32_t r1, int32_t m) {
  if (S.ctl[kMsfDone]) return;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int32_t c = -1;
  uint64_t key = kMsfNone, ab = kMsfNone;
  if (i < r1) {
    const int32_t v = (int32_t)i;
    if (!kPhaseB) {
      key = S.ckey[v];
      ab = key == kMsfNone ? kMsfNone : pack_ab(v, S.coth[v]);
      if (v >= r0) {
        const uint64_t rk = S.rkey[v - r0];
        if (rk != kMsfNone) {
          const uint64_t rab = pack_ab(S.roth[v - r0], v);
          if (edge_lt(rk, rab, key, ab)) { key = rk; ab = rab; }
        }
      }
      S.vkey[v] = key;
      S.vab[v] = ab;
    } else {
      key = S.vkey[v];
      ab = S.vab[v];
    }
    if (key != kMsfNone) c = S.comp[v];
    if (!FAMSA_EXPECT(c < r1)) c = -1;
  }
  // warp-aggregated atomics: lanes of one component reduce first
  const unsigned grp = __match_any_sync(0xffffffffu, c);
  const int leader = __ffs(grp) - 1;
  const int lane = threadIdx.x & 31;
  if (!kPhaseB) {
    const uint64_t g = group_min64(grp, key);
    if (lane == leader && c >= 0 && g < S.bkey[c]) atomicMin((unsigned long long *)&S.bkey[c], g);
  } else {
    const uint64_t want = c >= 0 ? S.bkey[c] : kMsfNone;
    const uint64_t mine = (c >= 0 && key == want) ? ab : kMsfNone;
    const uint64_t g = group_min64(grp, mine);
    if (lane == leader && c >= 0 && g != kMsfNone && g < S.bab[c])
      atomicMin((unsigned long long *)&S.bab[c], g);
  }
  // previous tree edges: both endpoint components
  if (i >= r1 && i < (int64_t)r1 + m) {
    const int32_t e = (int32_t)(i - r1);
    const int32_t a = S.ma[e], b = S.mb[e];
    const bool in = FAMSA_EXPECT(a >= 0 && a < r1 && b >= 0 && b < r1);
    const int32_t ca = in ? S.comp[a] : 0, cb = in ? S.comp[b] : 0;
    if (ca != cb && FAMSA_EXPECT(ca >= 0 && ca < r1 && cb >= 0 && cb < r1)) {
      const uint64_t ek = S.mkey[e];
      if (!kPhaseB) {
        if (ek < S.bkey[ca]) atomicMin((unsigned long long *)&S.bkey[ca], ek);
        if (ek < S.bkey[cb]) atomicMin((unsigned long long *)&S.bkey[cb], ek);
      } else {
        const uint64_t eab = pack_ab(a, b);
        if (ek == S.bkey[ca] && eab < S.bab[ca]) atomicMin((unsigned long long *)&S.bab[ca], eab);
        if (ek == S.bkey[cb] && eab < S.bab[cb]) atomicMin((unsigned long long *)&S.bab[cb], eab);
      }
    }
  }
}

// Each component root hooks onto the component across its lightest edge and
// records that edge (a mutually chosen edge once, by the smaller root, which
// stays a root).
__global__ void k_msf_hook(MsfState S, int32_t r1) {
  if (S.ctl[kMsfDone]) return;
  const int32_t c = (int32_t)(blockIdx.x * blockDim.x + threadIdx.x);
  if (c >= r1 || S.comp[c] != c) return;
  const uint64_t bk = S.bkey[c];
  if (bk == kMsfNone) {
    S.par[c] = c;
    return;
  }
  const uint64_t ab = S.bab[c];
  const int32_t a = (int32_t)(ab >> 32), b = (int32_t)(ab & 0xffffffffu);
  if (!FAMSA_EXPECT(a >= 0 && a < r1 && b >= 0 && b < r1)) {
    S.par[c] = c;
    return;
  }
  const int32_t ca = S.comp[a];
  const int32_t o = ca == c ? S.comp[b] : ca;
  if (!FAMSA_EXPECT(o >= 0 && o < r1 && o != c)) {
    S.par[c] = c;
    return;
  }
  const bool mutual = S.bkey[o] == bk && S.bab[o] == ab;
  S.par[c] = (mutual && c < o) ? c : o;
  if (!mutual || c < o) {
    const int32_t slot = atomicAdd(&S.ctl[kMsfCount], 1);
    if (slot < S.cap) {
      S.nkey[slot] = bk;
      S.na[slot] = a;
      S.nb[slot] = b;
    } else {
      atomicOr(&S.ctl[kMsfErr], 1);
    }
  }
}

// Every point follows the hooks to its new root; the per-component minima are
// cleared for the next round.  The tree is complete at r1 - 1 edges.
__global__ void k_msf_jump(MsfState S, int32_t r1) {
  if (S.ctl[kMsfDone]) return;
  const int32_t v = (int32_t)(blockIdx.x * blockDim.x + threadIdx.x);
  if (v < r1) {
    int32_t x = S.comp[v];
    for (int32_t it = 0; it < r1 && FAMSA_EXPECT(x >= 0 && x < r1) && S.par[x] != x; ++it) x = S.par[x];
    (void)FAMSA_EXPECT(x >= 0 && x < r1 && S.par[x] == x);  // the walk ended at a root
    S.comp[v] = x;
    S.bkey[v] = kMsfNone;
    S.bab[v] = kMsfNone;
  }
  if (v == 0 && S.ctl[kMsfCount] >= r1 - 1) S.ctl[kMsfDone] = 1;
}

__global__ void k_msf_begin(MsfState S, int32_t r1) {
  const int32_t v = (int32_t)(blockIdx.x * blockDim.x + threadIdx.x);
  if (v < r1) {
    S.comp[v] = v;
    S.bkey[v] = kMsfNone;
    S.bab[v] = kMsfNone;
  }
  if (v == 0) {
    S.ctl[kMsfCount] = 0;
    S.ctl[kMsfDone] = 0;
  }
}

// a block that ended with fewer than r1 - 1 edges left the tree unfinished
__global__ void k_msf_end(MsfState S, int32_t r1) {
  if (S.ctl[kMsfCount] != r1 - 1) atomicOr(&S.ctl[kMsfErr], 2);
}

// ---- the leaf order from the finished tree

struct ByEdge {
  const uint64_t *key;
  const int32_t *a, *b;
  __device__ bool operator()(int32_t x, int32_t y) const {
    if (key[x] != key[y]) return key[x] < key[y];
    if (a[x] != a[y]) return a[x] < a[y];
    return b[x] < b[y];
  }
};

__global__ void k_msf_iota(int32_t *o, int32_t n) {
  const int32_t i = (int32_t)(blockIdx.x * blockDim.x + threadIdx.x);
  if (i < n) o[i] = i;
}

__global__ void k_msf_msort(const int32_t *in, int32_t *out, int32_t n, int32_t width, ByEdge cmp) {
  const int32_t i = (int32_t)(blockIdx.x * blockDim.x + threadIdx.x);
  if (i < n) msort_at(i, in, out, n, width, cmp);
}

__device__ __forceinline__ uint64_t gap_code(uint64_t key) { return key == kMsfInf ? KeysNarrow::kInf : key; }

// the edges in sorted order, gathered so that the joins read them in sequence
__global__ void k_msf_gather(int32_t n, const int32_t *order, const uint64_t *mkey, const int32_t *ma,
                             const int32_t *mb, uint64_t *ek, int32_t *ea, int32_t *eb) {
  const int32_t i = (int32_t)(blockIdx.x * blockDim.x + threadIdx.x);
  if (i < n) {
    const int32_t e = order[i];
    if (!FAMSA_EXPECT(e >= 0 && e < n)) return;
    ek[i] = mkey[e];
    ea[i] = ma[e];
    eb[i] = mb[e];
  }
}

// gap p = the height of the join recorded after position p
__global__ void k_msf_gaps(int32_t n, const int32_t *gi, const uint64_t *ek, uint64_t *gap) {
  const int32_t p = (int32_t)(blockIdx.x * blockDim.x + threadIdx.x);
  if (p < n && FAMSA_EXPECT(gi[p] >= 0 && gi[p] < n)) gap[p] = gap_code(ek[gi[p]]);
}

// The joins in increasing order: a union-find (union by size) whose roots
// carry the head and tail of their leaf list.  At a join of x and y the list
// of x is followed by the list of y, and the index of the joining edge is
// recorded after the tail of x (gidx).  The final list (ranked in parallel,
// below) gives the leaf order and, per position, the edge whose height is
// its gap to the next position.
//
// The joins are sequential, so one thread commits them; the finds are not:
// the 32 lanes of warp 0 look up the roots of the next 32 edges' endpoints
// at once (read-only; union by size keeps every path below log2 k), and the
// committing lane only follows the few links that the joins in between
// added.  The other warps stage the next chunk of edges in shared memory.
// Index type I and the arrays' memory (shared memory for small k, global
// otherwise) are the caller's.
constexpr int kKrtThreads = 1024, kKrtChunk = 2048;

template <class I>
__device__ __forceinline__ void krt_run(int32_t k, const int32_t *ea, const int32_t *eb, I *par, I *head,
                                        I *tail, I *nxt, I *size, int32_t *gidx, int32_t *ord, int32_t *gi,
                                        int32_t *err, int32_t *ca, int32_t *cb, int32_t *sx, int32_t *sy) {
  for (int32_t v = threadIdx.x; v < k; v += kKrtThreads) {
    par[v] = (I)v; head[v] = (I)v; tail[v] = (I)v; nxt[v] = (I)v; size[v] = (I)1;
  }
  __syncthreads();
  if (*err) {
    // an unfinished tree: leave an in-bounds placeholder order for the
    // kernels that follow (the call reports the error)
    for (int32_t p = threadIdx.x; p < k; p += kKrtThreads) {
      ord[p] = p;
      if (p + 1 < k) gi[p] = 0;
    }
    return;
  }
  const int lane = threadIdx.x & 31;
  for (int32_t c0 = 0; c0 < k - 1; c0 += kKrtChunk) {
    const int32_t cn = min(kKrtChunk, k - 1 - c0);
    for (int32_t j = threadIdx.x; j < cn; j += kKrtThreads) {
      ca[j] = ea[c0 + j];
      cb[j] = eb[c0 + j];
    }
    __syncthreads();
    if (threadIdx.x < 32) {
      for (int32_t jb = 0; jb < cn; jb += 32) {
        const int32_t j = jb + lane;
        if (j < cn) {
          int32_t x = ca[j], y = cb[j];
          if (x < 0 || x >= k || y < 0 || y >= k) { x = 0; y = 0; }  // out of range: reported as a self join
          for (int it = 0; it < 64 && (int32_t)par[x] != x; ++it) x = par[x];
          for (int it = 0; it < 64 && (int32_t)par[y] != y; ++it) y = par[y];
          sx[lane] = x;
          sy[lane] = y;
        }
        __syncwarp();
        if (lane == 0) {
          const int32_t nb = min(32, cn - jb);
          for (int32_t l = 0; l < nb; ++l) {
            int32_t x = sx[l], y = sy[l];
            // the looked-up roots usually still are roots: read their records
            // and the root test at once, and walk (then re-read) only when a
            // join since the lookup moved one
            I px = par[x], py = par[y];
            I tx = tail[x], hy = head[y], hx = head[x], ty = tail[y];
            I sxz = size[x], syz = size[y];
            if ((int32_t)px != x || (int32_t)py != y) {
              while ((int32_t)par[x] != x) x = par[x];
              while ((int32_t)par[y] != y) y = par[y];
              tx = tail[x]; hy = head[y]; hx = head[x]; ty = tail[y];
              sxz = size[x]; syz = size[y];
            }
            if (x == y) { *err |= 4; break; }  // two points already joined: not a tree
            gidx[tx] = c0 + jb + l;
            nxt[tx] = hy;
            if (sxz < syz) {
              par[x] = (I)y; size[y] = (I)(sxz + syz); head[y] = hx;
            } else {
              par[y] = (I)x; size[x] = (I)(sxz + syz); tail[x] = ty;
            }
          }
        }
        __syncwarp();
      }
    }
    __syncthreads();
  }
  __syncthreads();
  if (*err) {
    for (int32_t p = threadIdx.x; p < k; p += kKrtThreads) {
      ord[p] = p;
      if (p + 1 < k) gi[p] = 0;
    }
    return;
  }
  // The joined list runs from the root's head through nxt to an element that
  // points to itself.  Its order comes from list ranking by pointer jumping
  // (Wyllie): every element's distance to the end, ceil(log2 k) rounds of
  // d(v) += d(J(v)), J(v) = J(J(v)), in the arrays the joins no longer need.
  // (One thread walking the list took 5 ms at k = 20,000, most of it waiting
  // on a global load per element.)
  I *J0 = par, *D0 = size, *J1 = tail, *D1 = head;
  for (int32_t v = threadIdx.x; v < k; v += kKrtThreads) {
    const I nv = nxt[v];
    J0[v] = nv;
    D0[v] = (I)((int32_t)nv == v ? 0 : 1);
  }
  __syncthreads();
  for (int32_t span = 1; span < k; span *= 2) {
    for (int32_t v = threadIdx.x; v < k; v += kKrtThreads) {
      const int32_t j = (int32_t)J0[v];
      J1[v] = J0[j];
      D1[v] = (I)((int32_t)D0[v] + (int32_t)D0[j]);
    }
    __syncthreads();
    I *t = J0; J0 = J1; J1 = t;
    t = D0; D0 = D1; D1 = t;
  }
  for (int32_t v = threadIdx.x; v < k; v += kKrtThreads) {
    const int32_t p = k - 1 - (int32_t)D0[v];
    ord[p] = v;
    if (p + 1 < k) gi[p] = gidx[v];
  }
}

constexpr int32_t kKrtSmemMax = 20480;  // 5 uint16 arrays + the edge chunk in shared memory

__global__ void __launch_bounds__(kKrtThreads) k_msf_krt_smem(int32_t k, const int32_t *ea, const int32_t *eb,
                                                              int32_t *gidx, int32_t *ord, int32_t *gi,
                                                              int32_t *ctl) {
  extern __shared__ int32_t krt_sm[];
  __shared__ int32_t err, sx[32], sy[32];
  if (threadIdx.x == 0) err = ctl[kMsfErr] ? 16 : 0;
  int32_t *ca = krt_sm, *cb = ca + kKrtChunk;
  uint16_t *par = reinterpret_cast<uint16_t *>(cb + kKrtChunk);
  uint16_t *head = par + k, *tail = head + k, *nxt = tail + k, *size = nxt + k;
  krt_run<uint16_t>(k, ea, eb, par, head, tail, nxt, size, gidx, ord, gi, &err, ca, cb, sx, sy);
  if (threadIdx.x == 0 && err) atomicOr(&ctl[kMsfErr], err);
}

__global__ void __launch_bounds__(kKrtThreads) k_msf_krt_global(int32_t k, const int32_t *ea, const int32_t *eb,
                                                                int32_t *w, int32_t *gidx, int32_t *ord,
                                                                int32_t *gi, int32_t *ctl) {
  __shared__ int32_t ca[kKrtChunk], cb[kKrtChunk];
  __shared__ int32_t err, sx[32], sy[32];
  if (threadIdx.x == 0) err = ctl[kMsfErr] ? 16 : 0;
  const int64_t K = k;
  krt_run<int32_t>(k, ea, eb, w, w + K, w + 2 * K, w + 3 * K, w + 4 * K, gidx, ord, gi, &err, ca, cb, sx, sy);
  if (threadIdx.x == 0 && err) atomicOr(&ctl[kMsfErr], err);
}


// ---- edge lists in and out (sharded pair sets)

__global__ void k_msf_no_candidates(MsfState S, int32_t n) {
  const int32_t v = (int32_t)(blockIdx.x * blockDim.x + threadIdx.x);
  if (v < n) S.ckey[v] = kMsfNone;
}

// caller edges (a, b, num / den) -> tree edges with order-code keys; a bad
// endpoint, a self loop or a distance outside the order codes' range sets
// error bit 8
__global__ void k_msf_from_fractions(int32_t m, int32_t k, const int32_t *a, const int32_t *b,
                                     const uint64_t *num, const uint32_t *den, uint64_t *mkey, int32_t *ma,
                                     int32_t *mb, int32_t *ctl) {
  const int32_t e = (int32_t)(blockIdx.x * blockDim.x + threadIdx.x);
  if (e >= m) return;
  int32_t x = a[e], y = b[e];
  const uint64_t p = num[e];
  const uint32_t q = den[e];
  const bool ok = x >= 0 && y >= 0 && x < k && y < k && x != y && (q == 0 || (q <= 32767 && p < (1ull << 32)));
  if (!ok) {
    atomicOr(&ctl[kMsfErr], 8);
    x = 0;
    y = 1 % k;
  }
  ma[e] = min(x, y);
  mb[e] = max(x, y);
  mkey[e] = q == 0 ? kMsfInf : order_code((uint32_t)p, q);
}

// tree edges -> caller labels (through perm, or as they are when perm is
// null), a < b, and the distance as a reduced fraction (+inf = 1 / 0)
__global__ void k_msf_to_fractions(int32_t m, const uint64_t *mkey, const int32_t *ma, const int32_t *mb,
                                   const int32_t *perm, int32_t *a, int32_t *b, uint64_t *num, uint32_t *den) {
  const int32_t e = (int32_t)(blockIdx.x * blockDim.x + threadIdx.x);
  if (e >= m) return;
  int32_t x = ma[e], y = mb[e];
  if (perm) { x = perm[x]; y = perm[y]; }
  a[e] = min(x, y);
  b[e] = max(x, y);
  const uint64_t key = mkey[e];
  if (key == kMsfInf) {
    num[e] = 1;
    den[e] = 0;
  } else {
    uint64_t p;
    uint32_t q;
    code_fraction(key, &p, &q);
    num[e] = p;
    den[e] = q;
  }
}

inline unsigned nblocks(int64_t n, int t) { return (unsigned)std::max<int64_t>((n + t - 1) / t, 1); }

}  // namespace

int msf_rounds(int32_t r1) {
  int r = 1;
  while ((1 << (r - 1)) < r1) ++r;  // ceil(log2 r1) + 1
  return r;
}

cudaError_t launch_msf_block(MsfState &S, const uint16_t *rowbuf, int64_t ld, int32_t r0, int32_t r1,
                             int32_t m, cudaStream_t st, int64_t *launches) {
  const int T = 256;
  int64_t L = 0;
  k_msf_begin<<<nblocks(r1, T), T, 0, st>>>(S, r1);
  ++L;
  const int rounds = msf_rounds(r1);
  for (int r = 0; r < rounds; ++r) {
    if (r == 0) k_msf_rowmin<true><<<(unsigned)(r1 - r0), kRowThreads, 0, st>>>(S, rowbuf, ld, r0, r1);
    else k_msf_rowmin<false><<<(unsigned)(r1 - r0), kRowThreads, 0, st>>>(S, rowbuf, ld, r0, r1);
    k_msf_colmin<<<nblocks(r1, kColX), dim3(kColX, kColY), 0, st>>>(S, ld, r0, r1);
    k_msf_cmin<false><<<nblocks((int64_t)r1 + m, T), T, 0, st>>>(S, r0, r1, m);
    k_msf_cmin<true><<<nblocks((int64_t)r1 + m, T), T, 0, st>>>(S, r0, r1, m);
    k_msf_hook<<<nblocks(r1, T), T, 0, st>>>(S, r1);
    k_msf_jump<<<nblocks(r1, T), T, 0, st>>>(S, r1);
    L += 6;
  }
  k_msf_end<<<1, 1, 0, st>>>(S, r1);
  ++L;
  // the new tree becomes the previous tree of the next block
  std::swap(S.mkey, S.nkey);
  std::swap(S.ma, S.na);
  std::swap(S.mb, S.nb);
  if (launches) *launches += L;
  return cudaGetLastError();
}

cudaError_t launch_msf_edges(MsfState &S, int32_t n, int32_t m, cudaStream_t st, int64_t *launches) {
  const int T = 256;
  int64_t L = 0;
  k_msf_begin<<<nblocks(n, T), T, 0, st>>>(S, n);
  k_msf_no_candidates<<<nblocks(n, T), T, 0, st>>>(S, n);
  L += 2;
  const int rounds = msf_rounds(n);
  for (int r = 0; r < rounds; ++r) {
    k_msf_cmin<false><<<nblocks((int64_t)n + m, T), T, 0, st>>>(S, n, n, m);
    k_msf_cmin<true><<<nblocks((int64_t)n + m, T), T, 0, st>>>(S, n, n, m);
    k_msf_hook<<<nblocks(n, T), T, 0, st>>>(S, n);
    k_msf_jump<<<nblocks(n, T), T, 0, st>>>(S, n);
    L += 4;
  }
  k_msf_end<<<1, 1, 0, st>>>(S, n);
  ++L;
  std::swap(S.mkey, S.nkey);
  std::swap(S.ma, S.na);
  std::swap(S.mb, S.nb);
  if (launches) *launches += L;
  return cudaGetLastError();
}

cudaError_t launch_msf_from_fractions(MsfState &S, int32_t m, int32_t k, const int32_t *a, const int32_t *b,
                                      const uint64_t *num, const uint32_t *den, cudaStream_t st) {
  if (m > 0) k_msf_from_fractions<<<nblocks(m, 256), 256, 0, st>>>(m, k, a, b, num, den, S.mkey, S.ma, S.mb, S.ctl);
  return cudaGetLastError();
}

cudaError_t launch_msf_to_fractions(const MsfState &S, int32_t m, const int32_t *perm, int32_t *a, int32_t *b,
                                    uint64_t *num, uint32_t *den, cudaStream_t st) {
  if (m > 0) k_msf_to_fractions<<<nblocks(m, 256), 256, 0, st>>>(m, S.mkey, S.ma, S.mb, perm, a, b, num, den);
  return cudaGetLastError();
}

cudaError_t launch_msf_leaf_order(const MsfState &S, int32_t k, int32_t *ord, uint64_t *gap, int32_t *idx_a,
                                  int32_t *idx_b, int32_t *work, uint64_t *ek, cudaStream_t st,
                                  int64_t *launches) {
  const int T = 256;
  const int32_t n = k - 1;
  int64_t L = 0;
  k_msf_iota<<<nblocks(n, T), T, 0, st>>>(idx_a, n);
  ++L;
  int32_t *a = idx_a, *b = idx_b;
  for (int64_t w = 1; w < n; w *= 2) {
    k_msf_msort<<<nblocks(n, T), T, 0, st>>>(a, b, n, (int32_t)w, ByEdge{S.mkey, S.ma, S.mb});
    std::swap(a, b);
    ++L;
  }
  // a: sorted edge order; b is free: the sorted endpoints go to b and work
  int32_t *ea = b, *eb = work, *gidx = work + k, *gi = work + 2 * (int64_t)k;
  k_msf_gather<<<nblocks(n, T), T, 0, st>>>(n, a, S.mkey, S.ma, S.mb, ek, ea, eb);
  ++L;
  if (k <= kKrtSmemMax) {
    const size_t smem = 2 * sizeof(int32_t) * kKrtChunk + 5 * sizeof(uint16_t) * (size_t)k;
    // the cap is per kernel, not per launch: set it to the largest size any
    // call needs, so that calls on other streams never lower it under a launch
    const size_t smem_max = 2 * sizeof(int32_t) * kKrtChunk + 5 * sizeof(uint16_t) * (size_t)kKrtSmemMax;
    cudaError_t e = cudaFuncSetAttribute(k_msf_krt_smem, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_max);
    if (e != cudaSuccess) return e;
    k_msf_krt_smem<<<1, kKrtThreads, smem, st>>>(k, ea, eb, gidx, ord, gi, S.ctl);
  } else {
    k_msf_krt_global<<<1, kKrtThreads, 0, st>>>(k, ea, eb, work + 3 * (int64_t)k, gidx, ord, gi, S.ctl);
  }
  k_msf_gaps<<<nblocks(n, T), T, 0, st>>>(n, gi, ek, gap);
  L += 2;
  if (launches) *launches += L;
  return cudaGetLastError();
}

}  // namespace famsa
