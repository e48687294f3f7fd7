// Single-linkage guide tree on the device: LCS row blocks streamed into a
// SLINK-equivalent row update, then the canonical pointer representation and
// the merge list.
//
// FAMSA Methods, "Determination of the guide tree": single linkage computed
// incrementally by SLINK (Sibson 1973) from similarity rows, stages I and II
// run together so only O(k) tree state is kept.  Pairs are ordered by the
// exact rational distance indel^2 / LCS (the paper's similarity LCS/indel^2,
// reversed), indel = |A| + |B| - 2 LCS.
//
// Row update (one new point n over the points already inserted).  The state
// is a leaf order of the current single-linkage dendrogram plus the gap
// between neighbours, gap[p] = u(ord[p], ord[p+1]), where u is the minimax
// (single-link) distance; in such an order u(x_p, x_q) = max(gap[p..q-1]).
// With d[p] = dist(ord[p], n), the minimax distance from n to each point is
//     D[q] = min over p of max(d[p], max gap between p and q)
// = min(Lf[q], Rf[q]) with Lf[q] = min(d[q], max(Lf[q-1], gap[q-1])) and
// Rf[q] = min(d[q], max(Rf[q+1], gap[q])): two scans whose steps are clamp
// functions x -> min(hi, max(x, lo)), closed under composition, so they run
// as parallel prefix scans.  Sibson's pointer representation then updates
// elementwise: lambda(j) = min(lambda(j), D(j)) and pi(j) = n iff
// D(j) <= lambda(j) (this is exactly lambda(j) = min_{l>j} u(j,l),
// pi(j) = max{l > j : u(j,l) <= lambda(j)} after n joins).
//
// Re-layout: with x0 the first minimum of D, the new leaf order is
// [positions < x0 sorted by D descending] n [positions >= x0 sorted by D
// ascending], both stable.  Usually D is already non-increasing before x0 and
// non-decreasing after it, so this is a shift; otherwise each side is a few
// sorted runs merged pairwise.  New gaps: min(max(D(x), D(y)), old gap if y
// followed x in the old order).
//
// Points are inserted in length-sorted order (the order the LCS kernels like);
// the final pointer representation is rebuilt in the caller's labels from the
// minimum spanning tree it encodes (edges (j, pi(j)) at height lambda(j)), by
// union-find over edges grouped by equal height.
#include <cooperative_groups.h>

#include <algorithm>
#include <vector>

#include "famsa_internal.cuh"

namespace cg = cooperative_groups;

namespace famsa {

// ----------------------------------------------------------------- keys
// Packed exact distance: (indel^2 << 16) | LCS.  indel^2 < 2^34, LCS <= 65535.
// LCS = 0 gives +inf, encoded (1 << 16) (num 1, den 0); 0 is num 0.
// Compare a < b by cross multiplication (products < 2^50).
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

struct Clamp {  // x -> min(hi, max(x, lo))
  uint64_t lo, hi;
};
__device__ __forceinline__ Clamp identity_clamp() { return Clamp{kKeyZero, kKeyInf}; }
// a then b
__device__ __forceinline__ Clamp compose(const Clamp &a, const Clamp &b) {
  return Clamp{kmax(a.lo, b.lo), kmin(b.hi, kmax(a.hi, b.lo))};
}
__device__ __forceinline__ Clamp shfl_clamp_up(const Clamp &c, int d) {
  return Clamp{__shfl_up_sync(0xffffffffu, c.lo, d), __shfl_up_sync(0xffffffffu, c.hi, d)};
}
__device__ __forceinline__ Clamp shfl_clamp_down(const Clamp &c, int d) {
  return Clamp{__shfl_down_sync(0xffffffffu, c.lo, d), __shfl_down_sync(0xffffffffu, c.hi, d)};
}

// ----------------------------------------------------------------- state
constexpr int kSlinkThreads = 1024;
constexpr int kMaxClusterCtas = 16;
constexpr int kRunsSmem = 2048;   // natural-run merge keeps up to this many run starts per side

struct SlinkState {
  // per position, double-buffered by insertion parity
  int32_t *ord[2];
  int32_t *olen[2];
  uint64_t *gap[2];
  // per position scratch
  uint64_t *D;
  uint64_t *mD[2];
  int32_t *mOrd[2];
  int32_t *mLen[2];
  int32_t *mOld[2];
  // per node (insertion labels)
  uint64_t *lam;
  int32_t *pi;
  // run starts (unsorted, appended) per side
  int32_t *runsA;
  int32_t *runsB;
  // control
  uint64_t *ctl;   // see ctl_* offsets
  const int32_t *slen;  // lengths in insertion (sorted) order
};

// ctl layout (uint64 words)
constexpr int kCtlAggL = 0;                           // 2 words per CTA
constexpr int kCtlAggR = kCtlAggL + 2 * kMaxClusterCtas;
constexpr int kCtlArg = kCtlAggR + 2 * kMaxClusterCtas;  // 2 words per CTA: key, pos
constexpr int kCtlCnt = kCtlArg + 2 * kMaxClusterCtas;   // 6 words: run counts A,B for 3 slots
constexpr int kCtlStats = kCtlCnt + 6;                    // 2 words: merges, rounds
constexpr int kCtlWords = kCtlStats + 4;

struct SlinkArgs {
  SlinkState s;
  const uint16_t *rowbuf;
  int64_t ld;
  int32_t r0, r1;
};

// Block-level exclusive scan of clamps in thread order (forward) or reverse
// thread order (backward).  Returns this thread's exclusive prefix and sets
// *total to the block's full composition.
template <bool kForward>
__device__ Clamp block_scan(Clamp v, Clamp *total, Clamp *sw) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  Clamp inc = v;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    if (kForward) {
      Clamp y = shfl_clamp_up(inc, d);
      if (lane >= d) inc = compose(y, inc);
    } else {
      Clamp y = shfl_clamp_down(inc, d);
      if (lane + d < 32) inc = compose(y, inc);
    }
  }
  Clamp exc;
  if (kForward) {
    exc = shfl_clamp_up(inc, 1);
    if (lane == 0) exc = identity_clamp();
    if (lane == 31) sw[warp] = inc;
  } else {
    exc = shfl_clamp_down(inc, 1);
    if (lane == 31) exc = identity_clamp();
    if (lane == 0) sw[warp] = inc;
  }
  __syncthreads();
  if (warp == 0) {
    Clamp w = lane < nw ? sw[lane] : identity_clamp();
    Clamp winc = w;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      if (kForward) {
        Clamp y = shfl_clamp_up(winc, d);
        if (lane >= d) winc = compose(y, winc);
      } else {
        Clamp y = shfl_clamp_down(winc, d);
        if (lane + d < 32) winc = compose(y, winc);
      }
    }
    Clamp wexc;
    if (kForward) {
      wexc = shfl_clamp_up(winc, 1);
      if (lane == 0) wexc = identity_clamp();
    } else {
      wexc = shfl_clamp_down(winc, 1);
      if (lane == nw - 1 || lane >= nw) wexc = identity_clamp();
    }
    if (lane < nw) sw[32 + lane] = wexc;
    if (kForward ? lane == nw - 1 : lane == 0) sw[64] = winc;
  }
  __syncthreads();
  Clamp res = compose(sw[32 + warp], exc);
  *total = sw[64];
  __syncthreads();
  return res;
}

// position range of this thread's chunk
__device__ __forceinline__ void chunk_of(int32_t m, int32_t tid, int32_t nthreads, int32_t *b,
                                         int32_t *e) {
  int32_t c = (m + nthreads - 1) / nthreads;
  int64_t bb = (int64_t)tid * c;
  *b = (int32_t)(bb < m ? bb : (int64_t)m);
  *e = (int32_t)(bb + c < m ? bb + c : (int64_t)m);
}

// first position in a sorted run list (smem) whose start is <= i: returns run index
__device__ __forceinline__ int32_t run_of(const int32_t *starts, int32_t nruns, int32_t i) {
  int32_t lo = 0, hi = nruns - 1;
  while (lo < hi) {
    int32_t mid = (lo + hi + 1) >> 1;
    if (starts[mid] <= i) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// in-place bitonic sort of n ints in shared memory (n <= cap, cap power of two)
__device__ void smem_sort(int32_t *a, int32_t n, int32_t cap) {
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

// One launch inserts points r0..r1-1 (insertion labels) with the rows of
// LCS values in rowbuf.  A thread-block cluster does every step together;
// cluster barriers separate the phases.
__global__ void __launch_bounds__(kSlinkThreads, 1) k_slink_rows(SlinkArgs a) {
  cg::cluster_group cluster = cg::this_cluster();
  const int32_t ncta = (int32_t)cluster.num_blocks();
  const int32_t cta = (int32_t)cluster.block_rank();
  const int32_t nthreads = ncta * blockDim.x;
  const int32_t tid = cta * blockDim.x + threadIdx.x;
  __shared__ Clamp sw[65];
  __shared__ int32_t sRunsA[kRunsSmem], sRunsB[kRunsSmem];
  __shared__ uint64_t sRed[64];
  __shared__ int32_t sRedPos[32];
  SlinkState &S = a.s;
  uint64_t *ctl = S.ctl;

  for (int32_t n = a.r0; n < a.r1; ++n) {
    const int32_t m = n;
    const int cur = n & 1, nxt = cur ^ 1;
    const int slot = n % 3, slot_next = (n + 1) % 3;
    const int32_t *ord = S.ord[cur];
    const int32_t *olen = S.olen[cur];
    const uint64_t *gap = S.gap[cur];
    const uint16_t *row = a.rowbuf + (int64_t)(n - a.r0) * a.ld;
    const uint32_t ln = (uint32_t)S.slen[n];
    int32_t cb, ce;
    chunk_of(m, tid, nthreads, &cb, &ce);

    // ---- phase A: distances, chunk summaries of both scans
    Clamp sl = identity_clamp(), sr = identity_clamp();
    for (int32_t q = cb; q < ce; ++q) {
      uint64_t d = make_key(row[ord[q]], (uint32_t)olen[q], ln);
      S.D[q] = d;
      Clamp f{q == 0 ? kKeyInf : gap[q - 1], d};
      sl = compose(sl, f);
    }
    for (int32_t q = ce - 1; q >= cb; --q) {
      Clamp f{q == m - 1 ? kKeyInf : gap[q], S.D[q]};
      sr = compose(sr, f);
    }
    Clamp totL, totR;
    Clamp preL = block_scan<true>(sl, &totL, sw);
    Clamp preR = block_scan<false>(sr, &totR, sw);
    if (threadIdx.x == 0) {
      ctl[kCtlAggL + 2 * cta] = totL.lo;
      ctl[kCtlAggL + 2 * cta + 1] = totL.hi;
      ctl[kCtlAggR + 2 * cta] = totR.lo;
      ctl[kCtlAggR + 2 * cta + 1] = totR.hi;
      // run counters rotate over three slots: insertion n counts into slot n % 3,
      // which every CTA has stopped reading two barriers before it is reset here
      if (cta == 0) ctl[kCtlCnt + 2 * slot_next] = 0, ctl[kCtlCnt + 2 * slot_next + 1] = 0;
    }
    cluster.sync();

    // ---- phase B: finish the scans, D, pointer update, first minimum
    {
      Clamp cl = identity_clamp(), cr = identity_clamp();
      for (int32_t c = 0; c < cta; ++c) cl = compose(cl, Clamp{ctl[kCtlAggL + 2 * c], ctl[kCtlAggL + 2 * c + 1]});
      for (int32_t c = ncta - 1; c > cta; --c) cr = compose(cr, Clamp{ctl[kCtlAggR + 2 * c], ctl[kCtlAggR + 2 * c + 1]});
      preL = compose(cl, preL);
      preR = compose(cr, preR);
    }
    uint64_t best = kKeyInf;
    int32_t bestpos = INT32_MAX;
    if (cb < ce) {
      uint64_t x = preL.hi;
      for (int32_t q = cb; q < ce; ++q) {
        uint64_t d = S.D[q];
        x = q == 0 ? d : kmin(d, kmax(x, gap[q - 1]));
        S.D[q] = x;
      }
      x = preR.hi;
      for (int32_t q = ce - 1; q >= cb; --q) {
        // S.D[q] holds Lf[q]; the R scan needs d[q] again
        uint64_t d = make_key(row[ord[q]], (uint32_t)olen[q], ln);
        x = q == m - 1 ? d : kmin(d, kmax(x, gap[q]));
        uint64_t Dq = kmin(S.D[q], x);
        S.D[q] = Dq;
        int32_t node = ord[q];
        uint64_t lam = S.lam[node];
        if (!klt(lam, Dq)) {  // D <= lambda
          S.lam[node] = Dq;
          S.pi[node] = n;
        }
        if (klt(Dq, best) || (!klt(best, Dq) && q < bestpos)) { best = Dq; bestpos = q; }
      }
    }
    // CTA argmin (value, then position)
    {
      const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
      for (int d = 16; d > 0; d >>= 1) {
        uint64_t ob = __shfl_down_sync(0xffffffffu, best, d);
        int32_t op = __shfl_down_sync(0xffffffffu, bestpos, d);
        if (klt(ob, best) || (!klt(best, ob) && op < bestpos)) { best = ob; bestpos = op; }
      }
      if (lane == 0) { sRed[warp] = best; sRedPos[warp] = bestpos; }
      __syncthreads();
      if (warp == 0) {
        best = lane < (int)(blockDim.x >> 5) ? sRed[lane] : kKeyInf;
        bestpos = lane < (int)(blockDim.x >> 5) ? sRedPos[lane] : INT32_MAX;
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) {
          uint64_t ob = __shfl_down_sync(0xffffffffu, best, d);
          int32_t op = __shfl_down_sync(0xffffffffu, bestpos, d);
          if (klt(ob, best) || (!klt(best, ob) && op < bestpos)) { best = ob; bestpos = op; }
        }
        if (lane == 0) {
          ctl[kCtlArg + 2 * cta] = best;
          ctl[kCtlArg + 2 * cta + 1] = (uint64_t)(uint32_t)bestpos;
        }
      }
    }
    if (tid == 0) {
      S.lam[n] = kKeyInf;
      S.pi[n] = n;
    }
    cluster.sync();

    // ---- phase C: speculative shift re-layout, run starts
    int32_t x0;
    {
      uint64_t b = kKeyInf;
      int32_t bp = INT32_MAX;
      for (int32_t c = 0; c < ncta; ++c) {
        uint64_t v = ctl[kCtlArg + 2 * c];
        int32_t p = (int32_t)(uint32_t)ctl[kCtlArg + 2 * c + 1];
        if (klt(v, b) || (!klt(b, v) && p < bp)) { b = v; bp = p; }
      }
      x0 = bp;
    }
    int32_t *nord = S.ord[nxt];
    int32_t *nlen = S.olen[nxt];
    uint64_t *ngap = S.gap[nxt];
    for (int32_t p = cb; p < ce; ++p) {
      const uint64_t Dp = S.D[p];
      const int32_t np = p < x0 ? p : p + 1;
      nord[np] = ord[p];
      nlen[np] = olen[p];
      if (p + 1 < m) {
        const uint64_t Dn = S.D[p + 1];
        if (p + 1 == x0) ngap[p] = Dp;  // last of the left side, then n
        else ngap[np] = kmin(kmax(Dp, Dn), gap[p]);
      }
      if (p == x0) {
        nord[x0] = n;
        nlen[x0] = (int32_t)ln;
        ngap[x0] = Dp;  // n, then old position x0
      }
      if (p >= 1 && p < x0 && klt(S.D[p - 1], Dp)) {
        uint64_t at = atomicAdd((unsigned long long *)&ctl[kCtlCnt + 2 * slot], 1ull);
        S.runsA[at] = p;
      }
      if (p > x0 && klt(Dp, S.D[p - 1])) {
        uint64_t at = atomicAdd((unsigned long long *)&ctl[kCtlCnt + 2 * slot + 1], 1ull);
        S.runsB[at] = p;
      }
    }
    cluster.sync();

    // ---- phase D (only when a side is not monotone): merge the sorted runs
    const int32_t nA = (int32_t)ctl[kCtlCnt + 2 * slot] + 1;      // runs on the left side
    const int32_t nB = (int32_t)ctl[kCtlCnt + 2 * slot + 1] + 1;  // runs on the right side
    if (nA > 1 || nB > 1) {
      const bool natural = nA <= kRunsSmem && nB <= kRunsSmem;
      if (natural) {
        // every CTA sorts the run starts into its own shared memory
        for (int32_t i = threadIdx.x; i < nA; i += blockDim.x) sRunsA[i] = i == 0 ? 0 : S.runsA[i - 1];
        for (int32_t i = threadIdx.x; i < nB; i += blockDim.x) sRunsB[i] = i == 0 ? x0 : S.runsB[i - 1];
        __syncthreads();
        int32_t capA = 1, capB = 1;
        while (capA < nA) capA <<= 1;
        while (capB < nB) capB <<= 1;
        smem_sort(sRunsA, nA, capA);
        smem_sort(sRunsB, nB, capB);
      }
      // initial buffers
      for (int32_t p = cb; p < ce; ++p) {
        S.mD[0][p] = S.D[p];
        S.mOrd[0][p] = ord[p];
        S.mLen[0][p] = olen[p];
        S.mOld[0][p] = p;
      }
      if (tid == 0) {
        ctl[kCtlStats] += 1;
      }
      cluster.sync();
      // pairwise merge rounds over both sides at once
      int src = 0;
      const int32_t sideLenA = x0, sideLenB = m - x0;
      for (int32_t width = 1;; width <<= 1) {
        // run count at this level per side
        int32_t runsA_now = natural ? (nA + width - 1) / width : (sideLenA + width - 1) / width;
        int32_t runsB_now = natural ? (nB + width - 1) / width : (sideLenB + width - 1) / width;
        if (runsA_now <= 1 && runsB_now <= 1) break;
        if (tid == 0) ctl[kCtlStats + 1] += 1;
        const int dst = src ^ 1;
        for (int32_t p = cb; p < ce; ++p) {
          const bool left = p < x0;
          const int32_t sbase = left ? 0 : x0;
          const int32_t slen_side = left ? sideLenA : sideLenB;
          const int32_t i = p - sbase;  // side-relative position
          int32_t rs, re, ps, pe, pairs;
          int32_t run;
          if (natural) {
            const int32_t *starts = left ? sRunsA : sRunsB;
            const int32_t nr = left ? nA : nB;
            int32_t r = run_of(starts, nr, p);
            run = r / width;
            int32_t r_first = run * width;
            rs = starts[r_first] - sbase;
            re = (r_first + width < nr) ? starts[r_first + width] - sbase : slen_side;
            int32_t prt = run ^ 1;
            int32_t pf = prt * width;
            if (pf < nr) {
              ps = starts[pf] - sbase;
              pe = (pf + width < nr) ? starts[pf + width] - sbase : slen_side;
              pairs = 1;
            } else {
              ps = pe = 0;
              pairs = 0;
            }
          } else {
            run = i / width;
            rs = run * width;
            re = min(rs + width, slen_side);
            int32_t prt = run ^ 1;
            ps = prt * width;
            pe = min(ps + width, slen_side);
            pairs = ps < slen_side;
          }
          const uint64_t v = S.mD[src][p];
          int32_t np = p;
          if (pairs) {
            // stable merge: left run first among equals.  Left side sorts by D
            // descending, right side ascending.
            const bool isLeftRun = (run & 1) == 0;
            int32_t lo = ps, hi = pe;
            while (lo < hi) {
              int32_t mid = (lo + hi) >> 1;
              uint64_t w = S.mD[src][sbase + mid];
              bool before;
              if (left) before = isLeftRun ? klt(v, w) : !klt(w, v);   // w > v  |  w >= v
              else before = isLeftRun ? klt(w, v) : !klt(v, w);        // w < v  |  w <= v
              if (before) lo = mid + 1; else hi = mid;
            }
            const int32_t cnt = lo - ps;
            const int32_t mstart = min(rs, ps);
            np = sbase + mstart + (i - rs) + cnt;
          }
          S.mD[dst][np] = v;
          S.mOrd[dst][np] = S.mOrd[src][p];
          S.mLen[dst][np] = S.mLen[src][p];
          S.mOld[dst][np] = S.mOld[src][p];
        }
        cluster.sync();
        src = dst;
      }
      // final order and gaps
      for (int32_t p = cb; p < ce; ++p) {
        const int32_t np = p < x0 ? p : p + 1;
        nord[np] = S.mOrd[src][p];
        nlen[np] = S.mLen[src][p];
        const uint64_t Dp = S.mD[src][p];
        if (p == x0 - 1) ngap[np] = Dp;
        if (p == x0) ngap[x0] = Dp;
        if (p + 1 < m && p + 1 != x0) {
          const uint64_t Dn = S.mD[src][p + 1];
          const int32_t o = S.mOld[src][p], on = S.mOld[src][p + 1];
          uint64_t g = kmax(Dp, Dn);
          if (on == o + 1) g = kmin(g, gap[o]);
          ngap[np] = g;
        }
        if (p == x0) {
          nord[x0] = n;
          nlen[x0] = (int32_t)ln;
        }
      }
      cluster.sync();
    }
  }
}

// ------------------------------------------------------------ finalise
// Comparison merge pass on indices: order by (key[idx], idx).
__global__ void k_merge_idx(const uint64_t *key, const int32_t *in, int32_t *out, int32_t n,
                            int32_t width) {
  int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int64_t run = i / width;
  int64_t start = run * width;
  int64_t pair_start = (run & ~1LL) * width;
  int64_t pstart = (run ^ 1) * width;
  int32_t x = in[i];
  if (pstart >= n) { out[i] = x; return; }
  int64_t pend = pstart + width < n ? pstart + width : (int64_t)n;
  uint64_t kx = key[x];
  int64_t lo = pstart, hi = pend;
  while (lo < hi) {
    int64_t mid = (lo + hi) >> 1;
    int32_t y = in[mid];
    uint64_t ky = key[y];
    bool yfirst = klt(ky, kx) || (!klt(kx, ky) && y < x);
    if (yfirst) lo = mid + 1; else hi = mid;
  }
  out[pair_start + (i - start) + (lo - pstart)] = x;
}

__global__ void k_iota(int32_t *a, int32_t n) {
  int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) a[i] = i;
}

// MST edges in original labels: edge j (insertion label) = (perm[j], perm[pi[j]]), weight lam[j]
__global__ void k_edges(const int32_t *pi, const uint64_t *lam, const int32_t *perm, int32_t k,
                        int32_t *eu, int32_t *ev, uint64_t *ew) {
  int32_t j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= k - 1) return;
  eu[j] = perm[j];
  ev[j] = perm[pi[j]];
  ew[j] = lam[j];
}

__device__ int32_t uf_find(int32_t *parent, int32_t x) {
  while (parent[x] != x) {
    int32_t p = parent[x];
    parent[x] = parent[p];
    x = p;
  }
  return x;
}

// Canonical pointer representation from the MST: edges in ascending weight,
// grouped by equal weight; after a group, every component that merged into a
// component with a larger maximum gets lambda = weight, pi = that maximum.
__global__ void k_canonical(const int32_t *order, const int32_t *eu, const int32_t *ev,
                            const uint64_t *ew, int32_t k, int32_t *parent, int32_t *cmax,
                            int32_t *stamp, int32_t *touched, int32_t *pi_out, uint64_t *lam_out) {
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  for (int32_t i = 0; i < k; ++i) {
    parent[i] = i; cmax[i] = i; stamp[i] = -1;
    pi_out[i] = k - 1; lam_out[i] = kKeyInf;
  }
  pi_out[k - 1] = k - 1;
  int32_t e = 0;
  while (e < k - 1) {
    const uint64_t h = ew[order[e]];
    int32_t g1 = e;
    while (g1 < k - 1 && !klt(h, ew[order[g1]]) && !klt(ew[order[g1]], h)) ++g1;
    int32_t nt = 0;
    for (int32_t t = e; t < g1; ++t) {
      int32_t a = uf_find(parent, eu[order[t]]), b = uf_find(parent, ev[order[t]]);
      if (stamp[a] != e) { stamp[a] = e; touched[nt++] = a; }
      if (stamp[b] != e) { stamp[b] = e; touched[nt++] = b; }
    }
    // remember each old component's maximum before merging (cmax of old roots)
    for (int32_t t = 0; t < nt; ++t) touched[2 * k + t] = cmax[touched[t]];
    for (int32_t t = e; t < g1; ++t) {
      int32_t a = uf_find(parent, eu[order[t]]), b = uf_find(parent, ev[order[t]]);
      if (a == b) continue;
      int32_t mx = max(cmax[a], cmax[b]);
      parent[a] = b;
      cmax[b] = mx;
    }
    for (int32_t t = 0; t < nt; ++t) {
      int32_t r = touched[t];
      int32_t oldmax = touched[2 * k + t];
      int32_t nm = cmax[uf_find(parent, r)];
      if (nm > oldmax) {
        pi_out[oldmax] = nm;
        lam_out[oldmax] = h;
      }
    }
    e = g1;
  }
}

// Merge list: j in (lambda, j) order; union-find of j and pi(j).
__global__ void k_merges(const int32_t *order, const int32_t *pi, const uint64_t *lam, int32_t k,
                         int32_t *parent, int32_t *cid, int32_t *csize, int32_t *merges,
                         uint64_t *hkey, int32_t *sizes) {
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  for (int32_t i = 0; i < k; ++i) { parent[i] = i; cid[i] = i; csize[i] = 1; }
  for (int32_t t = 0; t < k - 1; ++t) {
    int32_t j = order[t];
    int32_t a = uf_find(parent, j), b = uf_find(parent, pi[j]);
    int32_t ia = cid[a], ib = cid[b];
    merges[2 * t] = min(ia, ib);
    merges[2 * t + 1] = max(ia, ib);
    hkey[t] = lam[j];
    parent[a] = b;
    csize[b] += csize[a];
    cid[b] = k + t;
    sizes[t] = csize[b];
  }
}

__device__ uint64_t gcd_u64(uint64_t a, uint64_t b) {
  while (b) { uint64_t t = a % b; a = b; b = t; }
  return a;
}

// packed key -> reduced (num, den)
__global__ void k_reduce_keys(const uint64_t *key, int32_t n, uint64_t *num, uint32_t *den) {
  int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  uint64_t kk = key[i];
  uint64_t nu = kk >> 16;
  uint32_t de = (uint32_t)(kk & 0xffffu);
  if (de == 0) { nu = 1; }
  else if (nu == 0) { de = 1; }
  else {
    uint64_t g = gcd_u64(nu, de);
    nu /= g;
    de = (uint32_t)(de / g);
  }
  if (num) num[i] = nu;
  if (den) den[i] = de;
}

// ------------------------------------------------------------ host driver
static int pick_cluster(int *cl) {
  static int cached = 0;
  if (cached) { *cl = cached; return 0; }
  int want[2] = {16, 8};
  for (int w : want) {
    if (w > 8) {
      if (cudaFuncSetAttribute(k_slink_rows, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) {
        cudaGetLastError();
        continue;
      }
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(w, 1, 1);
    cfg.blockDim = dim3(kSlinkThreads, 1, 1);
    cudaLaunchAttribute attr;
    attr.id = cudaLaunchAttributeClusterDimension;
    attr.val.clusterDim.x = w;
    attr.val.clusterDim.y = 1;
    attr.val.clusterDim.z = 1;
    cfg.attrs = &attr;
    cfg.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, k_slink_rows, &cfg) == cudaSuccess && n >= 1) {
      cached = w;
      *cl = w;
      return 0;
    }
    cudaGetLastError();
  }
  return -1;
}

static int g_force_cluster = 0;

struct Scratch {
  std::vector<void *> ptrs;
  cudaStream_t st;
  cudaError_t err = cudaSuccess;
  template <typename T>
  T *get(size_t n) {
    void *p = nullptr;
    if (err != cudaSuccess) return nullptr;
    err = cudaMallocAsync(&p, std::max<size_t>(n, 1) * sizeof(T), st);
    if (err != cudaSuccess) return nullptr;
    ptrs.push_back(p);
    return static_cast<T *>(p);
  }
  void release() {
    for (void *p : ptrs) cudaFreeAsync(p, st);
    ptrs.clear();
  }
};

int slink_tree(Family *f, int32_t *pi_out, uint64_t *lnum_out, uint32_t *lden_out,
               int32_t *merges_out, uint64_t *hnum_out, uint32_t *hden_out, int32_t *sizes_out,
               bool out_on_device, cudaStream_t st) {
  const int32_t k = f->k;
  for (int i = 0; i < 16; ++i) f->stats[i] = 0;
  cudaError_t err = cudaSuccess;
  int cl = 0;
  if (g_force_cluster) cl = g_force_cluster;
  else if (pick_cluster(&cl) != 0) return FAMSA_ECUDA;

  // streams: LCS on one, the row update on a higher-priority one
  int prio_lo = 0, prio_hi = 0;
  cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi);
  cudaStream_t sA = nullptr, sB = nullptr;
  cudaEvent_t ev_start = nullptr, ev_end = nullptr, lcs_done[2] = {nullptr, nullptr},
              upd_done[2] = {nullptr, nullptr};
  Scratch sc;
  sc.st = st;
  int64_t launches = 0, lcs_launches = 0;
  int rc = FAMSA_OK;
  // timing events: per row block, LCS begin/end on sA and update begin/end on sB
  std::vector<cudaEvent_t> tev;
  auto timing_event = [&](cudaStream_t s) -> cudaError_t {
    cudaEvent_t e;
    cudaError_t r = cudaEventCreate(&e);
    if (r != cudaSuccess) return r;
    tev.push_back(e);
    return cudaEventRecord(e, s);
  };

#define CKE(x)                                       \
  do {                                               \
    cudaError_t e_ = (x);                            \
    if (e_ != cudaSuccess) { err = e_; goto done; }  \
  } while (0)

  CKE(cudaStreamCreateWithPriority(&sA, cudaStreamNonBlocking, prio_lo));
  CKE(cudaStreamCreateWithPriority(&sB, cudaStreamNonBlocking, prio_hi));
  CKE(cudaEventCreateWithFlags(&ev_start, cudaEventDisableTiming));
  CKE(cudaEventCreateWithFlags(&ev_end, cudaEventDisableTiming));
  for (int i = 0; i < 2; ++i) {
    CKE(cudaEventCreateWithFlags(&lcs_done[i], cudaEventDisableTiming));
    CKE(cudaEventCreateWithFlags(&upd_done[i], cudaEventDisableTiming));
  }
  {
    // state
    SlinkState S;
    for (int i = 0; i < 2; ++i) {
      S.ord[i] = sc.get<int32_t>(k + 1);
      S.olen[i] = sc.get<int32_t>(k + 1);
      S.gap[i] = sc.get<uint64_t>(k + 1);
      S.mD[i] = sc.get<uint64_t>(k + 1);
      S.mOrd[i] = sc.get<int32_t>(k + 1);
      S.mLen[i] = sc.get<int32_t>(k + 1);
      S.mOld[i] = sc.get<int32_t>(k + 1);
    }
    S.D = sc.get<uint64_t>(k + 1);
    S.lam = sc.get<uint64_t>(k);
    S.pi = sc.get<int32_t>(k);
    S.runsA = sc.get<int32_t>(k + 1);
    S.runsB = sc.get<int32_t>(k + 1);
    S.ctl = sc.get<uint64_t>(kCtlWords);
    S.slen = f->d_slen;
    // row blocks
    int32_t B = (int32_t)std::min<int64_t>(std::max<int64_t>((int64_t)(1 << 27) / std::max(k, 1), 64), 2048);
    B = std::min(B, std::max(k - 1, 1));
    const int64_t ld = k;
    uint16_t *rowbuf[2];
    rowbuf[0] = sc.get<uint16_t>((size_t)B * ld);
    rowbuf[1] = sc.get<uint16_t>((size_t)B * ld);
    std::vector<int32_t> h_iota(k), h_w(k);
    for (int32_t s = 0; s < k; ++s) { h_iota[s] = s; h_w[s] = (f->h_slen[s] + 63) / 64; }
    int32_t *d_iota = sc.get<int32_t>(k);
    // edges / finalisation buffers
    int32_t *eu = sc.get<int32_t>(k), *ev = sc.get<int32_t>(k);
    uint64_t *ew = sc.get<uint64_t>(k);
    int32_t *ordA = sc.get<int32_t>(k), *ordB = sc.get<int32_t>(k);
    int32_t *ufp = sc.get<int32_t>(k), *ufm = sc.get<int32_t>(k), *ufs = sc.get<int32_t>(k);
    int32_t *touched = sc.get<int32_t>(4 * (size_t)k);
    int32_t *cpi = sc.get<int32_t>(k);
    uint64_t *clam = sc.get<uint64_t>(k);
    int32_t *mrg = sc.get<int32_t>(2 * (size_t)k);
    uint64_t *hkey = sc.get<uint64_t>(k);
    int32_t *msz = sc.get<int32_t>(k);
    uint64_t *lnum_d = sc.get<uint64_t>(k), *hnum_d = sc.get<uint64_t>(k);
    uint32_t *lden_d = sc.get<uint32_t>(k), *hden_d = sc.get<uint32_t>(k);
    if (sc.err != cudaSuccess) { err = sc.err; goto done; }
    CKE(cudaMemcpyAsync(d_iota, h_iota.data(), sizeof(int32_t) * k, cudaMemcpyHostToDevice, st));
    CKE(cudaMemsetAsync(S.ctl, 0, sizeof(uint64_t) * kCtlWords, st));
    {
      // initial state: point 0 alone; lambda(0) = inf, pi(0) = 0
      std::vector<int32_t> z1 = {0};
      std::vector<uint64_t> inf1 = {kKeyInf};
      CKE(cudaMemcpyAsync(S.ord[1], z1.data(), sizeof(int32_t), cudaMemcpyHostToDevice, st));
      CKE(cudaMemcpyAsync(S.olen[1], f->d_slen, sizeof(int32_t), cudaMemcpyDeviceToDevice, st));
      CKE(cudaMemcpyAsync(S.lam, inf1.data(), sizeof(uint64_t), cudaMemcpyHostToDevice, st));
      CKE(cudaMemcpyAsync(S.pi, z1.data(), sizeof(int32_t), cudaMemcpyHostToDevice, st));
      CKE(cudaStreamSynchronize(st));
    }
    CKE(cudaEventRecord(ev_start, st));
    CKE(cudaStreamWaitEvent(sA, ev_start, 0));
    CKE(cudaStreamWaitEvent(sB, ev_start, 0));
    int64_t cells = 0, words = 0, pairs = 0;
    {
      // algorithmic counters: rows s (Peq side) against columns t < s
      int64_t colsum = 0;
      for (int32_t s = 0; s < k; ++s) {
        words += (int64_t)h_w[s] * colsum;
        cells += (int64_t)f->h_slen[s] * colsum;
        colsum += f->h_slen[s];
      }
      pairs = (int64_t)k * (k - 1) / 2;
    }
    int32_t blk = 0;
    for (int32_t r0 = 1; r0 < k; r0 += B, ++blk) {
      const int32_t r1 = std::min(r0 + B, k);
      const int buf = blk & 1;
      if (blk >= 2) CKE(cudaStreamWaitEvent(sA, upd_done[buf], 0));
      LcsBatch b;
      b.peq = f->d_peq;
      b.colres = f->d_colres;
      b.group_off = f->d_group_off;
      b.group_chunks = f->d_group_chunks;
      b.col_perm = f->d_perm;
      b.col_len = f->d_slen;
      b.n_cols = k;
      b.k = k;
      b.row_peq_off = f->d_peq_off + r0;
      b.row_len = f->d_slen + r0;
      b.row_id = d_iota + r0;
      b.row_orig = f->d_perm + r0;
      b.n_rows = r1 - r0;
      b.h_row_w = h_w.data() + r0;
      b.h_row_id = h_iota.data() + r0;
      b.mode = kOutRowbuf;
      b.out = rowbuf[buf];
      b.ld = ld;
      b.row0 = r0;
      b.triangle = true;
      CKE(timing_event(sA));
      CKE(launch_lcs(b, sA, &lcs_launches));
      CKE(timing_event(sA));
      CKE(cudaEventRecord(lcs_done[buf], sA));
      CKE(cudaStreamWaitEvent(sB, lcs_done[buf], 0));
      SlinkArgs args;
      args.s = S;
      args.rowbuf = rowbuf[buf];
      args.ld = ld;
      args.r0 = r0;
      args.r1 = r1;
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3(cl, 1, 1);
      cfg.blockDim = dim3(kSlinkThreads, 1, 1);
      cfg.stream = sB;
      cudaLaunchAttribute attr;
      attr.id = cudaLaunchAttributeClusterDimension;
      attr.val.clusterDim.x = cl;
      attr.val.clusterDim.y = 1;
      attr.val.clusterDim.z = 1;
      cfg.attrs = &attr;
      cfg.numAttrs = 1;
      CKE(timing_event(sB));
      CKE(cudaLaunchKernelEx(&cfg, k_slink_rows, args));
      ++launches;
      CKE(timing_event(sB));
      CKE(cudaEventRecord(upd_done[buf], sB));
    }
    // finalise on sB
    CKE(timing_event(sB));
    const int T = 256;
    unsigned nb = (unsigned)((k + T - 1) / T);
    if (k >= 2) {
      k_edges<<<nb, T, 0, sB>>>(S.pi, S.lam, f->d_perm, k, eu, ev, ew);
      k_iota<<<nb, T, 0, sB>>>(ordA, k - 1);
      launches += 2;
      for (int64_t w = 1; w < k - 1; w *= 2) {
        k_merge_idx<<<nb, T, 0, sB>>>(ew, ordA, ordB, k - 1, (int32_t)w);
        std::swap(ordA, ordB);
        ++launches;
      }
      k_canonical<<<1, 1, 0, sB>>>(ordA, eu, ev, ew, k, ufp, ufm, ufs, touched, cpi, clam);
      k_iota<<<nb, T, 0, sB>>>(ordA, k - 1);
      launches += 2;
      for (int64_t w = 1; w < k - 1; w *= 2) {
        k_merge_idx<<<nb, T, 0, sB>>>(clam, ordA, ordB, k - 1, (int32_t)w);
        std::swap(ordA, ordB);
        ++launches;
      }
      k_merges<<<1, 1, 0, sB>>>(ordA, cpi, clam, k, ufp, ufm, ufs, mrg, hkey, msz);
      k_reduce_keys<<<nb, T, 0, sB>>>(clam, k, lnum_d, lden_d);
      k_reduce_keys<<<nb, T, 0, sB>>>(hkey, k - 1, hnum_d, hden_d);
      launches += 3;
    } else {
      std::vector<int32_t> z = {0};
      std::vector<uint64_t> one = {1};
      std::vector<uint32_t> zero = {0};
      CKE(cudaMemcpyAsync(cpi, z.data(), sizeof(int32_t), cudaMemcpyHostToDevice, sB));
      CKE(cudaMemcpyAsync(lnum_d, one.data(), sizeof(uint64_t), cudaMemcpyHostToDevice, sB));
      CKE(cudaMemcpyAsync(lden_d, zero.data(), sizeof(uint32_t), cudaMemcpyHostToDevice, sB));
      CKE(cudaStreamSynchronize(sB));
    }
    CKE(cudaGetLastError());
    CKE(timing_event(sB));
    // outputs
    cudaMemcpyKind kind = out_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    if (pi_out) CKE(cudaMemcpyAsync(pi_out, cpi, sizeof(int32_t) * k, kind, sB));
    if (lnum_out) CKE(cudaMemcpyAsync(lnum_out, lnum_d, sizeof(uint64_t) * k, kind, sB));
    if (lden_out) CKE(cudaMemcpyAsync(lden_out, lden_d, sizeof(uint32_t) * k, kind, sB));
    if (k >= 2) {
      if (merges_out) CKE(cudaMemcpyAsync(merges_out, mrg, sizeof(int32_t) * 2 * (k - 1), kind, sB));
      if (hnum_out) CKE(cudaMemcpyAsync(hnum_out, hnum_d, sizeof(uint64_t) * (k - 1), kind, sB));
      if (hden_out) CKE(cudaMemcpyAsync(hden_out, hden_d, sizeof(uint32_t) * (k - 1), kind, sB));
      if (sizes_out) CKE(cudaMemcpyAsync(sizes_out, msz, sizeof(int32_t) * (k - 1), kind, sB));
    }
    uint64_t hstats[2] = {0, 0};
    CKE(cudaMemcpyAsync(hstats, S.ctl + kCtlStats, sizeof(uint64_t) * 2, cudaMemcpyDeviceToHost, sB));
    CKE(cudaEventRecord(ev_end, sB));
    CKE(cudaStreamWaitEvent(st, ev_end, 0));
    CKE(cudaEventSynchronize(ev_end));
    {
      // events: 4 per row block (LCS begin/end, update begin/end), then 2 for finalisation
      double lcs_ms = 0, upd_ms = 0, fin_ms = 0;
      const size_t nblk = (tev.size() - 2) / 4;
      for (size_t i = 0; i < nblk; ++i) {
        float a = 0, b = 0;
        cudaEventElapsedTime(&a, tev[4 * i], tev[4 * i + 1]);
        cudaEventElapsedTime(&b, tev[4 * i + 2], tev[4 * i + 3]);
        lcs_ms += a;
        upd_ms += b;
      }
      float c = 0;
      cudaEventElapsedTime(&c, tev[tev.size() - 2], tev[tev.size() - 1]);
      fin_ms = c;
      f->stats[7] = (int64_t)(lcs_ms * 1e6);
      f->stats[8] = (int64_t)(upd_ms * 1e6);
      f->stats[9] = (int64_t)(fin_ms * 1e6);
      f->stats[10] = lcs_launches;
    }
    launches += lcs_launches;
    f->stats[0] = launches;
    f->stats[1] = cells;
    f->stats[2] = words;
    f->stats[3] = pairs;
    f->stats[4] = (int64_t)hstats[0];
    f->stats[5] = (int64_t)hstats[1];
    f->stats[6] = k;
  }
done:
  if (err != cudaSuccess) {
    if (sA) cudaStreamSynchronize(sA);
    if (sB) cudaStreamSynchronize(sB);
    rc = status_from_cuda(err);
  }
  sc.release();
  if (sA) cudaStreamDestroy(sA);
  if (sB) cudaStreamDestroy(sB);
  if (ev_start) cudaEventDestroy(ev_start);
  if (ev_end) cudaEventDestroy(ev_end);
  for (int i = 0; i < 2; ++i) {
    if (lcs_done[i]) cudaEventDestroy(lcs_done[i]);
    if (upd_done[i]) cudaEventDestroy(upd_done[i]);
  }
  for (cudaEvent_t e : tev) cudaEventDestroy(e);
  return rc;
#undef CKE
}

}  // namespace famsa

extern "C" int famsa_debug_set_cluster(int ctas) {
  if (ctas != 0 && ctas != 1 && ctas != 2 && ctas != 4 && ctas != 8 && ctas != 16) return FAMSA_EINVAL;
  famsa::g_force_cluster = ctas;
  return FAMSA_OK;
}
