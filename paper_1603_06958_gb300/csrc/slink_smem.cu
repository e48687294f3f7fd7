// Row update with the state in the distributed shared memory of one cluster.
//
// CTA c of the cluster owns positions [c*P, (c+1)*P) of the dendrogram leaf
// order (84 bytes of state a position).  Per inserted point n there are two
// cluster barriers:
//   phase B   the clamp scans finish (CTA prefixes through DSMEM), giving D,
//             the pointer update and the monotonicity of both sides of the
//             first minimum x0; the LCS values of the next row are prefetched
//             with cp.async meanwhile;
//   phase C+A the new layout is built from the old one (a shift by one after
//             x0: each CTA reads at most one element of its left neighbour),
//             and the distances and scan summaries of point n+1 are computed
//             on it.
// When a side is not monotone it is a few sorted runs: each element's place
// in the stable merge of its side is found in one pass (its index in its own
// run plus, for every other run, the number of that run's elements that go
// before it: a search over every 16th value of D held locally, then a binary
// search through DSMEM inside a window of at most 15 values), two more
// barriers.  Runs beyond the local capacity fall back to pairwise merges in
// global memory.  When every
// length is at most 32767 a key is the exact order code floor(indel^2 * 2^30 /
// LCS), compared as a plain integer; else it is (indel^2 << 16) | LCS,
// compared by cross multiplication.
#include <mutex>

#include "slink_merge.cuh"

namespace famsa {

constexpr int kSmemThreads = 512;
constexpr size_t kSmemBytesPerPos = 6 * sizeof(uint64_t) + 9 * sizeof(int32_t);
constexpr int kLocalRuns = 16;     // run starts a CTA may hold per side (fast merge)
constexpr int kFastRuns = 16;      // runs per side the fast merge handles
constexpr size_t kStaticSmem = 24 * 1024;  // the kernel's static shared memory, with margin

// Dynamic shared memory: the per-position state, then every 2^shift-th D value
// of the whole order (the samples of the run-merge rank search).
size_t smem_dyn_bytes(int32_t P, int32_t k, int shift) {
  return (((size_t)P * kSmemBytesPerPos + 7) & ~(size_t)7) +
         (size_t)((k + (1 << shift) - 1) >> shift) * sizeof(uint64_t);
}

// The sample stride (16 .. 64) whose samples fit beside the state of P
// positions, or -1 when even the state does not fit.  Finer strides shorten
// the DSMEM searches of a run merge but cost more in gathering the samples
// from every CTA (stride 4 measured slower than 16 at k = 20,000).
int smem_sample_shift(int32_t P, int32_t k) {
  int device = 0, optin = 0;
  cudaGetDevice(&device);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
  for (int s = 4; s <= 6; ++s)
    if (smem_dyn_bytes(P, k, s) + kStaticSmem <= (size_t)optin) return s;
  return -1;
}

struct Slot {
  int32_t cnt_a, cnt_b;                         // local run starts (fast merge)
  int32_t run_a[kLocalRuns], run_b[kLocalRuns];
};
// phase B results of one CTA, pushed into every CTA of the cluster
struct BRes {
  uint64_t arg_key, first_D, last_D;
  int32_t arg_pos, min_asc, max_desc, pad;
};

__device__ __forceinline__ void cp_async4(void *smem_dst, const void *gmem_src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async_commit_wait() {
  asm volatile("cp.async.commit_group;\ncp.async.wait_all;\n" ::: "memory");
}
// the 16-bit LCS of point `node` out of the aligned 32-bit word that holds it
__device__ __forceinline__ uint32_t half_of(int32_t word, int32_t node) {
  return (node & 1) ? ((uint32_t)word >> 16) : ((uint32_t)word & 0xffffu);
}

template <class K>
__global__ void __launch_bounds__(kSmemThreads, 1) k_slink_smem(SmemArgs arg) {
  cg::cluster_group cluster = cg::this_cluster();
  const int32_t ncta = (int32_t)cluster.num_blocks();
  __shared__ SmemArgs sArgs;
  if (threadIdx.x == 0) sArgs = arg.batch ? arg.batch[blockIdx.x / ncta] : arg;
  __syncthreads();
  const SmemArgs &a = sArgs;
  const int32_t cta = (int32_t)cluster.block_rank();
  const int32_t P = a.P;
  const int32_t base = cta * P;
  const int32_t T = blockDim.x;
  const int32_t E = (P + T - 1) / T;
  const int32_t i0 = threadIdx.x * E;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = T >> 5;
  const int32_t tid = cta * T + threadIdx.x;
  const SlinkState &S = a.s;
  uint64_t *ctl = S.ctl;
  constexpr uint64_t INF = K::kInf;

  extern __shared__ __align__(16) uint64_t smem[];
  uint64_t *const gap0 = smem, *const lam0 = smem + 2 * P, *const X0 = smem + 4 * P;
  int32_t *const ibase = reinterpret_cast<int32_t *>(smem + 6 * P);
  int32_t *const ord0 = ibase, *const len0 = ibase + 2 * P, *const pi0 = ibase + 4 * P;
  int32_t *const raw = ibase + 6 * P;   // aligned 32-bit words holding next-row LCS values
  int32_t *const raw2 = ibase + 7 * P;  // next-row LCS values after a run merge
  int32_t *const nold = ibase + 8 * P;  // old position of each new position after a run merge
  // every 2^sshift-th D of the whole order, for the rank searches of a run merge
  uint64_t *const sSmp = reinterpret_cast<uint64_t *>(
      reinterpret_cast<char *>(smem) + (((size_t)P * kSmemBytesPerPos + 7) & ~(size_t)7));
  const int sshift = a.sshift;
#define gapS(b) (gap0 + (b) * P)
#define lamS(b) (lam0 + (b) * P)
#define ordS(b) (ord0 + (b) * P)
#define lenS(b) (len0 + (b) * P)
#define piS(b) (pi0 + (b) * P)
#define XS(b) (X0 + (b) * P)
  __shared__ Clamp sw[130];
  __shared__ Slot slot;
  // every CTA's scan totals and phase B results, written here by the CTA that
  // owns them (DSMEM stores before a cluster barrier) and read locally after it
  __shared__ Clamp sAggL[kMaxClusterCtas], sAggR[kMaxClusterCtas];
  __shared__ BRes sRes[kMaxClusterCtas];
  __shared__ Clamp sPre[2];
  __shared__ int32_t sRunsA[kRunsSmem], sRunsB[kRunsSmem];
  __shared__ uint64_t sRed[32];
  __shared__ int32_t sRedPos[32], sRedA[32], sRedD[32];
  __shared__ int32_t sX0, sViol, sRawN, sFast, sNA, sNB;
  __shared__ uint64_t sGprev;

  const bool timer = tid == 0;
  long long tB = 0, tC = 0, tD = 0, t_last = clock64();
  long long sub[14] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
  long long t_sub = t_last;
#define SUBT(i) if (timer) { long long t_ = clock64(); sub[i] += t_ - t_sub; t_sub = t_; }

  int dsel = 0;  // XS(dsel): distances of the point being inserted, XS(dsel^1): minimax D

  // phase A over the layout in buffer b (m points, distances in dd): block-level
  // exclusive prefixes of both scans, CTA totals to the slot
  Clamp preL, preR;
  auto scan_summaries = [&](int b, int32_t m, uint64_t gprev, const uint64_t *dd) {
    const int32_t mc = max(0, min(m - base, P));
    const int32_t i1 = min(i0 + E, mc);
    Clamp sl = identity_clamp<K>(), sr = identity_clamp<K>();
    for (int32_t i = i0; i < i1; ++i) {
      const int32_t p = base + i;
      const uint64_t g = p == 0 ? INF : (i == 0 ? gprev : gapS(b)[i - 1]);
      sl = compose<K>(sl, Clamp{g, dd[i]});
    }
    for (int32_t i = i1 - 1; i >= i0; --i) {
      const int32_t p = base + i;
      sr = compose<K>(sr, Clamp{p == m - 1 ? INF : gapS(b)[i], dd[i]});
    }
    Clamp totL, totR;
    block_scan2<K>(sl, sr, &preL, &preR, &totL, &totR, sw);
    if (threadIdx.x < ncta) {
      cluster.map_shared_rank(sAggL, (int)threadIdx.x)[cta] = totL;
      cluster.map_shared_rank(sAggR, (int)threadIdx.x)[cta] = totR;
    }
  };

  // ---- load the layout of r0 points into buffer 0, distances to point r0
  {
    const int b0 = a.r0 & 1;
    const uint16_t *row = a.rowbuf;
    const uint32_t ln = (uint32_t)S.slen[a.r0];
    uint64_t *dd = XS(0);
    for (int32_t i = threadIdx.x; i < P; i += T) {
      const int32_t p = base + i;
      if (p < a.r0) {
        const int32_t node = S.ord[b0][p];
        const int32_t l = S.olen[b0][p];
        ordS(0)[i] = node;
        lenS(0)[i] = l;
        lamS(0)[i] = S.lam[b0][p];
        piS(0)[i] = S.pi[b0][p];
        gapS(0)[i] = p + 1 < a.r0 ? S.gap[b0][p] : INF;
        dd[i] = K::make(row[node], (uint32_t)l, ln);
      }
    }
    cluster.sync();
    uint64_t gprev = INF;
    if (base > 0 && base < a.r0) gprev = cluster.map_shared_rank(gapS(0), cta - 1)[P - 1];
    if (threadIdx.x == 0) sGprev = gprev;
    scan_summaries(0, a.r0, gprev, dd);
    if (cta == 0 && threadIdx.x == 0) {
      const int s1 = (a.r0 + 1) % 3;
      ctl[kCtlCnt + 2 * s1] = 0;
      ctl[kCtlCnt + 2 * s1 + 1] = 0;
    }
    cluster.sync();
  }

  int cur = 0;
  for (int32_t n = a.r0; n < a.r1; ++n) {
    const int32_t m = n, m1 = n + 1;
    const int nxt = cur ^ 1;
    const int sl_now = n % 3;
    const int32_t mc = max(0, min(m - base, P));
    const int32_t i1 = min(i0 + E, mc);
    const bool has_next = n + 1 < a.r1;
    const uint16_t *row_next = a.rowbuf + (int64_t)(n + 1 - a.r0) * a.ld;
    int32_t *ord = ordS(cur);
    int32_t *len = lenS(cur);
    uint64_t *gap = gapS(cur);
    uint64_t *lam = lamS(cur);
    int32_t *pi = piS(cur);
    uint64_t *dd = XS(dsel);
    uint64_t *DD = XS(dsel ^ 1);
    const uint64_t gprev = sGprev;

    // ---- phase B: CTA prefixes, D, pointer update, prefetch, first minimum, monotonicity
    if (warp == 0) {
      Clamp aL = identity_clamp<K>(), aR = identity_clamp<K>();
      if (lane < ncta) {
        aL = sAggL[lane];
        aR = sAggR[lane];
      }
      for (int d = 1; d < ncta; d <<= 1) {  // lanes >= ncta hold the identity
        Clamp yf = shfl_clamp_up(aL, d);
        Clamp yb = shfl_clamp_down(aR, d);
        if (lane >= d) aL = compose<K>(yf, aL);
        if (lane + d < 32) aR = compose<K>(yb, aR);
      }
      Clamp exL = shfl_clamp_up(aL, 1);
      Clamp exR = shfl_clamp_down(aR, 1);
      if (lane == 0) exL = identity_clamp<K>();
      if (lane == 31) exR = identity_clamp<K>();
      if (lane == cta) { sPre[0] = exL; sPre[1] = exR; }
    }
    if (has_next) {
      for (int32_t i = i0; i < i1; ++i) cp_async4(&raw[i], row_next + (ord[i] & ~1));
      if (threadIdx.x == 0) cp_async4(&sRawN, row_next + (n & ~1));
    }
    __syncthreads();
    SUBT(0)
    const Clamp fullL = compose<K>(sPre[0], preL), fullR = compose<K>(sPre[1], preR);
    uint64_t best = INF;
    int32_t bestpos = INT32_MAX;
    if (i0 < i1) {
      uint64_t x = fullL.hi;
      for (int32_t i = i0; i < i1; ++i) {
        const int32_t p = base + i;
        const uint64_t g = p == 0 ? INF : (i == 0 ? gprev : gap[i - 1]);
        x = p == 0 ? dd[i] : kmin_t<K>(dd[i], kmax_t<K>(x, g));
        DD[i] = x;
      }
      x = fullR.hi;
      for (int32_t i = i1 - 1; i >= i0; --i) {
        const int32_t p = base + i;
        x = p == m - 1 ? dd[i] : kmin_t<K>(dd[i], kmax_t<K>(x, gap[i]));
        const uint64_t Dv = kmin_t<K>(DD[i], x);
        DD[i] = Dv;
        if (!K::lt(lam[i], Dv)) {  // D <= lambda: the point's pointer moves to n
          lam[i] = Dv;
          pi[i] = n;
        }
        if (K::lt(Dv, best) || (!K::lt(best, Dv) && p < bestpos)) { best = Dv; bestpos = p; }
      }
    }
    __syncthreads();
    SUBT(1)
    int32_t masc = INT32_MAX, mdesc = -1;
    for (int32_t i = max(i0, 1); i < i1; ++i) {
      const uint64_t x = DD[i - 1], y = DD[i];
      if (K::lt(x, y)) masc = min(masc, base + i);
      if (K::lt(y, x)) mdesc = max(mdesc, base + i);
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
      const uint64_t ob = __shfl_down_sync(0xffffffffu, best, d);
      const int32_t op = __shfl_down_sync(0xffffffffu, bestpos, d);
      if (K::lt(ob, best) || (!K::lt(best, ob) && op < bestpos)) { best = ob; bestpos = op; }
      masc = min(masc, __shfl_down_sync(0xffffffffu, masc, d));
      mdesc = max(mdesc, __shfl_down_sync(0xffffffffu, mdesc, d));
    }
    if (lane == 0) { sRed[warp] = best; sRedPos[warp] = bestpos; sRedA[warp] = masc; sRedD[warp] = mdesc; }
    __syncthreads();
    if (warp == 0) {
      best = lane < nw ? sRed[lane] : INF;
      bestpos = lane < nw ? sRedPos[lane] : INT32_MAX;
      masc = lane < nw ? sRedA[lane] : INT32_MAX;
      mdesc = lane < nw ? sRedD[lane] : -1;
      for (int d = red_top(nw); d > 0; d >>= 1) {
        const uint64_t ob = __shfl_down_sync(0xffffffffu, best, d);
        const int32_t op = __shfl_down_sync(0xffffffffu, bestpos, d);
        if (K::lt(ob, best) || (!K::lt(best, ob) && op < bestpos)) { best = ob; bestpos = op; }
        masc = min(masc, __shfl_down_sync(0xffffffffu, masc, d));
        mdesc = max(mdesc, __shfl_down_sync(0xffffffffu, mdesc, d));
      }
      BRes rr;
      rr.arg_key = __shfl_sync(0xffffffffu, best, 0);
      rr.arg_pos = __shfl_sync(0xffffffffu, bestpos, 0);
      rr.min_asc = __shfl_sync(0xffffffffu, masc, 0);
      rr.max_desc = __shfl_sync(0xffffffffu, mdesc, 0);
      rr.first_D = mc > 0 ? DD[0] : INF;
      rr.last_D = mc > 0 ? DD[mc - 1] : INF;
      rr.pad = 0;
      if (lane < ncta) cluster.map_shared_rank(sRes, lane)[cta] = rr;
    }
    SUBT(2)
    cluster.sync();
    SUBT(3)
    if (timer) { long long t = clock64(); tB += t - t_last; t_last = t; }

    // ---- phase C: first minimum and monotonicity of the whole order
    if (warp == 0) {
      uint64_t b = INF, f = INF, l = INF;
      int32_t bp = INT32_MAX, ma = INT32_MAX, md = -1;
      if (lane < ncta) {
        const BRes &o = sRes[lane];
        b = o.arg_key;
        bp = o.arg_pos;
        ma = o.min_asc;
        md = o.max_desc;
        f = o.first_D;
        l = o.last_D;
      }
      // the pair across the boundary between CTA lane-1 and CTA lane
      const uint64_t prevLast = __shfl_up_sync(0xffffffffu, l, 1);
      const int32_t pb = lane * P;
      if (lane >= 1 && lane < ncta && pb < m) {
        if (K::lt(prevLast, f)) ma = min(ma, pb);
        if (K::lt(f, prevLast)) md = max(md, pb);
      }
      for (int d = red_top(ncta); d > 0; d >>= 1) {
        const uint64_t ob = __shfl_down_sync(0xffffffffu, b, d);
        const int32_t op = __shfl_down_sync(0xffffffffu, bp, d);
        if (K::lt(ob, b) || (!K::lt(b, ob) && op < bp)) { b = ob; bp = op; }
        ma = min(ma, __shfl_down_sync(0xffffffffu, ma, d));
        md = max(md, __shfl_down_sync(0xffffffffu, md, d));
      }
      if (lane == 0) {
        sX0 = bp;
        sViol = (ma < bp || md > bp) ? 1 : 0;
      }
    }
    if (has_next) cp_async_commit_wait();
    __syncthreads();
    SUBT(4)
    const int32_t x0 = sX0;
    const bool violation = sViol != 0;
    const uint32_t ln = (uint32_t)S.slen[n];
    const uint32_t ln1 = has_next ? (uint32_t)S.slen[n + 1] : 0;
    const int32_t mc1 = max(0, min(m1 - base, P));
    const int32_t j1 = min(i0 + E, mc1);
    // old-position readers (local, or another CTA through DSMEM)
    auto getD = [&](int32_t q) -> uint64_t {
      return (q >= base && q < base + P) ? DD[q - base] : cluster.map_shared_rank(DD, q / P)[q % P];
    };
    auto getG = [&](int32_t q) -> uint64_t {
      return (q >= base && q < base + P) ? gap[q - base] : cluster.map_shared_rank(gap, q / P)[q % P];
    };

    if (!violation) {
      // the new gap after new position np (np < m)
      auto new_gap = [&](int32_t np) -> uint64_t {
        if (np < x0 - 1) return kmin_t<K>(kmax_t<K>(getD(np), getD(np + 1)), getG(np));
        if (np == x0 - 1) return getD(x0 - 1);
        if (np == x0) return getD(x0);
        return kmin_t<K>(kmax_t<K>(getD(np - 1), getD(np)), getG(np - 1));
      };
      int32_t *nord = ordS(nxt), *nlen = lenS(nxt), *npi = piS(nxt);
      uint64_t *ngap = gapS(nxt), *nlam = lamS(nxt);
      for (int32_t j = i0; j < j1; ++j) {
        const int32_t np = base + j;
        int32_t o_ord, o_len, o_pi;
        uint64_t o_lam;
        uint32_t o_raw = 0;
        if (np == x0) {
          o_ord = n; o_len = (int32_t)ln; o_lam = INF; o_pi = n;
          if (has_next) o_raw = half_of(sRawN, n);
        } else {
          const int32_t src = np < x0 ? np : np - 1;
          if (src >= base) {
            const int32_t s = src - base;
            o_ord = ord[s]; o_len = len[s]; o_lam = lam[s]; o_pi = pi[s];
            if (has_next) o_raw = half_of(raw[s], o_ord);
          } else {  // the last element of the previous CTA
            const int32_t r = cta - 1;
            o_ord = cluster.map_shared_rank(ord, r)[P - 1];
            o_len = cluster.map_shared_rank(len, r)[P - 1];
            o_lam = cluster.map_shared_rank(lam, r)[P - 1];
            o_pi = cluster.map_shared_rank(pi, r)[P - 1];
            if (has_next) o_raw = half_of(cluster.map_shared_rank(raw, r)[P - 1], o_ord);
          }
        }
        nord[j] = o_ord; nlen[j] = o_len; nlam[j] = o_lam; npi[j] = o_pi;
        if (np < m) ngap[j] = new_gap(np);
        if (has_next) dd[j] = K::make(o_raw, (uint32_t)o_len, ln1);
      }
      if (threadIdx.x == 0) sGprev = (base > 0 && base < m1) ? new_gap(base - 1) : INF;
      __syncthreads();
      SUBT(5)
      if (has_next) {
        scan_summaries(nxt, m1, sGprev, dd);
        if (cta == 0 && threadIdx.x == 0) {
          const int s2 = (n + 2) % 3;
          ctl[kCtlCnt + 2 * s2] = 0;
          ctl[kCtlCnt + 2 * s2 + 1] = 0;
        }
      }
      SUBT(6)
      cluster.sync();
      SUBT(7)
      if (timer) { long long t = clock64(); tC += t - t_last; t_last = t; }
    } else {
      if (tid == 0) ctl[kCtlStats] += 1;
      t_sub = timer ? clock64() : 0;
      // ---- run starts of this CTA's positions, sorted, into the slot
      if (threadIdx.x == 0) { slot.cnt_a = 0; slot.cnt_b = 0; }
      __syncthreads();
      {
        const uint64_t dprev = (i0 == 0 && base > 0 && mc > 0) ? cluster.map_shared_rank(DD, cta - 1)[P - 1] : INF;
        for (int32_t i = i0; i < i1; ++i) {
          const int32_t p = base + i;
          const uint64_t Dp = DD[i], Dq = i == 0 ? dprev : DD[i - 1];
          if (p >= 1 && p < x0 && K::lt(Dq, Dp)) {
            const int at = atomicAdd(&slot.cnt_a, 1);
            if (at < kLocalRuns) slot.run_a[at] = p;
          }
          if (p > x0 && K::lt(Dp, Dq)) {
            const int at = atomicAdd(&slot.cnt_b, 1);
            if (at < kLocalRuns) slot.run_b[at] = p;
          }
        }
      }
      __syncthreads();
      if (threadIdx.x == 0) {  // insertion sort of the (short) local lists
        for (int side = 0; side < 2; ++side) {
          int32_t *r = side ? slot.run_b : slot.run_a;
          const int c = min(side ? slot.cnt_b : slot.cnt_a, kLocalRuns);
          for (int x = 1; x < c; ++x) {
            const int32_t v = r[x];
            int y = x - 1;
            while (y >= 0 && r[y] > v) { r[y + 1] = r[y]; --y; }
            r[y + 1] = v;
          }
        }
      }
      cluster.sync();
      SUBT(8)
      // ---- gather the run lists of every CTA
      if (warp == 0) {
        int32_t ca = 0, cb = 0;
        if (lane < ncta) {
          const Slot *o = cluster.map_shared_rank(&slot, lane);
          ca = o->cnt_a;
          cb = o->cnt_b;
        }
        const bool over = __any_sync(0xffffffffu, ca > kLocalRuns || cb > kLocalRuns);
        int32_t pa = ca, pb = cb;  // inclusive prefixes
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
          const int32_t ya = __shfl_up_sync(0xffffffffu, pa, d), yb = __shfl_up_sync(0xffffffffu, pb, d);
          if (lane >= d) { pa += ya; pb += yb; }
        }
        const int32_t ta = __shfl_sync(0xffffffffu, pa, 31), tb = __shfl_sync(0xffffffffu, pb, 31);
        const int32_t nA = x0 > 0 ? 1 + ta : 0, nB = 1 + tb;
        const bool fast = !over && nA <= kFastRuns && nB <= kFastRuns;
        if (fast && lane < ncta) {
          const Slot *o = cluster.map_shared_rank(&slot, lane);
          for (int t = 0; t < ca; ++t) sRunsA[1 + pa - ca + t] = o->run_a[t];
          for (int t = 0; t < cb; ++t) sRunsB[1 + pb - cb + t] = o->run_b[t];
        }
        if (lane == 0) {
          sRunsA[0] = 0;
          sRunsB[0] = x0;
          sFast = fast ? 1 : 0;
          sNA = nA;
          sNB = nB;
        }
      }
      __syncthreads();
      const bool fast = sFast != 0;
      if (fast) {
        if (tid == 0) { ctl[kCtlStats + 6] += 1; ctl[kCtlStats + 7] += sNA + sNB; }
        SUBT(9)
        const int32_t nA = sNA, nB = sNB;
        const int32_t nsmp = (m + (1 << sshift) - 1) >> sshift;
        for (int32_t q = threadIdx.x; q < nsmp; q += T) sSmp[q] = getD(q << sshift);
        __syncthreads();
        SUBT(12)
        // ---- each element's place in the stable merge of its side
        uint64_t *nD = dd;  // D of the element now at each new position (old distances are dead)
        for (int32_t i = i0; i < i1; ++i) {
          const int32_t p = base + i;
          const uint64_t v = DD[i];
          const bool left = p < x0;
          const int32_t *starts = left ? sRunsA : sRunsB;
          const int32_t nr = left ? nA : nB;
          const int32_t side_end = left ? x0 : m;
          const int32_t r = run_of(starts, nr, p);
          int32_t idx = p - starts[r];
          for (int32_t r2 = 0; r2 < nr; ++r2) {
            if (r2 == r) continue;
            const int32_t s0 = starts[r2], e0 = r2 + 1 < nr ? starts[r2 + 1] : side_end;
            // before(w): w precedes v in the merged order (a true prefix of run r2)
            auto before = [&](uint64_t w) -> bool {
              if (left) return r2 < r ? !K::lt(w, v) : K::lt(v, w);
              return r2 < r ? !K::lt(v, w) : K::lt(w, v);
            };
            // samples at positions q * 2^sshift inside [s0, e0)
            const int32_t kStride = 1 << sshift;
            int32_t qa = (s0 + kStride - 1) >> sshift, qb = (e0 - 1) >> sshift;
            int32_t lo = qa, hi = qb + 1;  // first sample index with before() false
            while (lo < hi) {
              const int32_t mid = (lo + hi) >> 1;
              if (before(sSmp[mid])) lo = mid + 1; else hi = mid;
            }
            // the boundary lies in [wlo, whi): after the last true sample, up to the first false one
            const int32_t wlo = lo > qa ? ((lo - 1) << sshift) + 1 : s0;
            const int32_t whi = lo <= qb ? (lo << sshift) : e0;
            // binary search inside the window (fewer than 2^sshift positions)
            // through DSMEM: a few dependent loads measured faster than reading
            // the whole window, or three quarter points a round trip, with
            // independent loads (merges are bound by DSMEM traffic)
            int32_t wa = wlo, wb = whi;
            while (wa < wb) {
              const int32_t mid = (wa + wb) >> 1;
              if (before(getD(mid))) wa = mid + 1; else wb = mid;
            }
            const int32_t cnt = wa - s0;
            idx += cnt;
          }
          const int32_t np = left ? idx : x0 + 1 + idx;
          const int32_t cn = np / P, in = np - cn * P;
          // four stores: (node, pointer) packed into the free gap slot, lambda, D, old position;
          // lengths and next-row LCS values are gathered again from global memory
          cluster.map_shared_rank(gapS(nxt), cn)[in] = ((uint64_t)(uint32_t)pi[i] << 32) | (uint32_t)ord[i];
          cluster.map_shared_rank(lamS(nxt), cn)[in] = lam[i];
          cluster.map_shared_rank(nD, cn)[in] = v;
          cluster.map_shared_rank(nold, cn)[in] = p;
        }
        SUBT(13)
        if (tid == 0) {  // the new point at x0
          const int32_t cx = x0 / P, ix = x0 - cx * P;
          cluster.map_shared_rank(gapS(nxt), cx)[ix] = ((uint64_t)(uint32_t)n << 32) | (uint32_t)n;
          cluster.map_shared_rank(lamS(nxt), cx)[ix] = INF;
          cluster.map_shared_rank(nold, cx)[ix] = -1;
        }
        cluster.sync();
        SUBT(10)
        for (int32_t j = i0; j < j1; ++j) {
          const uint64_t w = gapS(nxt)[j];
          const int32_t o = (int32_t)(uint32_t)w;
          ordS(nxt)[j] = o;
          piS(nxt)[j] = (int32_t)(w >> 32);
          lenS(nxt)[j] = S.slen[o];
          if (has_next) raw2[j] = row_next[o];
        }
        __syncthreads();
        // ---- new gaps: max of the two D values, capped by the old gap if they were neighbours
        auto nDat = [&](int32_t q) -> uint64_t {
          return (q >= base && q < base + P) ? nD[q - base] : cluster.map_shared_rank(nD, q / P)[q % P];
        };
        auto nOldAt = [&](int32_t q) -> int32_t {
          return (q >= base && q < base + P) ? nold[q - base] : cluster.map_shared_rank(nold, q / P)[q % P];
        };
        auto merged_gap = [&](int32_t np) -> uint64_t {
          if (np == x0 - 1) return nDat(x0 - 1);
          if (np == x0) return nDat(x0 + 1);
          uint64_t g = kmax_t<K>(nDat(np), nDat(np + 1));
          const int32_t o = nOldAt(np), on = nOldAt(np + 1);
          if (on == o + 1) g = kmin_t<K>(g, getG(o));
          return g;
        };
        uint64_t *ngap = gapS(nxt);
        for (int32_t j = i0; j < j1; ++j) {
          const int32_t np = base + j;
          if (np < m) ngap[j] = merged_gap(np);
        }
        const uint64_t gnew = (base > 0 && base < m1) ? merged_gap(base - 1) : INF;
        if (threadIdx.x == 0) sGprev = gnew;
        __syncthreads();
        if (has_next) {
          // distances of point n+1 go to the other array: nD is still read by neighbours
          uint64_t *ddn = DD;
          for (int32_t j = i0; j < j1; ++j) ddn[j] = K::make((uint32_t)raw2[j], (uint32_t)lenS(nxt)[j], ln1);
          scan_summaries(nxt, m1, gnew, ddn);
          if (cta == 0 && threadIdx.x == 0) {
            const int s2 = (n + 2) % 3;
            ctl[kCtlCnt + 2 * s2] = 0;
            ctl[kCtlCnt + 2 * s2 + 1] = 0;
          }
        }
        cluster.sync();
        SUBT(11)
        dsel ^= 1;
      } else {
        // ---- fallback: pairwise run merges through global memory
        const uint64_t dprev = (i0 == 0 && base > 0 && mc > 0) ? cluster.map_shared_rank(DD, cta - 1)[P - 1] : INF;
        for (int32_t i = i0; i < i1; ++i) {
          const int32_t p = base + i;
          const uint64_t Dp = DD[i];
          S.mD[0][p] = Dp;
          S.mOrd[0][p] = ord[i];
          S.mLen[0][p] = len[i];
          S.mOld[0][p] = p;
          S.mLam[0][p] = lam[i];
          S.mPi[0][p] = pi[i];
          S.mRaw[0][p] = has_next ? (int32_t)half_of(raw[i], ord[i]) : 0;
          S.mGap[p] = gap[i];
          const uint64_t Dq = i == 0 ? dprev : DD[i - 1];
          if (p >= 1 && p < x0 && K::lt(Dq, Dp)) {
            const uint64_t at = atomicAdd((unsigned long long *)&ctl[kCtlCnt + 2 * sl_now], 1ull);
            S.runsA[at] = p;
          }
          if (p > x0 && K::lt(Dp, Dq)) {
            const uint64_t at = atomicAdd((unsigned long long *)&ctl[kCtlCnt + 2 * sl_now + 1], 1ull);
            S.runsB[at] = p;
          }
        }
        cluster.sync();
        const int32_t nA = (int32_t)ctl[kCtlCnt + 2 * sl_now] + 1;
        const int32_t nB = (int32_t)ctl[kCtlCnt + 2 * sl_now + 1] + 1;
        const bool natural = nA <= kRunsSmem && nB <= kRunsSmem;
        if (natural) {
          for (int32_t i = threadIdx.x; i < nA; i += T) sRunsA[i] = i == 0 ? 0 : S.runsA[i - 1];
          for (int32_t i = threadIdx.x; i < nB; i += T) sRunsB[i] = i == 0 ? x0 : S.runsB[i - 1];
          __syncthreads();
          int32_t capA = 1, capB = 1;
          while (capA < nA) capA <<= 1;
          while (capB < nB) capB <<= 1;
          smem_sort(sRunsA, nA, capA);
          smem_sort(sRunsB, nB, capB);
        }
        const int32_t cb = base + i0, ce = base + i1;
        const int src = merge_rounds<K>(S, cluster, m, x0, natural, sRunsA, nA, sRunsB, nB, cb, ce, tid == 0);
        for (int32_t p = cb; p < ce; ++p) {
          const int32_t np = p < x0 ? p : p + 1;
          const int32_t cn = np / P, in = np - cn * P;
          cluster.map_shared_rank(ordS(nxt), cn)[in] = S.mOrd[src][p];
          cluster.map_shared_rank(lenS(nxt), cn)[in] = S.mLen[src][p];
          cluster.map_shared_rank(lamS(nxt), cn)[in] = S.mLam[src][p];
          cluster.map_shared_rank(piS(nxt), cn)[in] = S.mPi[src][p];
          cluster.map_shared_rank(raw2, cn)[in] = S.mRaw[src][p];
          uint64_t *dgap = cluster.map_shared_rank(gapS(nxt), cn);
          const uint64_t Dp = S.mD[src][p];
          if (p == x0 - 1) dgap[in] = Dp;
          if (p + 1 < m && p + 1 != x0) {
            const uint64_t Dn = S.mD[src][p + 1];
            const int32_t o = S.mOld[src][p], on = S.mOld[src][p + 1];
            uint64_t g = kmax_t<K>(Dp, Dn);
            if (on == o + 1) g = kmin_t<K>(g, S.mGap[o]);
            dgap[in] = g;
          }
          if (p == x0) {
            const int32_t cx = x0 / P, ix = x0 - cx * P;
            cluster.map_shared_rank(ordS(nxt), cx)[ix] = n;
            cluster.map_shared_rank(lenS(nxt), cx)[ix] = (int32_t)ln;
            cluster.map_shared_rank(lamS(nxt), cx)[ix] = INF;
            cluster.map_shared_rank(piS(nxt), cx)[ix] = n;
            cluster.map_shared_rank(raw2, cx)[ix] = has_next ? (int32_t)half_of(sRawN, n) : 0;
            cluster.map_shared_rank(gapS(nxt), cx)[ix] = Dp;
          }
        }
        cluster.sync();
        if (has_next) {
          for (int32_t j = i0; j < j1; ++j) dd[j] = K::make((uint32_t)raw2[j], (uint32_t)lenS(nxt)[j], ln1);
          const uint64_t g = (base > 0 && base < m1) ? cluster.map_shared_rank(gapS(nxt), cta - 1)[P - 1] : INF;
          if (threadIdx.x == 0) sGprev = g;
          scan_summaries(nxt, m1, g, dd);
          if (cta == 0 && threadIdx.x == 0) {
            const int s2 = (n + 2) % 3;
            ctl[kCtlCnt + 2 * s2] = 0;
            ctl[kCtlCnt + 2 * s2 + 1] = 0;
          }
        }
        cluster.sync();
      }
      if (timer) { long long t = clock64(); tD += t - t_last; t_last = t; t_sub = t; }
    }
    cur = nxt;
  }

  // ---- store the layout of r1 points
  {
    const int b1 = a.r1 & 1;
    for (int32_t i = threadIdx.x; i < P; i += T) {
      const int32_t p = base + i;
      if (p < a.r1) {
        S.ord[b1][p] = ordS(cur)[i];
        S.olen[b1][p] = lenS(cur)[i];
        S.lam[b1][p] = lamS(cur)[i];
        S.pi[b1][p] = piS(cur)[i];
        if (p + 1 < a.r1) S.gap[b1][p] = gapS(cur)[i];
      }
    }
  }
  if (timer) {
    for (int i = 0; i < 14; ++i) atomicAdd((unsigned long long *)&ctl[kCtlStats + 8 + i], (unsigned long long)sub[i]);
    atomicAdd((unsigned long long *)&ctl[kCtlStats + 3], (unsigned long long)tB);
    atomicAdd((unsigned long long *)&ctl[kCtlStats + 4], (unsigned long long)tC);
    atomicAdd((unsigned long long *)&ctl[kCtlStats + 5], (unsigned long long)tD);
  }
#undef SUBT
#undef gapS
#undef lamS
#undef ordS
#undef lenS
#undef piS
#undef XS
}

static int g_smem_threads = kSmemThreads;

// Cluster size for the shared-memory kernel, or 0 when the family does not fit.
int smem_cluster_for(int32_t k, int force) {
  int device = 0, optin = 0;
  cudaGetDevice(&device);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
  (void)optin;
  // the smallest cluster that fits, but at least 16 CTAs from 16k points on
  // (per-insertion work then dominates the barrier cost)
  for (int c : {1, 2, 4, 8, 16}) {
    if (force && c != force) continue;
    if (!force && k >= 16384 && c < 16) continue;
    int32_t P = (k + c - 1) / c;
    if (smem_sample_shift(P, P * c) >= 0) return c;
  }
  return 0;
}

// Cluster size for one family on its own (latency): about 512 positions per
// CTA or fewer (measured on the plain recipe: k = 1,000 is fastest on 2 CTAs,
// 3,000 on 8, 6,000 and up on 16), never below the smallest that fits.
// Batches keep the smallest cluster that fits, which costs the fewest
// SM-seconds when many families share the GPU.
int smem_cluster_latency(int32_t k) {
  const int fit = smem_cluster_for(k, 0);
  if (fit == 0) return 0;
  int c = 1;
  while (c < 16 && (int64_t)c * 512 < k) c *= 2;
  c = c > fit ? c : fit;
  // the wider cluster must fit too (it always does when a narrower one fits: P shrinks)
  return smem_cluster_for(k, c) == c ? c : fit;
}

// The kernel's dynamic shared-memory cap and non-portable cluster permission
// are set once, to the device maxima: a per-launch value could be lowered by
// a concurrent caller between its setting and another caller's launch.
template <class K>
static cudaError_t smem_kernel_attributes() {
  static std::once_flag once;
  static cudaError_t result = cudaSuccess;
  std::call_once(once, [] {
    int device = 0, optin = 0;
    cudaFuncAttributes fa;
    cudaError_t e = cudaGetDevice(&device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, k_slink_smem<K>);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_slink_smem<K>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               optin - (int)fa.sharedSizeBytes);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_slink_smem<K>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    result = e;
  });
  return result;
}

template <class K>
static cudaError_t launch_smem_t(const SmemArgs &args, int cl, cudaStream_t st, int32_t n_clusters) {
  const size_t dyn = args.batch ? args.dyn_bytes : smem_dyn_bytes(args.P, args.P * cl, args.sshift);
  cudaError_t e = smem_kernel_attributes<K>();
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(cl * n_clusters), 1, 1);
  cfg.blockDim = dim3(g_smem_threads, 1, 1);
  cfg.dynamicSmemBytes = dyn;
  cfg.stream = st;
  // the stream's priority travels with the launch, so that a captured graph
  // node keeps it (graphs instantiated with node priorities)
  int prio = 0;
  cudaStreamGetPriority(st, &prio);
  cudaLaunchAttribute attr[2];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = cl;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  attr[1].id = cudaLaunchAttributePriority;
  attr[1].val.priority = prio;
  cfg.attrs = attr;
  cfg.numAttrs = 2;
  return cudaLaunchKernelEx(&cfg, k_slink_smem<K>, args);
}

cudaError_t launch_slink_smem(const SlinkState &S, const uint16_t *rowbuf, int64_t ld, int32_t r0,
                              int32_t r1, int cl, int32_t k, bool narrow, cudaStream_t st) {
  SmemArgs args;
  args.s = S;
  args.rowbuf = rowbuf;
  args.ld = ld;
  args.r0 = r0;
  args.r1 = r1;
  args.P = (k + cl - 1) / cl;
  args.sshift = smem_sample_shift(args.P, args.P * cl);
  args.batch = nullptr;
  args.dyn_bytes = 0;
  if (args.sshift < 0) return cudaErrorInvalidValue;
  return narrow ? launch_smem_t<KeysNarrow>(args, cl, st, 1) : launch_smem_t<KeysWide>(args, cl, st, 1);
}

cudaError_t launch_slink_smem_batch(const SmemArgs *d_args, int32_t n_clusters, int cl, size_t dyn_bytes,
                                    bool narrow, cudaStream_t st) {
  if (n_clusters <= 0) return cudaSuccess;
  SmemArgs args = {};
  args.dyn_bytes = dyn_bytes;  // the largest need of the launch's families
  args.batch = d_args;
  return narrow ? launch_smem_t<KeysNarrow>(args, cl, st, n_clusters)
                : launch_smem_t<KeysWide>(args, cl, st, n_clusters);
}

// narrow keys (num << 32 | den) -> wide keys (num << 16 | den), in place
__global__ void k_widen_keys(uint64_t *key, int32_t n) {
  int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) key[i] = KeysNarrow::wide(key[i]);
}

cudaError_t widen_keys(uint64_t *key, int32_t n, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  k_widen_keys<<<(n + 255) / 256, 256, 0, st>>>(key, n);
  return cudaGetLastError();
}

}  // namespace famsa

extern "C" int famsa_debug_set_update_threads(int threads) {
  if (threads != 0 && threads != 128 && threads != 256 && threads != 512) return FAMSA_EINVAL;
  famsa::g_smem_threads = threads ? threads : famsa::kSmemThreads;
  return FAMSA_OK;
}
