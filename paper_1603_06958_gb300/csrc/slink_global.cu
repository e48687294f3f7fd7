// Row update with the state in global memory (any family size).
//
// One launch inserts points r0..r1-1 (insertion labels) using the LCS rows in
// rowbuf.  A thread-block cluster runs every step; cluster barriers separate
// the phases: distances + scan summaries | scans, D, pointer update, first
// minimum | re-layout | run merges (when a side is not monotone).
#include <mutex>

#include "slink_merge.cuh"

namespace famsa {


struct GlobalArgs {
  SlinkState s;
  const uint16_t *rowbuf;
  int64_t ld;
  int32_t r0, r1;
};

// Positions are dealt out as rows of 32 consecutive positions, a contiguous
// run of rows per warp: every load and store of a row is one coalesced
// warp access, and the clamp scans run across the 32 lanes of a row (warp
// shuffles) with the warp's running prefix carried from row to row.
struct GBest {
  uint64_t key;
  int32_t pos, pad;
};

// Each warp stages tiles of 32 * kE consecutive positions in shared memory
// with coalesced loads; each lane then runs the clamp steps over kE
// consecutive positions of the tile, and one warp scan over the 32 lane
// totals joins them.  Shared arrays are padded one slot per lane block so
// that the lanes' strided accesses do not collide in one bank.
template <class K, int kThreads, int kE>
__global__ void __launch_bounds__(kThreads, 1) k_slink_global(GlobalArgs a) {
  cg::cluster_group cluster = cg::this_cluster();
  constexpr int kWarps = kThreads / 32;
  constexpr int32_t kTile = 32 * kE;
  constexpr int32_t kNP = 32 * (kE + 1);  // padded slots of one tile array
  extern __shared__ __align__(16) uint64_t gsm[];
  const int32_t ncta = (int32_t)cluster.num_blocks();
  const int32_t cta = (int32_t)cluster.block_rank();
  const int32_t nthreads = ncta * blockDim.x;
  const int32_t tid = cta * blockDim.x + threadIdx.x;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int32_t gw = cta * kWarps + warp, nwarps = ncta * kWarps;
  // this warp's tile arrays: sD, sX, sL, sG (uint64), sI0, sI1 (int32)
  uint64_t *const sD = gsm + (size_t)warp * (4 * kNP + 1 + kNP);
  uint64_t *const sX = sD + kNP;
  uint64_t *const sL = sX + kNP;
  uint64_t *const sG = sL + kNP;  // kNP + 1 slots
  int32_t *const sI0 = reinterpret_cast<int32_t *>(sG + kNP + 1);
  int32_t *const sI1 = sI0 + kNP;
  auto sidx = [](int32_t k) { return k + k / kE; };
  auto gidx = [](int32_t k) { return k + k / kE; };
  __shared__ Clamp sWL[kWarps], sWR[kWarps];                 // warp totals, then exclusive prefixes
  __shared__ Clamp sAggL[kMaxClusterCtas], sAggR[kMaxClusterCtas];  // every CTA's totals (pushed)
  __shared__ Clamp sCtaPre[2];
  __shared__ GBest sBest[kMaxClusterCtas];                  // every CTA's first minimum (pushed)
  __shared__ uint64_t sWBest[kWarps];
  __shared__ int32_t sWBestPos[kWarps];
  __shared__ int32_t sRunsA[kRunsSmem], sRunsB[kRunsSmem];
  const SlinkState &S = a.s;
  uint64_t *ctl = S.ctl;
  constexpr uint64_t INF = K::kInf;

  // cycles of one thread per phase (A distances + summaries, B scans + pointer
  // update, C re-layout, D run merges), for the counters of famsa_last_stats
  const bool timer = tid == 0;
  long long tA = 0, tB = 0, tC = 0, tD = 0, t_last = clock64();
  long long sub[12] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
  long long t_sub = t_last;
#define GSUB(i) if (timer) { const long long t_ = clock64(); sub[i] += t_ - t_sub; t_sub = t_; }
  for (int32_t n = a.r0; n < a.r1; ++n) {
    const int32_t m = n;
    const int cur = m & 1, nxt = cur ^ 1;
    const int slot = n % 3, slot_next = (n + 1) % 3;
    const int32_t *ord = S.ord[cur];
    const int32_t *olen = S.olen[cur];
    const uint64_t *gap = S.gap[cur];
    uint64_t *lam = S.lam[cur];
    int32_t *pi = S.pi[cur];
    uint64_t *dd = S.mD[1];  // distances to n; free until a run merge, which starts after phase B
    const uint16_t *row = a.rowbuf + (int64_t)(n - a.r0) * a.ld;
    const uint32_t ln = (uint32_t)S.slen[n];
    const int32_t nrows = (m + 31) >> 5;
    const int32_t rpw = (nrows + nwarps - 1) / nwarps;
    const int32_t row_b = min(gw * rpw, nrows), row_e = min(row_b + rpw, nrows);

    // ---- phase A: distances, warp totals of both scans (L in position order, R reversed)
    const int32_t wpos_b = row_b << 5, wpos_e = min(row_e << 5, m);
    {
      Clamp wL = identity_clamp<K>(), wR = identity_clamp<K>();
      for (int32_t tb = wpos_b; tb < wpos_e; tb += kTile) {
        const int32_t te = min(tb + kTile, wpos_e);
#pragma unroll
        for (int j = 0; j < kE; ++j) {
          const int32_t k = 32 * j + lane, p = tb + k;
          if (p < te) {
            sI0[sidx(k)] = ord[p];
            sI1[sidx(k)] = olen[p];
          }
        }
#pragma unroll
        for (int j = 0; j <= kE; ++j) {
          const int32_t k = 32 * j + lane;
          if (k <= kTile) {
            const int32_t q = tb - 1 + k;  // the gap between positions q and q+1
            sG[gidx(k)] = (q < 0 || q >= m - 1) ? INF : gap[q];
          }
        }
        __syncwarp();
        Clamp tL = identity_clamp<K>(), tR = identity_clamp<K>();
        {
          uint16_t rv[kE];
#pragma unroll
          for (int i = 0; i < kE; ++i) {
            const int32_t k = lane * kE + i;
            if (tb + k < te) rv[i] = row[sI0[sidx(k)]];
          }
#pragma unroll
          for (int i = 0; i < kE; ++i) {
            const int32_t k = lane * kE + i;
            if (tb + k < te) {
              const uint64_t d = K::make(rv[i], (uint32_t)sI1[sidx(k)], ln);
              sD[sidx(k)] = d;
              tL = compose<K>(tL, Clamp{sG[gidx(k)], d});
              tR = compose<K>(Clamp{sG[gidx(k + 1)], d}, tR);
            }
          }
        }
        __syncwarp();
#pragma unroll
        for (int j = 0; j < kE; ++j) {
          const int32_t k = 32 * j + lane, p = tb + k;
          if (p < te) dd[p] = sD[sidx(k)];
        }
#pragma unroll
        for (int s = 1; s < 32; s <<= 1) {
          const Clamp yL = shfl_clamp_down(tL, s), yR = shfl_clamp_down(tR, s);
          if (lane + s < 32) {
            tL = compose<K>(tL, yL);
            tR = compose<K>(yR, tR);
          }
        }
        wL = compose<K>(wL, shfl_clamp_idx(tL, 0));
        wR = compose<K>(shfl_clamp_idx(tR, 0), wR);
        __syncwarp();
      }
      GSUB(0)
      if (lane == 0) {
        sWL[warp] = wL;
        sWR[warp] = wR;
      }
      __syncthreads();
      GSUB(1)
      if (warp == 0) {
        // exclusive prefixes of the warps (L from the left, R from the right) and CTA totals
        Clamp vL = lane < kWarps ? sWL[lane] : identity_clamp<K>();
        Clamp vR = lane < kWarps ? sWR[lane] : identity_clamp<K>();
        Clamp iL = vL, iR = vR;
#pragma unroll
        for (int s = 1; s < 32; s <<= 1) {
          const Clamp yL = shfl_clamp_up(iL, s), yR = shfl_clamp_down(iR, s);
          if (lane >= s) iL = compose<K>(yL, iL);
          if (lane + s < 32) iR = compose<K>(yR, iR);
        }
        Clamp eL = shfl_clamp_up(iL, 1), eR = shfl_clamp_down(iR, 1);
        if (lane == 0) eL = identity_clamp<K>();
        if (lane == 31) eR = identity_clamp<K>();
        if (lane < kWarps) {
          sWL[lane] = eL;
          sWR[lane] = eR;
        }
        const Clamp totL = shfl_clamp_idx(iL, 31), totR = shfl_clamp_idx(iR, 0);
        if (lane < ncta) {
          cluster.map_shared_rank(sAggL, lane)[cta] = totL;
          cluster.map_shared_rank(sAggR, lane)[cta] = totR;
        }
        // run counters rotate over three slots; slot (n+1)%3 was last read two
        // barriers ago by every CTA
        if (cta == 0 && lane == 0) ctl[kCtlCnt + 2 * slot_next] = 0, ctl[kCtlCnt + 2 * slot_next + 1] = 0;
      }
    }
    GSUB(2)
    cluster.sync();
    if (timer) { const long long t_ = clock64(); tA += t_ - t_last; t_last = t_; }
    GSUB(3)

    // ---- phase B: finish the scans, D, pointer update, first minimum
    if (threadIdx.x == 0) {
      Clamp cl = identity_clamp<K>(), cr = identity_clamp<K>();
      for (int32_t c = 0; c < cta; ++c) cl = compose<K>(cl, sAggL[c]);
      for (int32_t c = ncta - 1; c > cta; --c) cr = compose<K>(cr, sAggR[c]);
      sCtaPre[0] = cl;
      sCtaPre[1] = cr;
    }
    __syncthreads();
    GSUB(4)
    uint64_t best = INF;
    int32_t bestpos = INT32_MAX;
    {
      // forward: Lf of every position, tile by tile
      Clamp run = compose<K>(sCtaPre[0], sWL[warp]);
      for (int32_t tb = wpos_b; tb < wpos_e; tb += kTile) {
        const int32_t te = min(tb + kTile, wpos_e);
#pragma unroll
        for (int j = 0; j < kE; ++j) {
          const int32_t k = 32 * j + lane, p = tb + k;
          if (p < te) sD[sidx(k)] = dd[p];
        }
#pragma unroll
        for (int j = 0; j <= kE; ++j) {
          const int32_t k = 32 * j + lane;
          if (k <= kTile) {
            const int32_t q = tb - 1 + k;
            sG[gidx(k)] = (q < 0 || q >= m - 1) ? INF : gap[q];
          }
        }
        __syncwarp();
        Clamp t = identity_clamp<K>();
#pragma unroll
        for (int i = 0; i < kE; ++i) {
          const int32_t k = lane * kE + i;
          if (tb + k < te) t = compose<K>(t, Clamp{sG[gidx(k)], sD[sidx(k)]});
        }
        Clamp inc = t;
#pragma unroll
        for (int s = 1; s < 32; s <<= 1) {
          const Clamp y = shfl_clamp_up(inc, s);
          if (lane >= s) inc = compose<K>(y, inc);
        }
        Clamp ex = shfl_clamp_up(inc, 1);
        if (lane == 0) ex = identity_clamp<K>();
        uint64_t x = compose<K>(run, ex).hi;
#pragma unroll
        for (int i = 0; i < kE; ++i) {
          const int32_t k = lane * kE + i;
          if (tb + k < te) {
            x = kmin_t<K>(sD[sidx(k)], kmax_t<K>(x, sG[gidx(k)]));
            sX[sidx(k)] = x;
          }
        }
        run = compose<K>(run, shfl_clamp_idx(inc, 31));
        __syncwarp();
#pragma unroll
        for (int j = 0; j < kE; ++j) {
          const int32_t k = 32 * j + lane, p = tb + k;
          if (p < te) S.D[p] = sX[sidx(k)];  // Lf
        }
        __syncwarp();
      }
      // backward: Rf, D, the pointer update and the first minimum, tiles from the right
      GSUB(5)
      run = compose<K>(sCtaPre[1], sWR[warp]);
      const int32_t ntiles = (wpos_e - wpos_b + kTile - 1) / kTile;
      for (int32_t ti = ntiles - 1; ti >= 0; --ti) {
        const int32_t tb = wpos_b + ti * kTile;
        const int32_t te = min(tb + kTile, wpos_e);
#pragma unroll
        for (int j = 0; j < kE; ++j) {
          const int32_t k = 32 * j + lane, p = tb + k;
          if (p < te) {
            sD[sidx(k)] = dd[p];
            sX[sidx(k)] = S.D[p];
            sL[sidx(k)] = lam[p];
            sI0[sidx(k)] = pi[p];
          }
        }
#pragma unroll
        for (int j = 0; j <= kE; ++j) {
          const int32_t k = 32 * j + lane;
          if (k <= kTile) {
            const int32_t q = tb - 1 + k;
            sG[gidx(k)] = (q < 0 || q >= m - 1) ? INF : gap[q];
          }
        }
        __syncwarp();
        Clamp t = identity_clamp<K>();
#pragma unroll
        for (int i = kE - 1; i >= 0; --i) {
          const int32_t k = lane * kE + i;
          if (tb + k < te) t = compose<K>(t, Clamp{sG[gidx(k + 1)], sD[sidx(k)]});
        }
        Clamp inc = t;
#pragma unroll
        for (int s = 1; s < 32; s <<= 1) {
          const Clamp y = shfl_clamp_down(inc, s);
          if (lane + s < 32) inc = compose<K>(y, inc);
        }
        Clamp ex = shfl_clamp_down(inc, 1);
        if (lane == 31) ex = identity_clamp<K>();
        uint64_t x = compose<K>(run, ex).hi;
#pragma unroll
        for (int i = kE - 1; i >= 0; --i) {
          const int32_t k = lane * kE + i;
          const int32_t p = tb + k;
          if (p < te) {
            x = kmin_t<K>(sD[sidx(k)], kmax_t<K>(x, sG[gidx(k + 1)]));
            const uint64_t Dq = kmin_t<K>(sX[sidx(k)], x);
            sX[sidx(k)] = Dq;
            if (!K::lt(sL[sidx(k)], Dq)) {  // D <= lambda: the point's pointer moves to n
              sL[sidx(k)] = Dq;
              sI0[sidx(k)] = n;
            }
            if (K::lt(Dq, best) || (!K::lt(best, Dq) && p < bestpos)) { best = Dq; bestpos = p; }
          }
        }
        run = compose<K>(run, shfl_clamp_idx(inc, 0));
        __syncwarp();
#pragma unroll
        for (int j = 0; j < kE; ++j) {
          const int32_t k = 32 * j + lane, p = tb + k;
          if (p < te) {
            S.D[p] = sX[sidx(k)];
            lam[p] = sL[sidx(k)];
            pi[p] = sI0[sidx(k)];
          }
        }
        __syncwarp();
      }
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
      const uint64_t ob = __shfl_down_sync(0xffffffffu, best, d);
      const int32_t op = __shfl_down_sync(0xffffffffu, bestpos, d);
      if (K::lt(ob, best) || (!K::lt(best, ob) && op < bestpos)) { best = ob; bestpos = op; }
    }
    if (lane == 0) { sWBest[warp] = best; sWBestPos[warp] = bestpos; }
    __syncthreads();
    GSUB(6)
    if (warp == 0) {
      best = lane < kWarps ? sWBest[lane] : INF;
      bestpos = lane < kWarps ? sWBestPos[lane] : INT32_MAX;
#pragma unroll
      for (int d = 16; d > 0; d >>= 1) {
        const uint64_t ob = __shfl_down_sync(0xffffffffu, best, d);
        const int32_t op = __shfl_down_sync(0xffffffffu, bestpos, d);
        if (K::lt(ob, best) || (!K::lt(best, ob) && op < bestpos)) { best = ob; bestpos = op; }
      }
      GBest gb;
      gb.key = __shfl_sync(0xffffffffu, best, 0);
      gb.pos = __shfl_sync(0xffffffffu, bestpos, 0);
      gb.pad = 0;
      if (lane < ncta) cluster.map_shared_rank(sBest, lane)[cta] = gb;
    }
    GSUB(7)
    cluster.sync();
    if (timer) { const long long t_ = clock64(); tB += t_ - t_last; t_last = t_; }
    GSUB(8)

    // ---- phase C: speculative shift re-layout, run starts (coalesced over the CTA's positions)
    int32_t x0;
    {
      uint64_t b = INF;
      int32_t bp = INT32_MAX;
      for (int32_t c = 0; c < ncta; ++c) {
        const uint64_t v = sBest[c].key;
        const int32_t p = sBest[c].pos;
        if (K::lt(v, b) || (!K::lt(b, v) && p < bp)) { b = v; bp = p; }
      }
      x0 = bp;
    }
    int32_t *nord = S.ord[nxt];
    int32_t *nlen = S.olen[nxt];
    uint64_t *ngap = S.gap[nxt];
    uint64_t *nlam = S.lam[nxt];
    int32_t *npi = S.pi[nxt];
    {
      const int32_t cta_b = min(cta * kWarps * rpw, nrows) << 5;
      const int32_t cta_e = min(min((cta + 1) * kWarps * rpw, nrows) << 5, m);
      for (int32_t p = cta_b + (int32_t)threadIdx.x; p < cta_e; p += kThreads) {
        const uint64_t Dp = S.D[p];
        const int32_t np = p < x0 ? p : p + 1;
        nord[np] = ord[p];
        nlen[np] = olen[p];
        nlam[np] = lam[p];
        npi[np] = pi[p];
        if (p + 1 < m) {
          const uint64_t Dn = S.D[p + 1];
          if (p + 1 == x0) ngap[p] = Dp;  // last of the left side, then n
          else ngap[np] = kmin_t<K>(kmax_t<K>(Dp, Dn), gap[p]);
        }
        if (p == x0) {
          nord[x0] = n;
          nlen[x0] = (int32_t)ln;
          nlam[x0] = INF;
          npi[x0] = n;
          ngap[x0] = Dp;  // n, then old position x0
        }
        if (p >= 1 && p < x0 && K::lt(S.D[p - 1], Dp)) {
          const uint64_t at = atomicAdd((unsigned long long *)&ctl[kCtlCnt + 2 * slot], 1ull);
          S.runsA[at] = p;
        }
        if (p > x0 && K::lt(Dp, S.D[p - 1])) {
          const uint64_t at = atomicAdd((unsigned long long *)&ctl[kCtlCnt + 2 * slot + 1], 1ull);
          S.runsB[at] = p;
        }
      }
    }
    GSUB(9)
    cluster.sync();
    if (timer) { const long long t_ = clock64(); tC += t_ - t_last; t_last = t_; }
    GSUB(10)

    // run merges: per-thread chunks of positions
    int32_t cb, ce;
    chunk_of(m, tid, nthreads, &cb, &ce);
    // ---- phase D (only when a side is not monotone): merge the sorted runs
    const int32_t nA = (int32_t)ctl[kCtlCnt + 2 * slot] + 1;
    const int32_t nB = (int32_t)ctl[kCtlCnt + 2 * slot + 1] + 1;
    if (nA > 1 || nB > 1) {
      const bool natural = nA <= kRunsSmem && nB <= kRunsSmem;
      if (natural) {
        for (int32_t i = threadIdx.x; i < nA; i += blockDim.x) sRunsA[i] = i == 0 ? 0 : S.runsA[i - 1];
        for (int32_t i = threadIdx.x; i < nB; i += blockDim.x) sRunsB[i] = i == 0 ? x0 : S.runsB[i - 1];
        __syncthreads();
        int32_t capA = 1, capB = 1;
        while (capA < nA) capA <<= 1;
        while (capB < nB) capB <<= 1;
        smem_sort(sRunsA, nA, capA);
        smem_sort(sRunsB, nB, capB);
      }
      for (int32_t p = cb; p < ce; ++p) {
        S.mD[0][p] = S.D[p];
        S.mOrd[0][p] = ord[p];
        S.mLen[0][p] = olen[p];
        S.mOld[0][p] = p;
        S.mLam[0][p] = lam[p];
        S.mPi[0][p] = pi[p];
        S.mRaw[0][p] = 0;
      }
      if (tid == 0) ctl[kCtlStats] += 1;
      cluster.sync();
      const int src = merge_rounds<K>(S, cluster, m, x0, natural, sRunsA, nA, sRunsB, nB, cb, ce, tid == 0);
      for (int32_t p = cb; p < ce; ++p) {
        const int32_t np = p < x0 ? p : p + 1;
        nord[np] = S.mOrd[src][p];
        nlen[np] = S.mLen[src][p];
        nlam[np] = S.mLam[src][p];
        npi[np] = S.mPi[src][p];
        const uint64_t Dp = S.mD[src][p];
        if (p == x0 - 1) ngap[np] = Dp;
        if (p == x0) ngap[x0] = Dp;
        if (p + 1 < m && p + 1 != x0) {
          const uint64_t Dn = S.mD[src][p + 1];
          const int32_t o = S.mOld[src][p], on = S.mOld[src][p + 1];
          uint64_t g = kmax_t<K>(Dp, Dn);
          if (on == o + 1) g = kmin_t<K>(g, gap[o]);
          ngap[np] = g;
        }
        if (p == x0) {
          nord[x0] = n;
          nlen[x0] = (int32_t)ln;
          nlam[x0] = INF;
          npi[x0] = n;
        }
      }
      cluster.sync();
      if (timer) { const long long t_ = clock64(); tD += t_ - t_last; t_last = t_; }
    }
    GSUB(11)
  }
  if (timer) {
    atomicAdd((unsigned long long *)&ctl[kCtlStats + 2], (unsigned long long)tA);
    atomicAdd((unsigned long long *)&ctl[kCtlStats + 3], (unsigned long long)tB);
    atomicAdd((unsigned long long *)&ctl[kCtlStats + 4], (unsigned long long)tC);
    atomicAdd((unsigned long long *)&ctl[kCtlStats + 5], (unsigned long long)tD);
    for (int i = 0; i < 12; ++i) atomicAdd((unsigned long long *)&ctl[kCtlStats + 8 + i], (unsigned long long)sub[i]);
  }
#undef GSUB
}

// -1 (default): by the number of points of the row block (512 threads below
// 100,000 -- measured 13-17 % faster at 30,000-49,000 -- and 1,024 above, 6 %
// faster at 150,000); 0: 1,024 threads a CTA, tiles of 4 per lane; 1: 512, tiles of 8
static int g_global_variant = -1;

template <int T, int E>
constexpr size_t global_smem_bytes() {
  // per warp: 4 arrays of 32 (E + 1) uint64, one more gap slot, 2 arrays of 32 (E + 1) int32 (as uint64 pairs)
  return (size_t)(T / 32) * (4 * 32 * (E + 1) + 1 + 32 * (E + 1)) * sizeof(uint64_t);
}

template <class K, int T, int E>
static cudaError_t global_kernel_attributes() {
  static std::once_flag once;
  static cudaError_t result = cudaSuccess;
  std::call_once(once, [] {
    cudaError_t e = cudaFuncSetAttribute(k_slink_global<K, T, E>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)global_smem_bytes<T, E>());
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_slink_global<K, T, E>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    result = e;
  });
  return result;
}

template <class K, int T, int E>
static cudaError_t launch_global_t(const GlobalArgs &args, int cl, cudaStream_t st) {
  cudaError_t e = global_kernel_attributes<K, T, E>();
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(cl, 1, 1);
  cfg.blockDim = dim3(T, 1, 1);
  cfg.dynamicSmemBytes = global_smem_bytes<T, E>();
  cfg.stream = st;
  int prio = 0;  // kept by a captured graph node (see launch_smem_t)
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
  return cudaLaunchKernelEx(&cfg, k_slink_global<K, T, E>, args);
}

cudaError_t launch_slink_global(const SlinkState &S, const uint16_t *rowbuf, int64_t ld, int32_t r0,
                                int32_t r1, int cl, bool narrow, cudaStream_t st) {
  GlobalArgs args;
  args.s = S;
  args.rowbuf = rowbuf;
  args.ld = ld;
  args.r0 = r0;
  args.r1 = r1;
  const int v = g_global_variant >= 0 ? g_global_variant : (r1 < 100000 ? 1 : 0);
  if (narrow)
    return v == 1 ? launch_global_t<KeysNarrow, 512, 8>(args, cl, st) : launch_global_t<KeysNarrow, 1024, 4>(args, cl, st);
  return v == 1 ? launch_global_t<KeysWide, 512, 8>(args, cl, st) : launch_global_t<KeysWide, 1024, 4>(args, cl, st);
}

int max_cluster_global() {
  static int cached = 0;
  if (cached) return cached;
  if (global_kernel_attributes<KeysWide, 1024, 4>() != cudaSuccess) {
    cudaGetLastError();
    return 1;
  }
  for (int w : {16, 8, 4, 2, 1}) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(w, 1, 1);
    cfg.blockDim = dim3(1024, 1, 1);
    cfg.dynamicSmemBytes = global_smem_bytes<1024, 4>();
    cudaLaunchAttribute attr;
    attr.id = cudaLaunchAttributeClusterDimension;
    attr.val.clusterDim.x = w;
    attr.val.clusterDim.y = 1;
    attr.val.clusterDim.z = 1;
    cfg.attrs = &attr;
    cfg.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, k_slink_global<KeysWide, 1024, 4>, &cfg) == cudaSuccess && n >= 1) {
      cached = w;
      return w;
    }
    cudaGetLastError();
  }
  return 1;
}

}  // namespace famsa

extern "C" int famsa_debug_set_global_variant(int v) {
  if (v < -1 || v > 1) return FAMSA_EINVAL;
  famsa::g_global_variant = v;
  return FAMSA_OK;
}
