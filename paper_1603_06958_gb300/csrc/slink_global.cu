// Row update with the state in global memory (any family size).
//
// One launch inserts points r0..r1-1 (insertion labels) using the LCS rows in
// rowbuf.  A thread-block cluster runs every step; cluster barriers separate
// the phases: distances + scan summaries | scans, D, pointer update, first
// minimum | re-layout.
#include "slink_merge.cuh"

namespace famsa {

struct GlobalArgs {
  SlinkState s;
  const uint16_t *rowbuf;
  int64_t ld;
  int32_t r0, r1;
};

__global__ void __launch_bounds__(kSlinkThreads, 1) k_slink_global(GlobalArgs a) {
  cg::cluster_group cluster = cg::this_cluster();
  const int32_t ncta = (int32_t)cluster.num_blocks();
  const int32_t cta = (int32_t)cluster.block_rank();
  const int32_t nthreads = ncta * blockDim.x;
  const int32_t tid = cta * blockDim.x + threadIdx.x;
  __shared__ Clamp sw[130];
  __shared__ int32_t sRunsA[kRunsSmem], sRunsB[kRunsSmem];
  __shared__ uint64_t sRed[32];
  __shared__ int32_t sRedPos[32];
  SlinkState &S = a.s;
  uint64_t *ctl = S.ctl;

  for (int32_t n = a.r0; n < a.r1; ++n) {
    const int32_t m = n;
    const int cur = m & 1, nxt = cur ^ 1;
    const int slot = n % 3, slot_next = (n + 1) % 3;
    const int32_t *ord = S.ord[cur];
    const int32_t *olen = S.olen[cur];
    const uint64_t *gap = S.gap[cur];
    uint64_t *lam = S.lam[cur];
    int32_t *pi = S.pi[cur];
    const uint16_t *row = a.rowbuf + (int64_t)(n - a.r0) * a.ld;
    const uint32_t ln = (uint32_t)S.slen[n];
    int32_t cb, ce;
    chunk_of(m, tid, nthreads, &cb, &ce);

    // ---- phase A: distances, chunk summaries of both scans
    Clamp sl = identity_clamp(), sr = identity_clamp();
    for (int32_t q = cb; q < ce; ++q) {
      uint64_t d = make_key(row[ord[q]], (uint32_t)olen[q], ln);
      S.D[q] = d;
      sl = compose(sl, Clamp{q == 0 ? kKeyInf : gap[q - 1], d});
    }
    for (int32_t q = ce - 1; q >= cb; --q) sr = compose(sr, Clamp{q == m - 1 ? kKeyInf : gap[q], S.D[q]});
    Clamp preL, preR, totL, totR;
    block_scan2(sl, sr, &preL, &preR, &totL, &totR, sw);
    if (threadIdx.x == 0) {
      ctl[kCtlAggL + 2 * cta] = totL.lo;
      ctl[kCtlAggL + 2 * cta + 1] = totL.hi;
      ctl[kCtlAggR + 2 * cta] = totR.lo;
      ctl[kCtlAggR + 2 * cta + 1] = totR.hi;
      // run counters rotate over three slots; slot (n+1)%3 was last read two
      // barriers ago by every CTA
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
        uint64_t d = make_key(row[ord[q]], (uint32_t)olen[q], ln);
        x = q == m - 1 ? d : kmin(d, kmax(x, gap[q]));
        uint64_t Dq = kmin(S.D[q], x);
        S.D[q] = Dq;
        if (!klt(lam[q], Dq)) {  // D <= lambda: the point's pointer moves to n
          lam[q] = Dq;
          pi[q] = n;
        }
        if (klt(Dq, best) || (!klt(best, Dq) && q < bestpos)) { best = Dq; bestpos = q; }
      }
    }
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
        const int nw = blockDim.x >> 5;
        best = lane < nw ? sRed[lane] : kKeyInf;
        bestpos = lane < nw ? sRedPos[lane] : INT32_MAX;
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
    uint64_t *nlam = S.lam[nxt];
    int32_t *npi = S.pi[nxt];
    for (int32_t p = cb; p < ce; ++p) {
      const uint64_t Dp = S.D[p];
      const int32_t np = p < x0 ? p : p + 1;
      nord[np] = ord[p];
      nlen[np] = olen[p];
      nlam[np] = lam[p];
      npi[np] = pi[p];
      if (p + 1 < m) {
        const uint64_t Dn = S.D[p + 1];
        if (p + 1 == x0) ngap[p] = Dp;  // last of the left side, then n
        else ngap[np] = kmin(kmax(Dp, Dn), gap[p]);
      }
      if (p == x0) {
        nord[x0] = n;
        nlen[x0] = (int32_t)ln;
        nlam[x0] = kKeyInf;
        npi[x0] = n;
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
      const int src = merge_rounds(S, cluster, m, x0, natural, sRunsA, nA, sRunsB, nB, cb, ce, tid == 0);
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
          uint64_t g = kmax(Dp, Dn);
          if (on == o + 1) g = kmin(g, gap[o]);
          ngap[np] = g;
        }
        if (p == x0) {
          nord[x0] = n;
          nlen[x0] = (int32_t)ln;
          nlam[x0] = kKeyInf;
          npi[x0] = n;
        }
      }
      cluster.sync();
    }
  }
}

cudaError_t launch_slink_global(const SlinkState &S, const uint16_t *rowbuf, int64_t ld, int32_t r0,
                                int32_t r1, int cl, cudaStream_t st) {
  GlobalArgs args;
  args.s = S;
  args.rowbuf = rowbuf;
  args.ld = ld;
  args.r0 = r0;
  args.r1 = r1;
  if (cl > 8) cudaFuncSetAttribute(k_slink_global, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(cl, 1, 1);
  cfg.blockDim = dim3(kSlinkThreads, 1, 1);
  cfg.stream = st;
  cudaLaunchAttribute attr;
  attr.id = cudaLaunchAttributeClusterDimension;
  attr.val.clusterDim.x = cl;
  attr.val.clusterDim.y = 1;
  attr.val.clusterDim.z = 1;
  cfg.attrs = &attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_slink_global, args);
}

int max_cluster_global() {
  static int cached = 0;
  if (cached) return cached;
  for (int w : {16, 8, 4, 2, 1}) {
    if (w > 8 &&
        cudaFuncSetAttribute(k_slink_global, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) {
      cudaGetLastError();
      continue;
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
    if (cudaOccupancyMaxActiveClusters(&n, k_slink_global, &cfg) == cudaSuccess && n >= 1) {
      cached = w;
      return w;
    }
    cudaGetLastError();
  }
  return 1;
}

}  // namespace famsa
