// Run-merge re-layout shared by the row-update kernels.
//
// After point n joins, the new leaf order is [positions < x0 sorted by D
// descending] n [positions >= x0 sorted by D ascending], both stable, where
// x0 is the first minimum of D.  When a side is not already monotone, it
// consists of a few sorted runs; they are merged pairwise here, in global
// memory, one cluster barrier per round.
#pragma once

#include "slink_common.cuh"

namespace famsa {

// Merge rounds over positions [0, m) held in S.m*[0]; the run starts of both
// sides are in sRunsA[0..nA) / sRunsB[0..nB) (sorted) when natural, else
// every element starts as its own run.  Threads own positions [cb, ce).
// Returns the buffer index holding the merged order.
template <class K = KeysWide>
__device__ __forceinline__ int merge_rounds(const SlinkState &S, cg::cluster_group &cluster, int32_t m,
                                            int32_t x0, bool natural, const int32_t *sRunsA,
                                            int32_t nA, const int32_t *sRunsB, int32_t nB,
                                            int32_t cb, int32_t ce, bool count_rounds) {
  int src = 0;
  const int32_t sideLenA = x0, sideLenB = m - x0;
  for (int32_t width = 1;; width <<= 1) {
    int32_t runsA_now = natural ? (nA + width - 1) / width : (sideLenA + width - 1) / width;
    int32_t runsB_now = natural ? (nB + width - 1) / width : (sideLenB + width - 1) / width;
    if (runsA_now <= 1 && runsB_now <= 1) break;
    if (count_rounds) S.ctl[kCtlStats + 1] += 1;
    const int dst = src ^ 1;
    for (int32_t p = cb; p < ce; ++p) {
      const bool left = p < x0;
      const int32_t sbase = left ? 0 : x0;
      const int32_t slen_side = left ? sideLenA : sideLenB;
      const int32_t i = p - sbase;
      int32_t rs, ps = 0, pe = 0, run;
      bool pairs;
      if (natural) {
        const int32_t *starts = left ? sRunsA : sRunsB;
        const int32_t nr = left ? nA : nB;
        int32_t r = run_of(starts, nr, p);
        run = r / width;
        rs = starts[run * width] - sbase;
        int32_t pf = (run ^ 1) * width;
        pairs = pf < nr;
        if (pairs) {
          ps = starts[pf] - sbase;
          pe = (pf + width < nr) ? starts[pf + width] - sbase : slen_side;
        }
      } else {
        run = i / width;
        rs = run * width;
        ps = (run ^ 1) * width;
        pe = min(ps + width, slen_side);
        pairs = ps < slen_side;
      }
      const uint64_t v = S.mD[src][p];
      int32_t np = p;
      if (pairs) {
        const int32_t cnt = merge_count<K>(S.mD[src], sbase, ps, pe, v, left, (run & 1) == 0);
        np = sbase + min(rs, ps) + (i - rs) + cnt;
      }
      S.mD[dst][np] = v;
      S.mOrd[dst][np] = S.mOrd[src][p];
      S.mLen[dst][np] = S.mLen[src][p];
      S.mOld[dst][np] = S.mOld[src][p];
      S.mLam[dst][np] = S.mLam[src][p];
      S.mPi[dst][np] = S.mPi[src][p];
      S.mRaw[dst][np] = S.mRaw[src][p];
    }
    cluster.sync();
    src = dst;
  }
  return src;
}

}  // namespace famsa
