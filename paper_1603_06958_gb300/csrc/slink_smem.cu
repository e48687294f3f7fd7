// Row update with the state in the distributed shared memory of one cluster.
//
// Same steps as the global-memory kernel, for families whose per-position
// state (72 bytes a position) fits in the shared memory of the cluster's
// CTAs: CTA c owns positions [c*P, (c+1)*P) of the leaf order, phases
// exchange a handful of values per CTA through DSMEM, and the common
// re-layout (a shift by one after x0) moves elements with DSMEM stores.  The
// rare run-merge re-layout goes through global memory.  The layout is loaded
// from global memory at the start of a launch and stored back at its end.
#include "slink_merge.cuh"

namespace famsa {

struct SmemArgs {
  SlinkState s;
  const uint16_t *rowbuf;
  int64_t ld;
  int32_t r0, r1;
  int32_t P;  // positions per CTA
};

constexpr size_t kSmemBytesPerPos = 6 * sizeof(uint64_t) + 6 * sizeof(int32_t);

size_t smem_bytes_for(int32_t P) { return (size_t)P * kSmemBytesPerPos; }

struct Slot {
  uint64_t aggL_lo, aggL_hi, aggR_lo, aggR_hi;
  uint64_t arg_key, first_D, last_D;
  int32_t arg_pos, min_asc, max_desc, pad;
};

__global__ void __launch_bounds__(kSlinkThreads, 1) k_slink_smem(SmemArgs a) {
  cg::cluster_group cluster = cg::this_cluster();
  const int32_t ncta = (int32_t)cluster.num_blocks();
  const int32_t cta = (int32_t)cluster.block_rank();
  const int32_t P = a.P;
  const int32_t base = cta * P;
  const int32_t T = blockDim.x;
  const int32_t E = (P + T - 1) / T;
  const int32_t i0 = threadIdx.x * E;
  const int32_t tid = cta * T + threadIdx.x;
  SlinkState &S = a.s;
  uint64_t *ctl = S.ctl;

  extern __shared__ __align__(16) uint64_t smem[];
  // buffer b of each per-position array (computed, not indexed, to stay in registers)
  uint64_t *const gap0 = smem, *const lam0 = smem + 2 * P;
  uint64_t *dd = smem + 4 * P;
  uint64_t *DD = smem + 5 * P;
  int32_t *const ibase = reinterpret_cast<int32_t *>(smem + 6 * P);
  int32_t *const ord0 = ibase, *const len0 = ibase + 2 * P, *const pi0 = ibase + 4 * P;
#define gapS(b) (gap0 + (b) * P)
#define lamS(b) (lam0 + (b) * P)
#define ordS(b) (ord0 + (b) * P)
#define lenS(b) (len0 + (b) * P)
#define piS(b) (pi0 + (b) * P)
  __shared__ Clamp sw[130];
  __shared__ Slot slot;
  __shared__ int32_t sRunsA[kRunsSmem], sRunsB[kRunsSmem];
  __shared__ uint64_t sRed[32];
  __shared__ int32_t sRedPos[32], sRedA[32], sRedD[32];

  // load the layout of r0 points
  {
    const int b0 = a.r0 & 1;
    for (int32_t i = threadIdx.x; i < P; i += T) {
      const int32_t p = base + i;
      if (p < a.r0) {
        ordS(0)[i] = S.ord[b0][p];
        lenS(0)[i] = S.olen[b0][p];
        lamS(0)[i] = S.lam[b0][p];
        piS(0)[i] = S.pi[b0][p];
        gapS(0)[i] = p + 1 < a.r0 ? S.gap[b0][p] : kKeyInf;
      }
    }
  }
  cluster.sync();

  int cur = 0;
  const bool timer = tid == 0;
  long long tA = 0, tB = 0, tC = 0, tD = 0, t_last = clock64();
  for (int32_t n = a.r0; n < a.r1; ++n) {
    const int32_t m = n;
    const int nxt = cur ^ 1;
    const int sl_now = n % 3, sl_next = (n + 1) % 3;
    const int32_t mc = max(0, min(m - base, P));
    const int32_t i1 = min(i0 + E, mc);
    const uint16_t *row = a.rowbuf + (int64_t)(n - a.r0) * a.ld;
    const uint32_t ln = (uint32_t)S.slen[n];
    int32_t *ord = ordS(cur);
    int32_t *len = lenS(cur);
    uint64_t *gap = gapS(cur);
    uint64_t *lam = lamS(cur);
    int32_t *pi = piS(cur);

    // ---- phase A: distances and scan summaries
    uint64_t gprev = kKeyInf;  // gap between position base-1 and base (owned by the previous CTA)
    if (i0 == 0 && base > 0 && mc > 0) gprev = cluster.map_shared_rank(gapS(cur), cta - 1)[P - 1];
    Clamp cl_sum = identity_clamp(), cr_sum = identity_clamp();
    for (int32_t i = i0; i < i1; ++i) {
      const int32_t p = base + i;
      const uint64_t d = make_key(row[ord[i]], (uint32_t)len[i], ln);
      dd[i] = d;
      const uint64_t g = p == 0 ? kKeyInf : (i == 0 ? gprev : gap[i - 1]);
      cl_sum = compose(cl_sum, Clamp{g, d});
    }
    for (int32_t i = i1 - 1; i >= i0; --i) {
      const int32_t p = base + i;
      cr_sum = compose(cr_sum, Clamp{p == m - 1 ? kKeyInf : gap[i], dd[i]});
    }
    Clamp preL, preR, totL, totR;
    block_scan2(cl_sum, cr_sum, &preL, &preR, &totL, &totR, sw);
    if (threadIdx.x == 0) {
      slot.aggL_lo = totL.lo;
      slot.aggL_hi = totL.hi;
      slot.aggR_lo = totR.lo;
      slot.aggR_hi = totR.hi;
      if (cta == 0) ctl[kCtlCnt + 2 * sl_next] = 0, ctl[kCtlCnt + 2 * sl_next + 1] = 0;
    }
    cluster.sync();
    if (timer) { long long t = clock64(); tA += t - t_last; t_last = t; }

    // ---- phase B: scans, D, pointer update, first minimum, monotonicity
    {
      Clamp cl = identity_clamp(), cr = identity_clamp();
      for (int32_t c = 0; c < cta; ++c) {
        const Slot *o = cluster.map_shared_rank(&slot, c);
        cl = compose(cl, Clamp{o->aggL_lo, o->aggL_hi});
      }
      for (int32_t c = ncta - 1; c > cta; --c) {
        const Slot *o = cluster.map_shared_rank(&slot, c);
        cr = compose(cr, Clamp{o->aggR_lo, o->aggR_hi});
      }
      preL = compose(cl, preL);
      preR = compose(cr, preR);
    }
    uint64_t best = kKeyInf;
    int32_t bestpos = INT32_MAX;
    if (i0 < i1) {
      uint64_t x = preL.hi;
      for (int32_t i = i0; i < i1; ++i) {
        const int32_t p = base + i;
        const uint64_t g = p == 0 ? kKeyInf : (i == 0 ? gprev : gap[i - 1]);
        x = p == 0 ? dd[i] : kmin(dd[i], kmax(x, g));
        DD[i] = x;
      }
      x = preR.hi;
      for (int32_t i = i1 - 1; i >= i0; --i) {
        const int32_t p = base + i;
        x = p == m - 1 ? dd[i] : kmin(dd[i], kmax(x, gap[i]));
        const uint64_t Dv = kmin(DD[i], x);
        DD[i] = Dv;
        if (!klt(lam[i], Dv)) {  // D <= lambda: the point's pointer moves to n
          lam[i] = Dv;
          pi[i] = n;
        }
        if (klt(Dv, best) || (!klt(best, Dv) && p < bestpos)) { best = Dv; bestpos = p; }
      }
    }
    __syncthreads();
    int32_t masc = INT32_MAX, mdesc = -1;
    for (int32_t i = max(i0, 1); i < i1; ++i) {
      const uint64_t x = DD[i - 1], y = DD[i];
      if (klt(x, y)) masc = min(masc, base + i);
      if (klt(y, x)) mdesc = max(mdesc, base + i);
    }
    {
      const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = T >> 5;
#pragma unroll
      for (int d = 16; d > 0; d >>= 1) {
        uint64_t ob = __shfl_down_sync(0xffffffffu, best, d);
        int32_t op = __shfl_down_sync(0xffffffffu, bestpos, d);
        if (klt(ob, best) || (!klt(best, ob) && op < bestpos)) { best = ob; bestpos = op; }
        masc = min(masc, __shfl_down_sync(0xffffffffu, masc, d));
        mdesc = max(mdesc, __shfl_down_sync(0xffffffffu, mdesc, d));
      }
      if (lane == 0) { sRed[warp] = best; sRedPos[warp] = bestpos; sRedA[warp] = masc; sRedD[warp] = mdesc; }
      __syncthreads();
      if (warp == 0) {
        best = lane < nw ? sRed[lane] : kKeyInf;
        bestpos = lane < nw ? sRedPos[lane] : INT32_MAX;
        masc = lane < nw ? sRedA[lane] : INT32_MAX;
        mdesc = lane < nw ? sRedD[lane] : -1;
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) {
          uint64_t ob = __shfl_down_sync(0xffffffffu, best, d);
          int32_t op = __shfl_down_sync(0xffffffffu, bestpos, d);
          if (klt(ob, best) || (!klt(best, ob) && op < bestpos)) { best = ob; bestpos = op; }
          masc = min(masc, __shfl_down_sync(0xffffffffu, masc, d));
          mdesc = max(mdesc, __shfl_down_sync(0xffffffffu, mdesc, d));
        }
        if (lane == 0) {
          slot.arg_key = best;
          slot.arg_pos = bestpos;
          slot.min_asc = masc;
          slot.max_desc = mdesc;
          slot.first_D = mc > 0 ? DD[0] : kKeyInf;
          slot.last_D = mc > 0 ? DD[mc - 1] : kKeyInf;
        }
      }
    }
    cluster.sync();
    if (timer) { long long t = clock64(); tB += t - t_last; t_last = t; }

    // ---- phase C: re-layout
    int32_t x0 = INT32_MAX;
    bool violation = false;
    {
      uint64_t b = kKeyInf;
      int32_t minAsc = INT32_MAX, maxDesc = -1;
      uint64_t prevLast = kKeyInf;
      for (int32_t c = 0; c < ncta; ++c) {
        const Slot *o = cluster.map_shared_rank(&slot, c);
        const uint64_t v = o->arg_key;
        const int32_t p = o->arg_pos;
        if (klt(v, b) || (!klt(b, v) && p < x0)) { b = v; x0 = p; }
        minAsc = min(minAsc, o->min_asc);
        maxDesc = max(maxDesc, o->max_desc);
        const int32_t pb = c * P;  // boundary pair (pb - 1, pb)
        if (c > 0 && pb < m) {
          const uint64_t f = o->first_D;
          if (klt(prevLast, f)) minAsc = min(minAsc, pb);
          if (klt(f, prevLast)) maxDesc = max(maxDesc, pb);
        }
        prevLast = o->last_D;
      }
      violation = minAsc < x0 || maxDesc > x0;
    }
    const int32_t cb = base + i0, ce = base + i1;
    if (!violation) {
      for (int32_t i = i0; i < i1; ++i) {
        const int32_t p = base + i;
        const int32_t np = p < x0 ? p : p + 1;
        const int32_t cn = np / P, in = np - cn * P;
        int32_t *dord = cluster.map_shared_rank(ordS(nxt), cn);
        int32_t *dlen = cluster.map_shared_rank(lenS(nxt), cn);
        uint64_t *dlam = cluster.map_shared_rank(lamS(nxt), cn);
        int32_t *dpi = cluster.map_shared_rank(piS(nxt), cn);
        uint64_t *dgap = cluster.map_shared_rank(gapS(nxt), cn);
        dord[in] = ord[i];
        dlen[in] = len[i];
        dlam[in] = lam[i];
        dpi[in] = pi[i];
        const uint64_t Dp = DD[i];
        if (p + 1 < m) {
          const uint64_t Dn = i + 1 < P ? DD[i + 1] : cluster.map_shared_rank(DD, cta + 1)[0];
          if (p + 1 == x0) dgap[in] = Dp;  // last of the left side, then n
          else dgap[in] = kmin(kmax(Dp, Dn), gap[i]);
        }
        if (p == x0) {
          // new position x0 = old position x0 belongs to this CTA
          ordS(nxt)[i] = n;
          lenS(nxt)[i] = (int32_t)ln;
          lamS(nxt)[i] = kKeyInf;
          piS(nxt)[i] = n;
          gapS(nxt)[i] = Dp;  // n, then old position x0
        }
      }
      cluster.sync();
      if (timer) { long long t = clock64(); tC += t - t_last; t_last = t; }
    } else {
      // run starts of both sides, element copies for the global-memory merge
      const uint64_t dprev = (i0 == 0 && base > 0 && mc > 0) ? cluster.map_shared_rank(DD, cta - 1)[P - 1] : kKeyInf;
      for (int32_t i = i0; i < i1; ++i) {
        const int32_t p = base + i;
        const uint64_t Dp = DD[i];
        S.mD[0][p] = Dp;
        S.mOrd[0][p] = ord[i];
        S.mLen[0][p] = len[i];
        S.mOld[0][p] = p;
        S.mLam[0][p] = lam[i];
        S.mPi[0][p] = pi[i];
        S.mGap[p] = gap[i];
        const uint64_t Dq = i == 0 ? dprev : DD[i - 1];
        if (p >= 1 && p < x0 && klt(Dq, Dp)) {
          uint64_t at = atomicAdd((unsigned long long *)&ctl[kCtlCnt + 2 * sl_now], 1ull);
          S.runsA[at] = p;
        }
        if (p > x0 && klt(Dp, Dq)) {
          uint64_t at = atomicAdd((unsigned long long *)&ctl[kCtlCnt + 2 * sl_now + 1], 1ull);
          S.runsB[at] = p;
        }
      }
      if (tid == 0) ctl[kCtlStats] += 1;
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
      const int src = merge_rounds(S, cluster, m, x0, natural, sRunsA, nA, sRunsB, nB, cb, ce, tid == 0);
      for (int32_t p = cb; p < ce; ++p) {
        const int32_t np = p < x0 ? p : p + 1;
        const int32_t cn = np / P, in = np - cn * P;
        int32_t *dord = cluster.map_shared_rank(ordS(nxt), cn);
        int32_t *dlen = cluster.map_shared_rank(lenS(nxt), cn);
        uint64_t *dlam = cluster.map_shared_rank(lamS(nxt), cn);
        int32_t *dpi = cluster.map_shared_rank(piS(nxt), cn);
        uint64_t *dgap = cluster.map_shared_rank(gapS(nxt), cn);
        dord[in] = S.mOrd[src][p];
        dlen[in] = S.mLen[src][p];
        dlam[in] = S.mLam[src][p];
        dpi[in] = S.mPi[src][p];
        const uint64_t Dp = S.mD[src][p];
        if (p == x0 - 1) dgap[in] = Dp;
        if (p + 1 < m && p + 1 != x0) {
          const uint64_t Dn = S.mD[src][p + 1];
          const int32_t o = S.mOld[src][p], on = S.mOld[src][p + 1];
          uint64_t g = kmax(Dp, Dn);
          if (on == o + 1) g = kmin(g, S.mGap[o]);
          dgap[in] = g;
        }
        if (p == x0) {
          const int32_t cx = x0 / P, ix = x0 - cx * P;
          cluster.map_shared_rank(ordS(nxt), cx)[ix] = n;
          cluster.map_shared_rank(lenS(nxt), cx)[ix] = (int32_t)ln;
          cluster.map_shared_rank(lamS(nxt), cx)[ix] = kKeyInf;
          cluster.map_shared_rank(piS(nxt), cx)[ix] = n;
          cluster.map_shared_rank(gapS(nxt), cx)[ix] = Dp;
        }
      }
      cluster.sync();
      if (timer) { long long t = clock64(); tD += t - t_last; t_last = t; }
    }
    cur = nxt;
  }
  if (timer) {
    atomicAdd((unsigned long long *)&ctl[kCtlStats + 2], (unsigned long long)tA);
    atomicAdd((unsigned long long *)&ctl[kCtlStats + 3], (unsigned long long)tB);
    atomicAdd((unsigned long long *)&ctl[kCtlStats + 4], (unsigned long long)tC);
    atomicAdd((unsigned long long *)&ctl[kCtlStats + 5], (unsigned long long)tD);
  }

  // store the layout of r1 points
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
#undef gapS
#undef lamS
#undef ordS
#undef lenS
#undef piS
}

// Cluster size for the shared-memory kernel, or 0 when the family does not fit.
int smem_cluster_for(int32_t k, int force) {
  int device = 0, optin = 0;
  cudaGetDevice(&device);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
  const size_t static_bytes = 24 * 1024;
  for (int c : {1, 2, 4, 8, 16}) {
    if (force && c != force) continue;
    int32_t P = (k + c - 1) / c;
    if (smem_bytes_for(P) + static_bytes <= (size_t)optin) return c;
  }
  return 0;
}

cudaError_t launch_slink_smem(const SlinkState &S, const uint16_t *rowbuf, int64_t ld, int32_t r0,
                              int32_t r1, int cl, int32_t k, cudaStream_t st) {
  SmemArgs args;
  args.s = S;
  args.rowbuf = rowbuf;
  args.ld = ld;
  args.r0 = r0;
  args.r1 = r1;
  args.P = (k + cl - 1) / cl;
  size_t dyn = smem_bytes_for(args.P);
  cudaError_t e = cudaFuncSetAttribute(k_slink_smem, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
  if (e != cudaSuccess) return e;
  if (cl > 8) {
    e = cudaFuncSetAttribute(k_slink_smem, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(cl, 1, 1);
  cfg.blockDim = dim3(kSlinkThreads, 1, 1);
  cfg.dynamicSmemBytes = dyn;
  cfg.stream = st;
  cudaLaunchAttribute attr;
  attr.id = cudaLaunchAttributeClusterDimension;
  attr.val.clusterDim.x = cl;
  attr.val.clusterDim.y = 1;
  attr.val.clusterDim.z = 1;
  cfg.attrs = &attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_slink_smem, args);
}

}  // namespace famsa
