// famsa_slink_tree host driver: LCS row blocks on one stream, the SLINK row
// update on a second (higher-priority) stream, kRowBuffers row blocks in
// flight so the LCS of the next blocks overlaps the row update of block b,
// then the parallel finalisation.
//
// FAMSA Methods, "Determination of the guide tree": stages I and II run
// together -- each similarity row feeds the single-linkage update as soon as
// it exists, so the k x k matrix is never stored (O(k) tree state plus a few
// row blocks).
//
// Points are inserted in the family's length-sorted order (the order the LCS
// kernels prefer); the single-linkage tree does not depend on the insertion
// order, and the outputs are produced in the caller's labels by the
// finalisation.
#include <algorithm>
#include <cstdio>
#include <vector>

#include "slink_msf.cuh"

namespace famsa {

static int g_force_cluster = 0;
// 0 automatic, 1 shared-memory insertion kernel, 2 global-memory insertion
// kernel, 3 minimum-spanning-tree rebuild per row block (automatic whenever
// every length is <= 32767; the insertion kernels take longer sequences)
static int g_update_path = 0;
static int g_row_block = 0;  // rows per row block (0 automatic)
static int g_serial = 0;       // 1: no overlap of LCS and row update (timing studies)

int slink_tree(Family *f, int32_t *pi_out, uint64_t *lnum_out, uint32_t *lden_out,
               int32_t *merges_out, uint64_t *hnum_out, uint32_t *hden_out, int32_t *sizes_out,
               bool out_on_device, cudaStream_t st) {
  const int32_t k = f->k;
  for (int i = 0; i < kStatsLen; ++i) f->stats[i] = 0;
  cudaError_t err = cudaSuccess;

  // which row update, and the insertion kernels' cluster size
  const bool narrow = f->max_len <= 32767;
  int path = g_update_path, cl = 0;
  if (path == 0 && narrow) path = 3;
  if (path == 3 && !narrow) return FAMSA_EINVAL;
  const bool msf = path == 3;
  if (!msf && path != 2) {
    cl = g_force_cluster ? smem_cluster_for(k, g_force_cluster) : smem_cluster_latency(k);
    if (cl > max_cluster_global()) cl = 0;
    if (cl == 0 && path == 1) return FAMSA_EINVAL;
    path = cl ? 1 : 2;
  }
  if (path == 2) cl = g_force_cluster ? g_force_cluster : max_cluster_global();
  // every row update compares exact order codes floor(num * 2^30 / den) when
  // every indel^2 fits in 32 bits and every LCS in 15 (all lengths <= 32767)

  int prio_lo = 0, prio_hi = 0;
  cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi);
  cudaStream_t sA = nullptr, sB = nullptr;
  cudaEvent_t ev_start = nullptr, ev_end = nullptr, lcs_done[kRowBuffers] = {}, upd_done[kRowBuffers] = {};
  Scratch sc;
  sc.st = st;
  int64_t launches = 0, lcs_launches = 0;
  int rc = FAMSA_OK;
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
  for (int i = 0; i < kRowBuffers; ++i) {
    CKE(cudaEventCreateWithFlags(&lcs_done[i], cudaEventDisableTiming));
    CKE(cudaEventCreateWithFlags(&upd_done[i], cudaEventDisableTiming));
  }
  {
    SlinkState S = {};
    MsfState M = {};
    const size_t kp = (size_t)k + 1;
    if (!msf) {
      for (int i = 0; i < 2; ++i) {
        S.ord[i] = sc.get<int32_t>(kp);
        S.olen[i] = sc.get<int32_t>(kp);
        S.gap[i] = sc.get<uint64_t>(kp);
        S.lam[i] = sc.get<uint64_t>(kp);
        S.pi[i] = sc.get<int32_t>(kp);
        S.mD[i] = sc.get<uint64_t>(kp);
        S.mOrd[i] = sc.get<int32_t>(kp);
        S.mLen[i] = sc.get<int32_t>(kp);
        S.mOld[i] = sc.get<int32_t>(kp);
        S.mLam[i] = sc.get<uint64_t>(kp);
        S.mPi[i] = sc.get<int32_t>(kp);
        S.mRaw[i] = sc.get<int32_t>(kp);
      }
      S.D = sc.get<uint64_t>(kp);
      S.mGap = sc.get<uint64_t>(kp);
      S.runsA = sc.get<int32_t>(kp);
      S.runsB = sc.get<int32_t>(kp);
      S.ctl = sc.get<uint64_t>(kCtlWords);
    }
    S.slen = f->d_slen;
    // row blocks: about 128 MB of 16-bit LCS values per buffer for the
    // insertion kernels; the tree rebuild costs a few passes over its block,
    // so it takes blocks up to 8x larger (fewer, larger launches)
    const int64_t budget = msf ? (int64_t)1 << 29 : (int64_t)1 << 26;
    int32_t B = (int32_t)std::min<int64_t>(std::max<int64_t>(budget / std::max(k, 1), 64), 2048);
    if (g_row_block) B = g_row_block;
    B = std::min(B, std::max(k - 1, 1));
    const int64_t ld = (k + 1) & ~1;  // even: rows start on 4-byte boundaries
    uint16_t *rowbuf[kRowBuffers];
    for (int i = 0; i < kRowBuffers; ++i) rowbuf[i] = sc.get<uint16_t>((size_t)B * ld);
    int32_t *msf_ord = nullptr, *msf_ia = nullptr, *msf_ib = nullptr, *msf_work = nullptr;
    uint64_t *msf_gap = nullptr, *msf_gafter = nullptr;
    if (msf) {
      M.comp = sc.get<int32_t>(kp);
      M.par = sc.get<int32_t>(kp);
      M.rkey = sc.get<uint64_t>((size_t)B);
      M.roth = sc.get<int32_t>((size_t)B);
      M.ckey = sc.get<uint64_t>(kp);
      M.coth = sc.get<int32_t>(kp);
      M.vkey = sc.get<uint64_t>(kp);
      M.vab = sc.get<uint64_t>(kp);
      M.bkey = sc.get<uint64_t>(kp);
      M.bab = sc.get<uint64_t>(kp);
      M.mkey = sc.get<uint64_t>(kp);
      M.ma = sc.get<int32_t>(kp);
      M.mb = sc.get<int32_t>(kp);
      M.nkey = sc.get<uint64_t>(kp);
      M.na = sc.get<int32_t>(kp);
      M.nb = sc.get<int32_t>(kp);
      M.cap = (int32_t)kp;
      M.ctl = sc.get<int32_t>(kMsfCtlWords);
      M.keys = sc.get<uint64_t>((size_t)B * ld);
      M.slen = f->d_slen;
      msf_ord = sc.get<int32_t>(kp);
      msf_ia = sc.get<int32_t>(kp);
      msf_ib = sc.get<int32_t>(kp);
      msf_work = sc.get<int32_t>(8 * kp);
      msf_gap = sc.get<uint64_t>(kp);
      msf_gafter = sc.get<uint64_t>(kp);
    }
    std::vector<int32_t> h_iota(k), h_w(k);
    for (int32_t s = 0; s < k; ++s) { h_iota[s] = s; h_w[s] = (f->h_slen[s] + 63) / 64; }
    int32_t *d_iota = sc.get<int32_t>(k);
    // finalisation buffers
    FinBufs FB = alloc_fin_bufs(sc, k);
    if (sc.err != cudaSuccess) { err = sc.err; goto done; }
    CKE(cudaMemcpyAsync(d_iota, h_iota.data(), sizeof(int32_t) * k, cudaMemcpyHostToDevice, st));
    if (msf) {
      CKE(cudaMemsetAsync(M.ctl, 0, sizeof(int32_t) * kMsfCtlWords, st));
    } else {
      CKE(cudaMemsetAsync(S.ctl, 0, sizeof(uint64_t) * kCtlWords, st));
      // the layout of one point (point 0): buffer 1
      std::vector<int32_t> z1 = {0};
      std::vector<uint64_t> inf1 = {narrow ? KeysNarrow::kInf : KeysWide::kInf};
      CKE(cudaMemcpyAsync(S.ord[1], z1.data(), sizeof(int32_t), cudaMemcpyHostToDevice, st));
      CKE(cudaMemcpyAsync(S.olen[1], f->d_slen, sizeof(int32_t), cudaMemcpyDeviceToDevice, st));
      CKE(cudaMemcpyAsync(S.lam[1], inf1.data(), sizeof(uint64_t), cudaMemcpyHostToDevice, st));
      CKE(cudaMemcpyAsync(S.pi[1], z1.data(), sizeof(int32_t), cudaMemcpyHostToDevice, st));
      CKE(cudaStreamSynchronize(st));
    }
    CKE(cudaEventRecord(ev_start, st));
    CKE(cudaStreamWaitEvent(sA, ev_start, 0));
    CKE(cudaStreamWaitEvent(sB, ev_start, 0));
    int64_t cells = 0, words = 0, pairs = (int64_t)k * (k - 1) / 2;
    {
      // algorithmic counters: each row s (its Peq words) against columns t < s
      int64_t colsum = 0;
      for (int32_t s = 0; s < k; ++s) {
        words += (int64_t)h_w[s] * colsum;
        cells += (int64_t)f->h_slen[s] * colsum;
        colsum += f->h_slen[s];
      }
    }
    int32_t blk = 0;
    // the first block is an eighth of the others: the row update can start
    // once its few, short rows are done.  A family of up to 2,048 points is
    // one block (B = k - 1): its whole LCS is short, and one set of tree
    // rounds (about 55 launches) costs less than overlapping three.
    const bool one_block = msf && !g_row_block && k <= 2048;
    const int32_t B0 = g_row_block || one_block ? B : std::min(B, std::max(B / 8, 64));  // the buffers hold B rows
    for (int32_t r0 = 1, r1 = 0; r0 < k; r0 = r1, ++blk) {
      {
        // the last block is a quarter of the others, so that little row
        // update work is left once the last LCS block is done
        int32_t take = blk == 0 ? B0 : B;
        const int32_t rem = k - r0, tail_rows = std::max(B / 4, 1);
        if (msf && !g_row_block && !one_block && rem > tail_rows && rem <= take + tail_rows) take = rem - tail_rows;
        r1 = std::min(r0 + take, k);
      }
      char tname[64];
      snprintf(tname, sizeof tname, "row block %d: rows %d-%d", blk, r0, r1 - 1);
      TraceRange trace(tname);
      const int buf = blk % kRowBuffers;
      if (blk >= kRowBuffers) CKE(cudaStreamWaitEvent(sA, upd_done[buf], 0));
      if (g_serial && blk >= 1) CKE(cudaStreamWaitEvent(sA, upd_done[(blk - 1) % kRowBuffers], 0));
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
      CKE(timing_event(sB));
      if (msf) {
        CKE(launch_msf_block(M, rowbuf[buf], ld, r0, r1, r0 - 1, sB, &launches));
      } else {
        if (path == 1) CKE(launch_slink_smem(S, rowbuf[buf], ld, r0, r1, cl, k, narrow, sB));
        else CKE(launch_slink_global(S, rowbuf[buf], ld, r0, r1, cl, narrow, sB));
        ++launches;
      }
      CKE(timing_event(sB));
      CKE(cudaEventRecord(upd_done[buf], sB));
    }
    // finalisation from the layout of k points (buffer k & 1), keys in the wide packing
    TraceRange trace_fin("leaf order and finalisation");
    CKE(timing_event(sB));
    // (the streamed lambda is widened for the debug export; the finalisation
    // widens the gaps itself)
    if (narrow && !msf) CKE(widen_keys(S.lam[k & 1], k, sB));
    if (k >= 2 && msf) {
      // the finished tree -> a dendrogram leaf order and its gaps
      CKE(launch_msf_leaf_order(M, k, msf_ord, msf_gap, msf_ia, msf_ib, msf_work, msf_gafter, sB, &launches));
      CKE(launch_finalize(msf_ord, msf_gap, f->d_perm, k, FB, sB, &launches, true));
    } else if (k >= 2) {
      CKE(launch_finalize(S.ord[k & 1], S.gap[k & 1], f->d_perm, k, FB, sB, &launches, narrow));
    } else {
      std::vector<int32_t> z = {0};
      std::vector<uint64_t> one = {1};
      std::vector<uint32_t> zero = {0};
      CKE(cudaMemcpyAsync(FB.pi, z.data(), sizeof(int32_t), cudaMemcpyHostToDevice, sB));
      CKE(cudaMemcpyAsync(FB.lnum, one.data(), sizeof(uint64_t), cudaMemcpyHostToDevice, sB));
      CKE(cudaMemcpyAsync(FB.lden, zero.data(), sizeof(uint32_t), cudaMemcpyHostToDevice, sB));
      CKE(cudaStreamSynchronize(sB));
    }
    CKE(cudaGetLastError());
    CKE(timing_event(sB));
    {
      cudaMemcpyKind kind = out_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
      if (pi_out) CKE(cudaMemcpyAsync(pi_out, FB.pi, sizeof(int32_t) * k, kind, sB));
      if (lnum_out) CKE(cudaMemcpyAsync(lnum_out, FB.lnum, sizeof(uint64_t) * k, kind, sB));
      if (lden_out) CKE(cudaMemcpyAsync(lden_out, FB.lden, sizeof(uint32_t) * k, kind, sB));
      if (k >= 2) {
        if (merges_out) CKE(cudaMemcpyAsync(merges_out, FB.merges, sizeof(int32_t) * 2 * (k - 1), kind, sB));
        if (hnum_out) CKE(cudaMemcpyAsync(hnum_out, FB.hnum, sizeof(uint64_t) * (k - 1), kind, sB));
        if (hden_out) CKE(cudaMemcpyAsync(hden_out, FB.hden, sizeof(uint32_t) * (k - 1), kind, sB));
        if (sizes_out) CKE(cudaMemcpyAsync(sizes_out, FB.sizes, sizeof(int32_t) * (k - 1), kind, sB));
      }
    }
    if (msf) {
      int32_t mctl[kMsfCtlWords] = {0};
      CKE(cudaMemcpyAsync(mctl, M.ctl, sizeof(mctl), cudaMemcpyDeviceToHost, sB));
      CKE(cudaEventRecord(ev_end, sB));
      CKE(cudaStreamWaitEvent(st, ev_end, 0));
      CKE(cudaEventSynchronize(ev_end));
      f->stats[18] = 1;
      f->dbg_state.clear();  // no insertion state on this path
      // a tree that did not come out with k - 1 edges, or a join of two
      // points already joined, is an internal error
      if (mctl[kMsfErr]) rc = FAMSA_ECUDA;
    } else {
      // the insertion-label pointer representation (debug export) and counters
      std::vector<int32_t> ordh(k), pih(k);
      std::vector<uint64_t> lamh(k);
      const int bk = k & 1;
      CKE(cudaMemcpyAsync(ordh.data(), S.ord[bk], sizeof(int32_t) * k, cudaMemcpyDeviceToHost, sB));
      CKE(cudaMemcpyAsync(pih.data(), S.pi[bk], sizeof(int32_t) * k, cudaMemcpyDeviceToHost, sB));
      CKE(cudaMemcpyAsync(lamh.data(), S.lam[bk], sizeof(uint64_t) * k, cudaMemcpyDeviceToHost, sB));
      uint64_t hstats[24] = {0};
      CKE(cudaMemcpyAsync(hstats, S.ctl + kCtlStats, sizeof(uint64_t) * 24, cudaMemcpyDeviceToHost, sB));
      f->stats[18] = narrow ? 1 : 0;
      for (int i = 0; i < 16; ++i) f->sub_kcycles[i] = (int64_t)(hstats[8 + i] / 1000);
      f->stats[19] = (int64_t)hstats[6];
      f->stats[20] = (int64_t)hstats[7];
      CKE(cudaEventRecord(ev_end, sB));
      CKE(cudaStreamWaitEvent(st, ev_end, 0));
      CKE(cudaEventSynchronize(ev_end));
      f->dbg_state.assign(4 * (size_t)k, 0);
      for (int32_t p = 0; p < k; ++p) {
        const int32_t node = ordh[p];
        f->dbg_state[4 * (size_t)node] = f->h_perm[node];
        f->dbg_state[4 * (size_t)node + 1] = pih[p];
        f->dbg_state[4 * (size_t)node + 2] = (int64_t)lamh[p];
      }
      f->stats[4] = (int64_t)hstats[0];
      f->stats[5] = (int64_t)hstats[1];
      // phase cycle counters of the shared-memory kernel (CTA 0, thread 0), in kilocycles
      for (int i = 0; i < 4; ++i) f->stats[14 + i] = (int64_t)(hstats[2 + i] / 1000);
    }
    {
      // events: 4 per row block (LCS begin/end, update begin/end), then 2 for finalisation
      double lcs_ms = 0, upd_ms = 0;
      const size_t nblk = (tev.size() - 2) / 4;
      for (size_t i = 0; i < nblk; ++i) {
        float x = 0, y = 0;
        cudaEventElapsedTime(&x, tev[4 * i], tev[4 * i + 1]);
        cudaEventElapsedTime(&y, tev[4 * i + 2], tev[4 * i + 3]);
        lcs_ms += x;
        upd_ms += y;
      }
      float z = 0;
      cudaEventElapsedTime(&z, tev[tev.size() - 2], tev[tev.size() - 1]);
      f->stats[7] = (int64_t)(lcs_ms * 1e6);
      f->stats[8] = (int64_t)(upd_ms * 1e6);
      f->stats[9] = (int64_t)(z * 1e6);
      f->stats[10] = lcs_launches;
      f->stats[12] = path;
      f->stats[13] = cl;
    }
    launches += lcs_launches;
    f->stats[0] = launches;
    f->stats[1] = cells;
    f->stats[2] = words;
    f->stats[3] = pairs;
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
  for (int i = 0; i < kRowBuffers; ++i) {
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

extern "C" int famsa_debug_set_serial(int on) {
  famsa::g_serial = on ? 1 : 0;
  return FAMSA_OK;
}

extern "C" int famsa_debug_sub_kcycles(const famsa_family *fh, int64_t *out16) {
  if (!fh || !out16) return FAMSA_EINVAL;
  const famsa::Family *f = reinterpret_cast<const famsa::Family *>(fh);
  for (int i = 0; i < 16; ++i) out16[i] = f->sub_kcycles[i];
  return FAMSA_OK;
}

extern "C" int famsa_debug_set_row_block(int rows) {
  if (rows < 0 || rows > 2048) return FAMSA_EINVAL;
  famsa::g_row_block = rows;
  return FAMSA_OK;
}

extern "C" int famsa_debug_set_update_path(int path) {
  if (path < 0 || path > 3) return FAMSA_EINVAL;
  famsa::g_update_path = path;
  return FAMSA_OK;
}

extern "C" int famsa_debug_order_code(uint32_t num, uint32_t den, uint64_t *code) {
  if (!code || den == 0 || den > 32767) return FAMSA_EINVAL;
  *code = famsa::order_code(num, den);
  return FAMSA_OK;
}

extern "C" int famsa_debug_code_fraction(uint64_t code, uint64_t *num, uint32_t *den) {
  if (!num || !den) return FAMSA_EINVAL;
  famsa::code_fraction(code, num, den);
  return FAMSA_OK;
}

extern "C" int famsa_debug_insertion_state(const famsa_family *fh, int32_t *perm, int32_t *pi,
                                           uint64_t *lam_num, uint32_t *lam_den) {
  if (!fh) return FAMSA_EINVAL;
  const famsa::Family *f = reinterpret_cast<const famsa::Family *>(fh);
  const int32_t k = f->k;
  if ((int64_t)f->dbg_state.size() != 4 * (int64_t)k) return FAMSA_EINVAL;
  for (int32_t j = 0; j < k; ++j) {
    const int64_t *e = &f->dbg_state[4 * (size_t)j];
    if (perm) perm[j] = (int32_t)e[0];
    if (pi) pi[j] = (int32_t)e[1];
    uint64_t key = (uint64_t)e[2];
    uint64_t num = key >> 16;
    uint32_t den = (uint32_t)(key & 0xffffu);
    if (den == 0) num = 1;
    else if (num == 0) den = 1;
    else {
      uint64_t a = num, b = den;
      while (b) { uint64_t t = a % b; a = b; b = t; }
      num /= a;
      den = (uint32_t)(den / a);
    }
    if (lam_num) lam_num[j] = num;
    if (lam_den) lam_den[j] = den;
  }
  return FAMSA_OK;
}
