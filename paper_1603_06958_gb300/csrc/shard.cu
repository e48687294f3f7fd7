// Sharding the pair set: famsa_msf_rows and famsa_tree_from_edges.
//
// FAMSA Methods, "Pairwise similarities calculation": the pairs are
// independent, and the paper spreads them over threads.  Single linkage
// ("Determination of the guide tree") depends only on a minimum spanning
// tree of the distance graph, and the minimum spanning tree of a union of
// edge sets is the minimum spanning tree of the union of their minimum
// spanning forests (an edge left out of a part's forest is the heaviest on a
// cycle of that part, and the cycle is still there in the union).  So the
// pair set splits into shards of rows -- one per GPU, say -- each reduced on
// its own device to a forest of fewer than k edges; one exchange of those
// edges and one more spanning-tree build on the union give exactly the tree
// of the whole family.
#include <algorithm>
#include <vector>

#include "slink_msf.cuh"

using namespace famsa;

namespace {

__global__ void k_iota(int32_t *o, int32_t n) {
  const int32_t i = (int32_t)(blockIdx.x * blockDim.x + threadIdx.x);
  if (i < n) o[i] = i;
}

// the tree-edge state for n points and up to m input edges
void alloc_msf(Scratch &sc, MsfState &M, int32_t n, int64_t m, int32_t block_rows, int64_t ld) {
  const size_t np = (size_t)n + 1, cap = (size_t)std::max<int64_t>(m, n) + 1;
  M.comp = sc.get<int32_t>(np);
  M.par = sc.get<int32_t>(np);
  M.rkey = sc.get<uint64_t>((size_t)std::max(block_rows, 1));
  M.roth = sc.get<int32_t>((size_t)std::max(block_rows, 1));
  M.ckey = sc.get<uint64_t>(np);
  M.coth = sc.get<int32_t>(np);
  M.vkey = sc.get<uint64_t>(np);
  M.vab = sc.get<uint64_t>(np);
  M.bkey = sc.get<uint64_t>(np);
  M.bab = sc.get<uint64_t>(np);
  M.mkey = sc.get<uint64_t>(cap);
  M.ma = sc.get<int32_t>(cap);
  M.mb = sc.get<int32_t>(cap);
  M.nkey = sc.get<uint64_t>(cap);
  M.na = sc.get<int32_t>(cap);
  M.nb = sc.get<int32_t>(cap);
  M.cap = (int32_t)cap;
  M.ctl = sc.get<int32_t>(kMsfCtlWords);
  M.keys = block_rows > 0 ? sc.get<uint64_t>((size_t)block_rows * ld) : nullptr;
}

int finish(Scratch &sc, cudaError_t err, cudaStream_t st) {
  if (err != cudaSuccess) cudaStreamSynchronize(st);
  sc.release();
  return status_from_cuda(err);
}

}  // namespace

#define CKS(x)                                       \
  do {                                               \
    cudaError_t e_ = (x);                            \
    if (e_ != cudaSuccess) return finish(sc, e_, st); \
  } while (0)

extern "C" int famsa_msf_rows(const famsa_family *fh, int32_t row_begin, int32_t row_end, int32_t *edge_a,
                              int32_t *edge_b, uint64_t *h_num, uint32_t *h_den, int out_on_device,
                              void *cuda_stream) {
  if (!fh || !edge_a || !edge_b || !h_num || !h_den) return FAMSA_EINVAL;
  Family *f = const_cast<Family *>(reinterpret_cast<const Family *>(fh));
  const int32_t k = f->k;
  if (row_begin < 1 || row_end > k || row_begin >= row_end) return FAMSA_EINVAL;
  if (f->max_len > 32767) return FAMSA_ERANGE;
  std::lock_guard<std::mutex> lk(f->mu);
  cudaStream_t st = (cudaStream_t)cuda_stream;
  Scratch sc;
  sc.st = st;
  const int32_t B = std::min<int32_t>(
      (int32_t)std::min<int64_t>(std::max<int64_t>(((int64_t)1 << 29) / std::max(k, 1), 64), 2048),
      row_end - row_begin);
  const int64_t ld = (k + 1) & ~1;
  uint16_t *rowbuf = sc.get<uint16_t>((size_t)B * ld);
  int32_t *d_iota = sc.get<int32_t>((size_t)k);
  MsfState M = {};
  alloc_msf(sc, M, row_end, row_end, B, ld);
  M.slen = f->d_slen;
  const int32_t n_out = row_end - 1;
  int32_t *oa = nullptr, *ob = nullptr;
  uint64_t *on = nullptr;
  uint32_t *od = nullptr;
  if (!out_on_device) {
    oa = sc.get<int32_t>(n_out);
    ob = sc.get<int32_t>(n_out);
    on = sc.get<uint64_t>(n_out);
    od = sc.get<uint32_t>(n_out);
  }
  if (sc.err != cudaSuccess) return finish(sc, sc.err, st);
  k_iota<<<(unsigned)((k + 255) / 256), 256, 0, st>>>(d_iota, k);
  CKS(cudaMemsetAsync(M.ctl, 0, sizeof(int32_t) * kMsfCtlWords, st));
  std::vector<int32_t> h_w(k), h_iota(k);
  for (int32_t s = 0; s < k; ++s) {
    h_w[s] = (f->h_slen[s] + 63) / 64;
    h_iota[s] = s;
  }
  int64_t launches = 0;
  for (int32_t r0 = row_begin, r1 = 0; r0 < row_end; r0 = r1) {
    r1 = std::min(r0 + B, row_end);
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
    b.out = rowbuf;
    b.ld = ld;
    b.row0 = r0;
    b.triangle = true;
    CKS(launch_lcs(b, st, &launches));
    // the shard's first block starts from no tree: its points below
    // row_begin are joined only through the shard's own rows
    CKS(launch_msf_block(M, rowbuf, ld, r0, r1, r0 == row_begin ? 0 : r0 - 1, st, &launches));
  }
  int32_t *da = out_on_device ? edge_a : oa, *db = out_on_device ? edge_b : ob;
  uint64_t *dn = out_on_device ? h_num : on;
  uint32_t *dd = out_on_device ? h_den : od;
  CKS(launch_msf_to_fractions(M, n_out, f->d_perm, da, db, dn, dd, st));
  int32_t mctl[kMsfCtlWords] = {0};
  CKS(cudaMemcpyAsync(mctl, M.ctl, sizeof(mctl), cudaMemcpyDeviceToHost, st));
  if (!out_on_device) {
    CKS(cudaMemcpyAsync(edge_a, oa, sizeof(int32_t) * n_out, cudaMemcpyDeviceToHost, st));
    CKS(cudaMemcpyAsync(edge_b, ob, sizeof(int32_t) * n_out, cudaMemcpyDeviceToHost, st));
    CKS(cudaMemcpyAsync(h_num, on, sizeof(uint64_t) * n_out, cudaMemcpyDeviceToHost, st));
    CKS(cudaMemcpyAsync(h_den, od, sizeof(uint32_t) * n_out, cudaMemcpyDeviceToHost, st));
  }
  CKS(cudaStreamSynchronize(st));
  sc.release();
  return mctl[kMsfErr] ? FAMSA_ECUDA : FAMSA_OK;
}

extern "C" int famsa_tree_from_edges(int32_t k, int64_t n_edges, const int32_t *edge_a, const int32_t *edge_b,
                                     const uint64_t *e_num, const uint32_t *e_den, int32_t *pi,
                                     uint64_t *lambda_num, uint32_t *lambda_den, int32_t *merges,
                                     uint64_t *h_num, uint32_t *h_den, int32_t *sizes, int on_device,
                                     void *cuda_stream) {
  if (k < 1 || n_edges < 0 || n_edges > INT32_MAX - 2) return FAMSA_EINVAL;
  if (n_edges > 0 && (!edge_a || !edge_b || !e_num || !e_den)) return FAMSA_EINVAL;
  if (k >= 2 && n_edges < k - 1) return FAMSA_EINVAL;  // cannot join all k points
  cudaStream_t st = (cudaStream_t)cuda_stream;
  Scratch sc;
  sc.st = st;
  const int32_t m = (int32_t)n_edges;
  const int32_t *ia = edge_a, *ib = edge_b;
  const uint64_t *in_num = e_num;
  const uint32_t *in_den = e_den;
  if (!on_device && m > 0) {
    int32_t *ta = sc.get<int32_t>(m), *tb = sc.get<int32_t>(m);
    uint64_t *tn = sc.get<uint64_t>(m);
    uint32_t *td = sc.get<uint32_t>(m);
    if (sc.err != cudaSuccess) return finish(sc, sc.err, st);
    CKS(cudaMemcpyAsync(ta, edge_a, sizeof(int32_t) * m, cudaMemcpyHostToDevice, st));
    CKS(cudaMemcpyAsync(tb, edge_b, sizeof(int32_t) * m, cudaMemcpyHostToDevice, st));
    CKS(cudaMemcpyAsync(tn, e_num, sizeof(uint64_t) * m, cudaMemcpyHostToDevice, st));
    CKS(cudaMemcpyAsync(td, e_den, sizeof(uint32_t) * m, cudaMemcpyHostToDevice, st));
    ia = ta; ib = tb; in_num = tn; in_den = td;
  }
  MsfState M = {};
  alloc_msf(sc, M, k, m, 0, 0);
  const size_t kp = (size_t)k + 1;
  int32_t *ord = sc.get<int32_t>(kp), *idx_a = sc.get<int32_t>(kp), *idx_b = sc.get<int32_t>(kp);
  int32_t *work = sc.get<int32_t>(8 * kp), *iota = sc.get<int32_t>(kp);
  uint64_t *gap = sc.get<uint64_t>(kp), *ek = sc.get<uint64_t>(kp);
  FinBufs FB = alloc_fin_bufs(sc, k);
  if (sc.err != cudaSuccess) return finish(sc, sc.err, st);
  CKS(cudaMemsetAsync(M.ctl, 0, sizeof(int32_t) * kMsfCtlWords, st));
  int64_t launches = 0;
  if (k >= 2) {
    k_iota<<<(unsigned)((k + 255) / 256), 256, 0, st>>>(iota, k);
    CKS(launch_msf_from_fractions(M, m, k, ia, ib, in_num, in_den, st));
    CKS(launch_msf_edges(M, k, m, st, &launches));
    CKS(launch_msf_leaf_order(M, k, ord, gap, idx_a, idx_b, work, ek, st, &launches));
    CKS(launch_finalize(ord, gap, iota, k, FB, st, &launches, true));
  } else {
    const int32_t z = 0;
    const uint64_t one = 1;
    const uint32_t zero = 0;
    CKS(cudaMemcpyAsync(FB.pi, &z, sizeof(z), cudaMemcpyHostToDevice, st));
    CKS(cudaMemcpyAsync(FB.lnum, &one, sizeof(one), cudaMemcpyHostToDevice, st));
    CKS(cudaMemcpyAsync(FB.lden, &zero, sizeof(zero), cudaMemcpyHostToDevice, st));
  }
  const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  if (pi) CKS(cudaMemcpyAsync(pi, FB.pi, sizeof(int32_t) * k, kind, st));
  if (lambda_num) CKS(cudaMemcpyAsync(lambda_num, FB.lnum, sizeof(uint64_t) * k, kind, st));
  if (lambda_den) CKS(cudaMemcpyAsync(lambda_den, FB.lden, sizeof(uint32_t) * k, kind, st));
  if (k >= 2) {
    if (merges) CKS(cudaMemcpyAsync(merges, FB.merges, sizeof(int32_t) * 2 * (k - 1), kind, st));
    if (h_num) CKS(cudaMemcpyAsync(h_num, FB.hnum, sizeof(uint64_t) * (k - 1), kind, st));
    if (h_den) CKS(cudaMemcpyAsync(h_den, FB.hden, sizeof(uint32_t) * (k - 1), kind, st));
    if (sizes) CKS(cudaMemcpyAsync(sizes, FB.sizes, sizeof(int32_t) * (k - 1), kind, st));
  }
  int32_t mctl[kMsfCtlWords] = {0};
  CKS(cudaMemcpyAsync(mctl, M.ctl, sizeof(mctl), cudaMemcpyDeviceToHost, st));
  CKS(cudaStreamSynchronize(st));
  sc.release();
  // bad edges, or edges that do not join all k points
  return mctl[kMsfErr] ? FAMSA_EINVAL : FAMSA_OK;
}
