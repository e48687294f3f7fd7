// C ABI entry points (declared in include/famsa_gpu.h).
#include <algorithm>
#include <cstring>
#include <numeric>
#include <vector>

#include "famsa_internal.cuh"

using famsa::Family;

namespace famsa {

// Per-family host metadata for LCS launches over the family's own rows.
struct RowList {
  std::vector<int32_t> w, id;
  int32_t *d_id = nullptr;
};

static void host_row_list(const Family *f, RowList &rl) {
  rl.w.resize(f->k);
  rl.id.resize(f->k);
  for (int32_t s = 0; s < f->k; ++s) {
    rl.w[s] = (f->h_slen[s] + 63) / 64;
    rl.id[s] = s;
  }
}

template <typename T>
static cudaError_t upload(const std::vector<T> &v, T **d, cudaStream_t st) {
  cudaError_t e = lib_malloc_async((void **)d, std::max<size_t>(v.size(), 1) * sizeof(T), st);
  if (e != cudaSuccess) { *d = nullptr; return e; }
  if (!v.empty()) e = cudaMemcpyAsync(*d, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, st);
  return e;
}

static void base_batch(const Family *f, LcsBatch &b) {
  b.peq = f->d_peq;
  b.colres = f->d_colres;
  b.group_off = f->d_group_off;
  b.group_chunks = f->d_group_chunks;
  b.col_perm = f->d_perm;
  b.col_len = f->d_slen;
  b.n_cols = f->k;
  b.k = f->k;
}

}  // namespace famsa

using namespace famsa;

extern "C" {

const char *famsa_strerror(int status) {
  switch (status) {
    case FAMSA_OK: return "success";
    case FAMSA_EINVAL: return "invalid argument (k < 1, NULL pointer, bad offsets, empty sequence, residue code >= 25 or bad range)";
    case FAMSA_ERANGE: return "out of range (sequence longer than 65535 or output larger than 2^31-1 entries)";
    case FAMSA_ENOMEM: return "out of memory";
    case FAMSA_ECUDA: return "CUDA error";
    case FAMSA_ETIMEOUT: return "device-side wait timed out";
    case FAMSA_ECANCELED: return "request cancelled before it started";
    case FAMSA_EBUSY: return "busy (queue full)";
    case FAMSA_ELIMIT: return "beyond the fixed scratch limits of famsa_lcs_query_noalloc (queries, or query length)";
    default: return "unknown status";
  }
}

int famsa_version(void) { return 10000; }

int famsa_encode_ascii(const char *text, int64_t n, uint8_t *codes, int64_t *bad_pos) {
  if (bad_pos) *bad_pos = -1;
  if (!text || !codes || n < 0) return FAMSA_EINVAL;
  static const char kAlphabet[] = "ACDEFGHIKLMNPQRSTVWYBZXUO";  // code = index
  int8_t table[256];
  for (int c = 0; c < 256; ++c) table[c] = -1;
  for (int i = 0; i < kCodes; ++i) {
    table[(unsigned char)kAlphabet[i]] = (int8_t)i;
    table[(unsigned char)(kAlphabet[i] - 'A' + 'a')] = (int8_t)i;
  }
  for (int64_t i = 0; i < n; ++i) {
    if (table[(unsigned char)text[i]] < 0) {
      if (bad_pos) *bad_pos = i;
      return FAMSA_EINVAL;
    }
  }
  for (int64_t i = 0; i < n; ++i) codes[i] = (uint8_t)table[(unsigned char)text[i]];
  return FAMSA_OK;
}

int famsa_pack_peq(const uint8_t *residues, const int64_t *offsets, int32_t k,
                   int residues_on_device, void *cuda_stream, famsa_family **out) {
  TraceRange trace("famsa_pack_peq");
  if (!out) return FAMSA_EINVAL;
  *out = nullptr;
  if (!residues || !offsets || k < 1) return FAMSA_EINVAL;
  if (!residues_on_device) {
    for (int32_t i = 0; i < k; ++i)
      if (offsets[i + 1] <= offsets[i]) return FAMSA_EINVAL;
    for (int32_t i = 0; i < k; ++i)
      if (offsets[i + 1] - offsets[i] > kMaxLen) return FAMSA_ERANGE;
  }
  Family *f = nullptr;
  int rc = pack_family(residues, offsets, k, residues_on_device != 0, (cudaStream_t)cuda_stream, &f);
  if (rc != FAMSA_OK) return rc;
  *out = reinterpret_cast<famsa_family *>(f);
  return FAMSA_OK;
}

int32_t famsa_family_size(const famsa_family *fh) {
  return fh ? reinterpret_cast<const Family *>(fh)->k : -1;
}

void famsa_free(famsa_family *fh) {
  if (!fh) return;
  Family *f = reinterpret_cast<Family *>(fh);
  {
    std::lock_guard<std::mutex> lk(f->mu);
    cudaDeviceSynchronize();
  }
  free_family(f);
}

int famsa_last_stats(const famsa_family *fh, int64_t *stats) {
  if (!fh || !stats) return FAMSA_EINVAL;
  const Family *f = reinterpret_cast<const Family *>(fh);
  for (int i = 0; i < kStatsLen; ++i) stats[i] = f->stats[i];
  stats[11] = f->pack_launches;
  return FAMSA_OK;
}

int famsa_lcs_allpairs(const famsa_family *fh, int32_t *lcs_out, int out_on_device,
                       void *cuda_stream) {
  TraceRange trace("famsa_lcs_allpairs");
  if (!fh || !lcs_out) return FAMSA_EINVAL;
  Family *f = const_cast<Family *>(reinterpret_cast<const Family *>(fh));
  std::lock_guard<std::mutex> lk(f->mu);
  cudaStream_t st = (cudaStream_t)cuda_stream;
  const int64_t k = f->k;
  const int64_t n = k * (k - 1) / 2;
  if (n > INT32_MAX) return FAMSA_ERANGE;
  if (n == 0) return FAMSA_OK;
  cudaError_t err = cudaSuccess;
  int32_t *d_out = lcs_out;
  RowList rl;
  host_row_list(f, rl);
  if (!out_on_device) {
    err = lib_malloc_async((void **)&d_out, sizeof(int32_t) * n, st);
    if (err != cudaSuccess) return status_from_cuda(err);
  }
  err = upload(rl.id, &rl.d_id, st);
  if (err == cudaSuccess) {
    LcsBatch b;
    base_batch(f, b);
    b.row_peq_off = f->d_peq_off;
    b.row_len = f->d_slen;
    b.row_id = rl.d_id;
    b.row_orig = f->d_perm;
    b.n_rows = f->k;
    b.h_row_w = rl.w.data();
    b.h_row_id = rl.id.data();
    b.mode = kOutTriOrig;
    b.out = d_out;
    b.triangle = true;
    int64_t launches = 0;
    err = launch_lcs(b, st, &launches);
  }
  if (err == cudaSuccess && !out_on_device)
    err = cudaMemcpyAsync(lcs_out, d_out, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, st);
  if (rl.d_id) cudaFreeAsync(rl.d_id, st);
  if (!out_on_device) cudaFreeAsync(d_out, st);
  if (err == cudaSuccess && !out_on_device) err = cudaStreamSynchronize(st);
  return status_from_cuda(err);
}

int famsa_lcs_rows(const famsa_family *fh, int32_t row_begin, int32_t row_end, int32_t *out,
                   int out_on_device, void *cuda_stream) {
  TraceRange trace("famsa_lcs_rows");
  if (!fh) return FAMSA_EINVAL;
  Family *f = const_cast<Family *>(reinterpret_cast<const Family *>(fh));
  if (row_begin < 0 || row_end < row_begin || row_end > f->k) return FAMSA_EINVAL;
  const int64_t n = ((int64_t)row_end * (row_end - 1) - (int64_t)row_begin * (row_begin - 1)) / 2;
  if (n > INT32_MAX) return FAMSA_ERANGE;
  if (n == 0) return FAMSA_OK;
  if (!out) return FAMSA_EINVAL;
  std::lock_guard<std::mutex> lk(f->mu);
  cudaStream_t st = (cudaStream_t)cuda_stream;
  // rows: sorted positions of the requested original rows, ascending (width nondecreasing)
  std::vector<int32_t> rank(f->k);
  for (int32_t s = 0; s < f->k; ++s) rank[f->h_perm[s]] = s;
  std::vector<int32_t> ids;
  for (int32_t i = std::max(row_begin, 1); i < row_end; ++i) ids.push_back(rank[i]);
  std::sort(ids.begin(), ids.end());
  const size_t m = ids.size();
  std::vector<int32_t> w(m), orig(m), len(m);
  for (size_t e = 0; e < m; ++e) {
    len[e] = f->h_slen[ids[e]];
    w[e] = (len[e] + 63) / 64;
    orig[e] = f->h_perm[ids[e]];
  }
  // per-entry Peq offsets are gathered on the device from the family's table
  cudaError_t err = cudaSuccess;
  int32_t *d_out = out, *d_ids = nullptr, *d_orig = nullptr, *d_len = nullptr;
  int64_t *d_po = nullptr;
  std::vector<int64_t> h_po(m);
  {
    std::vector<int64_t> all(f->k + 1);
    err = cudaMemcpyAsync(all.data(), f->d_peq_off, sizeof(int64_t) * (f->k + 1),
                          cudaMemcpyDeviceToHost, st);
    if (err == cudaSuccess) err = cudaStreamSynchronize(st);
    for (size_t e = 0; e < m; ++e) h_po[e] = all[ids[e]];
  }
  if (err == cudaSuccess && !out_on_device)
    err = lib_malloc_async((void **)&d_out, sizeof(int32_t) * n, st);
  if (err == cudaSuccess) err = upload(ids, &d_ids, st);
  if (err == cudaSuccess) err = upload(orig, &d_orig, st);
  if (err == cudaSuccess) err = upload(len, &d_len, st);
  if (err == cudaSuccess) err = upload(h_po, &d_po, st);
  if (err == cudaSuccess) {
    LcsBatch b;
    base_batch(f, b);
    b.row_peq_off = d_po;
    b.row_len = d_len;
    b.row_id = d_ids;
    b.row_orig = d_orig;
    b.n_rows = (int32_t)m;
    b.h_row_w = w.data();
    b.h_row_id = ids.data();
    b.mode = kOutRowsOrig;
    b.out = d_out;
    b.row0 = row_begin;
    b.triangle = false;
    int64_t launches = 0;
    err = launch_lcs(b, st, &launches);
  }
  if (err == cudaSuccess && !out_on_device)
    err = cudaMemcpyAsync(out, d_out, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, st);
  if (d_ids) cudaFreeAsync(d_ids, st);
  if (d_orig) cudaFreeAsync(d_orig, st);
  if (d_len) cudaFreeAsync(d_len, st);
  if (d_po) cudaFreeAsync(d_po, st);
  if (!out_on_device && d_out) cudaFreeAsync(d_out, st);
  if (err == cudaSuccess && !out_on_device) err = cudaStreamSynchronize(st);
  return status_from_cuda(err);
}

int famsa_lcs_query(const famsa_family *fh, const uint8_t *q, const int64_t *q_offsets,
                    int32_t nq, int q_on_device, int32_t *out, int out_on_device,
                    void *cuda_stream) {
  TraceRange trace("famsa_lcs_query");
  if (!fh || !q || !q_offsets || !out || nq < 1) return FAMSA_EINVAL;
  Family *f = const_cast<Family *>(reinterpret_cast<const Family *>(fh));
  std::lock_guard<std::mutex> lk(f->mu);
  cudaStream_t st = (cudaStream_t)cuda_stream;
  cudaError_t err = cudaSuccess;
  const uint8_t *d_q = q;
  const int64_t *d_qoff = q_offsets;
  uint8_t *own_q = nullptr;
  int64_t *own_off = nullptr;
  if (!q_on_device) {
    for (int32_t i = 0; i < nq; ++i)
      if (q_offsets[i + 1] <= q_offsets[i]) return FAMSA_EINVAL;
    int64_t total = q_offsets[nq];
    err = lib_malloc_async((void **)&own_q, std::max<int64_t>(total, 1), st);
    if (err == cudaSuccess) err = lib_malloc_async((void **)&own_off, sizeof(int64_t) * (nq + 1), st);
    if (err == cudaSuccess) err = cudaMemcpyAsync(own_q, q, total, cudaMemcpyHostToDevice, st);
    if (err == cudaSuccess)
      err = cudaMemcpyAsync(own_off, q_offsets, sizeof(int64_t) * (nq + 1), cudaMemcpyHostToDevice, st);
    if (err != cudaSuccess) {
      if (own_q) cudaFreeAsync(own_q, st);
      if (own_off) cudaFreeAsync(own_off, st);
      return status_from_cuda(err);
    }
    d_q = own_q;
    d_qoff = own_off;
  }
  uint32_t *qpeq = nullptr;
  int64_t *qpo = nullptr;
  int32_t *qlen = nullptr;
  std::vector<int32_t> h_len;
  int rc = pack_rows(d_q, d_qoff, nq, st, &qpeq, &qpo, &qlen, h_len);
  if (rc != FAMSA_OK) {
    if (own_q) cudaFreeAsync(own_q, st);
    if (own_off) cudaFreeAsync(own_off, st);
    cudaStreamSynchronize(st);
    return rc;
  }
  // rows sorted by width
  std::vector<int32_t> order(nq);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) { return h_len[a] < h_len[b]; });
  std::vector<int64_t> po_all(nq + 1, 0);
  for (int32_t i = 0; i < nq; ++i) po_all[i + 1] = po_all[i] + (h_len[i] + 63) / 64;
  std::vector<int32_t> w(nq), len(nq);
  std::vector<int64_t> po(nq);
  for (int32_t e = 0; e < nq; ++e) {
    int32_t i = order[e];
    len[e] = h_len[i];
    w[e] = (h_len[i] + 63) / 64;
    po[e] = po_all[i];
  }
  const int64_t n = (int64_t)nq * f->k;
  int32_t *d_out = out, *d_ids = nullptr, *d_len = nullptr;
  int64_t *d_po = nullptr;
  if (!out_on_device) err = lib_malloc_async((void **)&d_out, sizeof(int32_t) * n, st);
  if (err == cudaSuccess) err = upload(order, &d_ids, st);
  if (err == cudaSuccess) err = upload(len, &d_len, st);
  if (err == cudaSuccess) err = upload(po, &d_po, st);
  if (err == cudaSuccess) {
    LcsBatch b;
    base_batch(f, b);
    b.peq = qpeq;
    b.row_peq_off = d_po;
    b.row_len = d_len;
    b.row_id = d_ids;
    b.n_rows = nq;
    b.h_row_w = w.data();
    b.h_row_id = order.data();
    b.mode = kOutQuery;
    b.out = d_out;
    b.ld = f->k;
    b.triangle = false;
    int64_t launches = 0;
    err = launch_lcs(b, st, &launches);
  }
  if (err == cudaSuccess && !out_on_device)
    err = cudaMemcpyAsync(out, d_out, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, st);
  if (d_ids) cudaFreeAsync(d_ids, st);
  if (d_len) cudaFreeAsync(d_len, st);
  if (d_po) cudaFreeAsync(d_po, st);
  if (!out_on_device && d_out) cudaFreeAsync(d_out, st);
  cudaFreeAsync(qpeq, st);
  cudaFreeAsync(qpo, st);
  cudaFreeAsync(qlen, st);
  if (own_q) cudaFreeAsync(own_q, st);
  if (own_off) cudaFreeAsync(own_off, st);
  if (err == cudaSuccess && !out_on_device) err = cudaStreamSynchronize(st);
  return status_from_cuda(err);
}

int famsa_slink_tree(const famsa_family *fh, int32_t *pi, uint64_t *lambda_num,
                     uint32_t *lambda_den, int32_t *merges, uint64_t *h_num, uint32_t *h_den,
                     int32_t *sizes, int out_on_device, void *cuda_stream) {
  TraceRange trace("famsa_slink_tree");
  if (!fh) return FAMSA_EINVAL;
  Family *f = const_cast<Family *>(reinterpret_cast<const Family *>(fh));
  std::lock_guard<std::mutex> lk(f->mu);
  return slink_tree(f, pi, lambda_num, lambda_den, merges, h_num, h_den, sizes,
                    out_on_device != 0, (cudaStream_t)cuda_stream);
}

}  // extern "C"
