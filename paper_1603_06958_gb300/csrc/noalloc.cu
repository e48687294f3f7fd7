// famsa_lcs_query_noalloc: the query LCS (as famsa_lcs_query) with its
// scratch in a fixed device array instead of memory allocated per call.
//
// Who needs it: callers whose device memory is all handed out up front (a
// serving process that reserves its whole budget in its own arena, or runs
// next to another framework that owns the rest of the GPU) cannot get more
// at request time, and on a latency-bound request path an allocation may
// also wait for the device.  This variant uses only the caller's buffers and
// the fixed array below.
//
// The array holds the queries' match-bitmask (Peq) tables and the per-query
// row list the LCS kernels read.  Every call writes all of it that the call
// then reads, so the contents left by an earlier call do no harm; the only
// word that must start at zero (the validation status) is cleared by the
// first kernel of each call.
#include <mutex>

#include "famsa_gpu.h"
#include "famsa_internal.cuh"

namespace famsa {

constexpr int32_t kNoAllocMaxQueries = FAMSA_NOALLOC_MAX_QUERIES;
constexpr int32_t kNoAllocMaxLen = FAMSA_NOALLOC_MAX_LEN;
constexpr int32_t kNoAllocMaxW = (kNoAllocMaxLen + 63) / 64;
constexpr size_t kNoAllocPeqBytes =
    sizeof(uint32_t) * kPeqWordU32 * (size_t)kNoAllocMaxQueries * kNoAllocMaxW;
constexpr size_t kNoAllocMetaBytes = 4096;
constexpr size_t kNoAllocScratchBytes = kNoAllocPeqBytes + kNoAllocMetaBytes;
static_assert(kNoAllocScratchBytes == FAMSA_NOALLOC_SCRATCH_BYTES, "scratch size differs from the header");
static_assert(kNoAllocMaxQueries * (sizeof(int64_t) + 2 * sizeof(int32_t)) + sizeof(int32_t) <=
                  kNoAllocMetaBytes,
              "row list does not fit the metadata block");

// 1 MiB of Peq words plus 4 KiB of row list, one copy per device.
static __device__ __align__(256) uint8_t g_noalloc_scratch[kNoAllocScratchBytes];

struct NoAllocView {
  uint32_t *peq;      // [query][word][64] u32
  int64_t *peq_off;   // per query: first word of its Peq (query * W)
  int32_t *len;       // per query: length (0 when invalid)
  int32_t *id;        // per query: its index
  int32_t *status;    // bit 0: a bad length or residue code
};

static NoAllocView view_of(void *base) {
  uint8_t *b = static_cast<uint8_t *>(base);
  NoAllocView v;
  v.peq = reinterpret_cast<uint32_t *>(b);
  uint8_t *meta = b + kNoAllocPeqBytes;
  v.peq_off = reinterpret_cast<int64_t *>(meta);
  v.len = reinterpret_cast<int32_t *>(meta + sizeof(int64_t) * kNoAllocMaxQueries);
  v.id = v.len + kNoAllocMaxQueries;
  v.status = v.id + kNoAllocMaxQueries;
  return v;
}

// One block of kNoAllocMaxQueries threads: the row list of nq queries, each
// given W words, and the status cleared then set for bad lengths.
__global__ void k_noalloc_rows(const int64_t *q_off, int32_t nq, int32_t max_len, int32_t W,
                               NoAllocView v) {
  __shared__ int bad;
  if (threadIdx.x == 0) bad = 0;
  __syncthreads();
  const int32_t s = threadIdx.x;
  if (s < nq) {
    const int64_t l = q_off[s + 1] - q_off[s];
    const bool ok = l >= 1 && l <= max_len;
    if (!ok) atomicOr(&bad, 1);
    v.len[s] = ok ? (int32_t)l : 0;
    v.id[s] = s;
    v.peq_off[s] = (int64_t)s * W;
  }
  __syncthreads();
  if (threadIdx.x == 0) *v.status = bad;
}

// One warp per (query, word): bit b of plane h of code c is set iff
// residue 64*word + 32*h + b of the query is c; every word of the query's
// W-word slot is written (codes 25..31 and positions past the length are 0).
__global__ void k_noalloc_peq(const uint8_t *q, const int64_t *q_off, int32_t nq, int32_t W,
                              NoAllocView v) {
  const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (gw >= (int64_t)nq * W) return;
  const int32_t s = (int32_t)(gw / W), w = (int32_t)(gw - (int64_t)s * W);
  const int32_t len = v.len[s];
  const uint8_t *a = q + q_off[s];
  const int32_t p0 = w * 64 + lane, p1 = p0 + 32;
  const int c0 = p0 < len ? a[p0] : 255;
  const int c1 = p1 < len ? a[p1] : 255;
  const bool badc = (p0 < len && c0 >= kCodes) || (p1 < len && c1 >= kCodes);
  if (__any_sync(0xffffffffu, badc) && lane == 0) atomicOr(v.status, 1);
  uint32_t mylo = 0, myhi = 0;
#pragma unroll
  for (int c = 0; c < kCodes; ++c) {
    const uint32_t lo = __ballot_sync(0xffffffffu, c0 == c);
    const uint32_t hi = __ballot_sync(0xffffffffu, c1 == c);
    if (lane == c) { mylo = lo; myhi = hi; }
  }
  uint32_t *dst = v.peq + ((int64_t)s * W + w) * kPeqWordU32;
  dst[lane] = mylo;
  dst[32 + lane] = myhi;
}

constexpr int kNoAllocMaxDevices = 64;
static std::mutex g_noalloc_mu;       // the per-device address table
static std::mutex g_noalloc_call_mu;  // one call at a time owns the array
static void *g_noalloc_ptr[kNoAllocMaxDevices] = {nullptr};

// Device address of the array on the current device, looked up once per
// device (the first call on a device does this).
static int noalloc_scratch(void **out) {
  int dev = -1;
  cudaError_t err = cudaGetDevice(&dev);
  if (err != cudaSuccess) return status_from_cuda(err);
  if (dev < 0 || dev >= kNoAllocMaxDevices) return FAMSA_ECUDA;
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void *ptr = nullptr;
    err = cudaGetSymbolAddress((void **)&ptr, g_noalloc_scratch);
    if (err != cudaSuccess || !ptr) return FAMSA_ECUDA;
    g_noalloc_ptr[dev] = ptr;
  }
  *out = g_noalloc_ptr[dev];
  return FAMSA_OK;
}

}  // namespace famsa

using namespace famsa;

extern "C" int famsa_lcs_query_noalloc(const famsa_family *fh, const uint8_t *q,
                                       const int64_t *q_offsets, int32_t nq, int32_t max_len,
                                       int32_t *out, void *cuda_stream) {
  if (!fh || !q || !q_offsets || !out || nq < 1 || max_len < 1) return FAMSA_EINVAL;
  if (nq > kNoAllocMaxQueries || max_len > kNoAllocMaxLen) return FAMSA_ELIMIT;
  Family *f = const_cast<Family *>(reinterpret_cast<const Family *>(fh));
  void *base = nullptr;
  int rc = noalloc_scratch(&base);
  if (rc != FAMSA_OK) return rc;
  const NoAllocView v = view_of(base);
  const int32_t W = (max_len + 63) / 64;
  // held from the first launch until the stream has finished (the call waits
  // for it anyway), so calls from other threads cannot interleave their
  // kernels with this call's use of the shared array
  std::lock_guard<std::mutex> call_lk(g_noalloc_call_mu);
  std::lock_guard<std::mutex> lk(f->mu);
  cudaStream_t st = (cudaStream_t)cuda_stream;
  k_noalloc_rows<<<1, kNoAllocMaxQueries, 0, st>>>(q_offsets, nq, max_len, W, v);
  const int64_t warps = (int64_t)nq * W;
  const int T = 256;
  k_noalloc_peq<<<(unsigned)((warps * 32 + T - 1) / T), T, 0, st>>>(q, q_offsets, nq, W, v);
  cudaError_t err = cudaGetLastError();
  if (err != cudaSuccess) return status_from_cuda(err);
  // every query gets the same W, so the planner makes one launch
  int32_t h_w[kNoAllocMaxQueries];
  for (int32_t i = 0; i < nq; ++i) h_w[i] = W;
  LcsBatch b;
  b.peq = v.peq;
  b.row_peq_off = v.peq_off;
  b.row_len = v.len;
  b.row_id = v.id;
  b.n_rows = nq;
  b.h_row_w = h_w;
  b.colres = f->d_colres;
  b.group_off = f->d_group_off;
  b.group_chunks = f->d_group_chunks;
  b.col_perm = f->d_perm;
  b.col_len = f->d_slen;
  b.n_cols = f->k;
  b.k = f->k;
  b.mode = kOutQuery;
  b.out = out;
  b.ld = f->k;
  b.triangle = false;
  int64_t launches = 0;
  err = launch_lcs(b, st, &launches);
  if (err != cudaSuccess) return status_from_cuda(err);
  // the validation status comes back to the host (the call waits for its stream)
  int32_t h_status = 0;
  err = cudaMemcpyAsync(&h_status, v.status, sizeof(int32_t), cudaMemcpyDeviceToHost, st);
  if (err == cudaSuccess) err = cudaStreamSynchronize(st);
  if (err != cudaSuccess) return status_from_cuda(err);
  return h_status ? FAMSA_EINVAL : FAMSA_OK;
}
