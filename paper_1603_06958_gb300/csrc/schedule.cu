// famsa_progressive_schedule: the merge list in the form the progressive
// stage consumes.
//
// FAMSA Methods, "Progressive construction of the alignment": the third stage
// makes O(k) profile alignments in guide-tree order and spreads them over
// threads; at least half of them are degenerate -- one side a single
// sequence -- and take a simpler DP.  So the schedule gives each merge its
// level (1 + the larger level of its children; a sequence is level 0):
// merges of one level never use one another and can run at once, once the
// levels below are done.  The merges are ordered by (level, index), with the
// start of each level, and each is marked as two sequences, a sequence and a
// profile, or two profiles.
#include <algorithm>

#include "slink_common.cuh"

using namespace famsa;

namespace {

constexpr int kSchedThreads = 1024, kSchedChunk = 2048;
constexpr int32_t kSchedSmem = 50000;  // levels of up to this many merges live in shared memory

// Levels, in merge order (a child is always an earlier merge or a sequence).
// One thread walks the merges -- each level depends on the two before it in
// the tree -- while the block stages the next chunk of merges; the levels sit
// in shared memory when they fit.  A child id out of range sets *bad.
__global__ void __launch_bounds__(kSchedThreads) k_sched_levels(int32_t k, const int32_t *merges, int32_t *level,
                                                                int32_t *top_out, int32_t *bad_out, int use_smem) {
  extern __shared__ int32_t sm[];
  int32_t *ca = sm, *cb = ca + kSchedChunk;
  int32_t *lev = use_smem ? cb + kSchedChunk : level;
  const int32_t n = k - 1;
  int32_t top = 0, bad = 0;
  for (int32_t c0 = 0; c0 < n; c0 += kSchedChunk) {
    const int32_t cn = min(kSchedChunk, n - c0);
    for (int32_t j = threadIdx.x; j < cn; j += kSchedThreads) {
      ca[j] = merges[2 * (int64_t)(c0 + j)];
      cb[j] = merges[2 * (int64_t)(c0 + j) + 1];
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      for (int32_t j = 0; j < cn; ++j) {
        const int32_t t = c0 + j, a = ca[j], b = cb[j];
        int32_t la = 0, lb = 0;
        if (a < 0 || b < 0 || a >= k + t || b >= k + t) {
          bad = 1;
        } else {
          if (a >= k) la = lev[a - k];
          if (b >= k) lb = lev[b - k];
        }
        const int32_t l = 1 + max(la, lb);
        lev[t] = l;
        top = max(top, l);
      }
    }
    __syncthreads();
  }
  if (use_smem)
    for (int32_t t = threadIdx.x; t < n; t += kSchedThreads) level[t] = lev[t];
  if (threadIdx.x == 0) {
    *top_out = top;
    *bad_out = bad;
  }
}

__global__ void k_sched_kind(int32_t k, const int32_t *merges, const int32_t *sizes, int32_t *kind) {
  const int32_t t = (int32_t)(blockIdx.x * blockDim.x + threadIdx.x);
  if (t >= k - 1) return;
  const int32_t a = merges[2 * (int64_t)t], b = merges[2 * (int64_t)t + 1];
  const bool pa = a >= k && a < k + t && sizes[a - k] > 1;
  const bool pb = b >= k && b < k + t && sizes[b - k] > 1;
  kind[t] = (int32_t)pa + (int32_t)pb;
}

struct ByLevel {
  const int32_t *level;
  __device__ bool operator()(int32_t x, int32_t y) const {
    return level[x] != level[y] ? level[x] < level[y] : x < y;
  }
};

__global__ void k_sched_iota(int32_t *o, int32_t n) {
  const int32_t i = (int32_t)(blockIdx.x * blockDim.x + threadIdx.x);
  if (i < n) o[i] = i;
}

__global__ void k_sched_msort(const int32_t *in, int32_t *out, int32_t n, int32_t width, ByLevel cmp) {
  const int32_t i = (int32_t)(blockIdx.x * blockDim.x + threadIdx.x);
  if (i < n) msort_at(i, in, out, n, width, cmp);
}

// level l (1-based) starts at the first position of the sorted order that
// holds it; levels are 1..top without gaps (a level-l merge has a child at l-1)
__global__ void k_sched_starts(int32_t n, const int32_t *order, const int32_t *level, const int32_t *top,
                               int32_t *start) {
  const int32_t p = (int32_t)(blockIdx.x * blockDim.x + threadIdx.x);
  if (p >= n) return;
  const int32_t l = level[order[p]];
  if (p == 0 || level[order[p - 1]] != l) start[l - 1] = p;
  if (p == n - 1) start[*top] = n;
}

inline unsigned nb(int64_t n, int t) { return (unsigned)std::max<int64_t>((n + t - 1) / t, 1); }

}  // namespace

extern "C" int famsa_progressive_schedule(int32_t k, const int32_t *merges, const int32_t *sizes, int32_t *level,
                                          int32_t *order, int32_t *level_start, int32_t *kind,
                                          int32_t *n_levels, int on_device, void *cuda_stream) {
  if (k < 1 || !n_levels) return FAMSA_EINVAL;
  if (k >= 2 && (!merges || !sizes || !level || !order || !level_start || !kind)) return FAMSA_EINVAL;
  *n_levels = 0;
  if (k == 1) return FAMSA_OK;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  const int32_t n = k - 1;
  Scratch sc;
  sc.st = st;
  const int32_t *dm = merges, *ds = sizes;
  int32_t *dl = level, *dord = order, *dst = level_start, *dk = kind;
  if (!on_device) {
    int32_t *m2 = sc.get<int32_t>(2 * (size_t)n), *s2 = sc.get<int32_t>(n);
    dl = sc.get<int32_t>(n);
    dord = sc.get<int32_t>(n);
    dst = sc.get<int32_t>((size_t)n + 1);
    dk = sc.get<int32_t>(n);
    if (sc.err == cudaSuccess) {
      cudaMemcpyAsync(m2, merges, sizeof(int32_t) * 2 * (size_t)n, cudaMemcpyHostToDevice, st);
      cudaMemcpyAsync(s2, sizes, sizeof(int32_t) * (size_t)n, cudaMemcpyHostToDevice, st);
    }
    dm = m2;
    ds = s2;
  }
  int32_t *tmp = sc.get<int32_t>(n), *ctl = sc.get<int32_t>(2);
  if (sc.err != cudaSuccess) {
    cudaError_t e = sc.err;
    cudaStreamSynchronize(st);
    sc.release();
    return status_from_cuda(e);
  }
  const int use_smem = n <= kSchedSmem;
  const size_t smem = sizeof(int32_t) * (2 * kSchedChunk + (use_smem ? (size_t)n : 0));
  // the cap is per kernel: set the largest any call needs, so that calls on
  // other streams never lower it under this launch
  const size_t smem_max = sizeof(int32_t) * (2 * kSchedChunk + (size_t)kSchedSmem);
  cudaError_t err = cudaFuncSetAttribute(k_sched_levels, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_max);
  if (err == cudaSuccess) {
    k_sched_levels<<<1, kSchedThreads, smem, st>>>(k, dm, dl, ctl, ctl + 1, use_smem);
    k_sched_kind<<<nb(n, 256), 256, 0, st>>>(k, dm, ds, dk);
    k_sched_iota<<<nb(n, 256), 256, 0, st>>>(dord, n);
    int32_t *a = dord, *b = tmp;
    for (int64_t w = 1; w < n; w *= 2) {
      k_sched_msort<<<nb(n, 256), 256, 0, st>>>(a, b, n, (int32_t)w, ByLevel{dl});
      std::swap(a, b);
    }
    if (a != dord) cudaMemcpyAsync(dord, a, sizeof(int32_t) * (size_t)n, cudaMemcpyDeviceToDevice, st);
    k_sched_starts<<<nb(n, 256), 256, 0, st>>>(n, dord, dl, ctl, dst);
    err = cudaGetLastError();
  }
  int32_t hctl[2] = {0, 0};
  if (err == cudaSuccess) err = cudaMemcpyAsync(hctl, ctl, sizeof(hctl), cudaMemcpyDeviceToHost, st);
  if (err == cudaSuccess && !on_device) {
    cudaMemcpyAsync(level, dl, sizeof(int32_t) * (size_t)n, cudaMemcpyDeviceToHost, st);
    cudaMemcpyAsync(order, dord, sizeof(int32_t) * (size_t)n, cudaMemcpyDeviceToHost, st);
    cudaMemcpyAsync(kind, dk, sizeof(int32_t) * (size_t)n, cudaMemcpyDeviceToHost, st);
  }
  if (err == cudaSuccess) err = cudaStreamSynchronize(st);
  if (err == cudaSuccess && !on_device && !hctl[1])
    err = cudaMemcpy(level_start, dst, sizeof(int32_t) * ((size_t)hctl[0] + 1), cudaMemcpyDeviceToHost);
  if (err != cudaSuccess) cudaStreamSynchronize(st);
  sc.release();
  if (err != cudaSuccess) return status_from_cuda(err);
  if (hctl[1]) return FAMSA_EINVAL;
  *n_levels = hctl[0];
  return FAMSA_OK;
}
