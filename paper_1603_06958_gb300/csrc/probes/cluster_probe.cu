// Latency of the row update's building blocks on one thread-block cluster,
// in SM clocks per repetition (clock64 of thread 0 of CTA 0): the 512-thread
// block clamp scan with either key type, a cluster barrier alone and after
// every CTA pushed a clamp to every other CTA, and a chain of dependent loads
// from local shared memory and from another CTA's shared memory (DSMEM).
// These are the figures behind the choice of the order-code keys and of
// pushing the cross-CTA values before a barrier.
#include "famsa_probe.h"
#include "../slink_common.cuh"

namespace famsa {

constexpr int kProbeThreads = 512;
constexpr int kProbeSlots = 2048;

__device__ __forceinline__ uint64_t probe_key(uint32_t a, uint32_t b, bool narrow) {
  const uint32_t num = a % 100000u, den = 1u + b % 30000u;
  return narrow ? order_code(num, den) : (((uint64_t)num << 16) | den);
}

template <class K, int V>
__global__ void __launch_bounds__(kProbeThreads, 1) k_cluster_probe(int iters, unsigned long long *out,
                                                                    uint64_t *sink) {
  cg::cluster_group cluster = cg::this_cluster();
  const int ncta = (int)cluster.num_blocks();
  const int cta = (int)cluster.block_rank();
  __shared__ Clamp sw[130];
  __shared__ Clamp sAgg[kMaxClusterCtas];
  __shared__ uint64_t dd[kProbeSlots], gg[kProbeSlots];
  __shared__ uint32_t nxt[1024];
  const bool narrow = K::kInf == KeysNarrow::kInf;
  for (int i = threadIdx.x; i < kProbeSlots; i += blockDim.x) {
    dd[i] = probe_key(i * 7919u + cta, i, narrow);
    gg[i] = probe_key(i * 104729u, i + 3, narrow);
  }
  for (int i = threadIdx.x; i < 1024; i += blockDim.x) nxt[i] = (i * 97u + 13u) & 1023u;
  cluster.sync();
  uint64_t acc = 0;
  uint32_t idx = 0;
  const long long t0 = clock64();
  for (int it = 0; it < iters; ++it) {
    if (V == 0) {  // block scan of both clamp directions
      const int t = threadIdx.x;
      Clamp sl = Clamp{gg[t] ^ (acc & 1), dd[t]}, sr = Clamp{gg[t + 1], dd[t + 1] ^ (acc & 1)};
      Clamp pl, pr, tl, tr;
      block_scan2<K>(sl, sr, &pl, &pr, &tl, &tr, sw);
      acc += pl.hi ^ pr.lo ^ tl.hi ^ tr.lo;
      __syncthreads();
    } else if (V == 1) {  // cluster barrier alone
      cluster.sync();
      acc += 1;
    } else if (V == 2) {  // one clamp pushed to every CTA, then the barrier
      if ((int)threadIdx.x < ncta) cluster.map_shared_rank(sAgg, (int)threadIdx.x)[cta] = Clamp{acc, acc + 1};
      cluster.sync();
      acc += sAgg[(it + 1) % ncta].lo;
    } else if (V == 3) {  // dependent local shared-memory loads (thread 0 of CTA 0)
      if (threadIdx.x == 0 && cta == 0) idx = nxt[idx];
    } else {  // dependent loads from the next CTA's shared memory
      if (threadIdx.x == 0 && cta == 0) idx = cluster.map_shared_rank(nxt, 1 % ncta)[idx];
    }
  }
  const long long t1 = clock64();
  if (threadIdx.x == 0 && cta == 0) out[0] = (unsigned long long)(t1 - t0);
  sink[blockIdx.x * blockDim.x + threadIdx.x] = acc + idx;
  cluster.sync();
}

template <class K, int V>
static cudaError_t run_probe(int cl, int iters, unsigned long long *out, uint64_t *sink) {
  cudaError_t e = cudaFuncSetAttribute(k_cluster_probe<K, V>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)cl, 1, 1);
  cfg.blockDim = dim3(kProbeThreads, 1, 1);
  cudaLaunchAttribute attr;
  attr.id = cudaLaunchAttributeClusterDimension;
  attr.val.clusterDim.x = (unsigned)cl;
  attr.val.clusterDim.y = 1;
  attr.val.clusterDim.z = 1;
  cfg.attrs = &attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_cluster_probe<K, V>, iters, out, sink);
}

}  // namespace famsa

extern "C" int famsa_probe_cluster(int kind, int cluster_ctas, double *cycles) {
  using namespace famsa;
  if (kind < 0 || kind > 5 || !cycles) return FAMSA_EINVAL;
  if (cluster_ctas != 1 && cluster_ctas != 2 && cluster_ctas != 4 && cluster_ctas != 8 && cluster_ctas != 16)
    return FAMSA_EINVAL;
  const int iters = 4096;
  unsigned long long *out = nullptr;
  uint64_t *sink = nullptr;
  cudaError_t err = cudaMalloc((void **)&out, sizeof(unsigned long long));
  if (err == cudaSuccess) err = cudaMalloc((void **)&sink, sizeof(uint64_t) * kMaxClusterCtas * kProbeThreads);
  if (err == cudaSuccess) {
    switch (kind) {
      case 0: err = run_probe<KeysNarrow, 0>(cluster_ctas, iters, out, sink); break;
      case 1: err = run_probe<KeysWide, 0>(cluster_ctas, iters, out, sink); break;
      case 2: err = run_probe<KeysNarrow, 1>(cluster_ctas, iters, out, sink); break;
      case 3: err = run_probe<KeysNarrow, 2>(cluster_ctas, iters, out, sink); break;
      case 4: err = run_probe<KeysNarrow, 3>(cluster_ctas, iters, out, sink); break;
      default: err = run_probe<KeysNarrow, 4>(cluster_ctas, iters, out, sink); break;
    }
  }
  unsigned long long h = 0;
  if (err == cudaSuccess) err = cudaDeviceSynchronize();
  if (err == cudaSuccess) err = cudaMemcpy(&h, out, sizeof(h), cudaMemcpyDeviceToHost);
  cudaFree(out);
  cudaFree(sink);
  if (err != cudaSuccess) return (err == cudaErrorMemoryAllocation ? FAMSA_ENOMEM : FAMSA_ECUDA);
  *cycles = (double)h / iters;
  return FAMSA_OK;
}
