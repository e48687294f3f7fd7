// Integer pipe rates of the GPU, for the roofline of the LCS kernels.
//
// The bit-parallel LCS step needs LOP3 and 32-bit adds with carry, which
// issue on the ALU pipe only; IMAD issues on the FMA (heavy) pipe.  These
// kernels run many independent chains of one instruction kind (or an even
// LOP3/IMAD mix) so the measured instruction rate shows each pipe's width.
#include "../famsa_internal.cuh"
#include "famsa_probe.h"

namespace famsa {

constexpr int kPeakChains = 16;

template <int M>
__global__ void __launch_bounds__(256) k_int_peak(uint32_t seed, int iters, uint32_t *out) {
  uint32_t x[kPeakChains];
  const uint32_t y = seed * 7u + threadIdx.x, z = seed ^ (threadIdx.x * 13u);
#pragma unroll
  for (int i = 0; i < kPeakChains; ++i) x[i] = seed + i * 977u + threadIdx.x;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < kPeakChains; ++i) {
      if (M == 0 || (M == 3 && !(i & 1)))
        asm volatile("lop3.b32 %0, %0, %1, %2, 0x96;" : "+r"(x[i]) : "r"(y), "r"(z));
      else if (M == 1)
        asm volatile("{.reg .b32 t; add.u32 t, %0, %1; add.u32 %0, t, %2;}" : "+r"(x[i]) : "r"(y), "r"(z));
      else
        asm volatile("mad.lo.u32 %0, %0, %1, %2;" : "+r"(x[i]) : "r"(y), "r"(z));
    }
  }
  uint32_t s = 0;
#pragma unroll
  for (int i = 0; i < kPeakChains; ++i) s += x[i];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace famsa

extern "C" int famsa_probe_int_pipe_rate(int kind, double *inst_per_s) {
  using namespace famsa;
  if (kind < 0 || kind > 3 || !inst_per_s) return FAMSA_EINVAL;
  int dev = 0, sms = 0;
  cudaError_t err = cudaGetDevice(&dev);
  if (err == cudaSuccess) err = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (err != cudaSuccess) return (err == cudaErrorMemoryAllocation ? FAMSA_ENOMEM : FAMSA_ECUDA);
  const int blocks = sms * 8, threads = 256, iters = 8192;
  uint32_t *out = nullptr;
  err = cudaMalloc((void **)&out, sizeof(uint32_t) * blocks * threads);
  if (err != cudaSuccess) return (err == cudaErrorMemoryAllocation ? FAMSA_ENOMEM : FAMSA_ECUDA);
  cudaEvent_t a = nullptr, b = nullptr;
  float ms = 0.f;
  err = cudaEventCreate(&a);
  if (err == cudaSuccess) err = cudaEventCreate(&b);
  for (int rep = 0; rep < 2 && err == cudaSuccess; ++rep) {
    err = cudaEventRecord(a, 0);
    switch (kind) {
      case 0: k_int_peak<0><<<blocks, threads>>>(1u, iters, out); break;
      case 1: k_int_peak<1><<<blocks, threads>>>(1u, iters, out); break;
      case 2: k_int_peak<2><<<blocks, threads>>>(1u, iters, out); break;
      default: k_int_peak<3><<<blocks, threads>>>(1u, iters, out); break;
    }
    if (err == cudaSuccess) err = cudaGetLastError();
    if (err == cudaSuccess) err = cudaEventRecord(b, 0);
    if (err == cudaSuccess) err = cudaEventSynchronize(b);
    if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, a, b);
  }
  if (a) cudaEventDestroy(a);
  if (b) cudaEventDestroy(b);
  cudaFree(out);
  if (err != cudaSuccess) return (err == cudaErrorMemoryAllocation ? FAMSA_ENOMEM : FAMSA_ECUDA);
  *inst_per_s = (double)blocks * threads * iters * kPeakChains / (ms * 1e-3);
  return FAMSA_OK;
}
