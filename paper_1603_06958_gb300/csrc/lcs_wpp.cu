// Warp-per-pair LCS kernels (rows longer than the thread-per-pair limit).
#include "lcs_kernels.cuh"

namespace famsa {

template <int NW>
static cudaError_t go(const KParams &p, dim3 grid, cudaStream_t st) {
  size_t smem = (size_t)kCodes * 32 * NW * sizeof(uint64_t);
  cudaError_t e = cudaFuncSetAttribute(k_lcs_wpp<NW>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  k_lcs_wpp<NW><<<grid, kWppThreads, smem, st>>>(p);
  return cudaGetLastError();
}

cudaError_t launch_wpp(int NW, const KParams &p, dim3 grid, cudaStream_t st) {
  switch (NW) {
    case 1: return go<1>(p, grid, st);
    case 2: return go<2>(p, grid, st);
    case 4: return go<4>(p, grid, st);
    case 8: return go<8>(p, grid, st);
    case 16: return go<16>(p, grid, st);
    case 32: return go<32>(p, grid, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace famsa
