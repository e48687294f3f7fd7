// Generated by gen_lcs_tpp.py -- do not edit.
// Sliced LCS kernels for slice widths WL = 9..16 (64-bit words per warp).
#include "lcs_kernels.cuh"

namespace famsa {

template <int WL>
static cudaError_t go(int G, const KParams &p, dim3 grid, cudaStream_t st) {
  const size_t smem = slice_smem(WL, G);
  // the cap is per kernel: the largest any launch of it needs (16 slices),
  // so that launches from other threads never lower it under this one
  const size_t smem_max = slice_smem(WL, kSliceMaxG);
  if (smem_max > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_lcs_slice<WL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_max);
    if (e != cudaSuccess) return e;
  }
  k_lcs_slice<WL><<<grid, 32 * G, smem, st>>>(p);
  return cudaGetLastError();
}

cudaError_t launch_slice_b(int WL, int G, const KParams &p, dim3 grid, cudaStream_t st) {
  switch (WL) {
    case 9: return go<9>(G, p, grid, st);
    case 10: return go<10>(G, p, grid, st);
    case 11: return go<11>(G, p, grid, st);
    case 12: return go<12>(G, p, grid, st);
    case 13: return go<13>(G, p, grid, st);
    case 14: return go<14>(G, p, grid, st);
    case 15: return go<15>(G, p, grid, st);
    case 16: return go<16>(G, p, grid, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace famsa
