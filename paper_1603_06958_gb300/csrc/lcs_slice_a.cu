// Generated by gen_lcs_tpp.py -- do not edit.
// Sliced LCS kernels for slice widths WL = 1..8 (64-bit words per warp).
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

cudaError_t launch_slice_a(int WL, int G, const KParams &p, dim3 grid, cudaStream_t st) {
  switch (WL) {
    case 1: return go<1>(G, p, grid, st);
    case 2: return go<2>(G, p, grid, st);
    case 3: return go<3>(G, p, grid, st);
    case 4: return go<4>(G, p, grid, st);
    case 5: return go<5>(G, p, grid, st);
    case 6: return go<6>(G, p, grid, st);
    case 7: return go<7>(G, p, grid, st);
    case 8: return go<8>(G, p, grid, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace famsa
