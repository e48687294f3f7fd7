// Generated by gen_lcs_tpp.py -- do not edit.
// Thread-per-pair LCS kernels for row widths W = 17..24 (64-bit words),
// R rows per tile.
#include "lcs_kernels.cuh"

namespace famsa {

template <int W, int R>
static cudaError_t go(const KParams &p, dim3 grid, cudaStream_t st) {
  size_t smem = (size_t)R * W * kPeqWordU32 * sizeof(uint32_t);
  k_lcs_tpp<W, R><<<grid, kTppThreads, smem, st>>>(p);
  return cudaGetLastError();
}

cudaError_t launch_tpp_c(int W, int R, const KParams &p, dim3 grid, cudaStream_t st) {
  switch (W * 8 + R) {
    case 137: return go<17, 1>(p, grid, st);
    case 145: return go<18, 1>(p, grid, st);
    case 153: return go<19, 1>(p, grid, st);
    case 161: return go<20, 1>(p, grid, st);
    case 169: return go<21, 1>(p, grid, st);
    case 177: return go<22, 1>(p, grid, st);
    case 185: return go<23, 1>(p, grid, st);
    case 193: return go<24, 1>(p, grid, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace famsa
