// Generated by gen_lcs_tpp.py -- do not edit.
// Thread-per-pair LCS kernels for row widths W = 25..32 (64-bit words),
// R rows per tile.
#include "lcs_kernels.cuh"

namespace famsa {

template <int W, int R>
static cudaError_t go(const KParams &p, dim3 grid, cudaStream_t st) {
  size_t smem = (size_t)R * W * kPeqWordU32 * sizeof(uint32_t);
  k_lcs_tpp<W, R><<<grid, kTppThreads, smem, st>>>(p);
  return cudaGetLastError();
}

cudaError_t launch_tpp_d(int W, int R, const KParams &p, dim3 grid, cudaStream_t st) {
  switch (W * 8 + R) {
    case 201: return go<25, 1>(p, grid, st);
    case 209: return go<26, 1>(p, grid, st);
    case 217: return go<27, 1>(p, grid, st);
    case 225: return go<28, 1>(p, grid, st);
    case 233: return go<29, 1>(p, grid, st);
    case 241: return go<30, 1>(p, grid, st);
    case 249: return go<31, 1>(p, grid, st);
    case 257: return go<32, 1>(p, grid, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace famsa
