// Generated by gen_lcs_tpp.py -- do not edit.
// Thread-per-pair LCS kernels for row widths W = 9..16 (64-bit words),
// R rows per tile.
#include "lcs_kernels.cuh"

namespace famsa {

template <int W, int R>
static cudaError_t go(const KParams &p, dim3 grid, cudaStream_t st) {
  size_t smem = (size_t)R * W * kPeqWordU32 * sizeof(uint32_t);
  k_lcs_tpp<W, R><<<grid, kTppThreads, smem, st>>>(p);
  return cudaGetLastError();
}

cudaError_t launch_tpp_b(int W, int R, const KParams &p, dim3 grid, cudaStream_t st) {
  switch (W * 8 + R) {
    case 73: return go<9, 1>(p, grid, st);
    case 74: return go<9, 2>(p, grid, st);
    case 81: return go<10, 1>(p, grid, st);
    case 82: return go<10, 2>(p, grid, st);
    case 89: return go<11, 1>(p, grid, st);
    case 90: return go<11, 2>(p, grid, st);
    case 97: return go<12, 1>(p, grid, st);
    case 98: return go<12, 2>(p, grid, st);
    case 105: return go<13, 1>(p, grid, st);
    case 106: return go<13, 2>(p, grid, st);
    case 113: return go<14, 1>(p, grid, st);
    case 114: return go<14, 2>(p, grid, st);
    case 121: return go<15, 1>(p, grid, st);
    case 122: return go<15, 2>(p, grid, st);
    case 129: return go<16, 1>(p, grid, st);
    case 130: return go<16, 2>(p, grid, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace famsa
