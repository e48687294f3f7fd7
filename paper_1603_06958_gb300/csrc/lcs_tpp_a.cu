// Generated by gen_lcs_tpp.py -- do not edit.
// Thread-per-pair LCS kernels for row widths W = 1..8 (64-bit words),
// R rows per tile.
#include "lcs_kernels.cuh"

namespace famsa {

template <int W, int R>
static cudaError_t go(const KParams &p, dim3 grid, cudaStream_t st) {
  size_t smem = (size_t)R * W * kPeqWordU32 * sizeof(uint32_t);
  k_lcs_tpp<W, R><<<grid, kTppThreads, smem, st>>>(p);
  return cudaGetLastError();
}

cudaError_t launch_tpp_a(int W, int R, const KParams &p, dim3 grid, cudaStream_t st) {
  switch (W * 8 + R) {
    case 9: return go<1, 1>(p, grid, st);
    case 10: return go<1, 2>(p, grid, st);
    case 12: return go<1, 4>(p, grid, st);
    case 17: return go<2, 1>(p, grid, st);
    case 18: return go<2, 2>(p, grid, st);
    case 20: return go<2, 4>(p, grid, st);
    case 25: return go<3, 1>(p, grid, st);
    case 26: return go<3, 2>(p, grid, st);
    case 28: return go<3, 4>(p, grid, st);
    case 33: return go<4, 1>(p, grid, st);
    case 34: return go<4, 2>(p, grid, st);
    case 36: return go<4, 4>(p, grid, st);
    case 41: return go<5, 1>(p, grid, st);
    case 42: return go<5, 2>(p, grid, st);
    case 44: return go<5, 4>(p, grid, st);
    case 49: return go<6, 1>(p, grid, st);
    case 50: return go<6, 2>(p, grid, st);
    case 52: return go<6, 4>(p, grid, st);
    case 57: return go<7, 1>(p, grid, st);
    case 58: return go<7, 2>(p, grid, st);
    case 60: return go<7, 4>(p, grid, st);
    case 65: return go<8, 1>(p, grid, st);
    case 66: return go<8, 2>(p, grid, st);
    case 68: return go<8, 4>(p, grid, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace famsa
