// Thread-per-pair LCS kernels for row widths W = 1..10 (64-bit words).
#include "lcs_kernels.cuh"

namespace famsa {

template <int W>
static cudaError_t go(const KParams &p, dim3 grid, cudaStream_t st) {
  constexpr int R = TppRows<W>::R;
  size_t smem = (size_t)R * W * kPeqWordU32 * sizeof(uint32_t);
  k_lcs_tpp<W><<<grid, kTppThreads, smem, st>>>(p);
  return cudaGetLastError();
}

cudaError_t launch_tpp_a(int W, const KParams &p, dim3 grid, cudaStream_t st) {
  switch (W) {
    case 1: return go<1>(p, grid, st);
    case 2: return go<2>(p, grid, st);
    case 3: return go<3>(p, grid, st);
    case 4: return go<4>(p, grid, st);
    case 5: return go<5>(p, grid, st);
    case 6: return go<6>(p, grid, st);
    case 7: return go<7>(p, grid, st);
    case 8: return go<8>(p, grid, st);
    case 9: return go<9>(p, grid, st);
    case 10: return go<10>(p, grid, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace famsa
