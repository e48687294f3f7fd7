// Thread-per-pair LCS kernels for row widths W = 11..20 (64-bit words).
#include "lcs_kernels.cuh"

namespace famsa {

template <int W>
static cudaError_t go(const KParams &p, dim3 grid, cudaStream_t st) {
  constexpr int R = TppRows<W>::R;
  size_t smem = (size_t)R * W * kPeqWordU32 * sizeof(uint32_t);
  k_lcs_tpp<W><<<grid, kTppThreads, smem, st>>>(p);
  return cudaGetLastError();
}

cudaError_t launch_tpp_b(int W, const KParams &p, dim3 grid, cudaStream_t st) {
  switch (W) {
    case 11: return go<11>(p, grid, st);
    case 12: return go<12>(p, grid, st);
    case 13: return go<13>(p, grid, st);
    case 14: return go<14>(p, grid, st);
    case 15: return go<15>(p, grid, st);
    case 16: return go<16>(p, grid, st);
    case 17: return go<17>(p, grid, st);
    case 18: return go<18>(p, grid, st);
    case 19: return go<19>(p, grid, st);
    case 20: return go<20>(p, grid, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace famsa
