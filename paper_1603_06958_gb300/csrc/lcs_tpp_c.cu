// Thread-per-pair LCS kernels for row widths W = 21..32 (64-bit words).
#include "lcs_kernels.cuh"

namespace famsa {

template <int W>
static cudaError_t go(const KParams &p, dim3 grid, cudaStream_t st) {
  constexpr int R = TppRows<W>::R;
  size_t smem = (size_t)R * W * kPeqWordU32 * sizeof(uint32_t);
  k_lcs_tpp<W><<<grid, kTppThreads, smem, st>>>(p);
  return cudaGetLastError();
}

cudaError_t launch_tpp_c(int W, const KParams &p, dim3 grid, cudaStream_t st) {
  switch (W) {
    case 21: return go<21>(p, grid, st);
    case 22: return go<22>(p, grid, st);
    case 23: return go<23>(p, grid, st);
    case 24: return go<24>(p, grid, st);
    case 25: return go<25>(p, grid, st);
    case 26: return go<26>(p, grid, st);
    case 27: return go<27>(p, grid, st);
    case 28: return go<28>(p, grid, st);
    case 29: return go<29>(p, grid, st);
    case 30: return go<30>(p, grid, st);
    case 31: return go<31>(p, grid, st);
    case 32: return go<32>(p, grid, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace famsa
