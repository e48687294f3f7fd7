// Gap types, their set-size scaled costs, and gap-column insertion with the
// paper's type corrections.
//
// FAMSA Methods, "Gap types and costs determination": four gap types --
// terminal open (T_o), terminal extension (T_e), open (G_o), extension
// (G_e) -- with affine costs, all multiplied by
//     g_scale = 1 + log(k / g_l) / g_d   (g_l = 45, g_d = 7 by default),
// k the number of sequences of the input set.  When a column of gaps goes
// into a profile whose sequences already hold gaps, the inserted gap's type
// follows from its neighbours, and the gap after it may change (the six
// cases S1..S6 of that subsection).
//
// Alignment rows are m x n bytes: residue codes 0..24, FAMSA_GAP (255) for a
// gap.  Types: 0 residue, 1 T_o, 2 T_e, 3 G_o, 4 G_e.  The classification
// that S1..S6 preserve: gaps before the first residue or after the last one
// are terminal, the others are not; the first gap of a run opens it, the
// rest extend it (a row of gaps only is one terminal run).
#include <algorithm>
#include <cmath>

#include "famsa_internal.cuh"

namespace {

enum : uint8_t { kRes = 0, kTo = 1, kTe = 2, kGo = 3, kGe = 4 };
constexpr uint8_t kGap = 255;

// One CTA per row: first and last residue, then every cell from its left
// neighbour.
__global__ void k_gap_types(const uint8_t *aln, int32_t n, uint8_t *types) {
  const int64_t r = blockIdx.x;
  const uint8_t *row = aln + r * n;
  __shared__ int32_t first, last;
  if (threadIdx.x == 0) { first = n; last = -1; }
  __syncthreads();
  int32_t f = n, l = -1;
  for (int32_t j = threadIdx.x; j < n; j += blockDim.x)
    if (row[j] != kGap) { f = min(f, j); l = max(l, j); }
  atomicMin(&first, f);
  atomicMax(&last, l);
  __syncthreads();
  for (int32_t j = threadIdx.x; j < n; j += blockDim.x) {
    uint8_t t = kRes;
    if (row[j] == kGap) {
      const bool terminal = j < first || j > last;
      const bool opens = j == 0 || row[j - 1] != kGap;
      t = terminal ? (opens ? kTo : kTe) : (opens ? kGo : kGe);
    }
    types[r * n + j] = t;
  }
}

// Per row: the gap counts of each type times their costs, times g_scale.
__global__ void k_gap_cost(const uint8_t *types, int64_t m, int32_t n, double scale, double c_to, double c_te,
                           double c_go, double c_ge, double *cost) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= m) return;
  int64_t cnt[5] = {0, 0, 0, 0, 0};
  for (int32_t j = 0; j < n; ++j) cnt[types[r * n + j]]++;
  const double raw = c_to * (double)cnt[kTo] + c_te * (double)cnt[kTe] + c_go * (double)cnt[kGo] +
                     c_ge * (double)cnt[kGe];
  cost[r] = scale * raw;
}

// The type of a gap inserted between left neighbour L and right neighbour R
// (type values; 255 = no neighbour), and the new type of R (S1, S4).
__device__ __forceinline__ uint8_t inserted_type(uint8_t L, uint8_t *R) {
  constexpr uint8_t kNone = 255;
  if (*R == kTo) { *R = kTe; return kTo; }       // S1
  if (L == kTe) return kTe;                       // S2
  if (L == kTo) return kTe;                       // S6
  if (*R == kGo) { *R = kGe; return kGo; }       // S4
  if (L == kGo || L == kGe) return kGe;           // S3
  if (L == kNone || *R == kNone) return kTo;      // a new terminal run at an end of the row
  return kGo;                                     // S5
}

// One thread per row: the row with c gap columns inserted (positions pos[],
// ascending, each before original column pos[i]; equal positions give
// adjacent columns), types taken from the neighbours left to right.  The
// right neighbour of the insertions before column j is column j itself,
// whose type the insertions may correct (S1, S4) before it is written.
__global__ void k_gap_insert(const uint8_t *aln, const uint8_t *types, int64_t m, int32_t n, const int32_t *pos,
                             int32_t c, uint8_t *aln_out, uint8_t *types_out) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= m) return;
  const int64_t w = (int64_t)n + c;
  const uint8_t *a = aln + r * n, *t = types + r * n;
  uint8_t *ao = aln_out + r * w, *to = types_out + r * w;
  int32_t i = 0;
  int64_t o = 0;
  for (int32_t j = 0; j <= n; ++j) {
    uint8_t R = j < n ? t[j] : 255;
    while (i < c && pos[i] == j) {
      const uint8_t L = o > 0 ? to[o - 1] : 255;
      const uint8_t g = inserted_type(L, &R);
      ao[o] = kGap;
      to[o] = g;
      ++o;
      ++i;
    }
    if (j < n) {
      ao[o] = a[j];
      to[o] = R;
      ++o;
    }
  }
}

inline int status(cudaError_t e) { return famsa::status_from_cuda(e); }

}  // namespace

extern "C" int famsa_gap_types(const uint8_t *aln, int64_t m, int32_t n, uint8_t *types, void *cuda_stream) {
  if (m < 0 || n < 0 || (m > 0 && n > 0 && (!aln || !types))) return FAMSA_EINVAL;
  if (m == 0 || n == 0) return FAMSA_OK;
  if (m > INT32_MAX) return FAMSA_ERANGE;
  k_gap_types<<<(unsigned)m, 256, 0, (cudaStream_t)cuda_stream>>>(aln, n, types);
  return status(cudaGetLastError());
}

extern "C" double famsa_gap_scale(int64_t k, double g_l, double g_d) {
  if (k < 1 || !(g_l > 0) || g_d == 0) return NAN;
  return 1.0 + std::log((double)k / g_l) / g_d;
}

extern "C" int famsa_gap_cost(const uint8_t *types, int64_t m, int32_t n, int64_t k, const double *costs,
                              double g_l, double g_d, double *cost, void *cuda_stream) {
  if (m < 0 || n < 0 || !costs || k < 1 || !(g_l > 0) || g_d == 0) return FAMSA_EINVAL;
  if (m > 0 && (!types || !cost)) return FAMSA_EINVAL;
  if (m == 0) return FAMSA_OK;
  const double scale = famsa_gap_scale(k, g_l, g_d);
  const int T = 256;
  k_gap_cost<<<(unsigned)((m + T - 1) / T), T, 0, (cudaStream_t)cuda_stream>>>(
      types, m, n, scale, costs[0], costs[1], costs[2], costs[3], cost);
  return status(cudaGetLastError());
}

extern "C" int famsa_gap_insert(const uint8_t *aln, const uint8_t *types, int64_t m, int32_t n,
                                const int32_t *positions, int32_t c, uint8_t *aln_out, uint8_t *types_out,
                                void *cuda_stream) {
  if (m < 0 || n < 0 || c < 0 || (m > 0 && (!aln_out || !types_out)) || (m > 0 && n > 0 && (!aln || !types)) ||
      (c > 0 && !positions))
    return FAMSA_EINVAL;
  for (int32_t i = 0; i < c; ++i)
    if (positions[i] < 0 || positions[i] > n || (i > 0 && positions[i] < positions[i - 1])) return FAMSA_EINVAL;
  if (m == 0) return FAMSA_OK;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  int32_t *d_pos = nullptr;
  cudaError_t e = famsa::lib_malloc_async((void **)&d_pos, sizeof(int32_t) * (size_t)std::max(c, 1), st);
  if (e != cudaSuccess) return status(e);
  if (c > 0) e = cudaMemcpyAsync(d_pos, positions, sizeof(int32_t) * (size_t)c, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) {
    const int T = 128;
    k_gap_insert<<<(unsigned)((m + T - 1) / T), T, 0, st>>>(aln, types, m, n, d_pos, c, aln_out, types_out);
    e = cudaGetLastError();
  }
  cudaFreeAsync(d_pos, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);  // the host positions may go once the call returns
  return status(e);
}
