// Bit-parallel LCS kernels (sm_103a): thread-per-pair and warp-per-pair.
//
// FAMSA Methods, "Pairwise similarities calculation": the LCS length of A and
// B is computed bit-parallel, w = 64 DP cells per machine word, in
// O(|A||B|/w) time.  The recurrence over the bit-vector V (|A| bits, one per
// position of A, initially all ones) for each symbol b of B, with
// Peq_A[b] the match mask of b in A, is
//     V = (V + (V & Peq_A[b])) | (V & ~Peq_A[b])
// and LCS(A, B) = |A| - popcount(V restricted to the first |A| bits), which
// equals the number of zero bits of V over all words because bits past |A|
// never see a match and stay one.
//
// Threads do the paper's "several pairs per thread" vectorisation in the
// GPU's own way: a warp takes 32 column sequences of one length-sorted group
// against the same R row sequences, whose Peq planes sit in shared memory.
#pragma once

#include "famsa_internal.cuh"

namespace famsa {

#include "lcs_step.inc"

struct KParams {
  const uint32_t *peq;
  const int64_t *row_peq_off;
  const int32_t *row_len;
  const int32_t *row_id;
  const int32_t *row_orig;
  int32_t e0, e1;
  const uint8_t *colres;
  const int64_t *group_off;
  const int32_t *group_chunks;
  const int32_t *col_perm;
  const int32_t *col_len;
  int32_t n_cols, n_groups;
  int mode;
  void *out;
  int64_t ld;
  int32_t row0;
  int32_t k;
  int triangle;
  const int4 *items;        // batched families: one work item per CTA (else nullptr)
  const int64_t *row_base;  // kOutBatch output offsets per row entry
};

constexpr int kTppThreads = 128;  // 4 warps = 4 column groups per CTA
constexpr int kWppThreads = 256;  // 8 warps, one column each at a time
constexpr int kWppCols = 64;      // columns per warp-per-pair CTA

// Rows per thread-per-pair tile: the default, and the choices the batch
// autotuner may take (R * W <= 32 keeps the R x 2W words of V in registers).
constexpr int tpp_default_rows(int W) { return W <= 4 ? 4 : (W <= 8 ? 2 : 1); }
constexpr bool tpp_rows_allowed(int W, int R) { return (R == 1 || R == 2 || R == 4) && R * W <= 32; }

__device__ __forceinline__ int64_t tri_index(int64_t i, int64_t j, int64_t k) {
  return i * k - i * (i + 1) / 2 + (j - i - 1);
}

// Write one LCS result according to the output mode.
__device__ __forceinline__ void emit_lcs(const KParams &p, int32_t e, int32_t rid, int32_t t,
                                         int32_t L) {
  switch (p.mode) {
    case kOutTriOrig: {
      if (t >= rid) return;
      int64_t a = p.col_perm[t], b = p.col_perm[rid];
      int64_t i = a < b ? a : b, j = a < b ? b : a;
      if (FAMSA_EXPECT(i >= 0 && j < p.k && i != j)) static_cast<int32_t *>(p.out)[tri_index(i, j, p.k)] = L;
      return;
    }
    case kOutRowsOrig: {
      int64_t oc = p.col_perm[t], orr = p.row_orig[e];
      if (oc >= orr) return;
      int64_t base = (orr * (orr - 1) - (int64_t)p.row0 * (p.row0 - 1)) / 2;
      if (FAMSA_EXPECT(oc >= 0 && orr >= p.row0 && orr < p.k)) static_cast<int32_t *>(p.out)[base + oc] = L;
      return;
    }
    case kOutRowbuf: {
      if (t >= rid) return;
      if (FAMSA_EXPECT(rid >= p.row0 && t < p.ld))
        static_cast<uint16_t *>(p.out)[(int64_t)(rid - p.row0) * p.ld + t] = (uint16_t)L;
      return;
    }
    case kOutBatch: {
      if (t >= rid) return;
      if (FAMSA_EXPECT(p.row_base[e] + t >= 0)) static_cast<uint16_t *>(p.out)[p.row_base[e] + t] = (uint16_t)L;
      return;
    }
    default: {  // kOutQuery
      const int32_t c = p.col_perm[t];
      if (FAMSA_EXPECT(rid >= 0 && c >= 0 && c < p.ld)) static_cast<int32_t *>(p.out)[(int64_t)rid * p.ld + c] = L;
      return;
    }
  }
}

// ------------------------------------------------------------ thread per pair
// blockIdx.x: tile of R consecutive row entries; blockIdx.y: 128 consecutive
// sorted columns (4 groups of 32).  Each thread owns one column and runs the
// recurrence for all R rows of the tile at once (R independent carry chains).
// With a work list (batched families), work item blockIdx.x names the tile
// (at most R rows of one family) and its first column group instead.
// The explicit minimum of one CTA per SM matters: with it ptxas keeps more
// of a step's Peq words in flight (W = 7, R = 2: 84 registers instead of 55),
// which measured 4-5 % faster at every width than the bare thread bound.
template <int W, int R>
__global__ void __launch_bounds__(kTppThreads, 1) k_lcs_tpp(KParams p) {
  extern __shared__ __align__(16) uint32_t sPeq[];  // R * W * 64 u32
  int32_t tile_e, tile_end, gbase;
  if (p.items) {
    const int4 it = p.items[blockIdx.x];
    tile_e = it.x;
    tile_end = it.x + it.y;
    gbase = it.z;
  } else {
    tile_e = p.e0 + (int32_t)blockIdx.x * R;
    tile_end = min(tile_e + R, p.e1);
    gbase = (int32_t)blockIdx.y * 4;
  }
  int32_t last_e = tile_end - 1;
  int32_t col_limit = p.triangle ? p.row_id[last_e] : p.n_cols;
  if (gbase * kGroup >= col_limit) return;

  // stage the tile's Peq planes; rows shorter than W words are zero-padded
  if (threadIdx.x < R && tile_e + (int32_t)threadIdx.x < tile_end)
    (void)FAMSA_EXPECT((p.row_len[tile_e + threadIdx.x] + 63) / 64 <= W);  // a wider row would be cut
  for (int i = threadIdx.x; i < R * W * 16; i += kTppThreads) {
    int r = i / (W * 16), rem = i - r * (W * 16), w = rem >> 4;
    int32_t e = tile_e + r;
    uint4 v = make_uint4(0, 0, 0, 0);
    if (e < tile_end && w < (p.row_len[e] + 63) / 64)
      v = reinterpret_cast<const uint4 *>(p.peq + (p.row_peq_off[e] + w) * kPeqWordU32)[rem & 15];
    reinterpret_cast<uint4 *>(sPeq)[i] = v;
  }
  __syncthreads();

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int32_t g = gbase + warp;
  if (g >= p.n_groups || g * kGroup >= col_limit) return;

  uint32_t V[R][2 * W];
#pragma unroll
  for (int r = 0; r < R; ++r)
#pragma unroll
    for (int i = 0; i < 2 * W; ++i) V[r][i] = 0xffffffffu;

  const uint4 *src = reinterpret_cast<const uint4 *>(p.colres + p.group_off[g]) + lane;
  const int32_t nch = p.group_chunks[g];
  uint4 cur = __ldg(src);
  const char *sbase = reinterpret_cast<const char *>(sPeq);
  for (int32_t q = 0; q < nch; ++q) {
    uint4 nxt = cur;
    if (q + 1 < nch) nxt = __ldg(src + (int64_t)(q + 1) * kGroup);
    const uint32_t cw[4] = {cur.x, cur.y, cur.z, cur.w};
#pragma unroll
    for (int j = 0; j < 4; ++j) {
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        const uint32_t off = (cw[j] >> (8 * b)) & 0xffu;  // 4 * symbol
        const char *base = sbase + off;
#pragma unroll
        for (int r = 0; r < R; ++r) {
          uint32_t P[2 * W];
#pragma unroll
          for (int w = 0; w < W; ++w) {
            P[2 * w] = *reinterpret_cast<const uint32_t *>(base + (r * W + w) * 256);
            P[2 * w + 1] = *reinterpret_cast<const uint32_t *>(base + (r * W + w) * 256 + 128);
          }
          lcs_step<W>(V[r], P);
        }
      }
    }
    cur = nxt;
  }

  const int32_t t = g * kGroup + lane;
  if (t >= p.n_cols) return;
#pragma unroll
  for (int r = 0; r < R; ++r) {
    int32_t e = tile_e + r;
    if (e >= tile_end) break;
    int32_t L = 0;
#pragma unroll
    for (int i = 0; i < 2 * W; ++i) L += __popc(~V[r][i]);
    emit_lcs(p, e, p.row_id[e], t, L);
  }
}

// ------------------------------------------------------------ sliced pairs
// Rows too wide for one thread's registers are split into G slices of WL
// words; warp s of a CTA holds words [s*WL, (s+1)*WL) of the row's vector for
// the 32 columns of one group, so every lane of a warp reads the same Peq
// word (conflict free, as in thread-per-pair).  The add's carry crosses from
// slice s to s+1: warp s runs chunk q (16 symbols) of the columns at
// iteration q + s, collects the 16 carries out of its top word in a mask
// (bit 15 - j for symbol j), and after the CTA barrier warp s+1 takes them
// back in the same order as the carries into its bottom word.  Each step
// costs two operations beyond the recurrence's 6 per word, and each chunk
// one barrier; a CTA runs nch + G - 1 chunk iterations for nch chunks.
// Words past the row's length have Peq 0, so they stay all ones whatever
// carry arrives: the zero bits of all slices count the LCS.
constexpr int kSliceWords = 16;  // default words per slice (the largest instance)
constexpr int kSliceMaxG = 16;   // slices per CTA: 512 threads
constexpr int kSliceMaxW = kSliceWords * kSliceMaxG;  // 256 words = 16,384 residues
constexpr int kSliceMinW = 24;   // rows of at least this many words are sliced by default

template <int WL>
__global__ void __launch_bounds__(32 * kSliceMaxG, 1) k_lcs_slice(KParams p) {
  extern __shared__ __align__(16) uint32_t sSl[];
  const int G = (int)(blockDim.x >> 5);
  int32_t e, grp;
  if (p.items) {
    const int4 it = p.items[blockIdx.x];
    e = it.x;
    grp = it.z;
  } else {
    e = p.e0 + (int32_t)blockIdx.x;
    grp = (int32_t)blockIdx.y;
  }
  const int32_t rid = p.row_id[e];
  const int32_t col_limit = p.triangle ? rid : p.n_cols;
  if (grp >= p.n_groups || grp * kGroup >= col_limit) return;  // uniform over the CTA
  const int32_t Wr = (p.row_len[e] + 63) / 64;
  if (threadIdx.x == 0) (void)FAMSA_EXPECT(Wr <= G * WL && G <= kSliceMaxG && (int)blockDim.x == 32 * G);
  uint32_t *sPeq = sSl;                               // G * WL words x 64 u32
  uint32_t *sMask = sSl + G * WL * kPeqWordU32;       // [2][G][32] carry masks
  uint32_t *sSum = sMask + 2 * G * kGroup;            // [G][32] partial counts
  const uint4 *prow = reinterpret_cast<const uint4 *>(p.peq + p.row_peq_off[e] * kPeqWordU32);
  for (int i = threadIdx.x; i < G * WL * 16; i += blockDim.x) {
    uint4 v = make_uint4(0, 0, 0, 0);
    if ((i >> 4) < Wr) v = prow[i];
    reinterpret_cast<uint4 *>(sPeq)[i] = v;
  }
  __syncthreads();

  const int s = (int)(threadIdx.x >> 5), lane = (int)(threadIdx.x & 31);
  uint32_t V[2 * WL];
#pragma unroll
  for (int i = 0; i < 2 * WL; ++i) V[i] = 0xffffffffu;
  const uint4 *src = reinterpret_cast<const uint4 *>(p.colres + p.group_off[grp]) + lane;
  const int32_t nch = p.group_chunks[grp];
  const char *sbase = reinterpret_cast<const char *>(sPeq + s * WL * kPeqWordU32);
  uint4 cur = __ldg(src);
  for (int32_t it = 0; it < nch + G - 1; ++it) {
    const int32_t q = it - s;
    if (q >= 0 && q < nch) {  // uniform over the warp
      uint32_t cin = s > 0 ? sMask[((it + 1) & 1) * G * kGroup + (s - 1) * kGroup + lane] : 0u;
      uint32_t cout = 0;
      uint4 nxt = cur;
      if (q + 1 < nch) nxt = __ldg(src + (int64_t)(q + 1) * kGroup);
      const uint32_t cw[4] = {cur.x, cur.y, cur.z, cur.w};
#pragma unroll
      for (int j = 0; j < 4; ++j) {
#pragma unroll
        for (int b = 0; b < 4; ++b) {
          const char *base = sbase + ((cw[j] >> (8 * b)) & 0xffu);  // 4 * symbol
          uint32_t P[2 * WL];
#pragma unroll
          for (int w = 0; w < WL; ++w) {
            P[2 * w] = *reinterpret_cast<const uint32_t *>(base + w * 256);
            P[2 * w + 1] = *reinterpret_cast<const uint32_t *>(base + w * 256 + 128);
          }
          LcsSlice<WL>::run(V, P, cin, cout);
        }
      }
      sMask[(it & 1) * G * kGroup + s * kGroup + lane] = cout << 16;
      cur = nxt;
    }
    __syncthreads();
  }
  int32_t L = 0;
#pragma unroll
  for (int i = 0; i < 2 * WL; ++i) L += __popc(~V[i]);
  sSum[s * kGroup + lane] = (uint32_t)L;
  __syncthreads();
  if (s != 0) return;
  for (int j = 1; j < G; ++j) L += (int32_t)sSum[j * kGroup + lane];
  const int32_t t = grp * kGroup + lane;
  if (t < p.n_cols) emit_lcs(p, e, rid, t, L);
}

// shared memory of a slice launch: the row's planes, two mask buffers, the partial counts
constexpr size_t slice_smem(int WL, int G) {
  return (size_t)G * WL * kPeqWordU32 * 4 + (size_t)3 * G * kGroup * 4;
}

// ------------------------------------------------------------ warp per pair
// One row per CTA (Peq transposed to [symbol][word] in shared memory so the
// 32 lanes read 32 consecutive words); each warp runs whole columns.  Lane l
// holds words l, l+32, ..., the 64-bit add carries between lanes by a
// carry-lookahead over two ballots: with G = lanes whose word add overflowed
// and P = lanes whose sum is all ones, the carries into the lanes are
// ((G|P) + G + c_in) ^ P, and bit 32 of that sum carries into the next
// 32-word slice.
template <int NW>
__global__ void __launch_bounds__(kWppThreads) k_lcs_wpp(KParams p) {
  constexpr int WP = 32 * NW;
  extern __shared__ __align__(16) uint64_t sP[];  // kCodes * WP
  int32_t e, c_begin;
  if (p.items) {
    const int4 it = p.items[blockIdx.x];
    e = it.x;
    c_begin = it.z * kGroup;
  } else {
    e = p.e0 + (int32_t)blockIdx.x;
    c_begin = (int32_t)blockIdx.y * kWppCols;
  }
  const int32_t rid = p.row_id[e];
  const int32_t Wr = (p.row_len[e] + 63) / 64;
  if (threadIdx.x == 0) (void)FAMSA_EXPECT(Wr <= WP);
  const int32_t col_limit = p.triangle ? rid : p.n_cols;
  if (c_begin >= col_limit) return;
  const int32_t c_end = min(c_begin + kWppCols, col_limit);
  const uint32_t *prow = p.peq + p.row_peq_off[e] * kPeqWordU32;
  for (int i = threadIdx.x; i < kCodes * WP; i += kWppThreads) {
    int c = i / WP, w = i - c * WP;
    uint64_t v = 0;
    if (w < Wr)
      v = ((uint64_t)prow[w * kPeqWordU32 + 32 + c] << 32) | prow[w * kPeqWordU32 + c];
    sP[i] = v;
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int32_t t = c_begin + warp; t < c_end; t += kWppThreads / 32) {
    uint64_t V[NW];
#pragma unroll
    for (int j = 0; j < NW; ++j) V[j] = ~0ull;
    const int32_t g = t / kGroup, ln = t % kGroup;
    const uint4 *src = reinterpret_cast<const uint4 *>(p.colres + p.group_off[g]) + ln;
    const int32_t clen = p.col_len[t];
    for (int32_t q = 0; q * kChunk < clen; ++q) {
      const uint4 ch = __ldg(src + (int64_t)q * kGroup);
      const uint32_t cw[4] = {ch.x, ch.y, ch.z, ch.w};
      const int nb = min(kChunk, clen - q * kChunk);
#pragma unroll
      for (int b = 0; b < kChunk; ++b) {
        if (b >= nb) break;
        const uint32_t sym = ((cw[b >> 2] >> (8 * (b & 3))) & 0xffu) >> 2;
        const uint64_t *row = sP + sym * WP + lane;
        uint32_t cin = 0;
#pragma unroll
        for (int j = 0; j < NW; ++j) {
          const uint64_t P = row[j * 32];
          const uint64_t v = V[j];
          uint64_t s = v + (v & P);
          const uint32_t G = __ballot_sync(0xffffffffu, s < v);
          const uint32_t PP = __ballot_sync(0xffffffffu, s == ~0ull);
          const uint64_t tt = (uint64_t)(G | PP) + G + cin;
          const uint32_t C = (uint32_t)tt ^ PP;
          cin = (uint32_t)(tt >> 32);
          s += (C >> lane) & 1u;
          V[j] = s | (v & ~P);
        }
      }
    }
    int32_t L = 0;
#pragma unroll
    for (int j = 0; j < NW; ++j) L += __popcll(~V[j]);
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) L += __shfl_xor_sync(0xffffffffu, L, d);
    if (lane == 0) emit_lcs(p, e, rid, t, L);
  }
}

// per-width launchers (defined in the lcs_tpp_*.cu / lcs_wpp.cu units)
// thread-per-pair launch with R rows per tile (tpp_rows_allowed(W, R))
cudaError_t launch_tpp(int W, int R, const KParams &p, dim3 grid, cudaStream_t st);
// the R the launch planner uses for width W (autotuned, else the default)
int tpp_rows(int W);
void set_tpp_rows(int W, int R);
cudaError_t launch_wpp(int NW, const KParams &p, dim3 grid, cudaStream_t st);
// sliced launch: G slices of WL words per row, one column group per CTA (grid.y or items)
cudaError_t launch_slice(int WL, int G, const KParams &p, dim3 grid, cudaStream_t st);

// The kernel that runs rows of W words (lcs.cu): thread-per-pair (kw = W),
// sliced (kw = words per slice, g = slices) or warp-per-pair (kw = 64-bit
// words per lane).  Rows of one choice share a launch.
enum LcsKind : int { kLcsTpp = 0, kLcsSlice = 1, kLcsWpp = 2 };
struct LcsChoice {
  int kind, kw, g;
  bool operator==(const LcsChoice &o) const { return kind == o.kind && kw == o.kw && g == o.g; }
  bool operator!=(const LcsChoice &o) const { return !(*this == o); }
};
LcsChoice lcs_choice(int W);

}  // namespace famsa
