// Minimum-spanning-tree row update (slink_msf.cu): state and launch API.
#pragma once

#include "slink_common.cuh"

namespace famsa {

// Keys are exact order codes floor(indel^2 * 2^30 / LCS) (below 2^62 when
// every length is <= 32767); LCS = 0 (+infinity) sorts above all of them.
constexpr uint64_t kMsfInf = 1ull << 63;
constexpr uint64_t kMsfNone = ~0ull;  // no candidate edge
enum : int { kMsfCount = 0, kMsfDone = 1, kMsfErr = 2, kMsfCtlWords = 4 };

struct MsfState {
  int32_t *comp;                 // component root of each point
  int32_t *par;                  // hook target of each root in the current round
  uint64_t *rkey; int32_t *roth; // per block row: lightest edge to another component (key, column)
  uint64_t *ckey; int32_t *coth; // per point: lightest edge to a later block row in another component
  uint64_t *vkey, *vab;          // per point: its lightest candidate (key, a << 32 | b)
  uint64_t *bkey, *bab;          // per root: its component's lightest boundary edge
  uint64_t *mkey; int32_t *ma, *mb;  // the previous tree's edges (a < b)
  uint64_t *nkey; int32_t *na, *nb;  // the tree being built
  int32_t cap;                   // capacity of the edge arrays
  int32_t *ctl;                  // kMsfCount, kMsfDone, kMsfErr
  uint64_t *keys;                // block keys [row - r0][ld]
  const int32_t *slen;           // lengths in insertion order
};

// Rebuild the tree of points [0, r1) from the previous tree (m = r0 - 1 edges)
// and the block rows [r0, r1) of rowbuf; swaps the edge arrays in S.
cudaError_t launch_msf_block(MsfState &S, const uint16_t *rowbuf, int64_t ld, int32_t r0, int32_t r1,
                             int32_t m, cudaStream_t st, int64_t *launches);
// The finished tree (k - 1 edges in S.mkey/ma/mb) -> leaf order ord[k] and
// gaps gap[k - 1] (narrow order codes).  Scratch: idx_a, idx_b (k), work
// (8k int32), ek (k: the sorted keys).
cudaError_t launch_msf_leaf_order(const MsfState &S, int32_t k, int32_t *ord, uint64_t *gap, int32_t *idx_a,
                                  int32_t *idx_b, int32_t *work, uint64_t *ek, cudaStream_t st,
                                  int64_t *launches);
int msf_rounds(int32_t r1);
// The minimum spanning tree of points [0, n) from an edge list alone: the m
// edges in S.mkey/ma/mb (a graph that connects all n points) -> the n - 1
// tree edges, swapped into S.mkey/ma/mb.
cudaError_t launch_msf_edges(MsfState &S, int32_t n, int32_t m, cudaStream_t st, int64_t *launches);
// Caller edge lists <-> tree edges: distances as reduced fractions num / den
// (+inf = 1 / 0) on the caller's side, order codes inside; perm (optional)
// maps tree labels to the caller's on the way out.
cudaError_t launch_msf_from_fractions(MsfState &S, int32_t m, int32_t k, const int32_t *a, const int32_t *b,
                                      const uint64_t *num, const uint32_t *den, cudaStream_t st);
cudaError_t launch_msf_to_fractions(const MsfState &S, int32_t m, const int32_t *perm, int32_t *a, int32_t *b,
                                    uint64_t *num, uint32_t *den, cudaStream_t st);

}  // namespace famsa
