// Internal declarations of the GB300 FAMSA stage I+II library (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>

#include <mutex>
#include <vector>

#include "../../include/famsa_gpu.h"
#include "../../include/famsa_gpu_debug.h"

namespace famsa {

// ----------------------------------------------------------------- constants
constexpr int kCodes = 25;          // residue codes 0..24
constexpr int kCodeSlots = 32;      // Peq planes padded to 32 symbols (one bank per symbol)
constexpr int kPadCode = 31;        // column padding symbol: its Peq is 0 in every row
constexpr int kMaxLen = 65535;
enum : int { kBadArg = 1, kTooLong = 2 };  // validation status bits of the packing kernels
constexpr int kGroup = 32;          // columns per group (one warp)
constexpr int kChunk = 16;          // residues per interleaved chunk (one 16-byte load)
constexpr int kTppMaxW = 32;        // thread-per-pair handles rows of up to 32 words
constexpr int kStatsLen = 24;       // famsa_last_stats entries
// Row blocks of 16-bit LCS values in flight between the LCS kernels and the
// row update: the LCS may run this many blocks minus one ahead, so that it
// fills the early blocks' slack (where the row update is the longer) and the
// row update never waits on it later (where the LCS per block is the longer).
constexpr int kRowBuffers = 4;

// Peq layout (row side): for each sequence s and word w, 64 uint32:
//   [0..32)  low 32 bits of the mask for symbols 0..31
//   [32..64) high 32 bits
// so a thread reading symbol c touches bank c in each plane (conflict free).
constexpr int kPeqWordU32 = 64;

// Column layout: group g (sorted sequences 32g..32g+31), chunk q, lane l:
//   colres[group_off[g] + (q*32 + l)*16 + b] = 4 * code of residue 16q+b of
//   sequence 32g+l, or 4*kPadCode past its end.  Storing 4*code makes the
//   byte itself the shared-memory byte offset of the symbol's plane entry.

struct DeviceBuffer {
  void *ptr = nullptr;
  size_t bytes = 0;
};

// A packed family resident on the device.
struct Family {
  int32_t k = 0;
  int64_t total = 0;
  int32_t max_len = 0;
  int32_t max_w = 0;
  int device = 0;
  std::mutex mu;

  // original order
  int64_t *d_off = nullptr;      // k+1
  uint8_t *d_res = nullptr;      // total residues
  int32_t *d_len = nullptr;      // k lengths (original order)
  // sorted order: sorted position s -> original index perm[s]; rank = inverse
  int32_t *d_perm = nullptr;
  int32_t *d_rank = nullptr;
  int32_t *d_slen = nullptr;     // lengths in sorted order
  int64_t *d_peq_off = nullptr;  // word offset (units of 64 u32) of sorted sequence s
  uint32_t *d_peq = nullptr;     // sum_s W_s * 64 u32
  int64_t *d_group_off = nullptr;   // byte offset of column group g
  int32_t *d_group_chunks = nullptr;  // 16-residue chunks in group g
  uint8_t *d_colres = nullptr;
  int32_t n_groups = 0;
  int64_t peq_words = 0;
  int64_t colres_bytes = 0;

  // host copies used for launch planning
  std::vector<int32_t> h_slen;     // sorted lengths
  std::vector<int32_t> h_perm;

  // scratch reused across calls
  std::vector<DeviceBuffer> scratch;
  int64_t stats[kStatsLen] = {0};
  int64_t pack_launches = 0;
  int64_t sub_kcycles[16] = {0};
  // insertion-label pointer representation of the last tree build (debug export):
  // per point j: original label, pi, packed lambda key, 0
  std::vector<int64_t> dbg_state;
};

// Every device allocation of the library goes through lib_malloc_async
// (stream-ordered cudaMallocAsync), which counts them process-wide for
// famsa_debug_alloc_count.
cudaError_t lib_malloc_async(void **p, size_t bytes, cudaStream_t st);
// Allocation with an injectable failure hook (tests use it to check ENOMEM paths).
// Stream-ordered (cudaMallocAsync / cudaFreeAsync) on the calling thread's
// allocation stream, so that freeing never waits for the whole device.
cudaError_t dev_alloc(void **p, size_t bytes);
void dev_free(void *p);
// Sets the calling thread's allocation stream for its lifetime (default: the
// legacy stream).  Memory freed on a stream may be reused by later work of
// that stream at once: free only what no other stream still uses.
struct AllocStream {
  explicit AllocStream(cudaStream_t st);
  ~AllocStream();
  cudaStream_t prev;
};

// ------------------------------------------------------------ LCS launch API
enum OutMode : int {
  kOutTriOrig = 0,   // int32 at the i<j row-major index of the pair in original labels
  kOutRowsOrig = 1,  // int32 at rowoff(orig row) + orig col, only for orig col < orig row
  kOutRowbuf = 2,    // uint16 rowbuf[(row - row0) * ld + col], only for sorted col < sorted row
  kOutQuery = 3,     // int32 out[qrow * k + orig col]
  kOutBatch = 4,     // uint16 out[row_base[entry] + sorted col], only for sorted col < sorted row
};

// A batch of pairs for the LCS kernels: a list of row sequences (with their
// Peq) against the family's column groups.
struct LcsBatch {
  const uint32_t *peq = nullptr;       // row Peq base
  const int64_t *row_peq_off = nullptr;  // per row-list entry
  const int32_t *row_len = nullptr;      // per row-list entry (length)
  const int32_t *row_id = nullptr;       // per row-list entry: sorted id (tri/rowbuf) or query id
  const int32_t *row_orig = nullptr;     // per row-list entry: original label (rows mode)
  int32_t n_rows = 0;                    // entries in the row list
  // host view of the row list's W per entry, to plan launches (rows sorted by W)
  const int32_t *h_row_w = nullptr;
  // columns
  const uint8_t *colres = nullptr;
  const int64_t *group_off = nullptr;
  const int32_t *group_chunks = nullptr;
  const int32_t *col_perm = nullptr;     // sorted col -> original label
  const int32_t *col_len = nullptr;      // sorted col -> length
  int32_t n_cols = 0;
  const int32_t *h_row_id = nullptr;     // host copy of row_id (column bound per segment)
  // output
  int mode = kOutTriOrig;
  void *out = nullptr;
  int64_t ld = 0;        // rowbuf leading dimension / k for query
  int32_t row0 = 0;      // rowbuf: sorted id of its first row; rows mode: row_begin
  int32_t k = 0;         // family size (tri index)
  bool triangle = false; // restrict columns to sorted col < sorted row (by group bound)
  // batched families: an explicit work list replaces the launch planner's grid
  const int4 *items = nullptr;       // (first row entry, rows, first column group, unused)
  const int64_t *row_base = nullptr; // kOutBatch: output offset of each row entry
};

// Enqueue the LCS kernels for a batch; returns a CUDA error code.  Adds the
// number of kernel launches to *launches.
cudaError_t launch_lcs(const LcsBatch &b, cudaStream_t st, int64_t *launches);

// ------------------------------------------------------------ packing API
int pack_family(const uint8_t *residues, const int64_t *offsets, int32_t k, bool on_device,
                cudaStream_t st, Family **out);
void free_family(Family *f);

// Pack an arbitrary sequence list's Peq (query rows): writes peq (sum W*64 u32)
// and per-sequence offsets/lengths; returns FAMSA status.
int pack_rows(const uint8_t *d_res, const int64_t *d_off, int32_t n, cudaStream_t st,
              uint32_t **d_peq, int64_t **d_peq_off, int32_t **d_len, std::vector<int32_t> &h_len);

// ------------------------------------------------------------ tree API
int slink_tree(Family *f, int32_t *pi, uint64_t *lambda_num, uint32_t *lambda_den,
               int32_t *merges, uint64_t *h_num, uint32_t *h_den, int32_t *sizes,
               bool out_on_device, cudaStream_t st);

int status_from_cuda(cudaError_t e);

// An NVTX range for the lifetime of a scope: the entry points, each row
// block of a tree build, a batch's plan and graph launch and each served
// request show up by name on a profiler's timeline (nsys, ncu --nvtx).  With
// no profiler attached a push or pop costs next to nothing.
struct TraceRange {
  explicit TraceRange(const char *name) { nvtxRangePushA(name); }
  ~TraceRange() { nvtxRangePop(); }
  TraceRange(const TraceRange &) = delete;
  TraceRange &operator=(const TraceRange &) = delete;
};

// ------------------------------------------------------------ checked build
// Built with -DFAMSA_CHECKED (libfamsa_gpu_checked.so), kernels test the
// invariants their indexing relies on -- every index inside its buffer, every
// row inside its kernel's width, every component id inside its range -- and
// count each failure instead of trusting it; a failed check skips the access
// it guards.  It stands in for a memory checker.  The normal build compiles
// every check to nothing.  Each translation unit keeps its own counters
// (count, line of the first failure), read through famsa_debug_check_count.
using CheckReader = void (*)(unsigned long long *count_and_line);
int register_check_reader(CheckReader r);
void read_checks(unsigned long long *count, unsigned long long *first_line);

}  // namespace famsa

#ifdef FAMSA_CHECKED
namespace {
__device__ unsigned long long g_check_fail[2];  // failures, line of the first one
__device__ __forceinline__ bool famsa_expect(bool ok, int line) {
  if (!ok) {
    atomicAdd(&g_check_fail[0], 1ull);
    atomicCAS(&g_check_fail[1], 0ull, (unsigned long long)line);
  }
  return ok;
}
void read_checks_here(unsigned long long *v) {
  if (cudaMemcpyFromSymbol(v, g_check_fail, sizeof(g_check_fail)) != cudaSuccess) v[0] = v[1] = 0;
}
const int g_check_registered = famsa::register_check_reader(read_checks_here);
}  // namespace
#define FAMSA_EXPECT(cond) famsa_expect((cond), __LINE__)
#else
#define FAMSA_EXPECT(cond) true
#endif
