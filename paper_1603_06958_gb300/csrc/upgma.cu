// famsa_upgma_tree, famsa_nj_tree: UPGMA and neighbour joining over the
// family's LCS distances.
//
// FAMSA Methods, "Determination of the guide tree": UPGMA and neighbour
// joining are the guide trees the paper names beside single linkage, and it
// sets them against SLINK for memory -- they need the whole O(k^2) distance
// matrix, which 288 GB of HBM holds for families of tens of thousands.
//
// Distances are indel^2 / LCS as doubles (one correctly rounded division;
// +inf for LCS = 0).  UPGMA: every step takes the pair of live clusters in
// slots a < b with the smallest (d, a, b), keeps the merged cluster in slot
// a, and sets d(a, c) = (n_a * d(a, c) + n_b * d(b, c)) / (n_a + n_b) with
// each operation rounded on its own (no fused multiply-add), so the result
// is the plain sequential algorithm's bit for bit.
//
// Per row i the UPGMA state keeps its smallest (d(i, j), j) over live j > i.
// A step reads the smallest row minimum, rewrites row and column a, and then
// only rows whose minimum pointed at a or b, or that now see a smaller value
// at a, change; those pointing at a or b (usually few) are rescanned.
//
// Neighbour joining sums every row once (one thread per row, in increasing
// j as the sequential algorithm does), then keeps the sums by the update
// R(c) -= d(a, c) + d(b, c) - d(u, c) of each join; per step it recomputes
// every live pair's Q(a, b) = (r - 2) d(a, b) - R(a) - R(b), one CTA per
// live row, so a step is O(k^2) reads of the matrix and the tree O(k^3).
#include <algorithm>
#include <cmath>

#include "slink_common.cuh"

using namespace famsa;

namespace {

constexpr int32_t kNjMaxK = 32768;  // O(k^3) time: about a minute at this size

struct Upgma {
  double *D;         // k x k
  double *rval;      // per row: smallest d(i, j) over live j > i
  int32_t *rarg;     // its j (-1: no live j > i)
  int32_t *n;        // cluster sizes per slot
  int32_t *id;       // cluster id per slot
  uint8_t *live;
  int32_t *list;     // rows to rescan
  int32_t *ctl;      // [0] rescan count, [1] a, [2] b, [3] step
  double *pick_d;
  int32_t *merges;
  double *heights;
  int32_t *sizes;
  int32_t k;
};

__global__ void k_up_dist(const int32_t *tri, const int32_t *len, int32_t k, double *D) {
  const int64_t total = (int64_t)k * k;
  for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < total; x += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = x / k, j = x - i * k;
    double d = 0.0;
    if (j != i) {
      const int64_t a = min(i, j), b = max(i, j);
      const int32_t L = tri[a * k - a * (a + 1) / 2 + (b - a - 1)];
      const int64_t indel = (int64_t)len[i] + len[j] - 2 * (int64_t)L;
      d = L == 0 ? __longlong_as_double(0x7ff0000000000000LL) : __ddiv_rn((double)(indel * indel), (double)L);
    }
    D[x] = d;
  }
}

__device__ __forceinline__ bool pair_lt(double v1, int32_t j1, double v2, int32_t j2) {
  if (j2 < 0) return j1 >= 0;
  if (j1 < 0) return false;
  return v1 < v2 || (v1 == v2 && j1 < j2);
}

// smallest (D[i][j], j) over live j > i, one CTA per row
__device__ void row_min(const Upgma &U, int32_t i, double *sv, int32_t *sj) {
  double bv = 0.0;
  int32_t bj = -1;
  const double *row = U.D + (int64_t)i * U.k;
  for (int32_t j = i + 1 + threadIdx.x; j < U.k; j += blockDim.x)
    if (U.live[j] && pair_lt(row[j], j, bv, bj)) { bv = row[j]; bj = j; }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int d = 16; d > 0; d >>= 1) {
    const double v2 = __shfl_down_sync(0xffffffffu, bv, d);
    const int32_t j2 = __shfl_down_sync(0xffffffffu, bj, d);
    if (pair_lt(v2, j2, bv, bj)) { bv = v2; bj = j2; }
  }
  if (lane == 0) { sv[warp] = bv; sj[warp] = bj; }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w)
      if (pair_lt(sv[w], sj[w], bv, bj)) { bv = sv[w]; bj = sj[w]; }
    U.rval[i] = bv;
    U.rarg[i] = bj;
  }
  __syncthreads();
}

__global__ void k_up_rowmin_all(Upgma U) {
  __shared__ double sv[32];
  __shared__ int32_t sj[32];
  row_min(U, blockIdx.x, sv, sj);
}

// the smallest row minimum (d, a, b) over live rows: one CTA
__global__ void k_up_pick(Upgma U) {
  __shared__ double sv[32];
  __shared__ int32_t sa[32], sb[32];
  double bv = 0.0;
  int32_t ba = -1, bb = -1;
  for (int32_t i = threadIdx.x; i < U.k; i += blockDim.x) {
    if (!U.live[i] || U.rarg[i] < 0) continue;
    const double v = U.rval[i];
    if (ba < 0 || v < bv || (v == bv && (i < ba || (i == ba && U.rarg[i] < bb)))) { bv = v; ba = i; bb = U.rarg[i]; }
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int d = 16; d > 0; d >>= 1) {
    const double v2 = __shfl_down_sync(0xffffffffu, bv, d);
    const int32_t a2 = __shfl_down_sync(0xffffffffu, ba, d), b2 = __shfl_down_sync(0xffffffffu, bb, d);
    if (a2 >= 0 && (ba < 0 || v2 < bv || (v2 == bv && (a2 < ba || (a2 == ba && b2 < bb))))) { bv = v2; ba = a2; bb = b2; }
  }
  if (lane == 0) { sv[warp] = bv; sa[warp] = ba; sb[warp] = bb; }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) {
      const double v2 = sv[w];
      const int32_t a2 = sa[w], b2 = sb[w];
      if (a2 >= 0 && (ba < 0 || v2 < bv || (v2 == bv && (a2 < ba || (a2 == ba && b2 < bb))))) { bv = v2; ba = a2; bb = b2; }
    }
    U.ctl[0] = 0;
    U.ctl[1] = ba;
    U.ctl[2] = bb;
    *U.pick_d = bv;
  }
}

// row and column a of the merged cluster
__global__ void k_up_merge(Upgma U) {
  const int32_t a = U.ctl[1], b = U.ctl[2];
  if (a < 0) return;
  const double na = (double)U.n[a], nb = (double)U.n[b], nab = (double)(U.n[a] + U.n[b]);
  for (int32_t c = blockIdx.x * blockDim.x + threadIdx.x; c < U.k; c += gridDim.x * blockDim.x) {
    if (!U.live[c] || c == a || c == b) continue;
    const double x = __dmul_rn(na, U.D[(int64_t)a * U.k + c]);
    const double y = __dmul_rn(nb, U.D[(int64_t)b * U.k + c]);
    const double v = __ddiv_rn(__dadd_rn(x, y), nab);
    U.D[(int64_t)a * U.k + c] = v;
    U.D[(int64_t)c * U.k + a] = v;
  }
}

// the record of step t, and slot a takes the merged cluster
__global__ void k_up_book(Upgma U) {
  const int32_t a = U.ctl[1], b = U.ctl[2], t = U.ctl[3];
  if (a < 0) return;
  const int32_t ia = U.id[a], ib = U.id[b];
  U.merges[2 * t] = min(ia, ib);
  U.merges[2 * t + 1] = max(ia, ib);
  U.heights[t] = *U.pick_d;
  U.n[a] += U.n[b];
  U.sizes[t] = U.n[a];
  U.id[a] = U.k + t;
  U.live[b] = 0;
  U.ctl[3] = t + 1;
}

// row minima after the step: rows below a may see a new smallest value at a;
// rows whose minimum pointed at a or b, and row a itself, are rescanned
__global__ void k_up_fix(Upgma U) {
  const int32_t a = U.ctl[1], b = U.ctl[2];
  if (a < 0) return;
  const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= U.k || !U.live[i] || i > b) return;
  const int32_t r = U.rarg[i];
  bool rescan = i == a || r == a || r == b;
  if (!rescan && i < a) {
    const double v = U.D[(int64_t)i * U.k + a];
    if (pair_lt(v, a, U.rval[i], r)) { U.rval[i] = v; U.rarg[i] = a; }
  }
  if (rescan) U.list[atomicAdd(&U.ctl[0], 1)] = i;
}

__global__ void k_up_rescan(Upgma U) {
  __shared__ double sv[32];
  __shared__ int32_t sj[32];
  const int32_t cnt = U.ctl[0];
  for (int32_t x = blockIdx.x; x < cnt; x += gridDim.x) row_min(U, U.list[x], sv, sj);
}

__global__ void k_up_init(Upgma U) {
  const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < U.k) { U.n[i] = 1; U.id[i] = i; U.live[i] = 1; }
  if (i == 0) { U.ctl[0] = 0; U.ctl[1] = -1; U.ctl[2] = -1; U.ctl[3] = 0; }
}


// ------------------------------------------------------------ neighbour joining
struct Nj {
  double *D;        // k x k, symmetric
  double *R;        // per live slot: the sum of its distances to the other live slots
  double *rq;       // per live row i: smallest Q(i, j) over live j > i
  int32_t *rj;      // its j (-1: none)
  int32_t *n;       // cluster sizes per slot
  int32_t *id;      // cluster id per slot
  uint8_t *live;
  int32_t *list;    // the live slots, in no particular order (r of them at step k - r)
  int32_t *pos;     // a live slot's place in list
  int32_t *ctl;     // [0] a, [1] b, [2] an infinite distance seen
  double *dab;      // d(a, b) of the step
  int32_t *merges;
  double *lengths;
  int32_t *sizes;
  int32_t k;
};

__global__ void k_nj_init(Nj J) {
  const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < J.k) { J.n[i] = 1; J.id[i] = i; J.live[i] = 1; J.list[i] = i; J.pos[i] = i; }
  if (i == 0) { J.ctl[0] = -1; J.ctl[1] = -1; J.ctl[2] = 0; }
}

// neighbour joining is undefined with an infinite distance (a pair with LCS 0)
__global__ void k_nj_check(Nj J) {
  const int64_t total = (int64_t)J.k * J.k;
  for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < total; x += (int64_t)gridDim.x * blockDim.x)
    if (isinf(J.D[x])) J.ctl[2] = 1;
}

// the first row sums, R(i) over j != i in increasing j (thread i reads column
// i: coalesced across threads, and equal to row i since D is exactly symmetric)
__global__ void k_nj_rsum(Nj J) {
  const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= J.k) return;
  double s = 0.0;
  for (int32_t j = 0; j < J.k; ++j)
    if (j != i) s = __dadd_rn(s, J.D[(int64_t)j * J.k + i]);
  J.R[i] = s;
}

__device__ __forceinline__ bool q_lt(double v1, int32_t j1, double v2, int32_t j2) {
  if (j2 < 0) return j1 >= 0;
  if (j1 < 0) return false;
  return v1 < v2 || (v1 == v2 && j1 < j2);
}

// The order of finite doubles as unsigned integers: flip the sign bit of a
// non-negative value and every bit of a negative one (the two zeros, equal as
// doubles, share a key).  The scan below compares these on the integer ALU
// instead of issuing a fourth FP64 instruction per pair.
__device__ __forceinline__ uint64_t dkey(double q) {
  uint64_t b = (uint64_t)__double_as_longlong(q);
  if ((b << 1) == 0) b = 0;
  return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}

// live row list[blockIdx.x]: the smallest (Q(i, j), j) over live j > i
__global__ void k_nj_qrow(Nj J, double rm2) {
  __shared__ uint64_t sk[32];
  __shared__ double sv[32];
  __shared__ int32_t sj[32];
  const int32_t i = J.list[blockIdx.x];
  const double Ri = J.R[i];
  const double *row = J.D + (int64_t)i * J.k;
  uint64_t bk = ~0ull;
  double bv = 0.0;
  int32_t bj = -1;
  for (int32_t j = i + 1 + threadIdx.x; j < J.k; j += blockDim.x) {
    if (!J.live[j]) continue;
    const double q = __dsub_rn(__dsub_rn(__dmul_rn(rm2, row[j]), Ri), J.R[j]);
    const uint64_t kq = dkey(q);
    if (kq < bk) { bk = kq; bv = q; bj = j; }  // j ascends per thread: the first minimum stays
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int d = 16; d > 0; d >>= 1) {
    const uint64_t k2 = __shfl_down_sync(0xffffffffu, bk, d);
    const double v2 = __shfl_down_sync(0xffffffffu, bv, d);
    const int32_t j2 = __shfl_down_sync(0xffffffffu, bj, d);
    if (j2 >= 0 && (bj < 0 || k2 < bk || (k2 == bk && j2 < bj))) { bk = k2; bv = v2; bj = j2; }
  }
  if (lane == 0) { sk[warp] = bk; sv[warp] = bv; sj[warp] = bj; }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w)
      if (sj[w] >= 0 && (bj < 0 || sk[w] < bk || (sk[w] == bk && sj[w] < bj))) { bk = sk[w]; bv = sv[w]; bj = sj[w]; }
    J.rq[i] = bv;
    J.rj[i] = bj;
  }
}

// record step t (r clusters live): the pair (a, b) with the smallest
// (Q, a, b) (or, with two clusters left, the two), its branch lengths and
// R(u); slot a takes the new cluster, b leaves the live list
__global__ void k_nj_pick(Nj J, int32_t t, int32_t r) {
  __shared__ double sv[32];
  __shared__ int32_t sa[32], sb[32];
  double bv = 0.0;
  int32_t ba = -1, bb = -1;
  for (int32_t p = threadIdx.x; p < r; p += blockDim.x) {
    const int32_t i = J.list[p];
    const int32_t j = r > 2 ? J.rj[i] : 0;  // with two left, the lower slot wins
    if (j < 0) continue;
    const double v = r > 2 ? J.rq[i] : 0.0;
    if (ba < 0 || v < bv || (v == bv && (i < ba || (i == ba && j < bb)))) { bv = v; ba = i; bb = j; }
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int d = 16; d > 0; d >>= 1) {
    const double v2 = __shfl_down_sync(0xffffffffu, bv, d);
    const int32_t a2 = __shfl_down_sync(0xffffffffu, ba, d), b2 = __shfl_down_sync(0xffffffffu, bb, d);
    if (a2 >= 0 && (ba < 0 || v2 < bv || (v2 == bv && (a2 < ba || (a2 == ba && b2 < bb))))) { bv = v2; ba = a2; bb = b2; }
  }
  if (lane == 0) { sv[warp] = bv; sa[warp] = ba; sb[warp] = bb; }
  __syncthreads();
  if (threadIdx.x != 0) return;
  for (int w = 1; w < (int)(blockDim.x >> 5); ++w) {
    const double v2 = sv[w];
    const int32_t a2 = sa[w], b2 = sb[w];
    if (a2 >= 0 && (ba < 0 || v2 < bv || (v2 == bv && (a2 < ba || (a2 == ba && b2 < bb))))) { bv = v2; ba = a2; bb = b2; }
  }
  double da, db;
  if (r > 2) {
    const double dab = J.D[(int64_t)ba * J.k + bb];
    da = __dadd_rn(__dmul_rn(dab, 0.5), __ddiv_rn(__dsub_rn(J.R[ba], J.R[bb]), (double)(2 * (r - 2))));
    db = __dsub_rn(dab, da);
    *J.dab = dab;
    J.R[ba] = __dmul_rn(__dsub_rn(__dadd_rn(J.R[ba], J.R[bb]), __dmul_rn((double)r, dab)), 0.5);
  } else {
    bb = J.list[0] == ba ? J.list[1] : J.list[0];  // the other live slot
    da = __dmul_rn(J.D[(int64_t)ba * J.k + bb], 0.5);
    db = da;
  }
  const int32_t ia = J.id[ba], ib = J.id[bb];
  const bool lo_a = ia < ib;
  J.merges[2 * t] = lo_a ? ia : ib;
  J.merges[2 * t + 1] = lo_a ? ib : ia;
  J.lengths[2 * t] = lo_a ? da : db;
  J.lengths[2 * t + 1] = lo_a ? db : da;
  J.n[ba] += J.n[bb];
  J.sizes[t] = J.n[ba];
  J.id[ba] = J.k + t;
  J.live[bb] = 0;
  const int32_t p = J.pos[bb], last = J.list[r - 1];
  J.list[p] = last;
  J.pos[last] = p;
  J.ctl[0] = ba;
  J.ctl[1] = bb;
}

// row and column a of the new cluster and the other live rows' sums:
// d(a, c) = (d(a, c) + d(b, c) - d(a, b)) / 2, R(c) = R(c) - d(a, c) - d(b, c) + d(u, c)
__global__ void k_nj_merge(Nj J, int32_t nlive) {
  const int32_t a = J.ctl[0], b = J.ctl[1];
  const double dab = *J.dab;
  for (int32_t p = blockIdx.x * blockDim.x + threadIdx.x; p < nlive; p += gridDim.x * blockDim.x) {
    const int32_t c = J.list[p];
    if (c == a) continue;
    const double dac = J.D[(int64_t)a * J.k + c], dbc = J.D[(int64_t)b * J.k + c];
    const double v = __dmul_rn(__dsub_rn(__dadd_rn(dac, dbc), dab), 0.5);
    J.R[c] = __dadd_rn(__dsub_rn(__dsub_rn(J.R[c], dac), dbc), v);
    J.D[(int64_t)a * J.k + c] = v;
    J.D[(int64_t)c * J.k + a] = v;
  }
}
}  // namespace

// all pairs' LCS in caller labels (the i < j triangle), then the k x k distances
static cudaError_t family_distances(Family *f, Scratch &sc, double *D, int32_t *d_iota) {
  const int32_t k = f->k;
  cudaStream_t st = sc.st;
  int32_t *tri = sc.get<int32_t>((size_t)k * (k - 1) / 2);
  if (sc.err != cudaSuccess) return sc.err;
  std::vector<int32_t> h_w(k), h_id(k);
  for (int32_t s = 0; s < k; ++s) { h_w[s] = (f->h_slen[s] + 63) / 64; h_id[s] = s; }
  cudaError_t err = cudaMemcpyAsync(d_iota, h_id.data(), sizeof(int32_t) * k, cudaMemcpyHostToDevice, st);
  LcsBatch b;
  b.peq = f->d_peq;
  b.colres = f->d_colres;
  b.group_off = f->d_group_off;
  b.group_chunks = f->d_group_chunks;
  b.col_perm = f->d_perm;
  b.col_len = f->d_slen;
  b.n_cols = k;
  b.k = k;
  b.row_peq_off = f->d_peq_off;
  b.row_len = f->d_slen;
  b.row_id = d_iota;
  b.row_orig = f->d_perm;
  b.n_rows = k;
  b.h_row_w = h_w.data();
  b.h_row_id = h_id.data();
  b.mode = kOutTriOrig;
  b.out = tri;
  b.triangle = true;
  int64_t launches = 0;
  if (err == cudaSuccess) err = launch_lcs(b, st, &launches);
  if (err == cudaSuccess) {
    k_up_dist<<<152 * 16, 256, 0, st>>>(tri, f->d_len, k, D);
    err = cudaGetLastError();
  }
  // the host vectors above are read by the copy: wait before they go
  if (err == cudaSuccess) err = cudaStreamSynchronize(st);
  return err;
}

extern "C" int famsa_upgma_tree(const famsa_family *fh, int32_t *merges, double *heights, int32_t *sizes,
                                int on_device, void *cuda_stream) {
  if (!fh || !merges || !heights || !sizes) return FAMSA_EINVAL;
  Family *f = const_cast<Family *>(reinterpret_cast<const Family *>(fh));
  const int32_t k = f->k;
  if (k < 2) return FAMSA_OK;
  if ((int64_t)k * k > ((int64_t)1 << 34)) return FAMSA_ERANGE;  // the matrix alone would pass 128 GB
  std::lock_guard<std::mutex> lk(f->mu);
  cudaStream_t st = (cudaStream_t)cuda_stream;
  Scratch sc;
  sc.st = st;
  Upgma U;
  U.k = k;
  U.D = sc.get<double>((size_t)k * k);
  U.rval = sc.get<double>(k);
  U.rarg = sc.get<int32_t>(k);
  U.n = sc.get<int32_t>(k);
  U.id = sc.get<int32_t>(k);
  U.live = sc.get<uint8_t>(k);
  U.list = sc.get<int32_t>(k);
  U.ctl = sc.get<int32_t>(4);
  U.pick_d = sc.get<double>(1);
  int32_t *d_iota = sc.get<int32_t>(k);
  U.merges = on_device ? merges : sc.get<int32_t>(2 * (size_t)(k - 1));
  U.heights = on_device ? heights : sc.get<double>((size_t)(k - 1));
  U.sizes = on_device ? sizes : sc.get<int32_t>((size_t)(k - 1));
  cudaError_t err = sc.err;
  if (err == cudaSuccess) err = family_distances(f, sc, U.D, d_iota);
  if (err == cudaSuccess) {
    const unsigned nb = (unsigned)((k + 255) / 256);
    k_up_init<<<nb, 256, 0, st>>>(U);
    k_up_rowmin_all<<<(unsigned)k, 256, 0, st>>>(U);
    for (int32_t t = 0; t + 1 < k && err == cudaSuccess; ++t) {
      k_up_pick<<<1, 1024, 0, st>>>(U);
      k_up_merge<<<std::min<unsigned>(nb, 152), 256, 0, st>>>(U);
      k_up_book<<<1, 1, 0, st>>>(U);
      k_up_fix<<<nb, 256, 0, st>>>(U);
      k_up_rescan<<<152, 256, 0, st>>>(U);
      if ((t & 1023) == 0) err = cudaGetLastError();
    }
    if (err == cudaSuccess) err = cudaGetLastError();
  }
  if (err == cudaSuccess && !on_device) {
    err = cudaMemcpyAsync(merges, U.merges, sizeof(int32_t) * 2 * (size_t)(k - 1), cudaMemcpyDeviceToHost, st);
    if (err == cudaSuccess)
      err = cudaMemcpyAsync(heights, U.heights, sizeof(double) * (size_t)(k - 1), cudaMemcpyDeviceToHost, st);
    if (err == cudaSuccess)
      err = cudaMemcpyAsync(sizes, U.sizes, sizeof(int32_t) * (size_t)(k - 1), cudaMemcpyDeviceToHost, st);
  }
  if (err == cudaSuccess) err = cudaStreamSynchronize(st);
  else cudaStreamSynchronize(st);
  sc.release();
  return status_from_cuda(err);
}

extern "C" int famsa_nj_tree(const famsa_family *fh, int32_t *merges, double *lengths, int32_t *sizes,
                             int on_device, void *cuda_stream) {
  if (!fh || !merges || !lengths || !sizes) return FAMSA_EINVAL;
  Family *f = const_cast<Family *>(reinterpret_cast<const Family *>(fh));
  const int32_t k = f->k;
  if (k < 2) return FAMSA_OK;
  if (k > kNjMaxK) return FAMSA_ERANGE;
  std::lock_guard<std::mutex> lk(f->mu);
  cudaStream_t st = (cudaStream_t)cuda_stream;
  Scratch sc;
  sc.st = st;
  Nj J;
  J.k = k;
  J.D = sc.get<double>((size_t)k * k);
  J.R = sc.get<double>(k);
  J.rq = sc.get<double>(k);
  J.rj = sc.get<int32_t>(k);
  J.n = sc.get<int32_t>(k);
  J.id = sc.get<int32_t>(k);
  J.live = sc.get<uint8_t>(k);
  J.list = sc.get<int32_t>(k);
  J.pos = sc.get<int32_t>(k);
  J.ctl = sc.get<int32_t>(3);
  J.dab = sc.get<double>(1);
  int32_t *d_iota = sc.get<int32_t>(k);
  J.merges = on_device ? merges : sc.get<int32_t>(2 * (size_t)(k - 1));
  J.lengths = on_device ? lengths : sc.get<double>(2 * (size_t)(k - 1));
  J.sizes = on_device ? sizes : sc.get<int32_t>((size_t)(k - 1));
  cudaError_t err = sc.err;
  if (err == cudaSuccess) err = family_distances(f, sc, J.D, d_iota);
  int32_t inf = 0;
  if (err == cudaSuccess) {
    const unsigned nb = (unsigned)((k + 255) / 256);
    k_nj_init<<<nb, 256, 0, st>>>(J);
    k_nj_check<<<152 * 8, 256, 0, st>>>(J);
    err = cudaMemcpyAsync(&inf, J.ctl + 2, sizeof(int32_t), cudaMemcpyDeviceToHost, st);
    if (err == cudaSuccess) err = cudaStreamSynchronize(st);
  }
  if (err == cudaSuccess && !inf) {
    k_nj_rsum<<<(unsigned)((k + 63) / 64), 64, 0, st>>>(J);
    for (int32_t t = 0; t + 1 < k && err == cudaSuccess; ++t) {
      const int32_t r = k - t;  // live clusters
      if (r > 2) k_nj_qrow<<<(unsigned)r, 256, 0, st>>>(J, (double)(r - 2));
      k_nj_pick<<<1, 1024, 0, st>>>(J, t, r);
      if (r > 2) k_nj_merge<<<std::min<unsigned>((unsigned)((r + 254) / 255), 152), 256, 0, st>>>(J, r - 1);
      if ((t & 1023) == 0) err = cudaGetLastError();
    }
    if (err == cudaSuccess) err = cudaGetLastError();
  }
  if (err == cudaSuccess && !inf && !on_device) {
    err = cudaMemcpyAsync(merges, J.merges, sizeof(int32_t) * 2 * (size_t)(k - 1), cudaMemcpyDeviceToHost, st);
    if (err == cudaSuccess)
      err = cudaMemcpyAsync(lengths, J.lengths, sizeof(double) * 2 * (size_t)(k - 1), cudaMemcpyDeviceToHost, st);
    if (err == cudaSuccess)
      err = cudaMemcpyAsync(sizes, J.sizes, sizeof(int32_t) * (size_t)(k - 1), cudaMemcpyDeviceToHost, st);
  }
  if (err == cudaSuccess) err = cudaStreamSynchronize(st);
  else cudaStreamSynchronize(st);
  sc.release();
  if (err == cudaSuccess && inf) return FAMSA_ERANGE;
  return status_from_cuda(err);
}
