/*
 * CPU oracle for FAMSA stages I+II (test infrastructure only).
 *
 * Plain, slow, obviously correct restatements of what the GPU path computes.
 * Only the test suite, the smoke check and the benchmark's CPU-baseline arm
 * may load this library; the product path never does.  It shares no code,
 * header, table or helper with the CUDA library.
 *
 * What it computes (citations are to the FAMSA paper, Methods):
 *   - LCS length by the textbook dynamic-programming rule ("Pairwise
 *     similarities calculation": the LCS length is the maximal number of
 *     perfectly matching columns, computable by a straightforward DP rule).
 *     Matching is literal code equality (ambiguity codes match only
 *     themselves).
 *   - LCS length a second, independent way: the bit-parallel recurrence the
 *     paper applies in stage I (same subsection), written as plain scalar
 *     64-bit C with the carry rippled word by word.  It exists so that trees
 *     of families far too large for the DP can still be computed by the
 *     oracle; it is pinned against the DP and never against the GPU.
 *   - indel(A,B) = |A| + |B| - 2 LCS(A,B) and similarity = LCS / indel^2
 *     (the two displayed equations of that subsection).  The tree is keyed on
 *     the exact rational distance indel^2 / LCS, a strictly decreasing
 *     transform of the similarity; LCS = 0 gives +infinity, indel = 0 gives 0.
 *     Keys are compared by 128-bit cross multiplication, never in floating
 *     point.
 *   - single-linkage guide tree ("Determination of the guide tree") in
 *     Sibson's pointer representation (pi, lambda), three independent ways:
 *       (i)   Sibson's SLINK insertion, one point at a time in index order;
 *       (ii)  naive agglomeration: repeatedly merge the closest two clusters
 *             with the single-link update min(d(A,C), d(B,C));
 *       (iii) the definition: minimax (bottleneck) path distances by a
 *             Floyd-Warshall closure, then lambda(j) = min_{l>j} u(j,l) and
 *             pi(j) = max{ l > j : u(j,l) <= lambda(j) }.
 *   - merge list: indices sorted by (lambda, index) ascending, then
 *     union-find over (j, pi(j)) at height lambda(j); new cluster ids k+t.
 *
 * All functions return 0 on success and a negative value on bad arguments
 * or allocation failure.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef unsigned __int128 u128;

/* ------------------------------------------------------------ keys */
typedef struct { uint64_t num; uint32_t den; } okey; /* num/den, den == 0 means +inf */

static okey key_from_lcs(int32_t lcs, int32_t la, int32_t lb) {
  okey k;
  uint64_t indel = (uint64_t)(la + lb - 2 * lcs);
  k.num = indel * indel;
  k.den = (uint32_t)lcs;
  if (k.den == 0) k.num = 1; /* +inf, canonical */
  return k;
}
static const okey KEY_INF = {1, 0};

/* a < b */
static int key_lt(okey a, okey b) {
  if (a.den == 0) return 0;
  if (b.den == 0) return 1;
  return (u128)a.num * b.den < (u128)b.num * a.den;
}
static okey key_min(okey a, okey b) { return key_lt(b, a) ? b : a; }
static okey key_max(okey a, okey b) { return key_lt(a, b) ? b : a; }

static uint64_t gcd64(uint64_t a, uint64_t b) {
  while (b) { uint64_t t = a % b; a = b; b = t; }
  return a;
}
static void key_reduce(okey k, uint64_t *num, uint32_t *den) {
  if (k.den == 0) { *num = 1; *den = 0; return; }
  if (k.num == 0) { *num = 0; *den = 1; return; }
  uint64_t g = gcd64(k.num, k.den);
  *num = k.num / g;
  *den = (uint32_t)(k.den / g);
}

/* exposed for the comparator tests: returns -1, 0, 1 */
int oracle_key_cmp(uint64_t an, uint32_t ad, uint64_t bn, uint32_t bd) {
  okey a = {an, ad}, b = {bn, bd};
  if (a.den == 0 && a.num == 0) return -2;
  if (b.den == 0 && b.num == 0) return -2;
  if (key_lt(a, b)) return -1;
  if (key_lt(b, a)) return 1;
  return 0;
}

/* ------------------------------------------------------------ LCS by DP */
/* L[i][j] = L[i-1][j-1] + 1 if a_i == b_j else max(L[i-1][j], L[i][j-1]); two rows. */
static int32_t lcs_dp(const uint8_t *a, int32_t la, const uint8_t *b, int32_t lb, int32_t *row) {
  for (int32_t j = 0; j <= lb; ++j) row[j] = 0;
  for (int32_t i = 1; i <= la; ++i) {
    int32_t diag = 0; /* L[i-1][j-1] */
    for (int32_t j = 1; j <= lb; ++j) {
      int32_t up = row[j];      /* L[i-1][j] */
      int32_t left = row[j - 1]; /* L[i][j-1] (already overwritten) */
      int32_t v;
      if (a[i - 1] == b[j - 1]) v = diag + 1;
      else v = up > left ? up : left;
      diag = up;
      row[j] = v;
    }
  }
  return row[lb];
}

int32_t oracle_lcs(const uint8_t *a, int32_t la, const uint8_t *b, int32_t lb) {
  if (la < 0 || lb < 0) return -1;
  int32_t *row = (int32_t *)malloc(sizeof(int32_t) * (size_t)(lb + 1));
  if (!row) return -2;
  int32_t r = lcs_dp(a, la, b, lb, row);
  free(row);
  return r;
}

static int32_t max_len(const int64_t *off, int32_t k) {
  int32_t m = 0;
  for (int32_t i = 0; i < k; ++i) {
    int32_t l = (int32_t)(off[i + 1] - off[i]);
    if (l > m) m = l;
  }
  return m;
}

static void set_threads(int nthreads) {
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#else
  (void)nthreads;
#endif
}

int oracle_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* ------------------------------------------------------------ LCS, bit-parallel */
/*
 * The bit-parallel form of the same LCS length (FAMSA Methods, "Pairwise
 * similarities calculation": the LCS is computed with the bit-parallel
 * algorithm it cites, 64 DP cells per machine word).  Position p of A is bit
 * p % 64 of word p / 64 of a vector of W = ceil(|A| / 64) words.
 * Peq[c] has bit p set exactly when A[p] == c (any byte value c: matching is
 * literal equality).  V starts with every bit set; each symbol c of B, in
 * order, replaces V by
 *     V' = (V + (V & Peq[c])) | (V & ~Peq[c]),
 * where + adds the two W-word numbers, word 0 least significant, the carry
 * out of word w going into word w + 1 and the carry out of the last word
 * dropped.  The LCS length is the number of zero bits of V among the |A|
 * positions.  Bits above |A| in the last word stay one: Peq is zero there,
 * so both terms of the OR keep them set.
 */
#define BP_CODES 256

static void bp_peq(const uint8_t *a, int32_t la, int32_t W, uint64_t *peq /* [BP_CODES][W] */) {
  memset(peq, 0, sizeof(uint64_t) * (size_t)BP_CODES * (size_t)W);
  for (int32_t p = 0; p < la; ++p) peq[(size_t)a[p] * W + p / 64] |= (uint64_t)1 << (p % 64);
}

/* the recurrence for W words; V is the caller's W-word scratch */
static inline __attribute__((always_inline)) int32_t
bp_lcs_body(const uint64_t *peq, const int32_t W, int32_t la, const uint8_t *b, int32_t lb,
            uint64_t *V) {
  for (int32_t w = 0; w < W; ++w) V[w] = ~(uint64_t)0;
  for (int32_t i = 0; i < lb; ++i) {
    const uint64_t *P = peq + (size_t)b[i] * W;
    unsigned long long carry = 0;
    for (int32_t w = 0; w < W; ++w) {
      unsigned long long v = V[w], s, t;
      unsigned c1 = __builtin_uaddll_overflow(v, v & P[w], &s); /* V + (V & Peq[c]) */
      unsigned c2 = __builtin_uaddll_overflow(s, carry, &t);    /* + carry from word w - 1 */
      carry = c1 | c2;                                          /* at most one is set */
      V[w] = t | (v & ~P[w]);                                   /* | (V & ~Peq[c]) */
    }
  }
  int32_t ones = 0;
  for (int32_t p = 0; p < la; ++p) ones += (int32_t)((V[p / 64] >> (p % 64)) & 1);
  return la - ones;
}

/* The same function; small widths are spelled out as constants only so that the
   compiler keeps V in registers (about 1.5x faster on the host, same arithmetic). */
static int32_t bp_lcs(const uint64_t *peq, int32_t W, int32_t la, const uint8_t *b, int32_t lb,
                      uint64_t *V) {
  uint64_t R[8];
  switch (W) {
    case 1: return bp_lcs_body(peq, 1, la, b, lb, R);
    case 2: return bp_lcs_body(peq, 2, la, b, lb, R);
    case 3: return bp_lcs_body(peq, 3, la, b, lb, R);
    case 4: return bp_lcs_body(peq, 4, la, b, lb, R);
    case 5: return bp_lcs_body(peq, 5, la, b, lb, R);
    case 6: return bp_lcs_body(peq, 6, la, b, lb, R);
    case 7: return bp_lcs_body(peq, 7, la, b, lb, R);
    case 8: return bp_lcs_body(peq, 8, la, b, lb, R);
    default: return bp_lcs_body(peq, W, la, b, lb, V);
  }
}

static int32_t words_of(int32_t len) { return len > 0 ? (len + 63) / 64 : 1; }

int32_t oracle_lcs_bitpar(const uint8_t *a, int32_t la, const uint8_t *b, int32_t lb) {
  if (la < 0 || lb < 0) return -1;
  int32_t W = words_of(la);
  uint64_t *peq = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)BP_CODES * (size_t)W);
  uint64_t *V = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)W);
  if (!peq || !V) { free(peq); free(V); return -2; }
  bp_peq(a, la, W, peq);
  int32_t r = bp_lcs(peq, W, la, b, lb, V);
  free(peq);
  free(V);
  return r;
}

/* bit-parallel LCS for an explicit list of pairs; A = pa[t] is the Peq side */
int oracle_lcs_pairs_bitpar(const uint8_t *res, const int64_t *off, int32_t k, const int32_t *pa,
                            const int32_t *pb, int64_t npairs, int32_t *out, int nthreads) {
  if (k < 1 || npairs < 0) return -1;
  set_threads(nthreads);
  int32_t W = words_of(max_len(off, k));
  int bad = 0;
#pragma omp parallel
  {
    uint64_t *peq = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)BP_CODES * (size_t)W);
    uint64_t *V = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)W);
    if (!peq || !V) {
#pragma omp atomic write
      bad = 1;
    }
#pragma omp for schedule(dynamic, 64)
    for (int64_t t = 0; t < npairs; ++t) {
      if (!peq || !V) continue;
      int32_t i = pa[t], j = pb[t];
      int32_t la = (int32_t)(off[i + 1] - off[i]);
      int32_t wa = words_of(la);
      bp_peq(res + off[i], la, wa, peq);
      out[t] = bp_lcs(peq, wa, la, res + off[j], (int32_t)(off[j + 1] - off[j]), V);
    }
    free(peq);
    free(V);
  }
  return bad ? -2 : 0;
}

/* LCS for an explicit list of pairs (pa[t], pb[t]) */
int oracle_lcs_pairs(const uint8_t *res, const int64_t *off, int32_t k, const int32_t *pa,
                     const int32_t *pb, int64_t npairs, int32_t *out, int nthreads) {
  if (k < 1 || npairs < 0) return -1;
  set_threads(nthreads);
  int32_t ml = max_len(off, k);
  int bad = 0;
#pragma omp parallel
  {
    int32_t *row = (int32_t *)malloc(sizeof(int32_t) * (size_t)(ml + 1));
    if (!row) {
#pragma omp atomic write
      bad = 1;
    }
#pragma omp for schedule(dynamic, 64)
    for (int64_t t = 0; t < npairs; ++t) {
      if (!row) continue;
      int32_t i = pa[t], j = pb[t];
      out[t] = lcs_dp(res + off[i], (int32_t)(off[i + 1] - off[i]), res + off[j],
                      (int32_t)(off[j + 1] - off[j]), row);
    }
    free(row);
  }
  return bad ? -2 : 0;
}

/* all pairs i < j, row-major: index(i,j) = i*k - i*(i+1)/2 + (j - i - 1) */
int oracle_lcs_allpairs(const uint8_t *res, const int64_t *off, int32_t k, int32_t *out,
                        int nthreads) {
  if (k < 1) return -1;
  set_threads(nthreads);
  int32_t ml = max_len(off, k);
  int bad = 0;
#pragma omp parallel
  {
    int32_t *row = (int32_t *)malloc(sizeof(int32_t) * (size_t)(ml + 1));
    if (!row) {
#pragma omp atomic write
      bad = 1;
    }
#pragma omp for schedule(dynamic, 1)
    for (int32_t i = 0; i < k; ++i) {
      if (!row) continue;
      int64_t base = (int64_t)i * k - (int64_t)i * (i + 1) / 2;
      for (int32_t j = i + 1; j < k; ++j)
        out[base + (j - i - 1)] = lcs_dp(res + off[i], (int32_t)(off[i + 1] - off[i]),
                                         res + off[j], (int32_t)(off[j + 1] - off[j]), row);
    }
    free(row);
  }
  return bad ? -2 : 0;
}

/* LCS rows: for i in [r0, r1), j in [0, i): out[(sum_{r0<=i'<i} i') + j] */
int oracle_lcs_rows(const uint8_t *res, const int64_t *off, int32_t k, int32_t r0, int32_t r1,
                    int32_t *out, int nthreads) {
  if (k < 1 || r0 < 0 || r1 > k || r0 > r1) return -1;
  set_threads(nthreads);
  int32_t ml = max_len(off, k);
  int bad = 0;
#pragma omp parallel
  {
    int32_t *row = (int32_t *)malloc(sizeof(int32_t) * (size_t)(ml + 1));
    if (!row) {
#pragma omp atomic write
      bad = 1;
    }
#pragma omp for schedule(dynamic, 1)
    for (int32_t i = r0; i < r1; ++i) {
      if (!row) continue;
      int64_t base = ((int64_t)i * (i - 1) - (int64_t)r0 * (r0 - 1)) / 2;
      for (int32_t j = 0; j < i; ++j)
        out[base + j] = lcs_dp(res + off[i], (int32_t)(off[i + 1] - off[i]), res + off[j],
                               (int32_t)(off[j + 1] - off[j]), row);
    }
    free(row);
  }
  return bad ? -2 : 0;
}

/* ------------------------------------------------------------ trees */
static int64_t tri_index(int32_t i, int32_t j, int32_t k) { /* i < j */
  return (int64_t)i * k - (int64_t)i * (i + 1) / 2 + (j - i - 1);
}
static okey tri_key(const int32_t *lcs_tri, const int32_t *lens, int32_t k, int32_t i, int32_t j) {
  if (i > j) { int32_t t = i; i = j; j = t; }
  return key_from_lcs(lcs_tri[tri_index(i, j, k)], lens[i], lens[j]);
}

static void write_lambda(const okey *lam, int32_t k, uint64_t *lnum, uint32_t *lden) {
  for (int32_t j = 0; j < k; ++j) key_reduce(lam[j], &lnum[j], &lden[j]);
}

/*
 * (i) Sibson's SLINK.  Point n is inserted with M(j) = d(j, n) for j < n:
 *   pi(n) = n, lambda(n) = inf;
 *   for j = 0..n-1: if lambda(j) >= M(j): M(pi(j)) = min(M(pi(j)), lambda(j));
 *                   lambda(j) = M(j); pi(j) = n;
 *                 else M(pi(j)) = min(M(pi(j)), M(j));
 *   for j = 0..n-1: if lambda(j) >= lambda(pi(j)): pi(j) = n.
 * Distances come from a row callback so the k x k matrix need not exist.
 */
typedef void (*row_fn)(void *ctx, int32_t n, okey *M);

/* one insertion: point n joins points 0..n-1, whose distances to it are M[0..n-1] */
static void slink_insert(int32_t n, int32_t *pi, okey *lam, okey *M) {
  pi[n] = n;
  lam[n] = KEY_INF;
  for (int32_t j = 0; j < n; ++j) {
    int32_t p = pi[j];
    if (!key_lt(lam[j], M[j])) {
      M[p] = key_min(M[p], lam[j]);
      lam[j] = M[j];
      pi[j] = n;
    } else {
      M[p] = key_min(M[p], M[j]);
    }
  }
  for (int32_t j = 0; j < n; ++j)
    if (!key_lt(lam[j], lam[pi[j]])) pi[j] = n;
}

static int slink_core(int32_t k, row_fn fn, void *ctx, int32_t *pi, uint64_t *lnum,
                      uint32_t *lden) {
  okey *lam = (okey *)malloc(sizeof(okey) * (size_t)k);
  okey *M = (okey *)malloc(sizeof(okey) * (size_t)k);
  if (!lam || !M) { free(lam); free(M); return -2; }
  pi[0] = 0;
  lam[0] = KEY_INF;
  for (int32_t n = 1; n < k; ++n) {
    fn(ctx, n, M);
    slink_insert(n, pi, lam, M);
  }
  write_lambda(lam, k, lnum, lden);
  free(lam);
  free(M);
  return 0;
}

typedef struct { const int32_t *lcs_tri; const int32_t *lens; int32_t k; } tri_ctx;
static void tri_row(void *c, int32_t n, okey *M) {
  tri_ctx *t = (tri_ctx *)c;
  for (int32_t j = 0; j < n; ++j) M[j] = tri_key(t->lcs_tri, t->lens, t->k, j, n);
}

int oracle_slink_matrix(const int32_t *lcs_tri, const int32_t *lens, int32_t k, int32_t *pi,
                        uint64_t *lnum, uint32_t *lden) {
  if (k < 1) return -1;
  tri_ctx c = {lcs_tri, lens, k};
  return slink_core(k, tri_row, &c, pi, lnum, lden);
}

/* streamed: row n's LCS values are computed by DP when point n is inserted */
typedef struct {
  const uint8_t *res; const int64_t *off; int32_t k; int32_t *lcs; int32_t **rows; int nrows;
} dp_ctx;
static void dp_row(void *c, int32_t n, okey *M) {
  dp_ctx *t = (dp_ctx *)c;
  const uint8_t *a = t->res + t->off[n];
  int32_t la = (int32_t)(t->off[n + 1] - t->off[n]);
#pragma omp parallel for schedule(dynamic, 16)
  for (int32_t j = 0; j < n; ++j) {
#ifdef _OPENMP
    int32_t *row = t->rows[omp_get_thread_num()];
#else
    int32_t *row = t->rows[0];
#endif
    int32_t lb = (int32_t)(t->off[j + 1] - t->off[j]);
    int32_t L = lcs_dp(t->res + t->off[j], lb, a, la, row);
    M[j] = key_from_lcs(L, lb, la);
  }
}

int oracle_slink_streamed(const uint8_t *res, const int64_t *off, int32_t k, int32_t *pi,
                          uint64_t *lnum, uint32_t *lden, int nthreads) {
  if (k < 1) return -1;
  set_threads(nthreads);
  int nt = oracle_num_threads();
  int32_t ml = max_len(off, k);
  int32_t **rows = (int32_t **)calloc((size_t)nt, sizeof(int32_t *));
  if (!rows) return -2;
  int rc = 0;
  for (int t = 0; t < nt; ++t) {
    rows[t] = (int32_t *)malloc(sizeof(int32_t) * (size_t)(ml + 1));
    if (!rows[t]) rc = -2;
  }
  if (rc == 0) {
    dp_ctx c = {res, off, k, NULL, rows, nt};
    rc = slink_core(k, dp_row, &c, pi, lnum, lden);
  }
  for (int t = 0; t < nt; ++t) free(rows[t]);
  free(rows);
  return rc;
}

/*
 * Streamed SLINK whose rows come from the bit-parallel LCS.  Row n builds the
 * Peq table of sequence n once and runs every earlier sequence j < n through
 * it.  The pointer state is passed in and out (pi, and lambda as unreduced
 * num/den with den 0 = +inf) so that a run over a very large family can be
 * split into ranges of points [n0, n1) and saved in between; n0 == 0 starts
 * from the empty state.  Inserting the points of [0, k) in ranges gives the
 * same state as one call, since SLINK inserts one point at a time anyway.
 */
typedef struct {
  const uint8_t *res; const int64_t *off; uint64_t *peq; uint64_t **V;
} bp_ctx;
static void bp_row(void *c, int32_t n, okey *M) {
  bp_ctx *t = (bp_ctx *)c;
  int32_t la = (int32_t)(t->off[n + 1] - t->off[n]);
  int32_t wa = words_of(la);
  bp_peq(t->res + t->off[n], la, wa, t->peq);
#pragma omp parallel for schedule(dynamic, 256)
  for (int32_t j = 0; j < n; ++j) {
#ifdef _OPENMP
    uint64_t *V = t->V[omp_get_thread_num()];
#else
    uint64_t *V = t->V[0];
#endif
    int32_t lb = (int32_t)(t->off[j + 1] - t->off[j]);
    int32_t L = bp_lcs(t->peq, wa, la, t->res + t->off[j], lb, V);
    M[j] = key_from_lcs(L, lb, la);
  }
}

int oracle_slink_bitpar_range(const uint8_t *res, const int64_t *off, int32_t k, int32_t n0,
                              int32_t n1, int32_t *pi, uint64_t *lam_num, uint32_t *lam_den,
                              int nthreads) {
  if (k < 1 || n0 < 0 || n1 > k || n0 > n1) return -1;
  set_threads(nthreads);
  int nt = oracle_num_threads();
  int32_t W = words_of(max_len(off, k));
  okey *lam = (okey *)malloc(sizeof(okey) * (size_t)k);
  okey *M = (okey *)malloc(sizeof(okey) * (size_t)k);
  uint64_t *peq = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)BP_CODES * (size_t)W);
  uint64_t **V = (uint64_t **)calloc((size_t)nt, sizeof(uint64_t *));
  int rc = (lam && M && peq && V) ? 0 : -2;
  for (int t = 0; rc == 0 && t < nt; ++t) {
    V[t] = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)W);
    if (!V[t]) rc = -2;
  }
  if (rc == 0) {
    for (int32_t j = 0; j < n0; ++j) { lam[j].num = lam_num[j]; lam[j].den = lam_den[j]; }
    bp_ctx c = {res, off, peq, V};
    for (int32_t n = n0; n < n1; ++n) {
      if (n == 0) { pi[0] = 0; lam[0] = KEY_INF; continue; }
      bp_row(&c, n, M);
      slink_insert(n, pi, lam, M);
    }
    for (int32_t j = 0; j < n1; ++j) { lam_num[j] = lam[j].num; lam_den[j] = lam[j].den; }
  }
  if (V) for (int t = 0; t < nt; ++t) free(V[t]);
  free(V); free(peq); free(lam); free(M);
  return rc;
}

/* reduce keys to lowest terms (+inf = 1/0, zero = 0/1), as the tree functions output them */
int oracle_reduce_keys(const uint64_t *num, const uint32_t *den, int64_t n, uint64_t *rnum,
                       uint32_t *rden) {
  if (n < 0) return -1;
  for (int64_t t = 0; t < n; ++t) {
    okey q = {num[t], den[t]};
    key_reduce(q, &rnum[t], &rden[t]);
  }
  return 0;
}

/*
 * (ii) Naive O(k^3) agglomeration.  Active clusters carry their largest
 * index; the closest pair (ties: lowest (a, b) cluster indices) is merged at
 * height h with single-link distances min(d(A,C), d(B,C)).  Merging clusters
 * with largest indices a < b sets lambda(a) = h, pi(a) = b.  A final pass in
 * descending j replaces pi(j) by pi(pi(j)) while lambda(pi(j)) == lambda(j),
 * so that pi(j) is the largest index of j's cluster at height lambda(j).
 */
int oracle_slink_naive(const int32_t *lcs_tri, const int32_t *lens, int32_t k, int32_t *pi,
                       uint64_t *lnum, uint32_t *lden) {
  if (k < 1) return -1;
  okey *D = (okey *)malloc(sizeof(okey) * (size_t)k * (size_t)k);
  okey *lam = (okey *)malloc(sizeof(okey) * (size_t)k);
  int32_t *maxid = (int32_t *)malloc(sizeof(int32_t) * (size_t)k);
  char *alive = (char *)malloc((size_t)k);
  if (!D || !lam || !maxid || !alive) { free(D); free(lam); free(maxid); free(alive); return -2; }
  for (int32_t a = 0; a < k; ++a) {
    alive[a] = 1; maxid[a] = a; lam[a] = KEY_INF; pi[a] = a;
    for (int32_t b = 0; b < k; ++b)
      D[(size_t)a * k + b] = a == b ? KEY_INF : tri_key(lcs_tri, lens, k, a, b);
  }
  for (int32_t step = 0; step + 1 < k; ++step) {
    int32_t ba = -1, bb = -1;
    okey best = KEY_INF;
    for (int32_t a = 0; a < k; ++a) {
      if (!alive[a]) continue;
      for (int32_t b = a + 1; b < k; ++b) {
        if (!alive[b]) continue;
        okey d = D[(size_t)a * k + b];
        if (ba < 0 || key_lt(d, best)) { best = d; ba = a; bb = b; }
      }
    }
    /* clusters ba and bb merge at height best; keep slot ba */
    int32_t ma = maxid[ba], mb = maxid[bb];
    int32_t lo = ma < mb ? ma : mb, hi = ma < mb ? mb : ma;
    lam[lo] = best;
    pi[lo] = hi;
    maxid[ba] = hi;
    alive[bb] = 0;
    for (int32_t c = 0; c < k; ++c) {
      if (!alive[c] || c == ba) continue;
      okey m = key_min(D[(size_t)ba * k + c], D[(size_t)bb * k + c]);
      D[(size_t)ba * k + c] = m;
      D[(size_t)c * k + ba] = m;
    }
  }
  for (int32_t j = k - 2; j >= 0; --j) {
    while (pi[j] != k - 1 && pi[pi[j]] != pi[j] && !key_lt(lam[j], lam[pi[j]]) &&
           !key_lt(lam[pi[j]], lam[j]))
      pi[j] = pi[pi[j]];
  }
  write_lambda(lam, k, lnum, lden);
  free(D); free(lam); free(maxid); free(alive);
  return 0;
}

/*
 * (iii) The definition.  u = minimax closure of the complete graph:
 * u(i,j) = min over m of max(u(i,m), u(m,j)) (Floyd-Warshall order), then
 * lambda(j) = min_{l>j} u(j,l), pi(j) = max{ l > j : u(j,l) <= lambda(j) };
 * the last point is the root with pi = itself and lambda = +inf.
 */
int oracle_slink_definition(const int32_t *lcs_tri, const int32_t *lens, int32_t k, int32_t *pi,
                            uint64_t *lnum, uint32_t *lden) {
  if (k < 1) return -1;
  okey *U = (okey *)malloc(sizeof(okey) * (size_t)k * (size_t)k);
  okey *lam = (okey *)malloc(sizeof(okey) * (size_t)k);
  if (!U || !lam) { free(U); free(lam); return -2; }
  for (int32_t a = 0; a < k; ++a)
    for (int32_t b = 0; b < k; ++b)
      U[(size_t)a * k + b] = a == b ? (okey){0, 1} : tri_key(lcs_tri, lens, k, a, b);
  for (int32_t m = 0; m < k; ++m)
    for (int32_t a = 0; a < k; ++a)
      for (int32_t b = 0; b < k; ++b) {
        okey via = key_max(U[(size_t)a * k + m], U[(size_t)m * k + b]);
        if (key_lt(via, U[(size_t)a * k + b])) U[(size_t)a * k + b] = via;
      }
  for (int32_t j = 0; j < k; ++j) {
    okey best = KEY_INF;
    for (int32_t l = j + 1; l < k; ++l) best = key_min(best, U[(size_t)j * k + l]);
    lam[j] = best;
    int32_t p = j;
    for (int32_t l = j + 1; l < k; ++l)
      if (!key_lt(best, U[(size_t)j * k + l])) p = l;
    if (j == k - 1) { p = j; lam[j] = KEY_INF; }
    pi[j] = p;
  }
  write_lambda(lam, k, lnum, lden);
  free(U); free(lam);
  return 0;
}

/* minimax closure exposed for ultrametric tests: u as reduced (num, den) */
int oracle_minimax(const int32_t *lcs_tri, const int32_t *lens, int32_t k, uint64_t *unum,
                   uint32_t *uden) {
  if (k < 1) return -1;
  okey *U = (okey *)malloc(sizeof(okey) * (size_t)k * (size_t)k);
  if (!U) return -2;
  for (int32_t a = 0; a < k; ++a)
    for (int32_t b = 0; b < k; ++b)
      U[(size_t)a * k + b] = a == b ? (okey){0, 1} : tri_key(lcs_tri, lens, k, a, b);
  for (int32_t m = 0; m < k; ++m)
    for (int32_t a = 0; a < k; ++a)
      for (int32_t b = 0; b < k; ++b) {
        okey via = key_max(U[(size_t)a * k + m], U[(size_t)m * k + b]);
        if (key_lt(via, U[(size_t)a * k + b])) U[(size_t)a * k + b] = via;
      }
  for (size_t t = 0; t < (size_t)k * k; ++t) key_reduce(U[t], &unum[t], &uden[t]);
  free(U);
  return 0;
}

/* ------------------------------------------------------------ merges */
static int32_t uf_find(int32_t *parent, int32_t x) {
  while (parent[x] != x) { parent[x] = parent[parent[x]]; x = parent[x]; }
  return x;
}

/* insertion-free ordering: merge sort of indices by (lambda, j) */
static const uint64_t *g_num;
static const uint32_t *g_den;
static int order_lt(int32_t a, int32_t b) {
  okey ka = {g_num[a], g_den[a]}, kb = {g_num[b], g_den[b]};
  if (key_lt(ka, kb)) return 1;
  if (key_lt(kb, ka)) return 0;
  return a < b;
}
static void msort(int32_t *v, int32_t *tmp, int32_t n) {
  if (n < 2) return;
  int32_t h = n / 2;
  msort(v, tmp, h);
  msort(v + h, tmp, n - h);
  int32_t i = 0, j = h, t = 0;
  while (i < h && j < n) tmp[t++] = order_lt(v[j], v[i]) ? v[j++] : v[i++];
  while (i < h) tmp[t++] = v[i++];
  while (j < n) tmp[t++] = v[j++];
  memcpy(v, tmp, sizeof(int32_t) * (size_t)n);
}

/*
 * Merge list from the pointer representation: j in [0, k-1) sorted by
 * (lambda(j), j) ascending; for each, the clusters of j and pi(j) merge at
 * height lambda(j).  Output per merge t: (smaller id, larger id), the height
 * as a reduced fraction and the new cluster's size; the new cluster gets
 * id k + t.  lnum/lden are reduced fractions (as written by the tree
 * functions above).
 */
int oracle_merges(const int32_t *pi, const uint64_t *lnum, const uint32_t *lden, int32_t k,
                  int32_t *merges, uint64_t *hnum, uint32_t *hden, int32_t *sizes) {
  if (k < 1) return -1;
  if (k == 1) return 0;
  int32_t *ord = (int32_t *)malloc(sizeof(int32_t) * (size_t)k);
  int32_t *tmp = (int32_t *)malloc(sizeof(int32_t) * (size_t)k);
  int32_t *parent = (int32_t *)malloc(sizeof(int32_t) * (size_t)k);
  int32_t *cid = (int32_t *)malloc(sizeof(int32_t) * (size_t)k);
  int32_t *csize = (int32_t *)malloc(sizeof(int32_t) * (size_t)k);
  if (!ord || !tmp || !parent || !cid || !csize) {
    free(ord); free(tmp); free(parent); free(cid); free(csize);
    return -2;
  }
  for (int32_t j = 0; j < k; ++j) { ord[j] = j; parent[j] = j; cid[j] = j; csize[j] = 1; }
  g_num = lnum; g_den = lden;
  msort(ord, tmp, k - 1);
  for (int32_t t = 0; t < k - 1; ++t) {
    int32_t j = ord[t];
    int32_t a = uf_find(parent, j), b = uf_find(parent, pi[j]);
    int32_t ia = cid[a], ib = cid[b];
    merges[2 * t] = ia < ib ? ia : ib;
    merges[2 * t + 1] = ia < ib ? ib : ia;
    hnum[t] = lnum[j];
    hden[t] = lden[j];
    parent[a] = b;
    csize[b] += csize[a];
    cid[b] = k + t;
    sizes[t] = csize[b];
  }
  free(ord); free(tmp); free(parent); free(cid); free(csize);
  return 0;
}

/* ------------------------------------------------------------ sharded pair sets */
/*
 * Minimum spanning forest of the pairs (order[i], order[j]) with r0 <= i < r1
 * and j < i (order: a permutation of 0..k-1, the row order of the shard; NULL
 * means the identity), by Kruskal's algorithm: every such pair's exact key
 * by the DP, the pairs sorted by (key, smaller label, larger label), and each
 * pair taken when its points are not yet joined.  Writes the forest's edges
 * (a < b, reduced fractions) and returns their number, or a negative value.
 * Used for the sharded tree ("Pairwise similarities calculation" spreads the
 * pairs; single linkage depends only on a minimum spanning tree).
 */
typedef struct { okey key; int32_t a, b; } oedge;
static int edge_lt(const oedge *x, const oedge *y) {
  if (key_lt(x->key, y->key)) return 1;
  if (key_lt(y->key, x->key)) return 0;
  if (x->a != y->a) return x->a < y->a;
  return x->b < y->b;
}
static void esort(oedge *v, oedge *tmp, int64_t n) {
  if (n < 2) return;
  int64_t h = n / 2;
  esort(v, tmp, h);
  esort(v + h, tmp, n - h);
  int64_t i = 0, j = h, t = 0;
  while (i < h && j < n) tmp[t++] = edge_lt(&v[j], &v[i]) ? v[j++] : v[i++];
  while (i < h) tmp[t++] = v[i++];
  while (j < n) tmp[t++] = v[j++];
  memcpy(v, tmp, sizeof(oedge) * (size_t)n);
}

int64_t oracle_msf_rows(const uint8_t *res, const int64_t *off, int32_t k, const int32_t *order,
                        int32_t r0, int32_t r1, int32_t *ea, int32_t *eb, uint64_t *enum_,
                        uint32_t *eden, int nthreads) {
  if (k < 1 || r0 < 0 || r1 > k || r0 > r1) return -1;
  set_threads(nthreads);
  int64_t m = ((int64_t)r1 * (r1 - 1) - (int64_t)r0 * (r0 - 1)) / 2;
  oedge *E = (oedge *)malloc(sizeof(oedge) * (size_t)(m > 0 ? m : 1));
  oedge *T = (oedge *)malloc(sizeof(oedge) * (size_t)(m > 0 ? m : 1));
  int32_t *parent = (int32_t *)malloc(sizeof(int32_t) * (size_t)k);
  int32_t ml = max_len(off, k);
  if (!E || !T || !parent) { free(E); free(T); free(parent); return -2; }
  int bad = 0;
#pragma omp parallel
  {
    int32_t *row = (int32_t *)malloc(sizeof(int32_t) * (size_t)(ml + 1));
    if (!row) {
#pragma omp atomic write
      bad = 1;
    }
#pragma omp for schedule(dynamic, 1)
    for (int32_t i = r0; i < r1; ++i) {
      if (!row) continue;
      int64_t base = ((int64_t)i * (i - 1) - (int64_t)r0 * (r0 - 1)) / 2;
      int32_t x = order ? order[i] : i;
      int32_t lx = (int32_t)(off[x + 1] - off[x]);
      for (int32_t j = 0; j < i; ++j) {
        int32_t y = order ? order[j] : j;
        int32_t ly = (int32_t)(off[y + 1] - off[y]);
        int32_t L = lcs_dp(res + off[x], lx, res + off[y], ly, row);
        oedge e;
        e.key = key_from_lcs(L, lx, ly);
        e.a = x < y ? x : y;
        e.b = x < y ? y : x;
        E[base + j] = e;
      }
    }
    free(row);
  }
  if (bad) { free(E); free(T); free(parent); return -2; }
  esort(E, T, m);
  for (int32_t v = 0; v < k; ++v) parent[v] = v;
  int64_t n = 0;
  for (int64_t t = 0; t < m; ++t) {
    int32_t x = uf_find(parent, E[t].a), y = uf_find(parent, E[t].b);
    if (x == y) continue;
    parent[x] = y;
    ea[n] = E[t].a;
    eb[n] = E[t].b;
    key_reduce(E[t].key, &enum_[n], &eden[n]);
    ++n;
  }
  free(E); free(T); free(parent);
  return n;
}

/*
 * Single linkage of k points from an edge list alone: Sibson's SLINK over the
 * k x k matrix whose entries are the given edges' keys and +inf elsewhere
 * (the lightest key when an edge repeats).  When the edges contain a minimum
 * spanning tree of the complete distance graph, the single-link distances,
 * and so pi and lambda, are those of the complete graph.
 */
typedef struct { const okey *D; int32_t k; } dense_ctx;
static void dense_row(void *c, int32_t n, okey *M) {
  dense_ctx *t = (dense_ctx *)c;
  for (int32_t j = 0; j < n; ++j) M[j] = t->D[(size_t)j * t->k + n];
}

int oracle_slink_edges(int32_t k, int64_t m, const int32_t *ea, const int32_t *eb,
                       const uint64_t *enum_, const uint32_t *eden, int32_t *pi, uint64_t *lnum,
                       uint32_t *lden) {
  if (k < 1 || m < 0) return -1;
  okey *D = (okey *)malloc(sizeof(okey) * (size_t)k * (size_t)k);
  if (!D) return -2;
  for (size_t t = 0; t < (size_t)k * k; ++t) D[t] = KEY_INF;
  for (int64_t e = 0; e < m; ++e) {
    int32_t a = ea[e], b = eb[e];
    if (a < 0 || b < 0 || a >= k || b >= k || a == b) { free(D); return -1; }
    okey q = {enum_[e], eden[e]};
    if (q.den == 0) q = KEY_INF;
    D[(size_t)a * k + b] = key_min(D[(size_t)a * k + b], q);
    D[(size_t)b * k + a] = D[(size_t)a * k + b];
  }
  dense_ctx c = {D, k};
  int rc = slink_core(k, dense_row, &c, pi, lnum, lden);
  free(D);
  return rc;
}

/* ------------------------------------------------------------ progressive schedule */
/*
 * The merge list in the form the progressive stage consumes ("Progressive
 * construction of the alignment": O(k) profile alignments in guide-tree
 * order, spread over threads; at least half of them align a single sequence
 * with a profile).  Merge t joins clusters merges[2t] and merges[2t+1]
 * (ids < k are single sequences, k + t' the result of merge t').
 *   level[t] = 1 + the larger level of its two children (a sequence is at
 *     level 0): merges of one level never use one another, so each level can
 *     run at once, after the levels below it;
 *   order: the merges sorted by (level, t); level_start[l - 1] .. level_start[l]
 *     delimit level l in order (level_start has n_levels + 1 entries);
 *   kind[t]: 0 two single sequences, 1 one sequence and one profile, 2 two
 *     profiles (a child's size is 1 for a sequence, sizes[t'] for merge t').
 * Returns n_levels, or a negative value for a bad merge list.
 */
int32_t oracle_schedule(int32_t k, const int32_t *merges, const int32_t *sizes, int32_t *level,
                        int32_t *order, int32_t *level_start, int32_t *kind) {
  if (k < 1) return -1;
  int32_t n = k - 1, top = 0;
  for (int32_t t = 0; t < n; ++t) {
    int32_t la = 0, lb = 0, sa = 1, sb = 1;
    int32_t a = merges[2 * t], b = merges[2 * t + 1];
    if (a < 0 || b < 0 || a >= k + t || b >= k + t) return -1;
    if (a >= k) { la = level[a - k]; sa = sizes[a - k]; }
    if (b >= k) { lb = level[b - k]; sb = sizes[b - k]; }
    level[t] = 1 + (la > lb ? la : lb);
    kind[t] = (sa > 1) + (sb > 1);
    if (level[t] > top) top = level[t];
  }
  /* counting sort by level, stable in t */
  for (int32_t l = 0; l <= top; ++l) level_start[l] = 0;
  for (int32_t t = 0; t < n; ++t) level_start[level[t]]++;
  int32_t run = 0;
  for (int32_t l = 1; l <= top; ++l) {
    int32_t c = level_start[l];
    level_start[l - 1] = run;
    run += c;
  }
  level_start[top] = run;
  int32_t *fill = (int32_t *)malloc(sizeof(int32_t) * (size_t)(top + 1));
  if (!fill) return -2;
  for (int32_t l = 0; l < top; ++l) fill[l] = level_start[l];
  for (int32_t t = 0; t < n; ++t) order[fill[level[t] - 1]++] = t;
  free(fill);
  return top;
}

/* ------------------------------------------------------------ gap types and costs */
/*
 * "Gap types and costs determination": gaps are terminal open / extension
 * (T_o = 1, T_e = 2) or open / extension (G_o = 3, G_e = 4); 0 is a residue,
 * 255 a gap in the alignment rows (m x n bytes).  A gap before the row's
 * first residue or after its last one is terminal; the first gap of a run
 * opens it.
 */
enum { O_RES = 0, O_TO = 1, O_TE = 2, O_GO = 3, O_GE = 4 };
int oracle_gap_types(const uint8_t *aln, int64_t m, int32_t n, uint8_t *types) {
  if (m < 0 || n < 0) return -1;
  for (int64_t r = 0; r < m; ++r) {
    const uint8_t *a = aln + r * n;
    int32_t first = n, last = -1;
    for (int32_t j = 0; j < n; ++j)
      if (a[j] != 255) { if (first == n) first = j; last = j; }
    for (int32_t j = 0; j < n; ++j) {
      uint8_t t = O_RES;
      if (a[j] == 255) {
        int terminal = j < first || j > last;
        int opens = j == 0 || a[j - 1] != 255;
        t = terminal ? (opens ? O_TO : O_TE) : (opens ? O_GO : O_GE);
      }
      types[r * n + j] = t;
    }
  }
  return 0;
}

/*
 * Insertion of gap columns with the six corrections, one inserted gap at a
 * time from left to right (L: the type left of the new gap, R: the type right
 * of it, -1 at an end of the row):
 *   S1 R is T_o: the new gap is T_o and R becomes T_e;
 *   S2 L is T_e: the new gap is T_e;
 *   S3 inside (or closing) a run of G_o/G_e: G_e;
 *   S4 R is G_o: the new gap is G_o and R becomes G_e;
 *   S5 between residues: G_o;
 *   S6 L is T_o: the new gap is T_e;
 * and a gap that starts a new run at an end of the row is T_o.
 */
int oracle_gap_insert(const uint8_t *aln, const uint8_t *types, int64_t m, int32_t n, const int32_t *pos,
                      int32_t c, uint8_t *aln_out, uint8_t *types_out) {
  if (m < 0 || n < 0 || c < 0) return -1;
  for (int32_t i = 0; i < c; ++i)
    if (pos[i] < 0 || pos[i] > n || (i > 0 && pos[i] < pos[i - 1])) return -1;
  int64_t w = (int64_t)n + c;
  for (int64_t r = 0; r < m; ++r) {
    uint8_t *ao = aln_out + r * w, *to = types_out + r * w;
    /* start from the row as it is, then insert column by column */
    int64_t len = n;
    memcpy(ao, aln + r * n, (size_t)n);
    memcpy(to, types + r * n, (size_t)n);
    for (int32_t i = 0; i < c; ++i) {
      int64_t at = pos[i] + i; /* earlier insertions shifted the row */
      memmove(ao + at + 1, ao + at, (size_t)(len - at));
      memmove(to + at + 1, to + at, (size_t)(len - at));
      ++len;
      int L = at > 0 ? to[at - 1] : -1;
      int R = at + 1 < len ? to[at + 1] : -1;
      int g;
      if (R == O_TO) { g = O_TO; to[at + 1] = O_TE; }                 /* S1 */
      else if (L == O_TE) g = O_TE;                                    /* S2 */
      else if (L == O_GO || L == O_GE) g = O_GE;                       /* S3 */
      else if (R == O_GO) { g = O_GO; to[at + 1] = O_GE; }            /* S4 */
      else if (L == O_TO) g = O_TE;                                    /* S6 */
      else if (L < 0 || R < 0) g = O_TO;                               /* new terminal run */
      else g = O_GO;                                                   /* S5 */
      ao[at] = 255;
      to[at] = (uint8_t)g;
    }
  }
  return 0;
}

/* g_scale = 1 + log(k / g_l) / g_d, and per row g_scale * sum of count x cost */
double oracle_gap_scale(int64_t k, double g_l, double g_d) { return 1.0 + log((double)k / g_l) / g_d; }

int oracle_gap_cost(const uint8_t *types, int64_t m, int32_t n, int64_t k, const double *costs, double g_l,
                    double g_d, double *cost) {
  if (m < 0 || n < 0 || k < 1) return -1;
  double s = oracle_gap_scale(k, g_l, g_d);
  for (int64_t r = 0; r < m; ++r) {
    int64_t cnt[5] = {0, 0, 0, 0, 0};
    for (int32_t j = 0; j < n; ++j) cnt[types[r * n + j]]++;
    cost[r] = s * (costs[0] * (double)cnt[O_TO] + costs[1] * (double)cnt[O_TE] + costs[2] * (double)cnt[O_GO] +
                   costs[3] * (double)cnt[O_GE]);
  }
  return 0;
}

/* ------------------------------------------------------------ UPGMA */
/*
 * The alternative guide tree the paper names beside single linkage
 * ("Determination of the guide tree": UPGMA needs the whole O(k^2) matrix).
 * Distances d(i, j) = indel^2 / LCS as doubles (one correctly rounded
 * division; +inf for LCS = 0).  Plain UPGMA: while more than one cluster is
 * left, take the pair of clusters in slots a < b with the smallest
 * (d, a, b), record it, put the merged cluster in slot a and set, for every
 * other live slot c,
 *     d(a, c) = (n_a * d(a, c) + n_b * d(b, c)) / (n_a + n_b)
 * in exactly that order of operations (no fused multiply-add).  Merge t joins
 * the clusters of ids (smaller, larger), ids k + t' for earlier merges,
 * at height d(a, b), making a cluster of sizes[t] sequences.
 */
int oracle_distance_matrix(const uint8_t *res, const int64_t *off, int32_t k, double *D, int nthreads) {
  if (k < 1) return -1;
  int32_t *tri = (int32_t *)malloc(sizeof(int32_t) * (size_t)((int64_t)k * (k - 1) / 2 + 1));
  if (!tri) return -2;
  int rc = oracle_lcs_allpairs(res, off, k, tri, nthreads);
  if (rc == 0) {
    for (int32_t i = 0; i < k; ++i) {
      D[(size_t)i * k + i] = 0.0;
      for (int32_t j = i + 1; j < k; ++j) {
        int32_t L = tri[tri_index(i, j, k)];
        int64_t li = off[i + 1] - off[i], lj = off[j + 1] - off[j];
        int64_t indel = li + lj - 2 * (int64_t)L;
        double d = L == 0 ? INFINITY : (double)(indel * indel) / (double)L;
        D[(size_t)i * k + j] = d;
        D[(size_t)j * k + i] = d;
      }
    }
  }
  free(tri);
  return rc;
}

int oracle_upgma(int32_t k, const double *D0, int32_t *merges, double *heights, int32_t *sizes) {
  if (k < 1) return -1;
  double *D = (double *)malloc(sizeof(double) * (size_t)k * (size_t)k);
  int32_t *id = (int32_t *)malloc(sizeof(int32_t) * (size_t)k);
  int32_t *n = (int32_t *)malloc(sizeof(int32_t) * (size_t)k);
  char *alive = (char *)malloc((size_t)k);
  if (!D || !id || !n || !alive) { free(D); free(id); free(n); free(alive); return -2; }
  memcpy(D, D0, sizeof(double) * (size_t)k * (size_t)k);
  for (int32_t i = 0; i < k; ++i) { id[i] = i; n[i] = 1; alive[i] = 1; }
  for (int32_t t = 0; t + 1 < k; ++t) {
    int32_t ba = -1, bb = -1;
    double best = 0.0;
    for (int32_t a = 0; a < k; ++a) {
      if (!alive[a]) continue;
      for (int32_t b = a + 1; b < k; ++b) {
        if (!alive[b]) continue;
        double d = D[(size_t)a * k + b];
        if (ba < 0 || d < best) { best = d; ba = a; bb = b; }
      }
    }
    merges[2 * t] = id[ba] < id[bb] ? id[ba] : id[bb];
    merges[2 * t + 1] = id[ba] < id[bb] ? id[bb] : id[ba];
    heights[t] = best;
    double na = (double)n[ba], nb = (double)n[bb], nab = (double)(n[ba] + n[bb]);
    for (int32_t c = 0; c < k; ++c) {
      if (!alive[c] || c == ba || c == bb) continue;
      double x = na * D[(size_t)ba * k + c];
      double y = nb * D[(size_t)bb * k + c];
      double v = (x + y) / nab;
      D[(size_t)ba * k + c] = v;
      D[(size_t)c * k + ba] = v;
    }
    alive[bb] = 0;
    n[ba] += n[bb];
    id[ba] = k + t;
    sizes[t] = n[ba];
  }
  free(D); free(id); free(n); free(alive);
  return 0;
}

/*
 * Neighbour joining (Saitou & Nei 1987, in Studier & Keppler's form), the
 * other alternative to single linkage the paper names ("Determination of
 * the guide tree"), over the same distances as UPGMA.  With r clusters live:
 *     R(i)    = sum of d(i, j) over the live j != i;
 *     Q(a, b) = (r - 2) * d(a, b) - R(a) - R(b);
 * the pair of live slots a < b with the smallest (Q, a, b) is joined; its
 * branches are
 *     delta_a = d(a, b) / 2 + (R(a) - R(b)) / (2 (r - 2)),  delta_b = d(a, b) - delta_a;
 * the new cluster u takes slot a with d(u, c) = (d(a, c) + d(b, c) - d(a, b)) / 2
 * for every other live c.  The row sums start as sums in increasing j and
 * then follow the joins (Studier & Keppler's update, equal in exact
 * arithmetic to summing afresh):
 *     R(c) = R(c) - d(a, c) - d(b, c) + d(u, c)   for every other live c,
 *     R(u) = (R(a) + R(b) - r * d(a, b)) / 2.
 * When two clusters are left they are joined with d(a, b) / 2 on each branch
 * (the root of the guide tree).  Every operation is rounded on its own, in
 * exactly the order written (no fused multiply-add).  Merge t joins ids
 * (smaller, larger) with branch lengths[2t], lengths[2t+1] in that order,
 * making a cluster of sizes[t] sequences.  NJ is undefined with an infinite
 * distance (a pair with LCS 0): returns -3 then.
 */
int oracle_nj(int32_t k, const double *D0, int32_t *merges, double *lengths, int32_t *sizes) {
  if (k < 1) return -1;
  for (int64_t x = 0; x < (int64_t)k * k; ++x)
    if (!isfinite(D0[x])) return -3;
  double *D = (double *)malloc(sizeof(double) * (size_t)k * (size_t)k);
  double *R = (double *)malloc(sizeof(double) * (size_t)k);
  int32_t *id = (int32_t *)malloc(sizeof(int32_t) * (size_t)k);
  int32_t *n = (int32_t *)malloc(sizeof(int32_t) * (size_t)k);
  char *alive = (char *)malloc((size_t)k);
  if (!D || !R || !id || !n || !alive) { free(D); free(R); free(id); free(n); free(alive); return -2; }
  memcpy(D, D0, sizeof(double) * (size_t)k * (size_t)k);
  for (int32_t i = 0; i < k; ++i) {
    id[i] = i; n[i] = 1; alive[i] = 1;
    double s = 0.0;
    for (int32_t j = 0; j < k; ++j)
      if (j != i) s = s + D[(size_t)i * k + j];
    R[i] = s;
  }
  for (int32_t t = 0; t + 1 < k; ++t) {
    const int32_t r = k - t;
    int32_t ba = -1, bb = -1;
    double da, db;
    if (r == 2) {
      for (int32_t i = 0; i < k; ++i)
        if (alive[i]) { if (ba < 0) ba = i; else bb = i; }
      da = D[(size_t)ba * k + bb] * 0.5;
      db = da;
    } else {
      double best = 0.0;
      for (int32_t a = 0; a < k; ++a) {
        if (!alive[a]) continue;
        for (int32_t b = a + 1; b < k; ++b) {
          if (!alive[b]) continue;
          double q = (double)(r - 2) * D[(size_t)a * k + b];
          q = q - R[a];
          q = q - R[b];
          if (ba < 0 || q < best) { best = q; ba = a; bb = b; }
        }
      }
      const double dab = D[(size_t)ba * k + bb];
      da = dab * 0.5 + (R[ba] - R[bb]) / (double)(2 * (r - 2));
      db = dab - da;
      const double ru = ((R[ba] + R[bb]) - (double)r * dab) * 0.5;
      for (int32_t c = 0; c < k; ++c) {
        if (!alive[c] || c == ba || c == bb) continue;
        const double dac = D[(size_t)ba * k + c], dbc = D[(size_t)bb * k + c];
        const double v = ((dac + dbc) - dab) * 0.5;
        R[c] = ((R[c] - dac) - dbc) + v;
        D[(size_t)ba * k + c] = v;
        D[(size_t)c * k + ba] = v;
      }
      R[ba] = ru;
    }
    const int lo_a = id[ba] < id[bb];
    merges[2 * t] = lo_a ? id[ba] : id[bb];
    merges[2 * t + 1] = lo_a ? id[bb] : id[ba];
    lengths[2 * t] = lo_a ? da : db;
    lengths[2 * t + 1] = lo_a ? db : da;
    alive[bb] = 0;
    n[ba] += n[bb];
    id[ba] = k + t;
    sizes[t] = n[ba];
  }
  free(D); free(R); free(id); free(n); free(alive);
  return 0;
}
