/*
 * Seeded synthetic protein families (input generator only).
 *
 * This file holds none of the LCS or single-linkage arithmetic: it only
 * produces residue codes.  Both the CUDA path and the CPU oracle consume
 * its output.
 *
 * Recipe (one family):
 *   1. Root sequence: length fixed or drawn from a log-normal (median, sigma),
 *      clamped to [root_lo, root_hi]; residues drawn from the background.
 *   2. Tree: a random binary tree over k leaves by coalescent random joining
 *      (pick two active nodes uniformly, join them, repeat).
 *   3. Every branch: Poisson(sub_rate * len) substitutions at uniform sites
 *      (new residue drawn from the background, redrawn while equal to the
 *      old one), then Poisson(indel_rate * len) indel events, each an
 *      insertion or a deletion with probability 1/2 and a Geometric length
 *      with mean 3 on {1, 2, ...}; inserted residues come from the background.
 *   4. Leaves: optional duplication (a leaf copies an earlier leaf), optional
 *      terminal extension of U{ext_lo..ext_hi} background residues at a random
 *      terminus, clipping to [clip_lo, clip_hi] (truncate the C-terminus,
 *      pad the C-terminus with background residues), optional ambiguity
 *      replacement (each residue becomes X, B or Z with probability ambig).
 *
 * Background: amino-acid frequencies of Robinson & Robinson (1991),
 * Proc. Natl. Acad. Sci. USA 88:8880-8884, in parts per 100,000.
 *
 * Determinism: the generator must give the same bytes on x86-64 and AArch64.
 * All randomness is integer (xoshiro256**, seeded by splitmix64); the only
 * floating point is +,-,*,/ and sqrt (IEEE correctly rounded) plus frexp and
 * ldexp (exact), with the log/exp series written out below.  Build with
 * -ffp-contract=off so no fused multiply-add changes a rounding.
 *
 * Codes: 0..19 = A C D E F G H I K L M N P Q R S T V W Y, 20 = B, 21 = Z,
 * 22 = X, 23 = U, 24 = O.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
  uint64_t seed;
  int32_t k;
  int32_t root_len;      /* > 0: fixed root length; <= 0: log-normal draw */
  double root_median;
  double root_sigma;
  int32_t root_lo, root_hi;
  double sub_rate;       /* substitutions per site per branch */
  double indel_rate;     /* indel events per site per branch */
  int32_t clip_lo, clip_hi;
  double ext_frac;       /* fraction of leaves with a terminal extension */
  int32_t ext_lo, ext_hi;
  double ambig_frac;     /* per-residue probability of becoming X/B/Z */
  int32_t alphabet;      /* 0: 20 amino acids with background freqs; a>0: uniform over codes 0..a-1 */
  double dup_frac;       /* probability a leaf is replaced by a copy of an earlier leaf */
} synth_params;

/* ------------------------------------------------------------------ RNG */
typedef struct { uint64_t s[4]; } rng_t;

static uint64_t splitmix64(uint64_t *x) {
  uint64_t z = (*x += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
static void rng_seed(rng_t *r, uint64_t seed) {
  uint64_t x = seed;
  for (int i = 0; i < 4; ++i) r->s[i] = splitmix64(&x);
}
static inline uint64_t rotl(uint64_t x, int k) { return (x << k) | (x >> (64 - k)); }
static inline uint64_t rng_next(rng_t *r) {
  uint64_t *s = r->s;
  uint64_t res = rotl(s[1] * 5, 7) * 9;
  uint64_t t = s[1] << 17;
  s[2] ^= s[0]; s[3] ^= s[1]; s[1] ^= s[2]; s[0] ^= s[3];
  s[2] ^= t; s[3] = rotl(s[3], 45);
  return res;
}
/* uniform integer in [0, n), n >= 1, unbiased (rejection on the low word) */
static uint32_t rng_below(rng_t *r, uint32_t n) {
  uint64_t lim = (0x100000000ull / n) * n;
  for (;;) {
    uint64_t v = rng_next(r) >> 32;
    if (v < lim) return (uint32_t)(v % n);
  }
}
/* uniform double in (0, 1) */
static double rng_unif(rng_t *r) {
  return ((double)(rng_next(r) >> 11) + 0.5) * (1.0 / 9007199254740992.0);
}
/* Bernoulli with probability p, decided on a 32-bit integer threshold */
static int rng_bern(rng_t *r, double p) {
  if (p <= 0.0) return 0;
  if (p >= 1.0) return 1;
  uint64_t thr = (uint64_t)(p * 4294967296.0);
  return (rng_next(r) >> 32) < thr;
}

/* ------------------------------------------- deterministic log and exp */
static const double LN2 = 0.69314718055994530942;

static double det_log(double x) { /* x > 0 */
  int e;
  double m = frexp(x, &e);          /* x = m * 2^e, m in [0.5, 1) */
  double s = (m - 1.0) / (m + 1.0); /* log m = 2 atanh(s), |s| <= 1/3 */
  double s2 = s * s, term = s, sum = 0.0;
  for (int i = 1; i < 60; i += 2) { sum += term / (double)i; term *= s2; }
  return 2.0 * sum + (double)e * LN2;
}
static double det_exp(double x) {
  double kf = x / LN2;
  int k = (int)(kf >= 0 ? kf + 0.5 : kf - 0.5);
  double r = x - (double)k * LN2;   /* |r| <= ~ln2/2 */
  double term = 1.0, sum = 1.0;
  for (int i = 1; i < 30; ++i) { term *= r / (double)i; sum += term; }
  return ldexp(sum, k);
}
static double rng_normal(rng_t *r) { /* Marsaglia polar method */
  for (;;) {
    double u = 2.0 * rng_unif(r) - 1.0, v = 2.0 * rng_unif(r) - 1.0;
    double s = u * u + v * v;
    if (s > 0.0 && s < 1.0) return u * sqrt(-2.0 * det_log(s) / s);
  }
}
static uint32_t rng_poisson(rng_t *r, double mu) { /* inversion, mu small */
  if (mu <= 0.0) return 0;
  double p = det_exp(-mu), F = p, U = rng_unif(r);
  uint32_t x = 0;
  while (U > F && x < 100000) { ++x; p *= mu / (double)x; F += p; }
  return x;
}
static uint32_t rng_geom3(rng_t *r) { /* Geometric on {1,2,...}, mean 3 */
  uint32_t l = 1;
  while (rng_below(r, 3) != 0) ++l;
  return l;
}

/* ------------------------------------------------------- background */
/* A C D E F G H I K L M N P Q R S T V W Y */
static const uint32_t BG_PPK[20] = {7805, 1925, 5364, 6295, 3856, 7377, 2199, 5142, 5744, 9019,
                                    2243, 4487, 5203, 4264, 5129, 7120, 5841, 6441, 1330, 3216};
typedef struct { uint32_t cum[20]; uint32_t total; int alphabet; } bg_t;

static void bg_init(bg_t *b, int alphabet) {
  b->alphabet = alphabet;
  uint32_t c = 0;
  for (int i = 0; i < 20; ++i) { c += BG_PPK[i]; b->cum[i] = c; }
  b->total = c;
}
static uint8_t bg_draw(rng_t *r, const bg_t *b) {
  if (b->alphabet > 0) return (uint8_t)rng_below(r, (uint32_t)b->alphabet);
  uint32_t v = rng_below(r, b->total);
  int i = 0;
  while (v >= b->cum[i]) ++i;
  return (uint8_t)i;
}

/* ------------------------------------------------------- sequences */
typedef struct { uint8_t *d; int32_t n, cap; } seq_t;

static int seq_reserve(seq_t *s, int32_t cap) {
  if (cap <= s->cap) return 0;
  int32_t nc = s->cap ? s->cap : 64;
  while (nc < cap) nc *= 2;
  uint8_t *nd = (uint8_t *)realloc(s->d, (size_t)nc);
  if (!nd) return -1;
  s->d = nd; s->cap = nc;
  return 0;
}

static int mutate_branch(rng_t *r, const bg_t *bg, const synth_params *p, seq_t *s) {
  /* substitutions */
  uint32_t ns = rng_poisson(r, p->sub_rate * (double)s->n);
  for (uint32_t t = 0; t < ns && s->n > 0; ++t) {
    uint32_t site = rng_below(r, (uint32_t)s->n);
    uint8_t old = s->d[site], nw;
    int guard = 0;
    do { nw = bg_draw(r, bg); } while (nw == old && ++guard < 1000);
    s->d[site] = nw;
  }
  /* indels */
  uint32_t ni = rng_poisson(r, p->indel_rate * (double)s->n);
  for (uint32_t t = 0; t < ni; ++t) {
    uint32_t ins = rng_below(r, 2) == 0;
    uint32_t len = rng_geom3(r);
    if (ins) {
      uint32_t pos = rng_below(r, (uint32_t)s->n + 1);
      if (seq_reserve(s, s->n + (int32_t)len)) return -1;
      memmove(s->d + pos + len, s->d + pos, (size_t)(s->n - (int32_t)pos));
      for (uint32_t q = 0; q < len; ++q) s->d[pos + q] = bg_draw(r, bg);
      s->n += (int32_t)len;
    } else {
      uint32_t pos = rng_below(r, (uint32_t)s->n);
      if ((int32_t)(pos + len) > s->n) len = (uint32_t)(s->n - (int32_t)pos);
      if ((int32_t)len >= s->n) continue; /* never empty a sequence */
      memmove(s->d + pos, s->d + pos + len, (size_t)(s->n - (int32_t)(pos + len)));
      s->n -= (int32_t)len;
    }
  }
  return 0;
}

/*
 * Generate one family.  On success returns 0, sets *out_res to a malloc'd
 * buffer of offsets[k] residue codes (free with synth_free) and fills
 * offsets[0..k] (caller-allocated, k+1 entries).  Returns -1 on bad
 * parameters, -2 on allocation failure.
 */
int synth_family(const synth_params *p, uint8_t **out_res, int64_t *offsets) {
  if (!p || !out_res || !offsets || p->k < 1 || p->clip_lo < 1 || p->clip_hi < p->clip_lo ||
      p->alphabet < 0 || p->alphabet > 25)
    return -1;
  rng_t r;
  rng_seed(&r, p->seed * 0x9E3779B97F4A7C15ull + 0x5851F42D4C957F2Dull);
  bg_t bg;
  bg_init(&bg, p->alphabet);
  const int32_t k = p->k;
  const int32_t nn = 2 * k - 1;

  /* root length */
  int32_t root_len = p->root_len;
  if (root_len <= 0) {
    double z = rng_normal(&r);
    double len = p->root_median * det_exp(p->root_sigma * z);
    root_len = (int32_t)(len + 0.5);
  }
  if (p->root_lo > 0 && root_len < p->root_lo) root_len = p->root_lo;
  if (p->root_hi > 0 && root_len > p->root_hi) root_len = p->root_hi;
  if (root_len < 1) root_len = 1;

  /* coalescent tree: nodes 0..k-1 are leaves, k..2k-2 internal */
  int32_t *left = (int32_t *)malloc(sizeof(int32_t) * (size_t)nn);
  int32_t *right = (int32_t *)malloc(sizeof(int32_t) * (size_t)nn);
  int32_t *active = (int32_t *)malloc(sizeof(int32_t) * (size_t)k);
  seq_t *seqs = (seq_t *)calloc((size_t)nn, sizeof(seq_t));
  int32_t *stack = (int32_t *)malloc(sizeof(int32_t) * (size_t)nn);
  if (!left || !right || !active || !seqs || !stack) {
    free(left); free(right); free(active); free(seqs); free(stack);
    return -2;
  }
  for (int32_t i = 0; i < nn; ++i) left[i] = right[i] = -1;
  for (int32_t i = 0; i < k; ++i) active[i] = i;
  int32_t count = k, next = k;
  while (count > 1) {
    uint32_t i = rng_below(&r, (uint32_t)count);
    int32_t a = active[i];
    active[i] = active[--count];
    uint32_t j = rng_below(&r, (uint32_t)count);
    int32_t b = active[j];
    left[next] = a; right[next] = b;
    active[j] = next;
    ++next;
  }
  int32_t root = active[0];
  int rc = 0;

  /* root residues */
  if (seq_reserve(&seqs[root], root_len)) { rc = -2; goto done; }
  for (int32_t q = 0; q < root_len; ++q) seqs[root].d[q] = bg_draw(&r, &bg);
  seqs[root].n = root_len;

  /* evolve, depth first; a node's sequence is freed once both children hold copies */
  {
    int32_t sp = 0;
    stack[sp++] = root;
    while (sp > 0) {
      int32_t v = stack[--sp];
      if (left[v] < 0) continue; /* leaf: keep */
      int32_t ch[2] = {left[v], right[v]};
      for (int c = 0; c < 2; ++c) {
        seq_t *dst = &seqs[ch[c]];
        if (seq_reserve(dst, seqs[v].n)) { rc = -2; goto done; }
        memcpy(dst->d, seqs[v].d, (size_t)seqs[v].n);
        dst->n = seqs[v].n;
        if (mutate_branch(&r, &bg, p, dst)) { rc = -2; goto done; }
      }
      free(seqs[v].d); seqs[v].d = NULL; seqs[v].n = seqs[v].cap = 0;
      stack[sp++] = ch[1];
      stack[sp++] = ch[0];
    }
  }

  /* leaf post-processing in leaf index order */
  for (int32_t i = 0; i < k; ++i) {
    seq_t *s = &seqs[i];
    if (i > 0 && rng_bern(&r, p->dup_frac)) {
      int32_t src = (int32_t)rng_below(&r, (uint32_t)i);
      if (seq_reserve(s, seqs[src].n)) { rc = -2; goto done; }
      memcpy(s->d, seqs[src].d, (size_t)seqs[src].n);
      s->n = seqs[src].n;
      continue; /* an exact duplicate */
    }
    if (rng_bern(&r, p->ext_frac)) {
      int32_t el = p->ext_lo + (int32_t)rng_below(&r, (uint32_t)(p->ext_hi - p->ext_lo + 1));
      int n_term = rng_below(&r, 2) == 0;
      if (seq_reserve(s, s->n + el)) { rc = -2; goto done; }
      if (n_term) memmove(s->d + el, s->d, (size_t)s->n);
      for (int32_t q = 0; q < el; ++q) s->d[(n_term ? 0 : s->n) + q] = bg_draw(&r, &bg);
      s->n += el;
    }
    if (s->n > p->clip_hi) s->n = p->clip_hi;
    if (s->n < p->clip_lo) {
      if (seq_reserve(s, p->clip_lo)) { rc = -2; goto done; }
      while (s->n < p->clip_lo) s->d[s->n++] = bg_draw(&r, &bg);
    }
    if (p->ambig_frac > 0.0) {
      static const uint8_t AMB[3] = {22, 20, 21}; /* X B Z */
      for (int32_t q = 0; q < s->n; ++q)
        if (rng_bern(&r, p->ambig_frac)) s->d[q] = AMB[rng_below(&r, 3)];
    }
  }

  {
    int64_t total = 0;
    offsets[0] = 0;
    for (int32_t i = 0; i < k; ++i) { total += seqs[i].n; offsets[i + 1] = total; }
    uint8_t *res = (uint8_t *)malloc(total > 0 ? (size_t)total : 1);
    if (!res) { rc = -2; goto done; }
    for (int32_t i = 0; i < k; ++i) memcpy(res + offsets[i], seqs[i].d, (size_t)seqs[i].n);
    *out_res = res;
  }

done:
  for (int32_t i = 0; i < nn; ++i) free(seqs[i].d);
  free(seqs); free(left); free(right); free(active); free(stack);
  return rc;
}

void synth_free(void *ptr) { free(ptr); }

/* uniform draws for query batches and serving streams (same RNG, same determinism) */
int synth_uniform_ints(uint64_t seed, uint32_t n_below, int64_t count, uint32_t *out) {
  if (n_below < 1 || count < 0 || !out) return -1;
  rng_t r;
  rng_seed(&r, seed ^ 0xD1B54A32D192ED03ull);
  for (int64_t i = 0; i < count; ++i) out[i] = rng_below(&r, n_below);
  return 0;
}

/* log-uniform integers round(lo * (hi/lo)^f), f uniform in (0,1) (batched workload draws) */
int synth_log_uniform_ints(uint64_t seed, double lo, double hi, int64_t count, int32_t *out) {
  if (!(lo > 0.0) || hi < lo || count < 0 || !out) return -1;
  rng_t r;
  rng_seed(&r, seed ^ 0x2545F4914F6CDD1Dull);
  double llo = det_log(lo), lhi = det_log(hi);
  for (int64_t i = 0; i < count; ++i) {
    double v = det_exp(llo + rng_unif(&r) * (lhi - llo));
    out[i] = (int32_t)(v + 0.5);
  }
  return 0;
}
