/*
 * famsa_gpu.h -- C ABI of the GB300 (sm_103a) library for FAMSA stages I+II:
 * all-pairs LCS similarity over k protein sequences and the single-linkage
 * guide tree built from it.
 *
 * Paper: S. Deorowicz, A. Debudaj-Grabysz, A. Gudys, "Aligning 415 519
 * proteins in less than two hours on PC" (FAMSA).  Methods, subsections
 * "Pairwise similarities calculation" and "Determination of the guide tree".
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Residues are uint8 codes 0..24:
 *   0..19 = A C D E F G H I K L M N P Q R S T V W Y, 20 = B, 21 = Z, 22 = X,
 *   23 = U, 24 = O.  Codes match only themselves (an ambiguity code such as X
 *   matches X and nothing else).
 * A family is k >= 1 sequences given as one concatenated residue buffer and
 * int64 offsets[k+1] (sequence i is residues[offsets[i] .. offsets[i+1])).
 * Every sequence has length 1..65535.
 * Pointers flagged "on device" are CUDA device pointers of the current
 * device (for example torch tensors' data_ptr()); otherwise host pointers.
 * cuda_stream is a cudaStream_t (or NULL for the legacy default stream).
 * Calls are stream-ordered: a call returns once its work is enqueued, except
 * that a call whose output is on the host waits for its stream to finish.
 * The caller owns every input and output buffer; outputs are caller-allocated.
 * A handle may be used from several host threads: calls on one handle are
 * serialised by an internal mutex.  On error no output is guaranteed.
 *
 * Return values: FAMSA_OK or one of the codes below; famsa_strerror() gives
 * a message.
 */
#ifndef FAMSA_GPU_H
#define FAMSA_GPU_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  FAMSA_OK = 0,
  FAMSA_EINVAL = 1,   /* bad argument: k < 1, NULL pointer, offsets not
                         increasing, empty sequence, residue code >= 25,
                         row range outside [0, k] */
  FAMSA_ERANGE = 2,   /* a sequence longer than 65535, or an output with more
                         than 2^31 - 1 entries */
  FAMSA_ENOMEM = 3,   /* device or host allocation failed */
  FAMSA_ECUDA = 4,    /* a CUDA runtime call or kernel launch failed */
  FAMSA_ETIMEOUT = 5, /* a bounded device-side wait gave up */
  FAMSA_EBUSY = 6,    /* the serving queue is full */
  FAMSA_ELIMIT = 7,   /* beyond the fixed limits of famsa_lcs_query_noalloc */
  FAMSA_ECANCELED = 8 /* a serving request cancelled before it started */
} famsa_status;

/* Opaque handle: a packed family resident on the device.  It owns a device
 * copy of the residues, the per-sequence match-bitmask (Peq) tables, the
 * length-sorted column layout, and the scratch used by the tree build.  */
typedef struct famsa_family famsa_family;

/* Message for a status code; never NULL, static storage. */
const char *famsa_strerror(int status);

/* Library version as 10000*major + 100*minor + patch. */
int famsa_version(void);

/*
 * famsa_encode_ascii -- map protein letters to the residue codes every other
 * call takes (host only, no CUDA).  The paper's alphabet is the twenty amino
 * acids plus a few special symbols ("Pairwise similarities calculation"); the
 * reading here is codes 0-19 = A C D E F G H I K L M N P Q R S T V W Y and
 * 20 = B, 21 = Z, 22 = X, 23 = U, 24 = O.  Lowercase letters map like
 * uppercase; any other byte (gap '-', stop '*', digits, J, whitespace) is an
 * error, never a silent substitution.
 *   text      n bytes (host).
 *   codes     n bytes (host, caller-owned), written only on success.
 *   bad_pos   optional: the index of the first rejected byte, or -1.
 * Returns FAMSA_OK, or FAMSA_EINVAL for a NULL pointer, n < 0 or a rejected
 * byte.
 */
int famsa_encode_ascii(const char *text, int64_t n, uint8_t *codes, int64_t *bad_pos);

/*
 * famsa_pack_peq -- validate a family, copy it to the device and build its
 * match-bitmask tables ("Pairwise similarities calculation": the LCS is
 * computed bit-parallel, w = 64 DP cells per machine word, which needs for
 * every sequence A and symbol c the bitmask Peq_A[c] of the positions of A
 * holding c).
 *
 * residues, offsets: the family (see conventions); both on the device when
 *   residues_on_device != 0, else both on the host.
 * k: number of sequences, >= 1.
 * out: receives the new handle (set to NULL on error).
 *
 * Builds, on the device: bit p % 64 of word p / 64 of Peq_A[c] is set iff
 * A[p] == c (bits past |A| are 0); sequences ordered by (length, index); a
 * column layout of 32-sequence groups with 16-residue chunks interleaved so
 * a warp reads 512 contiguous bytes per chunk.  Synchronises cuda_stream
 * once (to read the validation status).
 * Errors: EINVAL, ERANGE (see above), ENOMEM, ECUDA.
 */
int famsa_pack_peq(const uint8_t *residues, const int64_t *offsets, int32_t k,
                   int residues_on_device, void *cuda_stream, famsa_family **out);

/* Number of sequences of a packed family (or -1 for NULL). */
int32_t famsa_family_size(const famsa_family *f);

/*
 * famsa_lcs_allpairs -- LCS length of every unordered pair.
 * lcs_out: k*(k-1)/2 int32, pairs i < j in row-major order: the pair (i, j)
 *   is at i*k - i*(i+1)/2 + (j - i - 1).  On the device iff
 *   out_on_device != 0.
 * Errors: EINVAL (NULL handle or output), ERANGE (k*(k-1)/2 > 2^31 - 1; use
 *   famsa_lcs_rows), ENOMEM, ECUDA.
 */
int famsa_lcs_allpairs(const famsa_family *f, int32_t *lcs_out, int out_on_device,
                       void *cuda_stream);

/*
 * famsa_lcs_rows -- a band of rows of the lower triangle, for streaming.
 * Rows i in [row_begin, row_end); row i lists LCS(i, j) for j = 0..i-1, and
 * the rows are concatenated: row i starts at
 *   (i*(i-1) - row_begin*(row_begin-1)) / 2.
 * out: that many int32, on the device iff out_on_device != 0.
 * Errors: EINVAL (range outside 0 <= row_begin <= row_end <= k), ERANGE
 *   (more than 2^31 - 1 outputs), ENOMEM, ECUDA.
 */
int famsa_lcs_rows(const famsa_family *f, int32_t row_begin, int32_t row_end, int32_t *out,
                   int out_on_device, void *cuda_stream);

/*
 * famsa_slink_tree -- the single-linkage guide tree ("Determination of the
 * guide tree": single linkage by SLINK, computed incrementally from the
 * similarity rows so the k x k matrix is never stored; similarity(A,B) =
 * LCS/indel^2 with indel = |A| + |B| - 2 LCS).
 *
 * Pairs are ordered by the exact rational distance indel^2 / LCS (a strictly
 * decreasing transform of the similarity): LCS = 0 gives +infinity, identical
 * sequences give 0.  Outputs, all in the caller's sequence numbering:
 *   pi[k], lambda_num[k], lambda_den[k]: Sibson's pointer representation.
 *     For j < k-1: lambda(j) = min over l > j of the single-link (minimax)
 *     distance u(j,l), pi(j) = max{ l > j : u(j,l) <= lambda(j) }.  The last
 *     point has pi = k-1 and lambda = +inf.  lambda is a reduced fraction
 *     num/den; +inf is (1, 0) and 0 is (0, 1).
 *   merges[2*(k-1)], h_num[k-1], h_den[k-1], sizes[k-1]: the merge list.
 *     Points j < k-1 are taken in (lambda(j), j) ascending order (a fixed
 *     lowest-index tie-break); merge t joins the clusters holding j and
 *     pi(j), records (smaller id, larger id), the height lambda(j) and the
 *     new size, and the new cluster gets id k + t (leaves are 0..k-1).
 * Any output pointer may be NULL to skip it.  Outputs are on the device iff
 * out_on_device != 0.  k == 1 gives pi = {0}, lambda = {(1,0)}, no merges.
 * Errors: EINVAL, ENOMEM, ECUDA, ETIMEOUT.
 */
int famsa_slink_tree(const famsa_family *f, int32_t *pi, uint64_t *lambda_num,
                     uint32_t *lambda_den, int32_t *merges, uint64_t *h_num, uint32_t *h_den,
                     int32_t *sizes, int out_on_device, void *cuda_stream);

/*
 * famsa_lcs_query -- LCS of query sequences against every member of a
 * resident family (the "Pairwise similarities calculation" applied to new
 * sequences; used by the serving loop).
 * q, q_offsets: nq query sequences in the family format (codes 0..24,
 *   lengths 1..65535), on the device iff q_on_device != 0.
 * out: nq*k int32, out[i*k + j] = LCS(query i, member j); on the device iff
 *   out_on_device != 0.
 * Errors: EINVAL, ERANGE, ENOMEM, ECUDA.
 */
int famsa_lcs_query(const famsa_family *f, const uint8_t *q, const int64_t *q_offsets,
                    int32_t nq, int q_on_device, int32_t *out, int out_on_device,
                    void *cuda_stream);

/*
 * famsa_upgma_tree -- UPGMA, the guide tree the paper names beside single
 * linkage and sets against it for memory ("Determination of the guide
 * tree": it needs the whole O(k^2) similarity matrix), over the family's
 * distances d = indel^2 / LCS as doubles (+inf for LCS = 0).  Each step
 * joins the live clusters in slots a < b with the smallest (d, a, b) and
 * sets d(a, c) = (n_a * d(a, c) + n_b * d(b, c)) / (n_a + n_b), each
 * operation rounded on its own (no fused multiply-add).
 *   merges (2(k-1)): merge t joins cluster ids (smaller, larger), ids < k
 *     the caller's sequences, k + t' the cluster of merge t'.
 *   heights (k-1 doubles): d(a, b) at merge t.  sizes (k-1): the new
 *     cluster's size.
 * On the device iff on_device != 0; the call waits for its stream.  It holds
 * the k x k matrix of doubles and the LCS triangle on the device (k = 20,000:
 * 4.0 GB).
 * Errors: EINVAL (NULL), ERANGE (k^2 above 2^34), ENOMEM, ECUDA.
 */
int famsa_upgma_tree(const famsa_family *f, int32_t *merges, double *heights, int32_t *sizes, int on_device,
                     void *cuda_stream);

/*
 * famsa_nj_tree -- neighbour joining, the other guide tree the paper names
 * beside single linkage ("Determination of the guide tree"), over the same
 * distances as famsa_upgma_tree.  With r clusters live, R(i) is the sum of
 * d(i, j) over the live j != i, and the live slots a < b with the smallest
 * (Q, a, b), Q = (r - 2) d(a, b) - R(a) - R(b), are joined with branches
 * delta_a = d(a, b) / 2 + (R(a) - R(b)) / (2 (r - 2)) and
 * delta_b = d(a, b) - delta_a; the new cluster u takes slot a with
 * d(u, c) = (d(a, c) + d(b, c) - d(a, b)) / 2.  The row sums are added in
 * increasing j once, then follow each join: R(c) = R(c) - d(a, c) - d(b, c)
 * + d(u, c), R(u) = (R(a) + R(b) - r d(a, b)) / 2.  The last two clusters
 * are joined with d(a, b) / 2 on each branch (the root).  Every operation is
 * rounded on its own, in that order (no fused multiply-add).
 *   merges (2(k-1)): merge t joins cluster ids (smaller, larger), as
 *     famsa_upgma_tree.
 *   lengths (2(k-1) doubles): the branch lengths to merges[2t] and
 *     merges[2t+1] (they may be negative: neighbour joining does not
 *     prevent it).  sizes (k-1): the new cluster's size.
 * On the device iff on_device != 0; the call waits for its stream.  It holds
 * the k x k matrix of doubles on the device; each step reads the live part
 * of it once, so the tree is O(k^3).
 * Errors: EINVAL (NULL), ERANGE (k above 32,768, or a pair with LCS 0: an
 *   infinite distance, for which neighbour joining is undefined), ENOMEM,
 *   ECUDA.
 */
int famsa_nj_tree(const famsa_family *f, int32_t *merges, double *lengths, int32_t *sizes, int on_device,
                  void *cuda_stream);

/*
 * famsa_progressive_schedule -- the merge list in the form the progressive
 * stage consumes ("Progressive construction of the alignment": O(k) profile
 * alignments in guide-tree order, spread over threads; at least half align a
 * single sequence with a profile, a simpler DP).
 *   merges (2(k-1)), sizes (k-1): as famsa_slink_tree / famsa_batch_tree
 *     write them (merge t joins ids merges[2t], merges[2t+1]; ids < k are
 *     sequences, k + t' the cluster made by merge t').
 *   level[t] (k-1): 1 + the larger level of merge t's two children (a
 *     sequence is level 0).  Merges of one level never use one another, so
 *     a level can run at once after the levels below it.
 *   order (k-1): the merges sorted by (level, t).
 *   level_start (k entries of room): level l is order[level_start[l-1] ..
 *     level_start[l]), l = 1..n_levels.
 *   kind[t] (k-1): 0 two single sequences, 1 a single sequence and a
 *     profile (the degenerate case), 2 two profiles.
 *   n_levels: host int32, the number of levels.
 * All other buffers on the device iff on_device != 0; the call waits for its
 * stream.
 * Errors: EINVAL (k < 1, NULL, a child id that is not a sequence or an
 *   earlier merge), ENOMEM, ECUDA.
 */
int famsa_progressive_schedule(int32_t k, const int32_t *merges, const int32_t *sizes, int32_t *level,
                               int32_t *order, int32_t *level_start, int32_t *kind,
                               int32_t *n_levels, int on_device, void *cuda_stream);

/*
 * Gap types and set-size scaled gap costs ("Gap types and costs
 * determination").  Four gap types with affine costs: terminal open (T_o),
 * terminal extension (T_e), open (G_o), extension (G_e); every cost is
 * multiplied by g_scale = 1 + log(k / g_l) / g_d (natural log; the paper's
 * defaults g_l = 45, g_d = 7), k the number of sequences of the input set.
 * Alignments are m rows of n bytes: residue codes, or FAMSA_GAP for a gap.
 * Type codes: 0 residue, 1 T_o, 2 T_e, 3 G_o, 4 G_e.  A gap before a row's
 * first residue or after its last is terminal, any other is not; the first
 * gap of a run opens it and the others extend it (a row of gaps only is one
 * terminal run).
 *
 * famsa_gap_types: those types for every cell (aln, types: m*n bytes ON THE
 *   DEVICE; stream-ordered).
 * famsa_gap_scale: g_scale for a set of k sequences (host; NaN for k < 1,
 *   g_l <= 0 or g_d == 0).
 * famsa_gap_cost: per row, g_scale(k) * (T_o*#T_o + T_e*#T_e + G_o*#G_o +
 *   G_e*#G_e), costs = {T_o, T_e, G_o, G_e} on the host, types and cost (m
 *   doubles) ON THE DEVICE; stream-ordered.
 * famsa_gap_insert: c gap columns inserted before original columns
 *   positions[0..c) (host, ascending, 0..n; equal positions give adjacent
 *   columns) into every row, with the types corrected as the paper's six
 *   cases S1..S6 say: the inserted gap takes its type from its neighbours,
 *   and a T_o or G_o right after it becomes T_e or G_e.  aln, types: m*n,
 *   aln_out, types_out: m*(n+c) bytes, ON THE DEVICE; the call waits for its
 *   stream.
 * Errors: EINVAL (NULL, negative sizes, positions out of range or not
 *   ascending), ERANGE (more than 2^31-1 rows for famsa_gap_types), ECUDA.
 */
#define FAMSA_GAP 255
int famsa_gap_types(const uint8_t *aln, int64_t m, int32_t n, uint8_t *types, void *cuda_stream);
double famsa_gap_scale(int64_t k, double g_l, double g_d);
int famsa_gap_cost(const uint8_t *types, int64_t m, int32_t n, int64_t k, const double *costs, double g_l,
                   double g_d, double *cost, void *cuda_stream);
int famsa_gap_insert(const uint8_t *aln, const uint8_t *types, int64_t m, int32_t n, const int32_t *positions,
                     int32_t c, uint8_t *aln_out, uint8_t *types_out, void *cuda_stream);

/*
 * Sharding the pair set across devices ("Pairwise similarities calculation":
 * the pairs are independent; "Determination of the guide tree": single
 * linkage).  Single linkage depends only on a minimum spanning tree of the
 * distance graph, and the minimum spanning tree of a union of edge sets is
 * the minimum spanning tree of the union of their minimum spanning forests.
 * So each device takes a range of rows, reduces the pairs of those rows to a
 * forest with famsa_msf_rows, the forests are exchanged (fewer than k edges
 * each), and famsa_tree_from_edges builds exactly the tree famsa_slink_tree
 * gives for the whole family.
 *
 * famsa_msf_rows -- the minimum spanning tree of the pairs (i, j) with i in
 * the rows [row_begin, row_end) and j < i, where rows are the points in the
 * family's internal order (1 <= row_begin < row_end <= k; rows [1, k) cover
 * every pair once, so any partition of them into ranges shards the pairs).
 * Those pairs join points 0..row_end-1, so the tree has row_end - 1 edges.
 *   edge_a[e] < edge_b[e]: the edge's two points in the caller's labels;
 *   h_num[e] / h_den[e]: its distance indel^2 / LCS in lowest terms
 *     (+inf = 1 / 0).  row_end - 1 entries each; on the device iff
 *     out_on_device != 0 (otherwise the call waits for its stream).
 * Errors: EINVAL (NULL, bad range), ERANGE (a sequence longer than 32767:
 *   the exact keys of this path need the shorter lengths), ENOMEM, ECUDA.
 */
int famsa_msf_rows(const famsa_family *f, int32_t row_begin, int32_t row_end, int32_t *edge_a,
                   int32_t *edge_b, uint64_t *h_num, uint32_t *h_den, int out_on_device,
                   void *cuda_stream);

/*
 * famsa_tree_from_edges -- the single-linkage tree of k points from any edge
 * list that contains a minimum spanning tree of their distance graph (for
 * example the union of the famsa_msf_rows forests of shards that cover rows
 * [1, k)).  Edges as famsa_msf_rows writes them: points 0..k-1, distances as
 * fractions with a denominator <= 32767 and a numerator below 2^32, or +inf.
 * Outputs as famsa_slink_tree (pi, lambda, merge list, sizes), in the labels
 * of the edges.  All buffers on the device iff on_device != 0; the call
 * waits for its stream.
 * Errors: EINVAL (k < 1, NULL, fewer than k - 1 edges, an edge that is out
 *   of range, a self loop, a distance outside the range above, or edges that
 *   do not join all k points; outputs then undefined), ENOMEM, ECUDA.
 */
int famsa_tree_from_edges(int32_t k, int64_t n_edges, const int32_t *edge_a, const int32_t *edge_b,
                          const uint64_t *e_num, const uint32_t *e_den, int32_t *pi,
                          uint64_t *lambda_num, uint32_t *lambda_den, int32_t *merges,
                          uint64_t *h_num, uint32_t *h_den, int32_t *sizes, int on_device,
                          void *cuda_stream);

/*
 * famsa_merge_similarity -- the merge heights as the paper's similarity
 * LCS / indel^2 ("Pairwise similarities calculation"), a double beside the
 * exact fractions the tree calls return.  A height num / den is the distance
 * indel^2 / LCS, so the similarity is den / num: +infinity for height 0
 * (identical sequences) and 0 for height +infinity (LCS 0).
 *   h_num, h_den: n heights as returned by famsa_slink_tree or
 *     famsa_batch_tree, ON THE DEVICE.
 *   similarity: n doubles ON THE DEVICE (caller-owned).
 * Stream-ordered on cuda_stream; returns after enqueue.
 * Errors: EINVAL (NULL pointer with n > 0, n < 0), ECUDA.
 */
int famsa_merge_similarity(const uint64_t *h_num, const uint32_t *h_den, int64_t n,
                           double *similarity, void *cuda_stream);

/*
 * famsa_lcs_query_noalloc -- famsa_lcs_query for callers that cannot
 * allocate device memory at call time.  The paper has no counterpart: it is
 * an interface of this library only.
 *
 * Some callers hand all their device memory out up front (a serving process
 * that reserves its whole budget in its own arena, or shares the GPU with a
 * framework that owns the rest of it), so a call that allocates fails or
 * takes memory they cannot spare; on a latency-bound request path an
 * allocation can also wait for the device.  This entry point allocates
 * nothing: its scratch (the queries' match-bitmask tables and row list) is
 * a fixed array of FAMSA_NOALLOC_SCRATCH_BYTES in the library's device
 * memory, one per device.
 *
 * q, q_offsets: nq query sequences in the family format, ON THE DEVICE.
 * nq: 1..FAMSA_NOALLOC_MAX_QUERIES.
 * max_len: an upper bound on every query's length, 1..FAMSA_NOALLOC_MAX_LEN
 *   (each query is computed with ceil(max_len / 64) words, so a tight bound
 *   is faster).
 * out: nq*k int32 ON THE DEVICE, out[i*k + j] = LCS(query i, member j), the
 *   same values famsa_lcs_query gives.
 * Errors: EINVAL (NULL argument, nq or max_len < 1, a query length outside
 *   1..max_len, a residue code >= 25: the last two found on the device, in
 *   which case out is undefined), ELIMIT (nq or max_len beyond the limits
 *   above; nothing is enqueued), ECUDA.
 * The call returns after its stream has finished (it reads the validation
 * status back).
 * Set-up: the first call on a device looks the array's address up on that
 * device (cudaGetSymbolAddress), so make that first call before any stream
 * capture on the device.
 * Sharing: every call on a device uses the same array, which keeps what the
 * last call wrote there; each call rewrites all of it that it reads.  Within
 * one process the library holds one lock from a call's first launch until its
 * stream has finished, so calls from several host threads (any handles, any
 * streams) run one after another.  GPU work that overlaps a call and touches
 * the array in another way -- a CUDA graph captured around a call and
 * replayed beside another call -- races on it: keep such replays serialised.
 */
#define FAMSA_NOALLOC_MAX_QUERIES 64
#define FAMSA_NOALLOC_MAX_LEN 4096
#define FAMSA_NOALLOC_SCRATCH_BYTES (1048576 + 4096)
int famsa_lcs_query_noalloc(const famsa_family *f, const uint8_t *q, const int64_t *q_offsets,
                            int32_t nq, int32_t max_len, int32_t *out, void *cuda_stream);

/*
 * Batched families -- the same stages I+II ("Pairwise similarities
 * calculation", "Determination of the guide tree") for many independent
 * families at once, so that small families do not leave the GPU idle.
 *
 * famsa_batch_pack -- validate and pack n_families families given as one
 * sequence list (the family format with n_seqs sequences) split by
 * family_offsets[n_families + 1] (HOST int64): family f is sequences
 * family_offsets[f] .. family_offsets[f+1]-1, at least one each,
 * family_offsets[0] = 0 and family_offsets[n_families] = n_seqs.
 * residues/offsets are on the device iff residues_on_device != 0.
 * Limits: n_seqs < 2^31, n_families <= 65535.  Errors: EINVAL, ERANGE,
 * ENOMEM, ECUDA.  Synchronises cuda_stream.
 */
typedef struct famsa_batch famsa_batch;
int famsa_batch_pack(const uint8_t *residues, const int64_t *offsets, int64_t n_seqs,
                     const int64_t *family_offsets, int32_t n_families, int residues_on_device,
                     void *cuda_stream, famsa_batch **out);

/*
 * famsa_batch_tree -- every family's single-linkage tree, exactly as
 * famsa_slink_tree gives it for that family alone, in the family's own
 * labels 0..k_f-1:
 *   pi, lambda_num, lambda_den: n_seqs entries; family f's at
 *     family_offsets[f];
 *   merges (2 per merge), h_num, h_den, sizes: n_seqs - n_families merges;
 *     family f's k_f - 1 merges start at merge family_offsets[f] - f, with
 *     cluster ids k_f + t local to the family.
 * Any output may be NULL.  Outputs on the device iff out_on_device != 0.
 * The first call builds the execution plan (work lists, buffers) and
 * captures the whole computation -- LCS launches per kernel width over all
 * families, the row update with one thread-block cluster per family, the
 * finalisation -- into one CUDA graph; every call launches that graph on
 * cuda_stream.  Errors: EINVAL, ENOMEM, ECUDA.
 */
int famsa_batch_tree(famsa_batch *b, int32_t *pi, uint64_t *lambda_num, uint32_t *lambda_den,
                     int32_t *merges, uint64_t *h_num, uint32_t *h_den, int32_t *sizes,
                     int out_on_device, void *cuda_stream);

/* Counters of the batch plan, stats[16] int64: 0 LCS cells (sum of |A||B|
 * over every family's pairs), 1 LCS word steps, 2 pairs, 3 LCS work items,
 * 4 kernel launches captured in the graph, 5 LCS kernel widths, 6 families
 * on the global-memory row update, 7..9 device time in ns of the LCS, the
 * row update and the finalisation in the last graph launch (this call waits
 * for that launch), 10 kernel widths the autotuner timed for this plan, 11
 * ns the autotuner took, 12 ns of host planning before the graph capture
 * (autotuner included), 13 ns of the capture, 14 ns of the graph
 * instantiation, 15 graph nodes.  Zero before the first tree.
 *
 * The autotuner: the first plan with at least 64 rows of a thread-per-pair
 * width times each allowed rows-per-tile choice (1, 2 or 4 rows, with rows
 * x words <= 32) on the same sample of its rows (about 4e9 word steps) and
 * keeps the default unless another choice is at least 2 % faster, for the
 * process, for batches and single families alike; results do not depend on
 * the choice. */
int famsa_batch_stats(const famsa_batch *b, int64_t *stats);

/* Release a batch and its device memory (NULL is ignored). */
void famsa_batch_free(famsa_batch *b);

/*
 * Serving loop -- guide-tree requests for new families and query batches
 * scored against resident families, run by a request queue with admission
 * by an HBM budget and continuous batching: each of `slots` worker threads
 * owns a CUDA stream and takes the first queued request that fits the free
 * part of the budget (a query also needs its family resident); requests
 * that arrive while others run start as soon as a slot and memory free up,
 * and their kernels overlap on the device.  A request that is older than
 * about one second is not overtaken.  A request larger than the whole
 * budget runs when nothing else does.  Each result equals the
 * single-request call (famsa_slink_tree / famsa_lcs_query) on the same
 * input, whatever runs beside it.  All inputs and outputs are host buffers;
 * inputs are copied at submission.  The calls below are thread-safe.
 *
 * famsa_server_create: budget in bytes of device memory for running and
 *   resident requests (estimated per request), slots in 1..64.  Uses the
 *   current device.
 * famsa_server_submit_tree: a family (see the conventions); keep_resident
 *   keeps its packed tables on the device for queries until released.
 * famsa_server_submit_query: nq queries against the family of an earlier
 *   tree request submitted with keep_resident (it may still be running).
 *   A query whose family fails ends with EINVAL.
 * famsa_server_wait: wait up to timeout_ms (< 0: forever) for a request;
 *   returns its status (FAMSA_OK or the error of its library call), or
 *   ETIMEOUT if it is still queued or running, EINVAL for an unknown id.
 * famsa_server_tree_result / famsa_server_query_result: copy a finished
 *   request's results, laid out as famsa_slink_tree / famsa_lcs_query give
 *   them (any tree output may be NULL).  EINVAL unless finished with OK.
 * famsa_server_request_info: info[7] int64 = status, kind (0 tree, 1 query),
 *   sequences (k or nq), ns from submission to start (-1 while queued), ns
 *   from submission to completion (-1 before), LCS cells, bytes reserved.
 * famsa_server_cancel: take a queued request out of the queue; its status
 *   becomes FAMSA_ECANCELED (queries queued against a cancelled tree request
 *   then fail with FAMSA_EINVAL).  A running request cannot be stopped (its
 *   kernels run to the end): FAMSA_EBUSY; unknown or finished: FAMSA_EINVAL.
 * famsa_server_release: forget a request and free a resident family (after
 *   its running queries end).
 * famsa_server_stats: stats[8] int64 = submitted, done, failed, queued,
 *   running, most running at once, bytes reserved now, most reserved.
 * famsa_server_destroy: fails queued requests, waits for running ones,
 *   frees everything.
 * Errors: EINVAL (bad argument or id), EBUSY (more than 2^20 queued).
 * The paper has no serving loop; this is the library's own scheduler.
 */
typedef struct famsa_server famsa_server;
int famsa_server_create(int64_t hbm_budget_bytes, int32_t slots, famsa_server **out);
int famsa_server_submit_tree(famsa_server *s, const uint8_t *residues, const int64_t *offsets,
                             int32_t k, int keep_resident, int64_t *request_id);
int famsa_server_submit_query(famsa_server *s, int64_t family_request, const uint8_t *q,
                              const int64_t *q_offsets, int32_t nq, int64_t *request_id);
int famsa_server_wait(famsa_server *s, int64_t request_id, int64_t timeout_ms);
int famsa_server_tree_result(famsa_server *s, int64_t request_id, int32_t *pi, uint64_t *lambda_num,
                             uint32_t *lambda_den, int32_t *merges, uint64_t *h_num, uint32_t *h_den,
                             int32_t *sizes);
int famsa_server_query_result(famsa_server *s, int64_t request_id, int32_t *out);
int famsa_server_request_info(famsa_server *s, int64_t request_id, int64_t *info);
int famsa_server_release(famsa_server *s, int64_t request_id);
int famsa_server_cancel(famsa_server *s, int64_t request_id);
int famsa_server_stats(famsa_server *s, int64_t *stats);
void famsa_server_destroy(famsa_server *s);

/* Release a handle and its device memory (NULL is ignored).  Waits for the
 * handle's pending work. */
void famsa_free(famsa_family *f);

/*
 * famsa_last_stats -- counters of the last famsa_slink_tree call on this
 * handle (for benchmarks).  stats[24] int64:
 *   0 kernel launches of the tree build, 1 LCS cells (sum of |A||B| over
 *   pairs), 2 LCS word steps (64-bit words of the Peq side times symbols of
 *   the other side, summed over pairs), 3 pairs, 4 insertions whose re-layout
 *   needed a run merge, 5 run-merge rounds, 6 points, 7 device time of the
 *   LCS kernels in ns (CUDA events around each row block), 8 device time of
 *   the row-update kernels in ns, 9 device time of the finalisation in ns,
 *   10 LCS kernel launches, 11 kernel launches of famsa_pack_peq for this
 *   handle, 12 row update (1 insertion in cluster shared memory, 2 insertion
 *   in global memory, 3 spanning-tree rebuild), 13 the cluster size of 1, 14..17 kilocycles spent by one thread of the
 *   shared-memory kernel in its phases (14 unused; 15 scans, pointer update
 *   and prefetch; 16 shift re-layout plus the next point's distances;
 *   17 run-merge re-layout), 18 1 when keys were exact order codes (every
 *   length <= 32767), 19 run merges done in shared memory, 20 the runs they
 *   merged (both sides), 21..23 reserved.
 * Returns EINVAL for NULL arguments.
 */
int famsa_last_stats(const famsa_family *f, int64_t *stats);

#ifdef __cplusplus
}
#endif

#endif /* FAMSA_GPU_H */
