/*
 * swgb.h -- C ABI of libswgb: batched Smith-Waterman local alignment with
 * affine gaps on one GB300 (sm_103a), for many-against-many protein search.
 *
 * The operation is the paper's alignment step (Sec. "Protein similarity
 * search pipeline", component (ii): batch alignment of the candidate pairs
 * found by shared k-mers; Sec. "Load balancing": a Smith-Waterman variant that
 * fills the whole score matrix of each pair; Sec. "How Performance Was
 * Measured": cell updates per second count the forward scoring pass).  The
 * problem statement it serves is Sec. "Overview of the Problem": a set of
 * query sequences aligned against a set of reference sequences (or a set
 * against itself), over candidate pairs (Sec. "Load balancing techniques":
 * each nonzero of the overlap matrix is one pairwise alignment).
 *
 * Scoring (integer throughout, "Performance Attributes" table):
 *   rows i walk the query, columns j the reference; a gap of length L costs
 *   gap_open + gap_extend * L;
 *     E(i,j) = max(E(i,j-1) - e, H(i,j-1) - o - e)
 *     F(i,j) = max(F(i-1,j) - e, H(i-1,j) - o - e)
 *     H(i,j) = max(0, H(i-1,j-1) + s(q_i, r_j), E(i,j), F(i,j))
 *   score S = max H.  The paper uses open 11 / extend 2 in its production
 *   run (program-parameters table); both are arguments here.
 * Record of a pair (0-based, inclusive coordinates):
 *   (q_end, r_end)     the row-major-first cell (smallest i, then j) with H = S;
 *   (q_start, r_start) from the local DP of the reversed prefixes
 *                      q[q_end..0], r[r_end..0]: its row-major-first cell
 *                      (a, b) with value S gives q_start = q_end - a,
 *                      r_start = r_end - b;
 *   S = 0 reports -1 in all four coordinates.
 * The paper fixes neither tie-breaks nor the start-finding pass; these are the
 * library's stated conventions, and results are identical (bit for bit) to a
 * plain int32 implementation of them.
 *
 * Residues are codes 0..23 in the order A R N D C Q E G H I L K M F P S T W Y
 * V B Z X * (NCBI BLOSUM order).  Sequence sets may also be loaded from ASCII
 * letters (case-insensitive; U and O read as X).
 *
 * Threading: a context owns device scratch reused by every call, so calls on
 * one context must be ordered (one stream, or caller-serialised).  Different
 * contexts are independent.  A sequence set (or index) may be read by the
 * calls of any context of its device at once; it must not be reloaded or
 * destroyed while such calls are in flight.
 */
#ifndef SWGB_H
#define SWGB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes (every int-returning call) ---- */
#define SWGB_OK 0
#define SWGB_EINVAL (-1)  /* null pointer, negative count, bad flags, penalty out of range */
#define SWGB_ERANGE (-2)  /* pair index outside its sequence set, or sequence too long */
#define SWGB_EBADRES (-3) /* a residue letter or code outside the alphabet */
#define SWGB_ENOMEM (-4)  /* a device or host allocation failed */
#define SWGB_ECUDA (-5)   /* a CUDA runtime call failed (message in swgb_last_error) */
#define SWGB_EINTERNAL (-6) /* the device detected an inconsistency in its own results */
#define SWGB_ETOOBIG (-7) /* a size exceeds a fixed limit (swgb_align_noalloc, swgb_discover, server) */
#define SWGB_ETIMEDOUT (-8) /* swgb_server_wait: the request did not finish in time */

#define SWGB_ALPHABET_SIZE 24
/* Longest sequence accepted (residues). */
#define SWGB_MAX_LENGTH 65536

/* ---- flags ---- */
/* swgb_seqset_create / swgb_seqset_load */
#define SWGB_SEQ_ASCII 0x1u   /* residues are ASCII letters; otherwise codes 0..23 */
#define SWGB_SEQ_DEVICE 0x2u  /* residues and offsets are device pointers; otherwise host */
#define SWGB_SEQ_COPY 0x4u    /* host residues go through the copy engines even when pinned */
/* swgb_params.flags */
#define SWGB_FORCE_INT32 0x1u /* every pair on the 32-bit path (no 16x2 packing) */
#define SWGB_TIMING 0x2u      /* record CUDA events around the forward and reverse kernels */

typedef struct swgb_ctx swgb_ctx;
typedef struct swgb_seqset swgb_seqset;
typedef struct swgb_server swgb_server;

/* One alignment result, 20 bytes. */
typedef struct {
    int32_t score;
    int32_t q_start;
    int32_t q_end;
    int32_t r_start;
    int32_t r_end;
} swgb_record;

/* Scoring parameters.
 *   matrix:     host pointer to 24 x 24 int8, row = query code, column =
 *               reference code (need not be symmetric).  Read during the call.
 *   gap_open:   o >= 0;  gap_extend: e >= 1.  The 8-bit query profile holds
 *               s + o + e, so max(matrix) + o + e must be <= 127.  A matrix
 *               with some s + o + e < 0 runs every pair on the 32-bit path
 *               (same results, about half the speed).
 *   flags:      SWGB_FORCE_INT32 | SWGB_TIMING. */
typedef struct {
    const int8_t* matrix;
    int32_t gap_open;
    int32_t gap_extend;
    uint32_t flags;
} swgb_params;

/* Counters of the last completed call on a context (see swgb_last_stats). */
typedef struct {
    int64_t n_pairs;         /* pairs in the call */
    int64_t n_int16_pairs;   /* forward pass on the packed 16x2 path */
    int64_t n_int32_pairs;   /* forward pass on the 32-bit path */
    int64_t n_reverse_pairs; /* pairs with score > 0 (reverse pass run) */
    int64_t forward_cells;   /* sum of lq * lr over the pairs */
    int64_t reverse_cells;   /* sum of (q_end + 1) * (r_end + 1) over scored pairs */
    float forward_ms;        /* forward DP kernels, CUDA events (SWGB_TIMING), else -1 */
    float reverse_ms;        /* reverse DP kernels, CUDA events (SWGB_TIMING), else -1 */
    float total_ms;          /* whole call on the stream (SWGB_TIMING), else -1 */
    int32_t kernel_launches; /* kernels the call launched */
    int64_t n_band_pairs;    /* reverse passes run over a band (swgb_set_band_min) */
    int64_t n_band_certified;/* of which the exactness certificate held (the others re-ran
                                over the whole rectangle) */
    int64_t forward_slots;   /* cell updates the forward DP kernels computed: wavefront steps x
                                tile rows x 2 pairs per register (fill and padding included) */
    int64_t reverse_slots;   /* likewise for the reverse pass, all its rounds */
} swgb_stats;

/* Creates a context on CUDA device `device` (made current on the calling
 * thread).  *out receives the context; the caller destroys it.
 * Errors: EINVAL (out NULL), ECUDA (no such device / CUDA failure), ENOMEM. */
int swgb_create(int device, swgb_ctx** out);

/* Frees the context and all its device scratch.  NULL is ignored. */
void swgb_destroy(swgb_ctx* ctx);

/* Message of the last failing call on ctx (empty string if none).  The
 * pointer stays valid until the next call on ctx. */
const char* swgb_last_error(const swgb_ctx* ctx);

/* Copies the library's BLOSUM62 (24 x 24 int8, row = query) into out[576]. */
void swgb_blosum62(int8_t* out);

/* Creates a sequence set on ctx's device from n_seqs sequences: sequence k is
 * residues[offsets[k] .. offsets[k+1]) (offsets has n_seqs + 1 entries,
 * non-decreasing, offsets[0] = 0 is not required).  flags: SWGB_SEQ_ASCII,
 * SWGB_SEQ_DEVICE.  The data are copied (and encoded) into library-owned
 * device memory on `stream` (a cudaStream_t, NULL = legacy default); the call
 * returns after the copy has completed, so the inputs may be reused.
 * The host reads only offsets[0] and offsets[n_seqs]: the offsets are checked
 * (non-decreasing, lengths up to SWGB_MAX_LENGTH), measured and rebased on
 * the device.  Host residues in pinned (page-locked) memory are read in place
 * by the encode kernel over the host link (the fastest load on an idle GPU);
 * other host residues, and pinned ones with SWGB_SEQ_COPY, are uploaded first
 * by the copy engines (in four concurrent parts from 64 MB on), so the upload
 * itself needs no SMs.
 * Errors: EINVAL, ERANGE (a sequence longer than SWGB_MAX_LENGTH, or offsets
 * decreasing), EBADRES (a letter/code outside the alphabet; such codes are
 * stored as 0), ENOMEM, ECUDA.  After ERANGE from the offsets the set is
 * empty. */
int swgb_seqset_create(swgb_ctx* ctx, const void* residues, const int64_t* offsets,
                       int64_t n_seqs, uint32_t flags, void* stream, swgb_seqset** out);

/* Replaces the content of an existing set (same rules as create); device
 * memory is reused when it is large enough. */
int swgb_seqset_load(swgb_seqset* set, const void* residues, const int64_t* offsets,
                     int64_t n_seqs, uint32_t flags, void* stream);

/* Number of sequences and longest length of a set. */
int swgb_seqset_info(const swgb_seqset* set, int64_t* n_seqs, int64_t* max_length);

/* Frees a sequence set.  NULL is ignored. */
void swgb_seqset_destroy(swgb_seqset* set);

/* Aligns n_pairs candidate pairs.  pairs: device int32 [n_pairs][2] =
 * (query index into `queries`, reference index into `refs`); out: device
 * swgb_record [n_pairs], written in pair order.  Both buffers are caller-owned
 * and must stay valid until the stream reaches the end of the call.  refs may
 * equal queries (one set against itself).  Asynchronous on `stream`: returns
 * after enqueueing; argument errors (EINVAL) are returned immediately, errors
 * found on the device (ERANGE for a pair index out of range, whose record is
 * written as zero score) are returned by swgb_sync.  Device scratch is grown
 * on demand by this call (it may allocate).
 * Errors: EINVAL, ENOMEM, ECUDA. */
int swgb_align(swgb_ctx* ctx, const swgb_seqset* queries, const swgb_seqset* refs,
               const int32_t* pairs, int64_t n_pairs, const swgb_params* params,
               swgb_record* out, void* stream);

/* Same as swgb_align with HOST pairs and HOST out: copies the pairs to the
 * device, aligns, copies the records back and waits for the stream.  Pinned
 * host buffers give asynchronous copies.  Returns the device status too. */
int swgb_align_host(swgb_ctx* ctx, const swgb_seqset* queries, const swgb_seqset* refs,
                    const int32_t* pairs_host, int64_t n_pairs, const swgb_params* params,
                    swgb_record* out_host, void* stream);

/* Waits for `stream`, then returns (and clears) the device-side status of the
 * calls issued on ctx: SWGB_OK, ERANGE or EINTERNAL; ECUDA if the stream
 * failed. */
int swgb_sync(swgb_ctx* ctx, void* stream);

/* Counters and (with SWGB_TIMING) kernel times of the last call; waits for
 * that call's stream.  Errors: EINVAL, ECUDA. */
int swgb_last_stats(swgb_ctx* ctx, swgb_stats* out);

/* Measures the issue rate of the packed 16x2 add-max instruction the forward
 * kernel is built on: *ops_per_clk_per_sm = instructions retired per SM clock
 * per SM, from a kernel of independent chains timed with the SM cycle
 * counter.  Also reports the SM count.  Synchronous.  Errors: EINVAL, ECUDA. */
int swgb_probe_addmax_rate(swgb_ctx* ctx, double* ops_per_clk_per_sm, int* sm_count);

/* ---- tile selection ----
 * Every pair gets the tile (G lanes x R reference rows per lane, and a chunk
 * count for long references) of least modelled cost
 *     (query length + G - 1) x chunks x G x (R + overhead),
 * where overhead is the per-step work of a lane counted in rows.  It is a
 * context setting (default 6), read by each swgb_align and swgb_plan_create. */
int swgb_set_tile_overhead(swgb_ctx* ctx, int overhead);  /* EINVAL unless 0..64 */
int swgb_get_tile_overhead(const swgb_ctx* ctx);          /* current value */

/* ---- banded reverse pass ----
 * The reverse pass (start coordinates) of a scored pair may run over a
 * staircase band of the reversed prefixes (la x lb) instead of their whole
 * rectangle (the paper's aligner fills the whole matrix, Sec. "Load
 * balancing"; the band is this library's).  On a 32-lane tile of 32 R rows
 * (R = 9..13), chunk c of the reversed reference streams only the query
 * positions [c 32 R - khi, (c + 1) 32 R + W - khi), which hold the diagonals
 * from min(0, lb - la) - m to max(0, lb - la) + m of the chunk's rows, with
 * W = |lb - la| + 2 m, khi = max(0, lb - la) + m and m = 64 + max(la, lb) / 32.
 * The DP there is anchored at the end cell.  The band's start is kept only
 * under an exactness certificate: every cell of the computed region through
 * which an alignment could leave it bounds that alignment's score by the
 * region's value there plus the forward pass's maximum over the reference
 * rows beyond it plus one gap opening; if every such bound at a position up
 * to the first cell of value S is below S, no alignment of score S leaves
 * the region first and its first cell of value S is the start of the
 * whole-matrix definition.  Otherwise the pair is re-run over the whole
 * rectangle, so the records never depend on the setting.  The forward pass
 * records those maxima (one int32 per forward lane, from a pool of at most
 * 512 MB per workspace; pairs past it keep the rectangle) for pairs whose
 * query and reference both have at least band_min residues on the packed
 * 16-bit path; a cost model picks per pair between the rectangle and the
 * band tiles.
 * band_min: 0 (off) or 32..65536; default 0; a context setting read by
 * swgb_align and swgb_plan_create, tuned by swgb_autotune. */
int swgb_set_band_min(swgb_ctx* ctx, int band_min);      /* EINVAL outside the range */
int swgb_get_band_min(const swgb_ctx* ctx);              /* current value */

/* What the last swgb_autotune measured (fastest of its timed calls each). */
typedef struct {
    int32_t tile_overhead;      /* chosen tile-cost overhead */
    int32_t band_min;           /* chosen band threshold (0 = no band) */
    float best_ms;              /* whole-call time at the chosen pair */
    float runner_up_ms;         /* best time of any other overhead at the chosen band_min */
    int32_t runner_up_overhead;
    float band_off_ms;          /* time with no band at the chosen overhead */
    int32_t candidates;         /* settings timed */
} swgb_tuning;
int swgb_last_tuning(const swgb_ctx* ctx, swgb_tuning* out);  /* EINVAL on NULL */

/* Times swgb_align on the given batch (device buffers, like swgb_align):
 * first the tile-cost overhead over 2 .. 40 (13 values) at the current
 * band_min, then band_min over {0, 256, 320, 384, 512, 768, 1024} at the
 * chosen overhead, then the overhead again at the chosen band_min; each
 * setting gets one warm-up call and the fastest of five timed calls.  Keeps
 * the fastest pair in ctx and reports the overhead and its whole-call time in
 * ms (swgb_last_tuning has the rest).  Synchronous; out receives the batch's
 * records, which do not depend on either setting.  Errors: those of
 * swgb_align. */
int swgb_autotune(swgb_ctx* ctx, const swgb_seqset* queries, const swgb_seqset* refs,
                  const int32_t* pairs, int64_t n_pairs, const swgb_params* params,
                  swgb_record* out, void* stream, int* best_overhead, float* best_ms);

/* ---- plans: one batch shape captured into a CUDA graph ----
 * The persistent launches of swgb_align (bucketing, forward and reverse DP
 * kernels on the context's streams) for fixed buffers, captured once into a
 * CUDA graph and replayed by swgb_plan_launch.  A plan owns its bucketing and
 * boundary workspace; it shares the context's status word and counters, so
 * swgb_sync and swgb_last_stats report its launches.  The buffers (sets,
 * pairs, out) must stay allocated while the plan exists; their CONTENTS may
 * change between launches (new pairs of the same count, sequences reloaded
 * into sets whose capacity and longest length do not grow; a plan captured
 * over queries of the 20 standard letters only refuses to launch, EINVAL,
 * once its query set holds other codes).  Launches of one
 * context (plans and swgb_align) must be ordered, as for swgb_align. */
typedef struct swgb_plan swgb_plan;

/* Captures the pipeline for (queries, refs, pairs[n_pairs], params, out).
 * Allocates the plan's workspace.  Errors: EINVAL, ENOMEM, ECUDA. */
int swgb_plan_create(swgb_ctx* ctx, const swgb_seqset* queries, const swgb_seqset* refs,
                     const int32_t* pairs, int64_t n_pairs, const swgb_params* params,
                     swgb_record* out, swgb_plan** plan);

/* Replays the captured pipeline on `stream` (asynchronous; device errors are
 * returned by swgb_sync).  Errors: EINVAL, ECUDA. */
int swgb_plan_launch(swgb_plan* plan, void* stream);

/* Frees a plan.  NULL is ignored. */
void swgb_plan_destroy(swgb_plan* plan);

/* ---- candidate discovery by shared k-mers ----
 * Sec. "Protein similarity search pipeline": the candidate pairs of a
 * many-against-many search are the nonzeros of the overlap matrix C = A A^T,
 * A being the sequence-by-k-mer matrix (k = 6 in the production run,
 * program-parameters table), and C(i, j) the number of k-mers the two
 * sequences share.  Sec. "Load balancing techniques": C is symmetric, so one
 * triangle is enough, and pairs below the common-k-mer threshold (2 in
 * production) are not aligned.  Definitions used here (the paper gives no
 * formula):
 *   K(s)    = the set of DISTINCT k-mers of s made of standard letters only
 *             (codes 0..19; a window touching B, Z, X or * forms no k-mer);
 *   C(i, j) = |K(s_i) intersect K(s_j)|.
 * swgb_discover finds every pair i < j of one set with C(i, j) >= min_shared.
 *   k:          1..6;  min_shared >= 1.
 *   pairs:      DEVICE int32 [capacity][2], receives (i, j), i < j, ordered by
 *               i then j (the order does not depend on scheduling);
 *   counts:     DEVICE int32 [capacity] receiving C(i, j), or NULL;
 *   capacity:   entries the buffers hold; the first min(found, capacity)
 *               pairs are written;
 *   *n_found:   the number of pairs found (may exceed capacity: call again
 *               with larger buffers).
 * Synchronous on `stream` (returns after the results are written).  Device
 * scratch is owned by the context and grown on demand (it may allocate;
 * about 9 bytes per residue + 8 bytes per possible k-mer value, 20^k).
 * Errors: EINVAL, ETOOBIG (a set of 2^32 residues or more), ENOMEM, ECUDA,
 * EINTERNAL. */
int swgb_discover(swgb_ctx* ctx, const swgb_seqset* set, int k, int min_shared, int32_t* pairs,
                  int32_t* counts, int64_t capacity, int64_t* n_found, void* stream);

/* ---- identity, coverage and the similarity filter ----
 * The production run keeps a pair in the similarity graph when its
 * alignment has identity >= 0.30 and coverage >= 0.70 (program-parameters
 * table); the paper defines neither measure.  Definitions used here:
 *   the global affine alignment (same scores and gaps as swgb_align, no zero
 *   floor) of the record's span q[q_start..q_end] x r[r_start..r_end] -- its
 *   optimum is the record's score -- is traced back from the span's end,
 *   preferring at a cell the diagonal, then a gap in the reference (a query
 *   residue against a gap), then a gap in the query, and inside a gap its
 *   opening before its extension;
 *   identity = identical columns / columns of that alignment;
 *   coverage = min((q_end - q_start + 1) / lq, (r_end - r_start + 1) / lr);
 *   pass     = identity >= id_num / id_den and coverage >= cov_num / cov_den,
 *              decided exactly in integers; a zero score never passes. */
typedef struct {
    int32_t id_num, id_den;    /* e.g. 3, 10 */
    int32_t cov_num, cov_den;  /* e.g. 7, 10 */
} swgb_thresholds;

typedef struct {
    int32_t matches;   /* identical columns (0 for a zero score) */
    int32_t columns;   /* alignment columns incl. gaps (0 for a zero score) */
    int32_t pass;      /* 1 if the pair passes the thresholds, else 0 */
} swgb_identity_record;

/* Identity and pass/fail of n_pairs records of swgb_align (same sets, same
 * pairs, same params).  pairs, records and out are DEVICE buffers, out is
 * swgb_identity_record [n_pairs] in pair order.  Synchronous on `stream`.
 * The span's DP runs forward carrying, per state, the (identical columns,
 * columns) of the path the preference above traces; no traceback matrix.
 * Device scratch (one work-list entry per pair, and one boundary column of
 * the longest query's rows per resident warp of the classes that split a
 * span into 256-column chunks) is owned by the context and grown on demand.
 * Errors: EINVAL, ENOMEM, ECUDA, ERANGE (a pair index or record coordinate
 * outside its sequences), EINTERNAL (a record whose span does not reach its
 * score, a span's chunk that waited too long for the previous chunk, or the
 * work lists disagreeing with their counts); a pair outside its sequences or
 * whose span does not reach its score gets -1, -1, 0. */
int swgb_identity(swgb_ctx* ctx, const swgb_seqset* queries, const swgb_seqset* refs,
                  const int32_t* pairs, const swgb_record* records, int64_t n_pairs,
                  const swgb_params* params, const swgb_thresholds* thresholds,
                  swgb_identity_record* out, void* stream);

/* Kernels launched by the last swgb_discover, swgb_identity,
 * swgb_pair_features, swgb_select_pairs or swgb_mlp_train call on ctx (-1 for
 * a NULL context). */
int swgb_search_launches(const swgb_ctx* ctx);

/* ---- resident k-mer index of a reference set ----
 * For the search of query sets against a fixed reference set (the paper's
 * problem statement allows two distinct sets, Sec. "Overview of the
 * Problem"): the references' distinct k-mers and their buckets (the columns
 * of the sequence-by-k-mer matrix, with first positions) stay in device
 * memory, so a query batch costs only its own k-mer sets and the join. */
typedef struct swgb_index swgb_index;

/* Builds the index of `refs` (which must outlive it) on ctx's device with k
 * in 1..6; about 12 bytes per reference residue + 4 (20^k + 1) bytes.
 * Synchronous on `stream`.  Errors: EINVAL, ETOOBIG, ENOMEM, ECUDA. */
int swgb_index_create(swgb_ctx* ctx, const swgb_seqset* refs, int k, void* stream,
                      swgb_index** out);
void swgb_index_destroy(swgb_index* index);
/* Reference count, k and device bytes held. */
int swgb_index_info(const swgb_index* index, int64_t* n_refs, int* k, int64_t* bytes);

/* Candidates of a query set against the index: every (query i, reference j)
 * with |K(q_i) intersect K(r_j)| >= min_shared (same K as swgb_discover),
 * ordered by (i, j), into DEVICE pairs [capacity][2] (and DEVICE counts
 * [capacity] or NULL); *n_found = their number (may exceed capacity).
 * Synchronous on `stream`.  Errors: as swgb_discover. */
int swgb_index_query(swgb_ctx* ctx, const swgb_index* index, const swgb_seqset* queries,
                     int min_shared, int32_t* pairs, int32_t* counts, int64_t capacity,
                     int64_t* n_found, void* stream);

/* swgb_pair_features for pairs (query i, reference j) of swgb_index_query,
 * using the index's tables for the references.  Synchronous on `stream`. */
int swgb_index_features(swgb_ctx* ctx, const swgb_index* index, const swgb_seqset* queries,
                        const int32_t* pairs, int64_t n_pairs, float* features, void* stream);

/* ---- the learned candidate filter ----
 * The paper keeps every candidate with at least two shared k-mers and notes
 * that few of them end in the similarity graph (Sec. "Blocked 2D Sparse
 * SUMMA"); the filter scores candidates from k-mer features with a small
 * network trained on the exact aligner's pass/fail labels, so that pairs it
 * predicts to fail are not aligned.  The paper has no such network: it is
 * this library's, defined below.
 *
 * Pair features (32 floats per pair (i of set A, j of set B)).  K(s) = the
 * distinct k-mers of standard letters of s with their FIRST start positions
 * p_s(x); for the c shared k-mers x: diagonal d(x) = p_i(x) - p_j(x),
 * D = li + lj - 2k + 1, bin(x) = floor(24 (d(x) + lj - k) / D), hist[0..23];
 * n_s(y) = occurrences of standard letter y.  Each feature is an integer
 * ratio num / den evaluated as the double quotient rounded to float (0 when
 * den = 0):
 *   0: c / (c + 16)            1: min(li, lj) / max(li, lj)
 *   2..25: hist[t] / c          26: sum_y |n_i(y) lj - n_j(y) li| / (2 li lj)
 *   27: li / (li + 256)         28: lj / (lj + 256)
 *   29: max_t hist[t] / c       30: c / min(|K(i)|, |K(j)|)
 *   31: (max d - min d) / D when c >= 2, else 0. */
int swgb_pair_features(swgb_ctx* ctx, const swgb_seqset* set_a, const swgb_seqset* set_b,
                       const int32_t* pairs, int64_t n_pairs, int k, float* features,
                       void* stream);
/* pairs: DEVICE int32 [n_pairs][2]; features: DEVICE float [n_pairs][32].
 * Pairs sorted by their first index share work (swgb_discover's order).
 * Synchronous on `stream`; may grow the context's scratch.
 * Errors: EINVAL, ERANGE (an index outside its set), ENOMEM, ECUDA. */

/* Network: 32 -> 64 -> 128 -> 1, ReLU, bfloat16 weights and activations,
 * float32 accumulation (x = bf16(features); a1 = bf16(relu(x W1 + b1));
 * a2 = bf16(relu(a1 W2 + b2)); logit = a2 . w3 + b3, with W1, W2 used as
 * their bfloat16 copies).  Parameters are float32, packed as W1 [32][64]
 * (row = input), b1 [64], W2 [64][128], b2 [128], w3 [128], b3 [1].
 * Training minimises the weighted mean binary cross-entropy of the logits
 * (weight pos_weight on label 1) with Adam (beta 0.9 / 0.999, eps 1e-8);
 * the gradient rounds dz2 = g3 w3 [z2 > 0] and dz1 = dz2 W2^T [z1 > 0] to
 * bfloat16 before their products. */
#define SWGB_MLP_PARAMS 10561
#define SWGB_FEATURES 32
typedef struct swgb_mlp swgb_mlp;

/* Creates a network on ctx's device with HOST parameters init[SWGB_MLP_PARAMS]
 * (the caller draws the initial values).  Errors: EINVAL, ENOMEM, ECUDA. */
int swgb_mlp_create(swgb_ctx* ctx, const float* init, swgb_mlp** out);
void swgb_mlp_destroy(swgb_mlp* mlp);
/* Replaces the parameters (HOST array) and resets the optimiser state. */
int swgb_mlp_set(swgb_mlp* mlp, const float* params);
/* Copies the parameters to HOST params[SWGB_MLP_PARAMS] (waits for the device). */
int swgb_mlp_get(swgb_mlp* mlp, float* params);
/* logits[p] for DEVICE features [n][32] into DEVICE logits [n]; asynchronous. */
int swgb_mlp_forward(swgb_mlp* mlp, const float* features, int64_t n, float* logits, void* stream);
/* Gradient of the loss over the DEVICE batch (features [n][32], labels [n]
 * of 0 / 1) into DEVICE grad [SWGB_MLP_PARAMS] and DEVICE loss [1], without
 * changing the parameters; asynchronous. */
int swgb_mlp_grad(swgb_mlp* mlp, const float* features, const float* labels, int64_t n,
                  float pos_weight, float* grad, float* loss, void* stream);
/* One pass over n samples in minibatches of `batch`: sample order[r] (a
 * DEVICE int32 permutation chosen by the caller, or NULL for 0..n-1) at
 * position r; an Adam step of learning rate lr per minibatch.  *mean_loss
 * (may be NULL) receives the mean of the minibatch losses.  Synchronous. */
int swgb_mlp_train(swgb_mlp* mlp, const float* features, const float* labels,
                   const int32_t* order, int64_t n, int64_t batch, float lr, float pos_weight,
                   float* mean_loss, void* stream);

/* The whole training loop: `epochs` passes of swgb_mlp_train, each in a
 * sample order the library draws from `seed` (a Fisher-Yates shuffle driven
 * by splitmix64, so a seed gives the same orders everywhere); pos_weight <= 0
 * means sqrt(negatives / positives) of the labels (each count at least 1).
 * losses: HOST float [epochs] receiving each epoch's mean minibatch loss, or
 * NULL.  Training is reproducible: the gradient adds the blocks' partial sums
 * in block order.  Synchronous; allocates a sample-order buffer.  Errors:
 * EINVAL, ENOMEM, ECUDA. */
int swgb_mlp_fit(swgb_mlp* mlp, const float* features, const float* labels, int64_t n, int epochs,
                 int64_t batch, float lr, float pos_weight, uint64_t seed, float* losses, void* stream);

/* The decision threshold for a target recall: the largest t such that the
 * logits >= t keep at least `recall` (0..1) of the positives of (DEVICE
 * features [n][32], DEVICE labels [n]): the k-th smallest positive logit,
 * k = floor((1 - recall) * positives); -infinity with no positive.
 * Synchronous; allocates a logits buffer.  Errors: EINVAL, ENOMEM, ECUDA. */
int swgb_mlp_calibrate(swgb_mlp* mlp, const float* features, const float* labels, int64_t n,
                       float recall, float* threshold, void* stream);

/* Keeps the pairs whose logit is >= threshold, in order: kept (DEVICE int32
 * [n_pairs][2]) receives them, kept_index (DEVICE int64 [n_pairs], or NULL)
 * their positions in `pairs`, *n_kept their number.  Synchronous. */
int swgb_select_pairs(swgb_ctx* ctx, const int32_t* pairs, const float* logits, int64_t n_pairs,
                      float threshold, int32_t* kept, int64_t* kept_index, int64_t* n_kept,
                      void* stream);

/* ---- serving: a query server over a resident reference set ----
 * The paper runs one batch job; this server answers a stream of requests
 * (batches of query sequences) against references kept on the device.  Each
 * request goes through the whole search: candidates from the resident
 * k-mer index (swgb_index_query), optionally the learned filter
 * (swgb_index_features, the network, swgb_select_pairs), exact alignment
 * (swgb_align) and identity / pass-fail (swgb_identity).
 *
 * Scheduling: `slots` worker threads, each with its own context and CUDA
 * stream.  A free worker admits the longest FIFO prefix of the waiting
 * requests that fits one batch (max_batch_queries, max_batch_residues) and
 * the device-memory budget (the reservations of the requests in flight,
 * reservation = 24 bytes per residue + candidates_per_query x 192 bytes per
 * query, stay within max_inflight_bytes; the blocked formation of the
 * overlap matrix bounds memory the same way, Sec. "Blocked 2D Sparse
 * SUMMA"), and runs it; the batches of different workers overlap on the
 * GPU.  Requests that arrive while others run are admitted as workers and
 * memory free up.  A request's results do not depend on the batch it joins
 * or on what runs beside it: every pair's computation is independent. */
typedef struct {
    int32_t slots;                 /* worker slots (batches in flight), 1..64 */
    int32_t max_batch_queries;     /* queries of one batch */
    int64_t max_batch_residues;    /* query residues of one batch */
    int64_t max_inflight_bytes;    /* budget of the in-flight reservations */
    int32_t candidates_per_query;  /* reservation model (see above) */
    int32_t min_shared;            /* common k-mers of a candidate */
    float threshold;               /* logit threshold of the filter */
    swgb_thresholds identity;      /* pass / fail thresholds */
} swgb_server_config;

#define SWGB_SERVER_STAGES 5

/* The results of one request (valid until swgb_server_release). */
typedef struct {
    int32_t status;                /* SWGB_OK or the failing call's code */
    int64_t n_pairs;               /* pairs aligned (kept by the filter) */
    int64_t n_candidates;          /* candidates before the filter */
    const int32_t* pairs;          /* [n_pairs][2]: (query index in the request, reference index), ordered */
    const int32_t* counts;         /* [n_pairs] common k-mers */
    const swgb_record* records;    /* [n_pairs] */
    const swgb_identity_record* identity;   /* [n_pairs] */
    double queue_ms;               /* submission to admission */
    double latency_ms;             /* submission to completion */
    int64_t batch_id;              /* the batch the request ran in */
    int32_t slot;                  /* the worker that ran it */
    const char* error;             /* message of a failed request ("" if none) */
    double stage_ms[SWGB_SERVER_STAGES];   /* host wall time of its batch's stages: loading the
                                              queries, candidates, filter, alignment + identity,
                                              results back */
} swgb_server_result;

/* Defaults: 3 slots, 4096 queries / 2^20 residues per batch, 4 GiB budget,
 * 256 candidates per query, min_shared 2, threshold 0, identity 3/10 and
 * coverage 7/10. */
void swgb_server_default_config(swgb_server_config* cfg);

/* Starts a server on CUDA device `device` over `refs` and its `index` (both
 * must outlive the server).  mlp_params: HOST float [SWGB_MLP_PARAMS] of a
 * trained network (copied), or NULL for no filter.  params->matrix is
 * copied.  Errors: EINVAL. */
int swgb_server_create(int device, const swgb_seqset* refs, const swgb_index* index,
                       const float* mlp_params, const swgb_params* params,
                       const swgb_server_config* cfg, swgb_server** out);
/* Stops the workers after the batches in flight and frees the server. */
void swgb_server_destroy(swgb_server* server);

/* Queues a request of n_queries HOST sequences (codes 0..23, offsets
 * n_queries + 1 entries; the data are copied) and returns its ticket.
 * Errors: EINVAL, ERANGE (decreasing offsets), EBADRES, ETOOBIG (larger than
 * one batch or than the whole budget). */
int swgb_server_submit(swgb_server* server, const uint8_t* codes, const int64_t* offsets,
                       int64_t n_queries, int64_t* ticket);
/* Waits up to timeout_ms (< 0: forever) for a request; fills *out.
 * Errors: EINVAL (unknown ticket), ETIMEDOUT. */
int swgb_server_wait(swgb_server* server, int64_t ticket, int64_t timeout_ms,
                     swgb_server_result* out);
/* Frees a finished request's results.  Errors: EINVAL. */
int swgb_server_release(swgb_server* server, int64_t ticket);
/* Most batches seen in flight at once, requests waiting, bytes reserved. */
int swgb_server_stats(swgb_server* server, int32_t* max_overlap, int64_t* pending,
                      int64_t* inflight_bytes);

/* ---- allocation-free variant ----
 * The paper has no counterpart of this call; it exists for callers that
 * cannot allocate device memory while they align -- code running inside a
 * memory pool or arena that already owns the device's memory, a framework
 * whose allocator must not be bypassed, or a service that must keep a fixed
 * footprint after start-up.  It runs the same kernels as swgb_align, but all
 * device scratch (bucketing arrays, work counters, status word, chunk-boundary
 * rows) lives in one fixed array compiled into the library, of
 * SWGB_NOALLOC_SCRATCH_BYTES; every GPU that loads the library holds that
 * array until the process exits.  It calls no cudaMalloc, cudaFree or other
 * allocating routine, and needs no context. */
#define SWGB_NOALLOC_SCRATCH_BYTES (32 << 20)
#define SWGB_NOALLOC_MAX_PAIRS (1 << 19)          /* pairs per call */
#define SWGB_NOALLOC_MAX_QUERY_LENGTH 4096        /* residues per query sequence */

/* Aligns n_pairs pairs like swgb_align, on the calling thread's current
 * device.  Every pointer is a caller-owned DEVICE pointer: q_codes/q_offsets
 * (n_q sequences, codes 0..23, offsets n_q + 1 entries), r_codes/r_offsets
 * (n_r sequences), pairs int32 [n_pairs][2], out swgb_record [n_pairs].
 * Offsets index the codes array from 0 (they are not rebased): they must be
 * non-negative and non-decreasing, and the last must not exceed the codes
 * the array holds (the library cannot see that size and does not check it).
 * params->matrix is a host pointer, as for swgb_align.  The query profile
 * always stages all 25 rows (the 24 codes and the pad), whatever letters the
 * queries use, so a batch of 20-letter queries keeps fewer DP blocks resident
 * per SM than swgb_align gives it; the records are the same.
 * The first call on a device resolves the array's device address and
 * configures the kernels; make that first call before any stream capture.
 * Every call shares the one array and it keeps the previous call's contents
 * (the call clears what must start at zero); calls that overlap on the GPU --
 * from several threads or streams at once -- race on it and must be
 * serialised by the caller.  Synchronous: returns after the stream has
 * finished the call.
 * Errors: EINVAL (bad argument or penalty), ETOOBIG (n_pairs above
 * SWGB_NOALLOC_MAX_PAIRS, a query longer than SWGB_NOALLOC_MAX_QUERY_LENGTH
 * or a reference longer than SWGB_MAX_LENGTH; nothing is launched), EBADRES
 * (a code >= 24), ERANGE (a negative or decreasing offset, or a pair index
 * out of range: that pair's record is zero), EINTERNAL, ECUDA. */
int swgb_align_noalloc(const uint8_t* q_codes, const int64_t* q_offsets, int64_t n_q,
                       const uint8_t* r_codes, const int64_t* r_offsets, int64_t n_r,
                       const int32_t* pairs, int64_t n_pairs, const swgb_params* params,
                       swgb_record* out, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* SWGB_H */
