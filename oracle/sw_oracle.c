/*
 * sw_oracle.c -- CPU oracle for local alignment with affine (Gotoh) gaps.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
 * call this file; only the tests, the package smoke check and the benchmark's
 * CPU-baseline leg use it.  It shares no code, header or table with the CUDA
 * library: its substitution table below is its own transcription.
 *
 * What it computes (the paper's alignment step, Sec. "Protein similarity
 * search pipeline" item (ii) "batch alignment of the discovered candidate
 * sequences", and Sec. "Load balancing": a Smith-Waterman variant that
 * computes the entire score matrix per candidate pair; integer scores per the
 * "Performance Attributes" table):
 *
 *   rows i = 0..lq-1 walk the query q, columns j = 0..lr-1 the reference r.
 *   A gap of length L costs  go + ge*L.
 *     E(i,j) = max(E(i,j-1) - ge, H(i,j-1) - go - ge)      (gap along r)
 *     F(i,j) = max(F(i-1,j) - ge, H(i-1,j) - go - ge)      (gap along q)
 *     H(i,j) = max(0, H(i-1,j-1) + s(q_i, r_j), E(i,j), F(i,j))
 *   with H = 0 and E = F = -infinity outside the matrix.
 *   score S = max H (0 if no cell is positive).
 *
 * The paper does not state tie-breaks or a start-finding pass; this oracle
 * uses these readings:
 *   end   (q_end, r_end): the first cell in row-major order (smallest i,
 *         then smallest j) with H = S.
 *   start (q_start, r_start): run the same local DP on the reversed prefixes
 *         q[q_end..0] and r[r_end..0]; the first cell (a, b) in row-major
 *         order with H' = S gives q_start = q_end - a, r_start = r_end - b.
 *   S = 0 gives all four coordinates = -1.
 * Every value is an int32; nothing is blocked, fused or reordered.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <pthread.h>

#define ORACLE_ALPHA 24

/* BLOSUM62 (Henikoff & Henikoff, PNAS 89:10915, 1992), integer half-bit
 * matrix as distributed by NCBI, letters in the order
 * A R N D C Q E G H I L K M F P S T W Y V B Z X *. */
static const int8_t ORACLE_BLOSUM62[ORACLE_ALPHA][ORACLE_ALPHA] = {
/*        A   R   N   D   C   Q   E   G   H   I   L   K   M   F   P   S   T   W   Y   V   B   Z   X   * */
/* A */ { 4, -1, -2, -2,  0, -1, -1,  0, -2, -1, -1, -1, -1, -2, -1,  1,  0, -3, -2,  0, -2, -1,  0, -4},
/* R */ {-1,  5,  0, -2, -3,  1,  0, -2,  0, -3, -2,  2, -1, -3, -2, -1, -1, -3, -2, -3, -1,  0, -1, -4},
/* N */ {-2,  0,  6,  1, -3,  0,  0,  0,  1, -3, -3,  0, -2, -3, -2,  1,  0, -4, -2, -3,  3,  0, -1, -4},
/* D */ {-2, -2,  1,  6, -3,  0,  2, -1, -1, -3, -4, -1, -3, -3, -1,  0, -1, -4, -3, -3,  4,  1, -1, -4},
/* C */ { 0, -3, -3, -3,  9, -3, -4, -3, -3, -1, -1, -3, -1, -2, -3, -1, -1, -2, -2, -1, -3, -3, -2, -4},
/* Q */ {-1,  1,  0,  0, -3,  5,  2, -2,  0, -3, -2,  1,  0, -3, -1,  0, -1, -2, -1, -2,  0,  3, -1, -4},
/* E */ {-1,  0,  0,  2, -4,  2,  5, -2,  0, -3, -3,  1, -2, -3, -1,  0, -1, -3, -2, -2,  1,  4, -1, -4},
/* G */ { 0, -2,  0, -1, -3, -2, -2,  6, -2, -4, -4, -2, -3, -3, -2,  0, -2, -2, -3, -3, -1, -2, -1, -4},
/* H */ {-2,  0,  1, -1, -3,  0,  0, -2,  8, -3, -3, -1, -2, -1, -2, -1, -2, -2,  2, -3,  0,  0, -1, -4},
/* I */ {-1, -3, -3, -3, -1, -3, -3, -4, -3,  4,  2, -3,  1,  0, -3, -2, -1, -3, -1,  3, -3, -3, -1, -4},
/* L */ {-1, -2, -3, -4, -1, -2, -3, -4, -3,  2,  4, -2,  2,  0, -3, -2, -1, -2, -1,  1, -4, -3, -1, -4},
/* K */ {-1,  2,  0, -1, -3,  1,  1, -2, -1, -3, -2,  5, -1, -3, -1,  0, -1, -3, -2, -2,  0,  1, -1, -4},
/* M */ {-1, -1, -2, -3, -1,  0, -2, -3, -2,  1,  2, -1,  5,  0, -2, -1, -1, -1, -1,  1, -3, -1, -1, -4},
/* F */ {-2, -3, -3, -3, -2, -3, -3, -3, -1,  0,  0, -3,  0,  6, -4, -2, -2,  1,  3, -1, -3, -3, -1, -4},
/* P */ {-1, -2, -2, -1, -3, -1, -1, -2, -2, -3, -3, -1, -2, -4,  7, -1, -1, -4, -3, -2, -2, -1, -2, -4},
/* S */ { 1, -1,  1,  0, -1,  0,  0,  0, -1, -2, -2,  0, -1, -2, -1,  4,  1, -3, -2, -2,  0,  0,  0, -4},
/* T */ { 0, -1,  0, -1, -1, -1, -1, -2, -2, -1, -1, -1, -1, -2, -1,  1,  5, -2, -2,  0, -1, -1,  0, -4},
/* W */ {-3, -3, -4, -4, -2, -2, -3, -2, -2, -3, -2, -3, -1,  1, -4, -3, -2, 11,  2, -3, -4, -3, -2, -4},
/* Y */ {-2, -2, -2, -3, -2, -1, -2, -3,  2, -1, -1, -2, -1,  3, -3, -2, -2,  2,  7, -1, -3, -2, -1, -4},
/* V */ { 0, -3, -3, -3, -1, -2, -2, -3, -3,  3,  1, -2,  1, -1, -2, -2,  0, -3, -1,  4, -3, -2, -1, -4},
/* B */ {-2, -1,  3,  4, -3,  0,  1, -1,  0, -3, -4,  0, -3, -3, -2,  0, -1, -4, -3, -3,  4,  1, -1, -4},
/* Z */ {-1,  0,  0,  1, -3,  3,  4, -2,  0, -3, -3,  1, -1, -3, -1,  0, -1, -3, -2, -2,  1,  4, -1, -4},
/* X */ { 0, -1, -1, -1, -2, -1, -1, -1, -1, -1, -1, -1, -1, -1, -2,  0,  0, -2, -1, -1, -1, -1, -1, -4},
/* * */ {-4, -4, -4, -4, -4, -4, -4, -4, -4, -4, -4, -4, -4, -4, -4, -4, -4, -4, -4, -4, -4, -4, -4,  1},
};

typedef struct {
    int32_t score, q_start, q_end, r_start, r_end;
} oracle_record;

/* Copies the oracle's own BLOSUM62 (24 x 24, row = query letter). */
void oracle_blosum62(int8_t* out)
{
    memcpy(out, ORACLE_BLOSUM62, sizeof(ORACLE_BLOSUM62));
}

static int32_t max2(int32_t a, int32_t b) { return a > b ? a : b; }

/* "Minus infinity" for E and F: low enough that subtracting gap costs many
 * times cannot wrap, and any real candidate beats it. */
#define ORACLE_NEG_INF (INT32_MIN / 4)

/*
 * Local Gotoh DP of a (rows) against b (columns), the recurrence in the file
 * header written out cell by cell.  Returns S and the row-major-first cell
 * (bi, bj) with H = S, or (-1, -1) when S = 0.  Returns -1 on allocation
 * failure (then *S is untouched).
 */
static int gotoh_local(const uint8_t* a, int64_t la, const uint8_t* b, int64_t lb,
                       const int8_t* mat, int32_t go, int32_t ge,
                       int32_t* S, int64_t* bi, int64_t* bj)
{
    int32_t* Hprev = (int32_t*)malloc(sizeof(int32_t) * (size_t)(lb + 1));
    int32_t* Fprev = (int32_t*)malloc(sizeof(int32_t) * (size_t)(lb + 1));
    int32_t* Hcur = (int32_t*)malloc(sizeof(int32_t) * (size_t)(lb + 1));
    int32_t* Fcur = (int32_t*)malloc(sizeof(int32_t) * (size_t)(lb + 1));
    if (!Hprev || !Fprev || !Hcur || !Fcur) {
        free(Hprev); free(Fprev); free(Hcur); free(Fcur);
        return -1;
    }
    /* row i = -1 (DP row 0): H = 0, F = -inf */
    for (int64_t j = 0; j <= lb; ++j) { Hprev[j] = 0; Fprev[j] = ORACLE_NEG_INF; }

    int32_t best = 0;
    int64_t best_i = -1, best_j = -1;
    for (int64_t i = 1; i <= la; ++i) {
        int32_t E = ORACLE_NEG_INF;     /* E(i, 0) */
        Hcur[0] = 0;                    /* H(i, 0) */
        Fcur[0] = ORACLE_NEG_INF;
        for (int64_t j = 1; j <= lb; ++j) {
            E = max2(E - ge, Hcur[j - 1] - go - ge);
            int32_t F = max2(Fprev[j] - ge, Hprev[j] - go - ge);
            int32_t D = Hprev[j - 1] + (int32_t)mat[a[i - 1] * ORACLE_ALPHA + b[j - 1]];
            int32_t H = max2(max2(0, D), max2(E, F));
            Hcur[j] = H;
            Fcur[j] = F;
            if (H > best) {          /* strict: keeps the row-major-first cell */
                best = H;
                best_i = i - 1;
                best_j = j - 1;
            }
        }
        int32_t* t;
        t = Hprev; Hprev = Hcur; Hcur = t;
        t = Fprev; Fprev = Fcur; Fcur = t;
    }
    free(Hprev); free(Fprev); free(Hcur); free(Fcur);
    *S = best;
    *bi = best_i;
    *bj = best_j;
    return 0;
}

/*
 * One pair: forward pass for (S, q_end, r_end), reverse pass for
 * (q_start, r_start).  Residues are codes 0..23.  Returns 0, or -1 on
 * allocation failure, or -2 if the reverse pass does not reach S (which the
 * reading in the header rules out; the check guards the oracle itself).
 */
int oracle_align_pair(const uint8_t* q, int64_t lq, const uint8_t* r, int64_t lr,
                      const int8_t* mat, int32_t go, int32_t ge, oracle_record* out)
{
    int32_t S;
    int64_t qe, re;
    if (gotoh_local(q, lq, r, lr, mat, go, ge, &S, &qe, &re) != 0) return -1;
    if (S == 0) {
        out->score = 0;
        out->q_start = out->q_end = out->r_start = out->r_end = -1;
        return 0;
    }
    uint8_t* qrev = (uint8_t*)malloc((size_t)(qe + 1));
    uint8_t* rrev = (uint8_t*)malloc((size_t)(re + 1));
    if (!qrev || !rrev) { free(qrev); free(rrev); return -1; }
    for (int64_t k = 0; k <= qe; ++k) qrev[k] = q[qe - k];
    for (int64_t k = 0; k <= re; ++k) rrev[k] = r[re - k];
    int32_t S2;
    int64_t a, b;
    int rc = gotoh_local(qrev, qe + 1, rrev, re + 1, mat, go, ge, &S2, &a, &b);
    free(qrev); free(rrev);
    if (rc != 0) return -1;
    if (S2 != S) return -2;
    out->score = S;
    out->q_end = (int32_t)qe;
    out->r_end = (int32_t)re;
    out->q_start = (int32_t)(qe - a);
    out->r_start = (int32_t)(re - b);
    return 0;
}

/* Forward pass only (score and end cell), for timing the forward leg. */
int oracle_forward_pair(const uint8_t* q, int64_t lq, const uint8_t* r, int64_t lr,
                        const int8_t* mat, int32_t go, int32_t ge,
                        int32_t* score, int64_t* q_end, int64_t* r_end)
{
    return gotoh_local(q, lq, r, lr, mat, go, ge, score, q_end, r_end);
}

/* ---- batch over pairs: one worker thread per core, pairs handed out by an
 * atomic counter; each pair is the plain per-pair call above. ---- */
typedef struct {
    const uint8_t* qres; const int64_t* qoff;
    const uint8_t* rres; const int64_t* roff;
    const int32_t* pairs; int64_t n_pairs;
    const int8_t* mat; int32_t go, ge;
    oracle_record* out;
    int64_t next;   /* shared counter */
    int status;     /* first error seen */
} batch_job;

static void* batch_worker(void* arg)
{
    batch_job* job = (batch_job*)arg;
    for (;;) {
        int64_t p = __atomic_fetch_add(&job->next, 1, __ATOMIC_RELAXED);
        if (p >= job->n_pairs) break;
        int32_t qi = job->pairs[2 * p], ri = job->pairs[2 * p + 1];
        const uint8_t* q = job->qres + job->qoff[qi];
        const uint8_t* r = job->rres + job->roff[ri];
        int64_t lq = job->qoff[qi + 1] - job->qoff[qi];
        int64_t lr = job->roff[ri + 1] - job->roff[ri];
        int rc = oracle_align_pair(q, lq, r, lr, job->mat, job->go, job->ge, &job->out[p]);
        if (rc != 0) {
            int expected = 0;
            __atomic_compare_exchange_n(&job->status, &expected, rc, 0,
                                        __ATOMIC_RELAXED, __ATOMIC_RELAXED);
        }
    }
    return NULL;
}

/*
 * Aligns pairs[p] = (query index, reference index) for p < n_pairs.
 * Sequences are concatenated codes with offsets (n + 1 entries).  Index
 * ranges are the caller's responsibility.  n_threads <= 1 runs inline.
 * Returns 0 or the first per-pair error.
 */
int oracle_align_batch(const uint8_t* qres, const int64_t* qoff,
                       const uint8_t* rres, const int64_t* roff,
                       const int32_t* pairs, int64_t n_pairs,
                       const int8_t* mat, int32_t go, int32_t ge,
                       oracle_record* out, int n_threads)
{
    batch_job job = {qres, qoff, rres, roff, pairs, n_pairs, mat, go, ge, out, 0, 0};
    if (n_threads <= 1) {
        batch_worker(&job);
        return job.status;
    }
    pthread_t* th = (pthread_t*)malloc(sizeof(pthread_t) * (size_t)n_threads);
    if (!th) return -1;
    int started = 0;
    for (int t = 0; t < n_threads; ++t) {
        if (pthread_create(&th[t], NULL, batch_worker, &job) != 0) break;
        ++started;
    }
    if (started == 0) batch_worker(&job);
    for (int t = 0; t < started; ++t) pthread_join(th[t], NULL);
    free(th);
    return job.status;
}
