/*
 * discovery_oracle.c -- CPU oracle for candidate discovery by shared k-mers
 * and for the identity of an alignment.  TEST INFRASTRUCTURE ONLY: the
 * product path never links or calls it, and it shares no code with it.
 *
 * Shared k-mers (Sec. "Protein similarity search pipeline" and "Load
 * balancing techniques": the overlap matrix C = A A^T of the sequence-by-k-mer
 * matrix A holds, per pair of sequences, their common k-mer count; pairs with
 * at least the common-k-mer threshold, 2 in the production parameters table,
 * are aligned; the matrix is symmetric, so only i < j is kept):
 *   K(s) = the set of distinct k-mers of s, a k-mer being k consecutive codes
 *          all below 20 (the standard letters; a k-mer touching B, Z, X or *
 *          is not formed), valued as a base-20 number, first letter most
 *          significant;
 *   C(i, j) = |K(s_i) intersect K(s_j)|.
 * The oracle keeps each K(s) as a sorted array and counts an intersection by
 * merging two of them.
 *
 * Identity and coverage (the thresholds 0.30 and 0.70 of the production
 * parameters table; the paper defines neither measure):
 *   the global affine alignment of the span q[qs..qe] x r[rs..re] of a local
 *   alignment record (its optimum is the record's score) is traced back from
 *   (qe, re): from H prefer the diagonal, then the gap in the reference (a
 *   query residue against a gap, from F), then the gap in the query (from E);
 *   inside a gap prefer the gap's opening over its extension.  identity =
 *   identical columns / columns; coverage = min((qe-qs+1)/lq, (re-rs+1)/lr).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <pthread.h>

#define STD_LETTERS 20

static int cmp_u32(const void* a, const void* b)
{
    uint32_t x = *(const uint32_t*)a, y = *(const uint32_t*)b;
    return x < y ? -1 : x > y;
}

/* K(s) into out (capacity n), sorted and distinct; returns |K(s)|. */
static int64_t kmer_set(const uint8_t* s, int64_t n, int k, uint32_t* out)
{
    int64_t m = 0;
    for (int64_t p = 0; p + k <= n; ++p) {
        uint32_t v = 0;
        int ok = 1;
        for (int t = 0; t < k; ++t) {
            if (s[p + t] >= STD_LETTERS) { ok = 0; break; }
            v = v * STD_LETTERS + s[p + t];
        }
        if (ok) out[m++] = v;
    }
    qsort(out, (size_t)m, sizeof(uint32_t), cmp_u32);
    int64_t u = 0;
    for (int64_t x = 0; x < m; ++x)
        if (u == 0 || out[u - 1] != out[x]) out[u++] = out[x];
    return u;
}

static int64_t merge_count(const uint32_t* a, int64_t na, const uint32_t* b, int64_t nb)
{
    int64_t x = 0, y = 0, c = 0;
    while (x < na && y < nb) {
        if (a[x] < b[y]) ++x;
        else if (a[x] > b[y]) ++y;
        else { ++c; ++x; ++y; }
    }
    return c;
}

int64_t oracle_shared_kmers(const uint8_t* a, int64_t la, const uint8_t* b, int64_t lb, int k)
{
    if (k < 1 || k > 6) return -1;
    uint32_t* ka = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)(la + 1));
    uint32_t* kb = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)(lb + 1));
    if (!ka || !kb) { free(ka); free(kb); return -1; }
    int64_t na = kmer_set(a, la, k, ka), nb = kmer_set(b, lb, k, kb);
    int64_t c = merge_count(ka, na, kb, nb);
    free(ka);
    free(kb);
    return c;
}

/* K(s) of every sequence of a set, kept for repeated queries. */
typedef struct {
    int64_t n;
    int64_t* start;   /* [n + 1] into sets */
    uint32_t* sets;
} kmer_index;

void* oracle_kmer_index(const uint8_t* res, const int64_t* off, int64_t n, int k)
{
    if (k < 1 || k > 6 || n < 0) return NULL;
    kmer_index* ix = (kmer_index*)calloc(1, sizeof(kmer_index));
    if (!ix) return NULL;
    ix->n = n;
    ix->start = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n + 1));
    ix->sets = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)(off[n] - off[0] + 1));
    if (!ix->start || !ix->sets) { free(ix->start); free(ix->sets); free(ix); return NULL; }
    int64_t m = 0;
    for (int64_t i = 0; i < n; ++i) {
        ix->start[i] = m;
        m += kmer_set(res + off[i], off[i + 1] - off[i], k, ix->sets + m);
    }
    ix->start[n] = m;
    return ix;
}

void oracle_kmer_index_free(void* h)
{
    kmer_index* ix = (kmer_index*)h;
    if (!ix) return;
    free(ix->start);
    free(ix->sets);
    free(ix);
}

/* Every j != i with C(i, j) >= min_shared, ascending; returns how many (the
 * first cap are written), or -1. */
int64_t oracle_candidates_of(const void* h, int64_t i, int min_shared, int32_t* js,
                             int32_t* counts, int64_t cap)
{
    const kmer_index* ix = (const kmer_index*)h;
    if (!ix || i < 0 || i >= ix->n) return -1;
    const uint32_t* a = ix->sets + ix->start[i];
    int64_t na = ix->start[i + 1] - ix->start[i], found = 0;
    for (int64_t j = 0; j < ix->n; ++j) {
        if (j == i) continue;
        int64_t c = merge_count(a, na, ix->sets + ix->start[j], ix->start[j + 1] - ix->start[j]);
        if (c >= min_shared) {
            if (found < cap) { js[found] = (int32_t)j; counts[found] = (int32_t)c; }
            ++found;
        }
    }
    return found;
}

typedef struct {
    const kmer_index* ix;
    int min_shared;
    int64_t i0, i1;
    int64_t n_out, cap;
    int32_t* pairs;
    int32_t* counts;
} all_job;

static void* all_worker(void* arg)
{
    all_job* J = (all_job*)arg;
    const kmer_index* ix = J->ix;
    for (int64_t i = J->i0; i < J->i1; ++i) {
        const uint32_t* a = ix->sets + ix->start[i];
        int64_t na = ix->start[i + 1] - ix->start[i];
        for (int64_t j = i + 1; j < ix->n; ++j) {
            int64_t c = merge_count(a, na, ix->sets + ix->start[j], ix->start[j + 1] - ix->start[j]);
            if (c >= J->min_shared) {
                if (J->n_out < J->cap) {
                    J->pairs[2 * J->n_out] = (int32_t)i;
                    J->pairs[2 * J->n_out + 1] = (int32_t)j;
                    J->counts[J->n_out] = (int32_t)c;
                }
                ++J->n_out;
            }
        }
    }
    return NULL;
}

/* Every pair i < j with C(i, j) >= min_shared, ordered by (i, j); returns
 * how many (the first cap are written), or -1.  Threads split the rows i. */
int64_t oracle_all_candidates(const void* h, int min_shared, int32_t* pairs, int32_t* counts,
                              int64_t cap, int n_threads)
{
    const kmer_index* ix = (const kmer_index*)h;
    if (!ix) return -1;
    if (n_threads < 1) n_threads = 1;
    if (n_threads > 64) n_threads = 64;
    all_job jobs[64];
    pthread_t th[64];
    int started[64];
    /* rows split by equal numbers of later sequences (work ~ n - i) */
    int64_t n = ix->n;
    double total = (double)n * (double)(n - 1) / 2.0;
    int64_t i = 0;
    for (int t = 0; t < n_threads; ++t) {
        double target = total * (t + 1) / n_threads, acc = (double)i * (2.0 * n - i - 1) / 2.0;
        int64_t e = i;
        while (e < n && acc < target) { acc += (double)(n - e - 1); ++e; }
        if (t == n_threads - 1) e = n;
        jobs[t].ix = ix; jobs[t].min_shared = min_shared;
        jobs[t].i0 = i; jobs[t].i1 = e; jobs[t].n_out = 0; jobs[t].cap = cap;
        jobs[t].pairs = (int32_t*)malloc(sizeof(int32_t) * 2 * (size_t)(cap > 0 ? cap : 1));
        jobs[t].counts = (int32_t*)malloc(sizeof(int32_t) * (size_t)(cap > 0 ? cap : 1));
        i = e;
    }
    for (int t = 0; t < n_threads; ++t) {
        started[t] = pthread_create(&th[t], NULL, all_worker, &jobs[t]) == 0;
        if (!started[t]) all_worker(&jobs[t]);
    }
    int64_t total_out = 0;
    for (int t = 0; t < n_threads; ++t) {
        if (started[t]) pthread_join(th[t], NULL);
    }
    int bad = 0;
    for (int t = 0; t < n_threads; ++t) {
        if (!jobs[t].pairs || !jobs[t].counts) bad = 1;
        int64_t m = jobs[t].n_out < jobs[t].cap ? jobs[t].n_out : jobs[t].cap;
        for (int64_t x = 0; x < m && !bad; ++x) {
            if (total_out + x < cap) {
                pairs[2 * (total_out + x)] = jobs[t].pairs[2 * x];
                pairs[2 * (total_out + x) + 1] = jobs[t].pairs[2 * x + 1];
                counts[total_out + x] = jobs[t].counts[x];
            }
        }
        total_out += jobs[t].n_out;
        free(jobs[t].pairs);
        free(jobs[t].counts);
    }
    return bad ? -1 : total_out;
}

/* ---- identity of a local alignment record ------------------------------- */

#define NEG_INF (-(1 << 28))

static int32_t imax(int32_t a, int32_t b) { return a > b ? a : b; }

/*
 * rec = {score, q_start, q_end, r_start, r_end}.  Writes the identical
 * columns and all columns of the traced alignment.  Returns 0; 1 for a zero
 * score (both outputs 0); -1 on bad arguments or memory; -2 when the span's
 * global optimum differs from the record's score.
 */
int oracle_span_identity(const uint8_t* q, int64_t lq, const uint8_t* r, int64_t lr,
                         const int32_t* rec, const int8_t* mat, int32_t go, int32_t ge,
                         int32_t* matches, int32_t* columns)
{
    *matches = 0;
    *columns = 0;
    if (rec[0] == 0) return 1;
    const int64_t qs = rec[1], qe = rec[2], rs = rec[3], re = rec[4];
    if (qs < 0 || qe < qs || qe >= lq || rs < 0 || re < rs || re >= lr) return -1;
    const int64_t n = qe - qs + 1, m = re - rs + 1;
    const int32_t oe = go + ge;
    /* matrices over (n + 1) x (m + 1): index 0 is the border before the span */
    const size_t cells = (size_t)(n + 1) * (size_t)(m + 1);
    int32_t* H = (int32_t*)malloc(sizeof(int32_t) * cells);
    int32_t* E = (int32_t*)malloc(sizeof(int32_t) * cells);
    int32_t* F = (int32_t*)malloc(sizeof(int32_t) * cells);
    if (!H || !E || !F) { free(H); free(E); free(F); return -1; }
#define AT(M, a, b) M[(size_t)(a) * (size_t)(m + 1) + (size_t)(b)]
    AT(H, 0, 0) = 0;
    AT(E, 0, 0) = NEG_INF;
    AT(F, 0, 0) = NEG_INF;
    for (int64_t b = 1; b <= m; ++b) {
        AT(E, 0, b) = -(oe + ge * (int32_t)(b - 1));
        AT(F, 0, b) = NEG_INF;
        AT(H, 0, b) = AT(E, 0, b);
    }
    for (int64_t a = 1; a <= n; ++a) {
        AT(F, a, 0) = -(oe + ge * (int32_t)(a - 1));
        AT(E, a, 0) = NEG_INF;
        AT(H, a, 0) = AT(F, a, 0);
        for (int64_t b = 1; b <= m; ++b) {
            AT(E, a, b) = imax(AT(E, a, b - 1) - ge, AT(H, a, b - 1) - oe);
            AT(F, a, b) = imax(AT(F, a - 1, b) - ge, AT(H, a - 1, b) - oe);
            const int32_t d = AT(H, a - 1, b - 1) + mat[q[qs + a - 1] * 24 + r[rs + b - 1]];
            AT(H, a, b) = imax(d, imax(AT(E, a, b), AT(F, a, b)));
        }
    }
    int rc = 0;
    if (AT(H, n, m) != rec[0]) {
        rc = -2;
    } else {
        int64_t a = n, b = m;
        int state = 0;   /* 0 = H, 1 = F (query residue vs gap), 2 = E (gap vs reference residue) */
        int32_t mt = 0, cols = 0;
        while (a > 0 || b > 0) {
            if (state == 0) {
                if (a > 0 && b > 0 &&
                    AT(H, a, b) == AT(H, a - 1, b - 1) + mat[q[qs + a - 1] * 24 + r[rs + b - 1]]) {
                    mt += q[qs + a - 1] == r[rs + b - 1];
                    ++cols;
                    --a;
                    --b;
                } else if (a > 0 && AT(H, a, b) == AT(F, a, b)) {
                    state = 1;
                } else {
                    state = 2;
                }
            } else if (state == 1) {
                ++cols;
                const int open = AT(F, a, b) == AT(H, a - 1, b) - oe;
                --a;
                state = open ? 0 : 1;
            } else {
                ++cols;
                const int open = AT(E, a, b) == AT(H, a, b - 1) - oe;
                --b;
                state = open ? 0 : 2;
            }
        }
        *matches = mt;
        *columns = cols;
    }
#undef AT
    free(H);
    free(E);
    free(F);
    return rc;
}
