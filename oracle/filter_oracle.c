/*
 * filter_oracle.c -- CPU oracle for the 32 features of a candidate pair that
 * the learned candidate filter reads.  TEST INFRASTRUCTURE ONLY: the product
 * path never links or calls it, and it shares no code with it.
 *
 * The paper prunes candidates only by their common k-mer count (threshold 2,
 * program-parameters table) and notes that few candidates end up in the
 * similarity graph (Sec. "Blocked 2D Sparse SUMMA"); the filter adds features
 * of the shared k-mers' diagonals, lengths and composition.  Definitions:
 *
 *   K(s)    distinct k-mers of s made of standard letters (codes 0..19), each
 *           with its FIRST start position p_s(x);
 *   shared  S = K(a) intersect K(b), c = |S|;
 *   d(x)    = p_a(x) - p_b(x), the diagonal of a shared k-mer, in
 *             [-(lb - k), la - k];
 *   D       = la + lb - 2k + 1 (the number of such diagonals);
 *   bin(x)  = floor(24 (d(x) + lb - k) / D), 0..23;  hist[t] = |{x: bin = t}|;
 *   n_s(y)  = occurrences of standard letter y in s.
 * Every feature is a ratio of two integers num / den, evaluated as the double
 * quotient rounded to float (0 where den is 0):
 *   f0      c / (c + 16)
 *   f1      min(la, lb) / max(la, lb)
 *   f2+t    hist[t] / c                                   t = 0..23
 *   f26     sum_y |n_a(y) lb - n_b(y) la| / (2 la lb)     composition distance
 *   f27     la / (la + 256)
 *   f28     lb / (lb + 256)
 *   f29     max_t hist[t] / c
 *   f30     c / min(|K(a)|, |K(b)|)
 *   f31     (max d - min d) / D                           (0 when c < 2)
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define STD_LETTERS 20
#define NBINS 24
#define NFEAT 32

typedef struct {
    uint32_t kmer;
    int64_t pos;
} entry;

static int cmp_entry(const void* x, const void* y)
{
    const entry* a = (const entry*)x;
    const entry* b = (const entry*)y;
    if (a->kmer != b->kmer) return a->kmer < b->kmer ? -1 : 1;
    return a->pos < b->pos ? -1 : (a->pos > b->pos);
}

/* K(s) with first positions, sorted by k-mer; returns |K(s)| (out holds n). */
static int64_t kmer_set_pos(const uint8_t* s, int64_t n, int k, entry* out)
{
    int64_t m = 0;
    for (int64_t p = 0; p + k <= n; ++p) {
        uint32_t v = 0;
        int ok = 1;
        for (int t = 0; t < k; ++t) {
            if (s[p + t] >= STD_LETTERS) { ok = 0; break; }
            v = v * STD_LETTERS + s[p + t];
        }
        if (ok) { out[m].kmer = v; out[m].pos = p; ++m; }
    }
    qsort(out, (size_t)m, sizeof(entry), cmp_entry);
    int64_t u = 0;
    for (int64_t x = 0; x < m; ++x)      /* the first of equal k-mers has the smallest position */
        if (u == 0 || out[u - 1].kmer != out[x].kmer) out[u++] = out[x];
    return u;
}

static float ratio(int64_t num, int64_t den)
{
    if (den == 0) return 0.0f;
    return (float)((double)num / (double)den);
}

/* The 32 features of the pair (a, b); returns 0, or -1 on bad k / memory. */
int oracle_pair_features(const uint8_t* a, int64_t la, const uint8_t* b, int64_t lb, int k,
                         float* out)
{
    if (k < 1 || k > 6) return -1;
    entry* ka = (entry*)malloc(sizeof(entry) * (size_t)(la + 1));
    entry* kb = (entry*)malloc(sizeof(entry) * (size_t)(lb + 1));
    if (!ka || !kb) { free(ka); free(kb); return -1; }
    const int64_t na = kmer_set_pos(a, la, k, ka), nb = kmer_set_pos(b, lb, k, kb);
    int64_t hist[NBINS] = {0};
    int64_t c = 0, dmin = 0, dmax = 0;
    const int64_t D = la + lb - 2 * (int64_t)k + 1;
    int64_t x = 0, y = 0;
    while (x < na && y < nb) {
        if (ka[x].kmer < kb[y].kmer) { ++x; continue; }
        if (ka[x].kmer > kb[y].kmer) { ++y; continue; }
        const int64_t d = ka[x].pos - kb[y].pos;
        hist[(NBINS * (d + lb - k)) / D] += 1;
        if (c == 0 || d < dmin) dmin = d;
        if (c == 0 || d > dmax) dmax = d;
        ++c;
        ++x;
        ++y;
    }
    int64_t na_c[STD_LETTERS] = {0}, nb_c[STD_LETTERS] = {0};
    for (int64_t p = 0; p < la; ++p) if (a[p] < STD_LETTERS) na_c[a[p]] += 1;
    for (int64_t p = 0; p < lb; ++p) if (b[p] < STD_LETTERS) nb_c[b[p]] += 1;
    int64_t comp = 0;
    for (int t = 0; t < STD_LETTERS; ++t) {
        const int64_t v = na_c[t] * lb - nb_c[t] * la;
        comp += v < 0 ? -v : v;
    }
    int64_t hmax = 0;
    for (int t = 0; t < NBINS; ++t) if (hist[t] > hmax) hmax = hist[t];
    out[0] = ratio(c, c + 16);
    out[1] = ratio(la < lb ? la : lb, la < lb ? lb : la);
    for (int t = 0; t < NBINS; ++t) out[2 + t] = ratio(hist[t], c);
    out[26] = ratio(comp, 2 * la * lb);
    out[27] = ratio(la, la + 256);
    out[28] = ratio(lb, lb + 256);
    out[29] = ratio(hmax, c);
    out[30] = ratio(c, na < nb ? na : nb);
    out[31] = c >= 2 ? ratio(dmax - dmin, D) : 0.0f;
    free(ka);
    free(kb);
    return 0;
}

/* Features of pairs[p] = (index into set A, index into set B) for p < n. */
int oracle_pair_features_batch(const uint8_t* res_a, const int64_t* off_a, const uint8_t* res_b,
                               const int64_t* off_b, const int32_t* pairs, int64_t n, int k,
                               float* out)
{
    for (int64_t p = 0; p < n; ++p) {
        const int32_t i = pairs[2 * p], j = pairs[2 * p + 1];
        const int rc = oracle_pair_features(res_a + off_a[i], off_a[i + 1] - off_a[i],
                                            res_b + off_b[j], off_b[j + 1] - off_b[j], k,
                                            out + (size_t)p * NFEAT);
        if (rc) return rc;
    }
    return 0;
}
