/*
 * workload_gen.c -- seeded synthetic protein-pair workloads.
 *
 * Holds no alignment arithmetic: it only draws sequences.  Both the CUDA
 * path's tests/benchmark and the CPU oracle consume what it writes.
 *
 * Every pair p owns an independent random stream: splitmix64 (Steele, Lea &
 * Flood, OOPSLA 2014) started from seed ^ mix(p), so any pair can be drawn
 * alone and pairs can be drawn in parallel with identical results.
 *
 * Per pair:
 *   query length  ~ uniform[lmin, lmax]  or  round(median * exp(sigma * N(0,1)))
 *                   clipped to [lmin, lmax];
 *   query residues ~ background table (20 standard letters);
 *   homologous pair (p < n_homologous): reference = mutate(query), where each
 *     query position, in order, draws u:
 *       u < indel_rate                      -> indel event: insertion or deletion
 *                                              (one fair bit), length L >= 1
 *                                              geometric with mean indel_mean;
 *                                              insertion emits L background
 *                                              residues then the position itself,
 *                                              deletion drops L positions starting
 *                                              here;
 *       u < indel_rate + subst_rate         -> substitution a -> b != a from the
 *                                              per-letter table (weights chosen by
 *                                              the caller);
 *       otherwise                           -> the residue is copied.
 *   unrelated pair: reference drawn like a query, independently.
 * A family set (wl_family_*) is one sequence set: families of copies, each
 * copy = mutate(the family's root).
 * The 16-bit sampling tables (background, substitution) are built by the
 * caller; this file only indexes them.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <pthread.h>

typedef struct {
    int64_t n_pairs;
    int64_t n_homologous;
    uint64_t seed;
    int32_t length_model;   /* 0 = uniform, 1 = log-normal */
    int32_t lmin, lmax;
    double median, sigma;
    double subst_rate, indel_rate, indel_mean;
} wl_params;

typedef struct {
    uint64_t s;
} wl_rng;

static uint64_t wl_next(wl_rng* r)
{
    uint64_t z = (r->s += 0x9E3779B97F4A7C15ULL);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* uniform in (0, 1) */
static double wl_unit(wl_rng* r)
{
    return ((double)(wl_next(r) >> 11) + 0.5) * (1.0 / 9007199254740992.0);
}

static void wl_seed(wl_rng* r, uint64_t seed, int64_t p)
{
    r->s = seed;
    uint64_t k = (uint64_t)p * 0xD1B54A32D192ED03ULL + 0x8CB92BA72F3D8DD7ULL;
    r->s ^= k;
    (void)wl_next(r);
}

static int32_t wl_length(wl_rng* r, const wl_params* P)
{
    if (P->length_model == 0) {
        uint64_t span = (uint64_t)(P->lmax - P->lmin + 1);
        return P->lmin + (int32_t)(wl_next(r) % span);
    }
    /* Box-Muller: one standard normal from two uniforms */
    double u1 = wl_unit(r), u2 = wl_unit(r);
    double z = sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2);
    double L = floor(P->median * exp(P->sigma * z) + 0.5);
    if (L < P->lmin) L = P->lmin;
    if (L > P->lmax) L = P->lmax;
    return (int32_t)L;
}

static uint8_t wl_background(wl_rng* r, const uint8_t* bg)
{
    return bg[wl_next(r) >> 48];
}

/* mutate(q) as described above, drawing from r; writes the residues to rbuf
 * when it is not NULL and returns the length. */
static int64_t wl_mutate(wl_rng* rng, const uint8_t* q, int32_t lq, const wl_params* P,
                         const uint8_t* bg, const uint8_t* sub, uint8_t* rbuf)
{
    int64_t lr = 0;
    double p_geo = 1.0 / P->indel_mean;   /* success probability */
    double log_fail = log(1.0 - p_geo);
    int32_t i = 0;
    while (i < lq) {
        double u = wl_unit(rng);
        if (u < P->indel_rate) {
            int insertion = (int)(wl_next(rng) >> 63);
            int64_t L = 1;
            if (p_geo < 1.0) L = 1 + (int64_t)floor(log(wl_unit(rng)) / log_fail);
            if (insertion) {
                for (int64_t k = 0; k < L; ++k) {
                    uint8_t c = wl_background(rng, bg);
                    if (rbuf) rbuf[lr] = c;
                    ++lr;
                }
                if (rbuf) rbuf[lr] = q[i];
                ++lr;
                ++i;
            } else {
                i += (int32_t)(L < (int64_t)(lq - i) ? L : (int64_t)(lq - i));
            }
        } else if (u < P->indel_rate + P->subst_rate) {
            uint8_t b = sub[(size_t)q[i] * 65536u + (wl_next(rng) >> 48)];
            if (rbuf) rbuf[lr] = b;
            ++lr;
            ++i;
        } else {
            if (rbuf) rbuf[lr] = q[i];
            ++lr;
            ++i;
        }
    }
    return lr;
}

/* Draws pair p.  Buffers may be NULL (lengths only); otherwise they must hold
 * the lengths a previous call reported. */
static void wl_pair(int64_t p, const wl_params* P, const uint8_t* bg, const uint8_t* sub,
                    uint8_t* qbuf, uint8_t* rbuf, int64_t* lq_out, int64_t* lr_out,
                    uint8_t* scratch)
{
    wl_rng rng;
    wl_seed(&rng, P->seed, p);
    int32_t lq = wl_length(&rng, P);
    /* the query is always materialised (into qbuf or scratch): a homologous
     * reference is derived from it */
    uint8_t* q = qbuf ? qbuf : scratch;
    for (int32_t i = 0; i < lq; ++i) q[i] = wl_background(&rng, bg);
    int64_t lr = 0;
    if (p < P->n_homologous) {
        lr = wl_mutate(&rng, q, lq, P, bg, sub, rbuf);
    } else {
        lr = wl_length(&rng, P);
        for (int64_t j = 0; j < lr; ++j) {
            uint8_t c = wl_background(&rng, bg);
            if (rbuf) rbuf[j] = c;
        }
    }
    *lq_out = lq;
    *lr_out = lr;
}

typedef struct {
    const wl_params* P;
    const uint8_t* bg;
    const uint8_t* sub;
    int64_t* q_len;          /* pass 1 */
    int64_t* r_len;
    const int64_t* q_off;    /* pass 2 */
    const int64_t* r_off;
    uint8_t* q_res;
    uint8_t* r_res;
    int64_t begin, end;
    int status;
} wl_job;

static void* wl_worker(void* arg)
{
    wl_job* J = (wl_job*)arg;
    uint8_t* scratch = (uint8_t*)malloc((size_t)J->P->lmax + 1);
    if (!scratch) { J->status = -1; return NULL; }
    for (int64_t p = J->begin; p < J->end; ++p) {
        int64_t lq, lr;
        if (J->q_res) {
            wl_pair(p, J->P, J->bg, J->sub, J->q_res + J->q_off[p], J->r_res + J->r_off[p],
                    &lq, &lr, scratch);
            if (lq != J->q_off[p + 1] - J->q_off[p] || lr != J->r_off[p + 1] - J->r_off[p]) {
                J->status = -2;
                break;
            }
        } else {
            wl_pair(p, J->P, J->bg, J->sub, NULL, NULL, &lq, &lr, scratch);
            J->q_len[p] = lq;
            J->r_len[p] = lr;
        }
    }
    free(scratch);
    return NULL;
}

static int wl_run(wl_job* proto, int n_threads)
{
    int64_t n = proto->P->n_pairs;
    if (n_threads < 1) n_threads = 1;
    if (n_threads > 256) n_threads = 256;
    wl_job jobs[256];
    pthread_t th[256];
    int started[256];
    for (int t = 0; t < n_threads; ++t) {
        jobs[t] = *proto;
        jobs[t].begin = n * t / n_threads;
        jobs[t].end = n * (t + 1) / n_threads;
        jobs[t].status = 0;
        started[t] = pthread_create(&th[t], NULL, wl_worker, &jobs[t]) == 0;
        if (!started[t]) wl_worker(&jobs[t]);
    }
    int st = 0;
    for (int t = 0; t < n_threads; ++t) {
        if (started[t]) pthread_join(th[t], NULL);
        if (jobs[t].status && !st) st = jobs[t].status;
    }
    return st;
}

/* Pass 1: per-pair query and reference lengths. */
int wl_lengths(const wl_params* P, const uint8_t* bg, const uint8_t* sub,
               int64_t* q_len, int64_t* r_len, int n_threads)
{
    wl_job J;
    memset(&J, 0, sizeof(J));
    J.P = P; J.bg = bg; J.sub = sub; J.q_len = q_len; J.r_len = r_len;
    return wl_run(&J, n_threads);
}

/* Pass 2: residues into buffers laid out by the offsets of pass 1. */
int wl_fill(const wl_params* P, const uint8_t* bg, const uint8_t* sub,
            const int64_t* q_off, const int64_t* r_off, uint8_t* q_res, uint8_t* r_res,
            int n_threads)
{
    wl_job J;
    memset(&J, 0, sizeof(J));
    J.P = P; J.bg = bg; J.sub = sub; J.q_off = q_off; J.r_off = r_off;
    J.q_res = q_res; J.r_res = r_res;
    return wl_run(&J, n_threads);
}

/* ---- families: one sequence set of n_pairs families x copies sequences ----
 * Sequence s belongs to family f = s / copies.  The family's root is drawn
 * like a query from the stream of (seed, f); sequence s is mutate(root) drawn
 * from the stream of (seed ^ kCopySalt, s), so every sequence can be drawn
 * alone, in parallel, with identical results. */
static const uint64_t kCopySalt = 0xC0B1E5C0B1E5C0B1ULL;

typedef struct {
    const wl_params* P;
    int64_t copies;
    const uint8_t* bg;
    const uint8_t* sub;
    int64_t* len;            /* pass 1 */
    const int64_t* off;      /* pass 2 */
    uint8_t* res;
    int64_t begin, end;
    int status;
} wl_fjob;

static void* wl_fworker(void* arg)
{
    wl_fjob* J = (wl_fjob*)arg;
    uint8_t* root = (uint8_t*)malloc((size_t)J->P->lmax + 1);
    if (!root) { J->status = -1; return NULL; }
    for (int64_t s = J->begin; s < J->end; ++s) {
        wl_rng rng;
        wl_seed(&rng, J->P->seed, s / J->copies);
        int32_t lroot = wl_length(&rng, J->P);
        for (int32_t i = 0; i < lroot; ++i) root[i] = wl_background(&rng, J->bg);
        wl_rng mr;
        wl_seed(&mr, J->P->seed ^ kCopySalt, s);
        uint8_t* out = J->res ? J->res + J->off[s] : NULL;
        int64_t l = wl_mutate(&mr, root, lroot, J->P, J->bg, J->sub, out);
        if (J->res) {
            if (l != J->off[s + 1] - J->off[s]) { J->status = -2; break; }
        } else {
            J->len[s] = l;
        }
    }
    free(root);
    return NULL;
}

static int wl_frun(wl_fjob* proto, int n_threads)
{
    int64_t n = proto->P->n_pairs * proto->copies;
    if (n_threads < 1) n_threads = 1;
    if (n_threads > 256) n_threads = 256;
    wl_fjob jobs[256];
    pthread_t th[256];
    int started[256];
    for (int t = 0; t < n_threads; ++t) {
        jobs[t] = *proto;
        jobs[t].begin = n * t / n_threads;
        jobs[t].end = n * (t + 1) / n_threads;
        jobs[t].status = 0;
        started[t] = pthread_create(&th[t], NULL, wl_fworker, &jobs[t]) == 0;
        if (!started[t]) wl_fworker(&jobs[t]);
    }
    int st = 0;
    for (int t = 0; t < n_threads; ++t) {
        if (started[t]) pthread_join(th[t], NULL);
        if (jobs[t].status && !st) st = jobs[t].status;
    }
    return st;
}

/* Pass 1 of a family set: the length of every sequence. */
int wl_family_lengths(const wl_params* P, int64_t copies, const uint8_t* bg, const uint8_t* sub,
                      int64_t* len, int n_threads)
{
    wl_fjob J;
    memset(&J, 0, sizeof(J));
    J.P = P; J.copies = copies; J.bg = bg; J.sub = sub; J.len = len;
    return wl_frun(&J, n_threads);
}

/* Pass 2 of a family set: residues laid out by the offsets of pass 1. */
int wl_family_fill(const wl_params* P, int64_t copies, const uint8_t* bg, const uint8_t* sub,
                   const int64_t* off, uint8_t* res, int n_threads)
{
    wl_fjob J;
    memset(&J, 0, sizeof(J));
    J.P = P; J.copies = copies; J.bg = bg; J.sub = sub; J.off = off; J.res = res;
    return wl_frun(&J, n_threads);
}
