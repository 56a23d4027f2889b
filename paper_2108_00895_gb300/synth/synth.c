/*
 * Seeded synthetic tf-idf corpora shaped like the paper's document collections
 * (Section 4.1: bag-of-words vectors, term frequency times log inverse document
 * frequency, stop words removed, every vector divided by its length).
 *
 * This file holds input generation only. It contains none of the clustering
 * arithmetic, and both the FP64 oracle and the CUDA path consume its output.
 *
 * Definition of a corpus (all randomness is counter-based, so the output does not
 * depend on the number of threads):
 *   nnz_i  = clip(round(exp(mu + sigma*z)), lo, hi), sigma = 1, mu = ln(mean) - 1/2,
 *            z standard normal (Box-Muller); hi is further capped at d/2. The length
 *            is drawn once per document; a redraw (below) keeps it.
 *   terms  = sequential Zipf(s) draws over ranks 1..d (P(r) ~ r^-s, term id r-1),
 *            repeats rejected, until nnz_i distinct terms are held.
 *   tf     = 1 + Poisson(1).
 *   df_t   = number of documents containing t;  w_it = tf_it * ln(N / df_t).
 *   Entries with df_t = N (idf 0, a "stop word") are dropped; a document left
 *   empty is redrawn with the next attempt counter and df is recounted.
 *   x_i    = w_i / ||w_i||_2 (computed in double, stored as float), columns ascending.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ---- counter-based random numbers (SplitMix64 finaliser as a keyed hash) ---- */
static inline uint64_t mix64(uint64_t z) {
    z ^= z >> 30; z *= 0xbf58476d1ce4e5b9ULL;
    z ^= z >> 27; z *= 0x94d049bb133111ebULL;
    z ^= z >> 31; return z;
}
static inline uint64_t rng_u64(uint64_t seed, uint64_t stream, uint64_t ctr) {
    uint64_t k = mix64(seed * 0x9E3779B97F4A7C15ULL + 0x632BE59BD9B4E019ULL);
    k = mix64(k ^ (stream * 0xD1B54A32D192ED03ULL + 0x8CB92BA72F3D8DD7ULL));
    return mix64(k + ctr * 0x9E3779B97F4A7C15ULL);
}
/* uniform in (0,1) */
static inline double rng_unit(uint64_t seed, uint64_t stream, uint64_t ctr) {
    return ((double)(rng_u64(seed, stream, ctr) >> 11) + 0.5) * (1.0 / 9007199254740992.0);
}

typedef struct { uint64_t seed, stream, ctr; } rstate;
static inline double next_unit(rstate *r) { return rng_unit(r->seed, r->stream, r->ctr++); }

/* ---- Walker/Vose alias table for the Zipf rank distribution ---- */
typedef struct { double *prob; int32_t *alias; int32_t n; } alias_t;

static int alias_build(alias_t *a, int32_t d, double s) {
    a->n = d;
    a->prob = (double *)malloc(sizeof(double) * (size_t)d);
    a->alias = (int32_t *)malloc(sizeof(int32_t) * (size_t)d);
    double *w = (double *)malloc(sizeof(double) * (size_t)d);
    int32_t *small = (int32_t *)malloc(sizeof(int32_t) * (size_t)d);
    int32_t *large = (int32_t *)malloc(sizeof(int32_t) * (size_t)d);
    if (!a->prob || !a->alias || !w || !small || !large) return -1;
    double h = 0.0;
    for (int32_t r = 0; r < d; ++r) { w[r] = pow((double)(r + 1), -s); h += w[r]; }
    int32_t ns = 0, nl = 0;
    for (int32_t r = 0; r < d; ++r) {
        w[r] = w[r] * (double)d / h;
        if (w[r] < 1.0) small[ns++] = r; else large[nl++] = r;
    }
    while (ns > 0 && nl > 0) {
        int32_t l = small[--ns], g = large[--nl];
        a->prob[l] = w[l]; a->alias[l] = g;
        w[g] = (w[g] + w[l]) - 1.0;
        if (w[g] < 1.0) small[ns++] = g; else large[nl++] = g;
    }
    while (nl > 0) { int32_t g = large[--nl]; a->prob[g] = 1.0; a->alias[g] = g; }
    while (ns > 0) { int32_t l = small[--ns]; a->prob[l] = 1.0; a->alias[l] = l; }
    free(w); free(small); free(large);
    return 0;
}
static void alias_free(alias_t *a) { free(a->prob); free(a->alias); }

static inline int32_t alias_draw(const alias_t *a, rstate *r) {
    double u = next_unit(r) * (double)a->n;
    int32_t b = (int32_t)u;
    if (b >= a->n) b = a->n - 1;
    double v = next_unit(r);
    return v < a->prob[b] ? b : a->alias[b];
}

static inline int32_t poisson1(rstate *r) {
    const double L = 0.36787944117144233; /* e^-1 */
    double p = 1.0; int32_t k = 0;
    do { ++k; p *= next_unit(r); } while (p > L);
    return k - 1;
}

static int cmp_i32(const void *a, const void *b) {
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

/* Draw one document's distinct terms (ascending) and term frequencies. */
static void draw_doc(const alias_t *zipf, uint64_t seed, int64_t doc, int32_t attempt,
                     int32_t n, int32_t *terms, int32_t *tfs, uint32_t *stamp, uint32_t tag) {
    rstate r = { seed, 0x100000000ULL + (uint64_t)doc * 64ULL + (uint64_t)attempt, 0 };
    int32_t got = 0;
    while (got < n) {
        int32_t t = alias_draw(zipf, &r);
        if (stamp[t] == tag) continue;
        stamp[t] = tag;
        terms[got++] = t;
    }
    qsort(terms, (size_t)n, sizeof(int32_t), cmp_i32);
    for (int32_t q = 0; q < n; ++q) tfs[q] = 1 + poisson1(&r);
}

/* Drawn length of a document (before dropping df = N terms); fixed across redraws. */
static int32_t draw_len(uint64_t seed, int64_t doc, double mu, int32_t lo, int32_t hi) {
    rstate r = { seed, (uint64_t)doc, 0 };
    double u1 = next_unit(&r), u2 = next_unit(&r);
    double z = sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2);
    double len = floor(exp(mu + z) + 0.5);
    return len < (double)lo ? lo : (len > (double)hi ? hi : (int32_t)len);
}

/*
 * Pass 1: returns the total number of stored entries E (after dropping df=N terms)
 * and keeps the drawn corpus in an opaque handle; pass 2 (synth_corpus_fill) writes
 * the CSR arrays. Returns NULL on allocation failure or invalid arguments.
 */
typedef struct {
    int64_t n_docs; int32_t n_terms;
    int64_t *off;      /* [N+1] offsets into terms/tfs (drawn entries) */
    int32_t *terms, *tfs, *len;
    int64_t *df;
    int64_t nnz_kept;
} synth_corpus;

synth_corpus *synth_corpus_draw(int64_t n_docs, int32_t n_terms, double nnz_mean,
                                int32_t nnz_lo, int32_t nnz_hi, double zipf_s, uint64_t seed) {
    if (n_docs < 1 || n_terms < 2 || nnz_mean <= 0.0 || nnz_lo < 1 || nnz_hi < nnz_lo) return NULL;
    int32_t hi = nnz_hi > n_terms / 2 ? n_terms / 2 : nnz_hi;
    int32_t lo = nnz_lo > hi ? hi : nnz_lo;
    if (lo < 1) lo = 1;
    const double mu = log(nnz_mean) - 0.5;
    alias_t zipf;
    if (alias_build(&zipf, n_terms, zipf_s) != 0) return NULL;

    synth_corpus *c = (synth_corpus *)calloc(1, sizeof(synth_corpus));
    c->n_docs = n_docs; c->n_terms = n_terms;
    c->off = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n_docs + 1));
    c->len = (int32_t *)malloc(sizeof(int32_t) * (size_t)n_docs);
    c->df = (int64_t *)calloc((size_t)n_terms, sizeof(int64_t));
    int32_t *attempt = (int32_t *)calloc((size_t)n_docs, sizeof(int32_t));
    char *pending = (char *)malloc((size_t)n_docs);
    if (!c->off || !c->len || !c->df || !attempt || !pending) { alias_free(&zipf); return NULL; }
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n_docs; ++i) c->len[i] = draw_len(seed, i, mu, lo, hi);
    c->off[0] = 0;
    for (int64_t i = 0; i < n_docs; ++i) c->off[i + 1] = c->off[i] + c->len[i];
    c->terms = (int32_t *)malloc(sizeof(int32_t) * (size_t)c->off[n_docs]);
    c->tfs = (int32_t *)malloc(sizeof(int32_t) * (size_t)c->off[n_docs]);
    if (!c->terms || !c->tfs) { alias_free(&zipf); return NULL; }
    memset(pending, 1, (size_t)n_docs);

    int nthreads = 1;
#ifdef _OPENMP
    nthreads = omp_get_max_threads();
#endif
    int64_t *df_part = (int64_t *)calloc((size_t)nthreads * (size_t)n_terms, sizeof(int64_t));

    for (int round = 0; round < 32; ++round) {
#pragma omp parallel
        {
            int tid = 0;
#ifdef _OPENMP
            tid = omp_get_thread_num();
#endif
            uint32_t *stamp = (uint32_t *)calloc((size_t)n_terms, sizeof(uint32_t));
            uint32_t tag = 0;
#pragma omp for schedule(dynamic, 256)
            for (int64_t i = 0; i < n_docs; ++i) {
                if (!pending[i]) continue;
                ++tag;
                if (tag == 0) { memset(stamp, 0, sizeof(uint32_t) * (size_t)n_terms); tag = 1; }
                draw_doc(&zipf, seed, i, attempt[i], c->len[i], c->terms + c->off[i],
                         c->tfs + c->off[i], stamp, tag);
            }
            free(stamp);
            int64_t *mydf = df_part + (size_t)tid * (size_t)n_terms;
            memset(mydf, 0, sizeof(int64_t) * (size_t)n_terms);
#pragma omp for schedule(static)
            for (int64_t i = 0; i < n_docs; ++i) {
                const int32_t *tt = c->terms + c->off[i];
                for (int32_t q = 0; q < c->len[i]; ++q) mydf[tt[q]]++;
            }
        }
        for (int32_t t = 0; t < n_terms; ++t) {
            int64_t s = 0;
            for (int p = 0; p < nthreads; ++p) s += df_part[(size_t)p * (size_t)n_terms + t];
            c->df[t] = s;
        }
        /* a document is empty iff all of its terms have df = N */
        int64_t n_empty = 0;
        for (int64_t i = 0; i < n_docs; ++i) {
            const int32_t *tt = c->terms + c->off[i];
            int keep = 0;
            for (int32_t q = 0; q < c->len[i]; ++q) if (c->df[tt[q]] < n_docs) { keep = 1; break; }
            pending[i] = (char)!keep;
            if (!keep) { attempt[i]++; n_empty++; }
        }
        if (n_empty == 0) break;
    }
    int64_t kept = 0;
    for (int64_t i = 0; i < n_docs; ++i) {
        const int32_t *tt = c->terms + c->off[i];
        for (int32_t q = 0; q < c->len[i]; ++q) kept += (c->df[tt[q]] < n_docs);
    }
    c->nnz_kept = kept;
    free(df_part); free(attempt); free(pending); alias_free(&zipf);
    return c;
}

int64_t synth_corpus_nnz(const synth_corpus *c) { return c ? c->nnz_kept : -1; }

/* Pass 2: write CSR (row_ptr[N+1], col_idx[E], values[E]) and free the handle. */
int synth_corpus_fill(synth_corpus *c, int64_t *row_ptr, int32_t *col_idx, float *values) {
    if (!c) return -1;
    const int64_t N = c->n_docs;
    /* row lengths after dropping df=N terms */
    row_ptr[0] = 0;
    for (int64_t i = 0; i < N; ++i) {
        const int32_t *tt = c->terms + c->off[i];
        int64_t n = 0;
        for (int32_t q = 0; q < c->len[i]; ++q) n += (c->df[tt[q]] < N);
        row_ptr[i + 1] = row_ptr[i] + n;
    }
#pragma omp parallel for schedule(dynamic, 256)
    for (int64_t i = 0; i < N; ++i) {
        const int32_t *tt = c->terms + c->off[i];
        const int32_t *tf = c->tfs + c->off[i];
        int64_t o = row_ptr[i];
        double ss = 0.0;
        for (int32_t q = 0; q < c->len[i]; ++q) {
            if (c->df[tt[q]] >= N) continue;
            double w = (double)tf[q] * log((double)N / (double)c->df[tt[q]]);
            ss += w * w;
        }
        double inv = 1.0 / sqrt(ss);
        for (int32_t q = 0; q < c->len[i]; ++q) {
            if (c->df[tt[q]] >= N) continue;
            double w = (double)tf[q] * log((double)N / (double)c->df[tt[q]]);
            col_idx[o] = tt[q];
            values[o] = (float)(w * inv);
            ++o;
        }
    }
    free(c->off); free(c->len); free(c->df); free(c->terms); free(c->tfs); free(c);
    return 0;
}

void synth_corpus_free(synth_corpus *c) {
    if (!c) return;
    free(c->off); free(c->len); free(c->df); free(c->terms); free(c->tfs); free(c);
}

/*
 * k distinct document ids by a seeded partial Fisher-Yates shuffle of 0..N-1.
 * Returns 0 on success, -1 on invalid arguments.
 */
int synth_init_ids(int64_t n_docs, int32_t k, uint64_t seed, int32_t *out) {
    if (k < 1 || (int64_t)k > n_docs) return -1;
    int32_t *perm = (int32_t *)malloc(sizeof(int32_t) * (size_t)n_docs);
    if (!perm) return -1;
    for (int64_t i = 0; i < n_docs; ++i) perm[i] = (int32_t)i;
    for (int32_t j = 0; j < k; ++j) {
        double u = rng_unit(seed, 0xF15E4ULL, (uint64_t)j);
        int64_t r = j + (int64_t)(u * (double)(n_docs - j));
        if (r >= n_docs) r = n_docs - 1;
        int32_t tmp = perm[j]; perm[j] = perm[r]; perm[r] = tmp;
        out[j] = perm[j];
    }
    free(perm);
    return 0;
}

/* Uniform doubles in (0,1) from the same counter generator, for seeded sampling. */
void synth_uniform(uint64_t seed, uint64_t stream, int64_t n, double *out) {
    for (int64_t i = 0; i < n; ++i) out[i] = rng_unit(seed, stream, (uint64_t)i);
}
