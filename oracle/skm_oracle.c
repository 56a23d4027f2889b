/*
 * FP64 CPU oracle for exact sparse spherical k-means.
 *
 * TEST INFRASTRUCTURE ONLY. This code checks the CUDA path; it is never part of it.
 * Only the test suite, the smoke check and the benchmark's CPU-baseline leg may load
 * it. It shares no code, header or table with the CUDA library.
 *
 * Paper: Knittel, Koch, Ertl, "Efficient Sparse Spherical k-Means for Document
 * Clustering", DocEng 2021.
 *
 * Conventions (all arithmetic in IEEE double, built with -ffp-contract=off):
 *   docs      CSR: row_ptr[N+1] (int64), col[E] (int32, strictly increasing per row),
 *             val[E] (float, >= 0, rows of unit L2 length).
 *   centroids term-major d x k: C[t*k + j] is entry t of centroid j.
 *   s_ij      = sum over the nonzeros t of x_i, in CSR order, of x_it * c_jt.
 *   argmax    ties go to the lowest centroid index.
 *
 * Readings of points the paper leaves open (each is restated where it is used):
 *   R1 "unchanged within a tolerance" (Sec. 3.1) is read with tolerance 0 and decided by
 *      membership: a centroid is unchanged iff no document joined or left its cluster.
 *   R2 an empty cluster keeps its previous centroid.
 *   R3 one iteration = assignment step, then centroid update; the loop starts from the
 *      centroids given by k initial documents.
 *   R4 the index threshold used for a query is the largest lambda strictly below the
 *      baseline similarity, after a relative safety factor for rounding (Sec. 3.2).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_MODE_PLAIN 0
#define OR_MODE_NCC 1
#define OR_MODE_NCC_INDEX 2
#define OR_MODE_INDEX 3

int oracle_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void oracle_set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/* Centroid entry as double; C is double (c_f32 = 0) or float (c_f32 = 1). */
static inline double cval(const void *C, int c_f32, size_t idx) {
    return c_f32 ? (double)((const float *)C)[idx] : ((const double *)C)[idx];
}

/* One similarity s_ij (Sec. 2: cosine = dot product of unit vectors). */
static double dot_one(const int64_t *row_ptr, const int32_t *col, const float *val, int64_t i,
                      const void *C, int c_f32, int32_t k, int32_t j) {
    double s = 0.0;
    for (int64_t p = row_ptr[i]; p < row_ptr[i + 1]; ++p)
        s += (double)val[p] * cval(C, c_f32, (size_t)col[p] * (size_t)k + (size_t)j);
    return s;
}

/*
 * Assignment step by its definition (Sec. 2): a_i = argmax_j s_ij over all k centroids.
 * Outputs (nullable except a): best score s1, runner-up score s2 (max over j != a_i;
 * -inf when k = 1).
 */
void oracle_assign(int64_t n_docs, const int64_t *row_ptr, const int32_t *col, const float *val,
                   int32_t d, int32_t k, const void *C, int c_f32,
                   int32_t *a, double *s1_out, double *s2_out) {
    (void)d;
#pragma omp parallel
    {
        double *s = (double *)malloc(sizeof(double) * (size_t)k);
#pragma omp for schedule(dynamic, 64)
        for (int64_t i = 0; i < n_docs; ++i) {
            for (int32_t j = 0; j < k; ++j) s[j] = 0.0;
            for (int64_t p = row_ptr[i]; p < row_ptr[i + 1]; ++p) {
                const double x = (double)val[p];
                const size_t base = (size_t)col[p] * (size_t)k;
                if (c_f32) {
                    const float *row = (const float *)C + base;
                    for (int32_t j = 0; j < k; ++j) s[j] += x * (double)row[j];
                } else {
                    const double *row = (const double *)C + base;
                    for (int32_t j = 0; j < k; ++j) s[j] += x * row[j];
                }
            }
            int32_t best = 0;
            for (int32_t j = 1; j < k; ++j) if (s[j] > s[best]) best = j;
            double second = -INFINITY;
            for (int32_t j = 0; j < k; ++j) if (j != best && s[j] > second) second = s[j];
            a[i] = best;
            if (s1_out) s1_out[i] = s[best];
            if (s2_out) s2_out[i] = second;
        }
        free(s);
    }
}

/* All k similarities of a set of docs (rows of out are docs; small inputs only). */
void oracle_scores(int64_t n_docs, const int64_t *row_ptr, const int32_t *col, const float *val,
                   int32_t k, const void *C, int c_f32, double *out) {
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < n_docs; ++i)
        for (int32_t j = 0; j < k; ++j)
            out[(size_t)i * (size_t)k + (size_t)j] = dot_one(row_ptr, col, val, i, C, c_f32, k, j);
}

/* Objective of an assignment (Sec. 2): sum_i s_{i,a_i}, summed over i ascending. */
double oracle_objective(int64_t n_docs, const int64_t *row_ptr, const int32_t *col,
                        const float *val, int32_t k, const void *C, int c_f32, const int32_t *a) {
    double tot = 0.0;
    for (int64_t i = 0; i < n_docs; ++i) tot += dot_one(row_ptr, col, val, i, C, c_f32, k, a[i]);
    return tot;
}

/*
 * Centroid update (Sec. 2): c_j = S_j / ||S_j||, S_j = sum of the member documents,
 * summed over members in ascending document order and the norm over terms ascending.
 * An empty cluster keeps its previous centroid (R2).
 *   C       in: previous centroids, out: new centroids (d x k double).
 *   changed out (nullable): 1 iff cluster j's membership differs between a_prev and a
 *           (R1); with a_prev == NULL every cluster that has members is changed.
 *   shift   out (nullable): max_j ||c_j(new) - c_j(old)||^2 (Sec. 4.1 stop rule).
 *   sizes   out (nullable): members per cluster.
 * Returns the number of changed clusters.
 */
int32_t oracle_update(int64_t n_docs, const int64_t *row_ptr, const int32_t *col, const float *val,
                      int32_t d, int32_t k, const int32_t *a, const int32_t *a_prev,
                      double *C, uint8_t *changed, double *shift, int64_t *sizes) {
    const size_t dk = (size_t)d * (size_t)k;
    double *S = (double *)calloc(dk, sizeof(double));
    int64_t *cnt = (int64_t *)calloc((size_t)k, sizeof(int64_t));
    uint8_t *chg = (uint8_t *)calloc((size_t)k, 1);
    if (!S || !cnt || !chg) { free(S); free(cnt); free(chg); return -1; }
    for (int64_t i = 0; i < n_docs; ++i) {
        const int32_t j = a[i];
        cnt[j]++;
        if (!a_prev) chg[j] = 1;
        else if (a_prev[i] != j) { chg[j] = 1; chg[a_prev[i]] = 1; }
        for (int64_t p = row_ptr[i]; p < row_ptr[i + 1]; ++p)
            S[(size_t)col[p] * (size_t)k + (size_t)j] += (double)val[p];
    }
    double max_shift = 0.0;
    int32_t n_changed = 0;
    for (int32_t j = 0; j < k; ++j) {
        n_changed += chg[j];
        if (cnt[j] == 0) continue;              /* R2: keep the previous centroid */
        double ss = 0.0;
        for (int32_t t = 0; t < d; ++t) {
            const double v = S[(size_t)t * (size_t)k + (size_t)j];
            ss += v * v;
        }
        const double nrm = sqrt(ss);
        double sh = 0.0;
        for (int32_t t = 0; t < d; ++t) {
            const size_t idx = (size_t)t * (size_t)k + (size_t)j;
            const double c = S[idx] / nrm;
            const double diff = c - C[idx];
            sh += diff * diff;
            C[idx] = c;
        }
        if (sh > max_shift) max_shift = sh;
    }
    if (changed) memcpy(changed, chg, (size_t)k);
    if (shift) *shift = max_shift;
    if (sizes) memcpy(sizes, cnt, sizeof(int64_t) * (size_t)k);
    free(S); free(cnt); free(chg);
    return n_changed;
}

/*
 * Centroids of selected clusters only (Sec. 2, same definition and summation order as
 * oracle_update): out[t * n_sel + q] = entry t of c_{sel[q]}; a cluster without members
 * gives a zero column. For checks on large collections where d x k would not fit.
 */
void oracle_centroids_subset(int64_t n_docs, const int64_t *row_ptr, const int32_t *col,
                             const float *val, int32_t d, const int32_t *a, int32_t n_sel,
                             const int32_t *sel, double *out) {
    memset(out, 0, sizeof(double) * (size_t)d * (size_t)n_sel);
    for (int32_t q = 0; q < n_sel; ++q) {
        const int32_t j = sel[q];
        for (int64_t i = 0; i < n_docs; ++i) {
            if (a[i] != j) continue;
            for (int64_t p = row_ptr[i]; p < row_ptr[i + 1]; ++p)
                out[(size_t)col[p] * (size_t)n_sel + (size_t)q] += (double)val[p];
        }
        double ss = 0.0;
        for (int32_t t = 0; t < d; ++t) {
            const double v = out[(size_t)t * (size_t)n_sel + (size_t)q];
            ss += v * v;
        }
        if (ss == 0.0) continue;
        const double nrm = sqrt(ss);
        for (int32_t t = 0; t < d; ++t) out[(size_t)t * (size_t)n_sel + (size_t)q] /= nrm;
    }
}

/* Initial centroids from k documents: c_j = x_{init_j} (R3). */
void oracle_init_centroids(const int64_t *row_ptr, const int32_t *col, const float *val,
                           int32_t d, int32_t k, const int32_t *init_ids, double *C) {
    memset(C, 0, sizeof(double) * (size_t)d * (size_t)k);
    for (int32_t j = 0; j < k; ++j) {
        const int64_t i = init_ids[j];
        for (int64_t p = row_ptr[i]; p < row_ptr[i + 1]; ++p)
            C[(size_t)col[p] * (size_t)k + (size_t)j] = (double)val[p];
    }
}

/* ------------------------------------------------------------------------------------
 * Dot product indexing structure (Sec. 3.2).
 *   G      general inverse index: term -> centroids with a nonzero entry at that term.
 *   P_lam  threshold index: term -> (centroid, minimum overlap count).
 * Both are stored as CSR over terms.
 * ---------------------------------------------------------------------------------- */
typedef struct {
    int32_t d, k;
    int64_t *g_ptr; int32_t *g_cent;                 /* G */
    int n_lam; double *lam;
    int64_t **p_ptr; int32_t **p_cent; int32_t **p_min;  /* P_lam per lambda */
} oracle_index;

typedef struct { double v; int32_t t; } vt_pair;
static int cmp_vt_desc(const void *x, const void *y) {
    const vt_pair *a = (const vt_pair *)x, *b = (const vt_pair *)y;
    if (a->v > b->v) return -1;
    if (a->v < b->v) return 1;
    return (a->t > b->t) - (a->t < b->t);        /* ties: term id ascending */
}

/*
 * Minimum overlap counts of one centroid for one lambda (Sec. 3.2, build steps 2-3).
 * v[0..m) sorted descending. minc[p] = smallest count q such that the squares of the q
 * entries starting at position p sum to at least lam^2 (an entry >= lam gives 1);
 * minc[p] = 0 where the threshold cannot be reached, and every later p is 0 too.
 * Linear version (the footnote): a window [p, end) whose squared sum is carried over,
 * adding each square once and subtracting it once.
 * The threshold is lam^2 (1 - 1e-12) so rounding cannot drop a valid candidate.
 */
void oracle_min_overlap_linear(int32_t m, const double *v, double lam, int32_t *minc) {
    const double thr = lam * lam * (1.0 - 1e-12);
    double sum = 0.0;
    int32_t end = 0;                     /* window is [p, end) */
    int stopped = 0;
    for (int32_t p = 0; p < m; ++p) {
        if (stopped) { minc[p] = 0; continue; }
        if (end < p) { end = p; sum = 0.0; }
        while (end < m && sum < thr) { sum += v[end] * v[end]; ++end; }
        if (sum < thr) { stopped = 1; minc[p] = 0; continue; }
        minc[p] = end - p;
        sum -= v[p] * v[p];
    }
}

/* The same counts by the direct O(m^2) reading of build step 3 (for cross-checking). */
void oracle_min_overlap_naive(int32_t m, const double *v, double lam, int32_t *minc) {
    const double thr = lam * lam * (1.0 - 1e-12);
    int stopped = 0;
    for (int32_t p = 0; p < m; ++p) {
        if (stopped) { minc[p] = 0; continue; }
        double sum = 0.0;
        int32_t q = p;
        while (q < m && sum < thr) { sum += v[q] * v[q]; ++q; }
        if (sum < thr) { stopped = 1; minc[p] = 0; continue; }
        minc[p] = q - p;
    }
}

void oracle_index_free(oracle_index *ix) {
    if (!ix) return;
    free(ix->g_ptr); free(ix->g_cent);
    for (int l = 0; l < ix->n_lam; ++l) { free(ix->p_ptr[l]); free(ix->p_cent[l]); free(ix->p_min[l]); }
    free(ix->p_ptr); free(ix->p_cent); free(ix->p_min); free(ix->lam);
    free(ix);
}

/* Build G and P_lam for every lambda from dense term-major centroids (Sec. 3.2). */
oracle_index *oracle_index_build(int32_t d, int32_t k, const double *C, int n_lam, const double *lam) {
    oracle_index *ix = (oracle_index *)calloc(1, sizeof(oracle_index));
    ix->d = d; ix->k = k; ix->n_lam = n_lam;
    ix->lam = (double *)malloc(sizeof(double) * (size_t)n_lam);
    memcpy(ix->lam, lam, sizeof(double) * (size_t)n_lam);
    /* G: nonzero pattern per term, centroids ascending */
    ix->g_ptr = (int64_t *)calloc((size_t)d + 1, sizeof(int64_t));
    for (int32_t t = 0; t < d; ++t) {
        int64_t c = 0;
        for (int32_t j = 0; j < k; ++j) c += (C[(size_t)t * (size_t)k + (size_t)j] != 0.0);
        ix->g_ptr[t + 1] = ix->g_ptr[t] + c;
    }
    ix->g_cent = (int32_t *)malloc(sizeof(int32_t) * (size_t)(ix->g_ptr[d] + 1));
    for (int32_t t = 0; t < d; ++t) {
        int64_t o = ix->g_ptr[t];
        for (int32_t j = 0; j < k; ++j)
            if (C[(size_t)t * (size_t)k + (size_t)j] != 0.0) ix->g_cent[o++] = j;
    }
    /* P_lam: per centroid, entries sorted by value descending, with min-overlap counts */
    ix->p_ptr = (int64_t **)calloc((size_t)n_lam, sizeof(int64_t *));
    ix->p_cent = (int32_t **)calloc((size_t)n_lam, sizeof(int32_t *));
    ix->p_min = (int32_t **)calloc((size_t)n_lam, sizeof(int32_t *));
    /* per centroid sorted entries */
    int64_t *cnt_j = (int64_t *)calloc((size_t)k + 1, sizeof(int64_t));
    for (int32_t t = 0; t < d; ++t)
        for (int64_t q = ix->g_ptr[t]; q < ix->g_ptr[t + 1]; ++q) cnt_j[ix->g_cent[q] + 1]++;
    for (int32_t j = 0; j < k; ++j) cnt_j[j + 1] += cnt_j[j];
    const int64_t nz = cnt_j[k];
    vt_pair *ent = (vt_pair *)malloc(sizeof(vt_pair) * (size_t)(nz + 1));
    int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * (size_t)(k + 1));
    memcpy(fill, cnt_j, sizeof(int64_t) * (size_t)(k + 1));
    for (int32_t t = 0; t < d; ++t)
        for (int64_t q = ix->g_ptr[t]; q < ix->g_ptr[t + 1]; ++q) {
            const int32_t j = ix->g_cent[q];
            ent[fill[j]].v = C[(size_t)t * (size_t)k + (size_t)j];
            ent[fill[j]].t = t;
            fill[j]++;
        }
    for (int32_t j = 0; j < k; ++j)
        qsort(ent + cnt_j[j], (size_t)(cnt_j[j + 1] - cnt_j[j]), sizeof(vt_pair), cmp_vt_desc);
    double *vbuf = (double *)malloc(sizeof(double) * (size_t)(nz + 1));
    int32_t *mbuf = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nz + 1));
    for (int l = 0; l < n_lam; ++l) {
        int64_t *pc = (int64_t *)calloc((size_t)d + 1, sizeof(int64_t));
        for (int32_t j = 0; j < k; ++j) {
            const int32_t m = (int32_t)(cnt_j[j + 1] - cnt_j[j]);
            for (int32_t p = 0; p < m; ++p) vbuf[cnt_j[j] + p] = ent[cnt_j[j] + p].v;
            oracle_min_overlap_linear(m, vbuf + cnt_j[j], lam[l], mbuf + cnt_j[j]);
            for (int32_t p = 0; p < m; ++p) if (mbuf[cnt_j[j] + p] > 0) pc[ent[cnt_j[j] + p].t + 1]++;
        }
        for (int32_t t = 0; t < d; ++t) pc[t + 1] += pc[t];
        int32_t *pcent = (int32_t *)malloc(sizeof(int32_t) * (size_t)(pc[d] + 1));
        int32_t *pmin = (int32_t *)malloc(sizeof(int32_t) * (size_t)(pc[d] + 1));
        int64_t *pf = (int64_t *)malloc(sizeof(int64_t) * (size_t)(d + 1));
        memcpy(pf, pc, sizeof(int64_t) * (size_t)(d + 1));
        for (int32_t j = 0; j < k; ++j) {             /* centroids ascending within a term */
            const int32_t m = (int32_t)(cnt_j[j + 1] - cnt_j[j]);
            for (int32_t p = 0; p < m; ++p) {
                const int32_t mc = mbuf[cnt_j[j] + p];
                if (mc <= 0) continue;
                const int32_t t = ent[cnt_j[j] + p].t;
                pcent[pf[t]] = j; pmin[pf[t]] = mc; pf[t]++;
            }
        }
        free(pf);
        ix->p_ptr[l] = pc; ix->p_cent[l] = pcent; ix->p_min[l] = pmin;
    }
    free(vbuf); free(mbuf); free(ent); free(fill); free(cnt_j);
    return ix;
}

/* Sizes of the structures (for reporting and tests). */
int64_t oracle_index_g_size(const oracle_index *ix) { return ix->g_ptr[ix->d]; }
int64_t oracle_index_p_size(const oracle_index *ix, int l) { return ix->p_ptr[l][ix->d]; }

/*
 * Index query (Sec. 3.2, query steps 1-2) for document i and threshold index l.
 * count[] (k ints, all zero on entry and on return) is scratch for the count map C.
 * Writes the candidate centroids, ascending, into cand; returns their number.
 */
int32_t oracle_index_query(const oracle_index *ix, int l, const int64_t *row_ptr, const int32_t *col,
                           int64_t i, int32_t *count, uint8_t *mark, int32_t *cand) {
    for (int64_t p = row_ptr[i]; p < row_ptr[i + 1]; ++p) {      /* step 1: overlap counts */
        const int32_t t = col[p];
        for (int64_t q = ix->g_ptr[t]; q < ix->g_ptr[t + 1]; ++q) count[ix->g_cent[q]]++;
    }
    int32_t nc = 0;
    const int64_t *pp = ix->p_ptr[l];
    for (int64_t p = row_ptr[i]; p < row_ptr[i + 1]; ++p) {      /* step 2: min-overlap test */
        const int32_t t = col[p];
        for (int64_t q = pp[t]; q < pp[t + 1]; ++q) {
            const int32_t j = ix->p_cent[l][q];
            if (!mark[j] && count[j] >= ix->p_min[l][q]) { mark[j] = 1; cand[nc++] = j; }
        }
    }
    for (int64_t p = row_ptr[i]; p < row_ptr[i + 1]; ++p) {      /* reset scratch */
        const int32_t t = col[p];
        for (int64_t q = ix->g_ptr[t]; q < ix->g_ptr[t + 1]; ++q) count[ix->g_cent[q]] = 0;
    }
    for (int32_t c = 0; c < nc; ++c) mark[cand[c]] = 0;
    /* ascending order (insertion sort; candidate lists are short) */
    for (int32_t a = 1; a < nc; ++a) {
        int32_t v = cand[a], b = a - 1;
        while (b >= 0 && cand[b] > v) { cand[b + 1] = cand[b]; --b; }
        cand[b + 1] = v;
    }
    return nc;
}

/* Python-friendly wrapper: build, query every doc for one lambda, free. */
int64_t oracle_index_candidates(int64_t n_docs, const int64_t *row_ptr, const int32_t *col,
                                int32_t d, int32_t k, const double *C, double lam,
                                int64_t *cand_ptr, int32_t *cand_out, int64_t cap) {
    oracle_index *ix = oracle_index_build(d, k, C, 1, &lam);
    int32_t *count = (int32_t *)calloc((size_t)k, sizeof(int32_t));
    uint8_t *mark = (uint8_t *)calloc((size_t)k, 1);
    int32_t *cand = (int32_t *)malloc(sizeof(int32_t) * (size_t)k);
    int64_t o = 0;
    cand_ptr[0] = 0;
    for (int64_t i = 0; i < n_docs; ++i) {
        const int32_t nc = oracle_index_query(ix, 0, row_ptr, col, i, count, mark, cand);
        for (int32_t c = 0; c < nc; ++c) { if (o < cap) cand_out[o] = cand[c]; ++o; }
        cand_ptr[i + 1] = o;
    }
    free(count); free(mark); free(cand);
    oracle_index_free(ix);
    return o;
}

/* Build-step check: P_lam entry count per lambda for the given centroids. */
int oracle_index_min_overlaps(int32_t m, const double *v_desc, double lam, int32_t *lin, int32_t *nai) {
    oracle_min_overlap_linear(m, v_desc, lam, lin);
    oracle_min_overlap_naive(m, v_desc, lam, nai);
    for (int32_t p = 0; p < m; ++p) if (lin[p] != nai[p]) return 1;
    return 0;
}

/* ------------------------------------------------------------------------------------
 * Lloyd loop (Sec. 2) with the optional accelerations of Sec. 3.
 *   mode       OR_MODE_PLAIN, OR_MODE_NCC (Sec. 3.1), OR_MODE_INDEX (Sec. 3.2) or
 *              OR_MODE_NCC_INDEX (both, Sec. 3.2 last paragraph).
 *   lam[n_lam] thresholds for the index modes (the paper uses 0.1, 0.25, 0.4, 0.6).
 *   index_min_changed  the index is used in an iteration only when more than this many
 *              clusters changed in the previous update (Sec. 4.3 suggests 100); -1 = always.
 *   shift_tol  stop when max_j ||c_j(new) - c_j(old)||^2 < shift_tol (Sec. 4.1); < 0 off.
 * Loop (R3): for t = 1..max_iter: assign; stop if no assignment changed (t > 1);
 * update; stop if the shift test passes.
 * Outputs: C (d x k, final centroids), a (final assignment), obj[t-1] = objective of
 * assignment t, n_changed_out[t-1] = docs whose assignment changed in step t,
 * sims_out[t-1] = similarities computed in step t (the paper's cost measure).
 * Returns the number of assignment steps performed, or -1 on allocation failure.
 * --------------------------------------------------------------------------------- */
int32_t oracle_fit(int64_t n_docs, const int64_t *row_ptr, const int32_t *col, const float *val,
                   int32_t d, int32_t k, const int32_t *init_ids, int32_t max_iter, double shift_tol,
                   int mode, int n_lam, const double *lam, int32_t index_min_changed,
                   double *C, int32_t *a, double *obj, int64_t *n_changed_out, int64_t *sims_out) {
    const int use_ncc = (mode == OR_MODE_NCC || mode == OR_MODE_NCC_INDEX);
    const int use_index = (mode == OR_MODE_INDEX || mode == OR_MODE_NCC_INDEX) && n_lam > 0;
    oracle_init_centroids(row_ptr, col, val, d, k, init_ids, C);
    int32_t *a_prev = (int32_t *)malloc(sizeof(int32_t) * (size_t)n_docs);
    double *s_prev = (double *)malloc(sizeof(double) * (size_t)n_docs);
    double *s_cur = (double *)malloc(sizeof(double) * (size_t)n_docs);
    uint8_t *changed = (uint8_t *)malloc((size_t)k);
    double *xnorm = (double *)malloc(sizeof(double) * (size_t)n_docs);
    if (!a_prev || !s_prev || !s_cur || !changed || !xnorm) return -1;
    for (int64_t i = 0; i < n_docs; ++i) {
        double ss = 0.0;
        for (int64_t p = row_ptr[i]; p < row_ptr[i + 1]; ++p) ss += (double)val[p] * (double)val[p];
        xnorm[i] = sqrt(ss);
    }
    int32_t n_changed_clusters = k;
    int32_t it = 0;
    for (int32_t t = 1; t <= max_iter; ++t) {
        it = t;
        const int have_prev = (t > 1);
        oracle_index *ix = NULL;
        if (use_index && have_prev &&
            (index_min_changed < 0 || n_changed_clusters > index_min_changed))
            ix = oracle_index_build(d, k, C, n_lam, lam);
        int64_t sims = 0;
#pragma omp parallel reduction(+ : sims)
        {
            double *s = (double *)malloc(sizeof(double) * (size_t)k);
            int32_t *count = (int32_t *)calloc((size_t)k, sizeof(int32_t));
            uint8_t *mark = (uint8_t *)calloc((size_t)k, 1);
            int32_t *cand = (int32_t *)malloc(sizeof(int32_t) * (size_t)k);
#pragma omp for schedule(dynamic, 64)
            for (int64_t i = 0; i < n_docs; ++i) {
                int32_t best = -1;
                double bs = -INFINITY;
                /* Sec. 3.1: a document whose cluster is unchanged is compared only with
                   changed centroids; its stored similarity stands for the rest. */
                const int ncc_skip = use_ncc && have_prev && !changed[a_prev[i]];
                if (ncc_skip) { best = a_prev[i]; bs = s_prev[i]; }
                if (ix) {
                    /* Sec. 3.2: the baseline is the similarity to the previous cluster. */
                    double sb;
                    if (ncc_skip) sb = bs;
                    else { sb = dot_one(row_ptr, col, val, i, C, 0, k, a_prev[i]); ++sims;
                           best = a_prev[i]; bs = sb; }
                    int l = -1;                      /* R4: largest lambda below the baseline */
                    for (int q = 0; q < n_lam; ++q)
                        if (lam[q] * xnorm[i] * (1.0 + 1e-11) < sb && (l < 0 || lam[q] > lam[l])) l = q;
                    if (l >= 0) {
                        const int32_t nc = oracle_index_query(ix, l, row_ptr, col, i, count, mark, cand);
                        for (int32_t c = 0; c < nc; ++c) {
                            const int32_t j = cand[c];
                            if (j == a_prev[i]) continue;
                            if (ncc_skip && !changed[j]) continue;   /* Sec. 3.2: combine with NCC */
                            const double v = dot_one(row_ptr, col, val, i, C, 0, k, j); ++sims;
                            if (v > bs || (v == bs && j < best)) { bs = v; best = j; }
                        }
                        a[i] = best; s_cur[i] = bs;
                        continue;
                    }
                    /* no threshold below the baseline: fall through to a scan */
                }
                if (ncc_skip) {
                    for (int32_t j = 0; j < k; ++j) {
                        if (!changed[j]) continue;
                        const double v = dot_one(row_ptr, col, val, i, C, 0, k, j); ++sims;
                        if (v > bs || (v == bs && j < best)) { bs = v; best = j; }
                    }
                } else {
                    for (int32_t j = 0; j < k; ++j) s[j] = 0.0;
                    for (int64_t p = row_ptr[i]; p < row_ptr[i + 1]; ++p) {
                        const double x = (double)val[p];
                        const double *row = C + (size_t)col[p] * (size_t)k;
                        for (int32_t j = 0; j < k; ++j) s[j] += x * row[j];
                    }
                    sims += k;
                    best = 0; bs = s[0];
                    for (int32_t j = 1; j < k; ++j) if (s[j] > bs) { bs = s[j]; best = j; }
                }
                a[i] = best; s_cur[i] = bs;
            }
            free(s); free(count); free(mark); free(cand);
        }
        if (ix) oracle_index_free(ix);
        double tot = 0.0;
        int64_t nch = 0;
        for (int64_t i = 0; i < n_docs; ++i) {
            tot += s_cur[i];
            nch += (!have_prev || a[i] != a_prev[i]);
        }
        if (obj) obj[t - 1] = tot;
        if (n_changed_out) n_changed_out[t - 1] = nch;
        if (sims_out) sims_out[t - 1] = sims;
        if (have_prev && nch == 0) break;                 /* Sec. 2: assignments unchanged */
        double shift = 0.0;
        n_changed_clusters = oracle_update(n_docs, row_ptr, col, val, d, k, a,
                                           have_prev ? a_prev : NULL, C, changed, &shift, NULL);
        memcpy(a_prev, a, sizeof(int32_t) * (size_t)n_docs);
        memcpy(s_prev, s_cur, sizeof(double) * (size_t)n_docs);
        if (shift_tol >= 0.0 && shift < shift_tol) break;  /* Sec. 4.1 stop rule */
    }
    free(a_prev); free(s_prev); free(s_cur); free(changed); free(xnorm);
    return it;
}

/* ------------------------------------------------------------------------------------
 * k-means++ seeding (Sec. 2 names the k-Means++ strategy as the usual initial assignment;
 * it draws each new seed with probability proportional to the squared distance to the
 * nearest seed drawn so far). For unit vectors ||x - c||^2 = 2 (1 - x . c), so the weight
 * of document i is proportional to dist_i = 1 - max over seeds of x_i . x_seed.
 * Readings (the paper does not spell the procedure out):
 *   K1 seed 0 is document floor(u_0 N); dist_i is computed in double, x_it * x_st summed
 *      over the document's nonzeros in CSR order (products and sums rounded separately;
 *      a product of two floats is exact in double);
 *   K2 the weights are integers w_i = floor(max(dist_i, 0) 2^32), 0 for documents already
 *      drawn; seed r is the smallest i whose inclusive prefix sum of w exceeds
 *      T = min(floor(u_r W), W - 1), W = sum of w; with W = 0 it is the smallest document
 *      not drawn yet.
 * u: k uniforms in [0, 1), the random numbers of the procedure. Returns 0, or -1 when a
 * buffer cannot be allocated.
 * ------------------------------------------------------------------------------------ */
int oracle_kmeanspp(int64_t n_docs, const int64_t *row_ptr, const int32_t *col, const float *val,
                    int32_t d, int32_t k, const double *u, int32_t *ids) {
    double *dist = (double *)malloc(sizeof(double) * (size_t)n_docs);
    double *seed = (double *)calloc((size_t)d, sizeof(double));   /* dense copy of the newest seed */
    unsigned char *drawn = (unsigned char *)calloc((size_t)n_docs, 1);
    if (!dist || !seed || !drawn) {
        free(dist);
        free(seed);
        free(drawn);
        return -1;
    }
    for (int64_t i = 0; i < n_docs; ++i) dist[i] = INFINITY;
    int64_t first = (int64_t)floor(u[0] * (double)n_docs);
    if (first >= n_docs) first = n_docs - 1;
    ids[0] = (int32_t)first;
    drawn[first] = 1;
    for (int32_t r = 1; r < k; ++r) {
        const int64_t s = ids[r - 1];
        for (int64_t p = row_ptr[s]; p < row_ptr[s + 1]; ++p) seed[col[p]] = (double)val[p];
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < n_docs; ++i) {
            double dot = 0.0;
            for (int64_t p = row_ptr[i]; p < row_ptr[i + 1]; ++p) dot += (double)val[p] * seed[col[p]];
            const double dd = 1.0 - dot;
            if (dd < dist[i]) dist[i] = dd;
        }
        for (int64_t p = row_ptr[s]; p < row_ptr[s + 1]; ++p) seed[col[p]] = 0.0;
        uint64_t W = 0;
        for (int64_t i = 0; i < n_docs; ++i)
            if (!drawn[i] && dist[i] > 0.0) W += (uint64_t)floor(dist[i] * 4294967296.0);
        int64_t pick = -1;
        if (W == 0) {
            for (int64_t i = 0; i < n_docs && pick < 0; ++i)
                if (!drawn[i]) pick = i;
        } else {
            uint64_t T = (uint64_t)floor(u[r] * (double)W);
            if (T >= W) T = W - 1;
            uint64_t run = 0;
            for (int64_t i = 0; i < n_docs; ++i) {
                if (!drawn[i] && dist[i] > 0.0) run += (uint64_t)floor(dist[i] * 4294967296.0);
                if (run > T) {
                    pick = i;
                    break;
                }
            }
        }
        ids[r] = (int32_t)pick;
        drawn[pick] = 1;
    }
    free(dist);
    free(seed);
    free(drawn);
    return 0;
}
