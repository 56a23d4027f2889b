/*
 * skm.h -- exact sparse spherical k-means on one GPU (sm_103a), C ABI.
 *
 * Method: Knittel, Koch, Ertl, "Efficient Sparse Spherical k-Means for Document
 * Clustering", DocEng 2021.
 *   - Sec. 2: documents and centroids are unit vectors; the assignment step gives each
 *     document the centroid of largest dot product (cosine similarity); the update step
 *     sets each centroid to the normalised sum of its members; the loop stops when no
 *     assignment changes (or on another criterion, Sec. 4.1).
 *   - Sec. 3.1 (non-changing clusters): a document whose cluster did not change in the
 *     last update is compared only with the centroids that did change.
 *
 * Conventions shared by every entry point:
 *   - Documents are CSR (skm_csr): row_ptr int64[N+1], col_idx int32[E] strictly
 *     increasing within a row and in [0, n_terms), values float[E] finite and >= 0,
 *     every row non-empty with L2 norm 1 +- 1e-5 (zero vectors are excluded, Sec. 4.1).
 *     Violations return SKM_ERR_INVALID; nothing aborts.
 *   - Centroids are a term-major n_terms x k matrix: entry (t, j) is term t of centroid j.
 *   - Ties in the argmax go to the lowest centroid index.
 *   - Arrays marked "host or device" follow skm_csr.on_device of the same call.
 *     The caller owns every array it passes; the library only borrows it for the call.
 *   - Calls are synchronous: when one returns, its outputs are written. Work is issued
 *     on the stream given in skm_config (NULL = the legacy default stream).
 *   - A context is not thread-safe; serialise calls on one context.
 *   - On any status other than SKM_OK, skm_last_error() describes the failure and the
 *     context stays usable (its centroids are those of the last successful update).
 */
#ifndef SKM_H
#define SKM_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define SKM_API __attribute__((visibility("default")))
#else
#define SKM_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct skm_ctx skm_ctx; /* opaque, owned by the library */

typedef enum {
    SKM_OK = 0,
    SKM_ERR_INVALID = 1, /* bad argument or malformed input */
    SKM_ERR_OOM = 2,     /* a device allocation failed */
    SKM_ERR_BUDGET = 3,  /* the request would exceed skm_config.mem_budget */
    SKM_ERR_CUDA = 4,    /* a CUDA call or kernel launch failed */
    SKM_ERR_STATE = 5,   /* call not valid in the context's state (e.g. no centroids yet) */
    SKM_ERR_TIMEOUT = 6  /* a bounded device wait gave up */
} skm_status;

enum { SKM_FP32 = 0, SKM_BF16 = 1 };          /* centroid storage for the scoring pass */
/* Sec. 3.1 skip off or on; NCC_INDEX adds the threshold index of Sec. 3.2 (skm_fit only) */
enum { SKM_PRUNE_NONE = 0, SKM_PRUNE_NCC = 1, SKM_PRUNE_NCC_INDEX = 2 };

/* Device memory provider. alloc returns NULL on failure; free receives the same size. */
typedef void *(*skm_alloc_fn)(size_t bytes, void *user);
typedef void (*skm_free_fn)(void *ptr, size_t bytes, void *user);

typedef struct {
    int32_t k;            /* clusters, >= 1 */
    int32_t precision;    /* SKM_FP32 or SKM_BF16: type of the centroid copy that is scored.
                             An FP32 master copy is always kept for rescoring and output. */
    int32_t prune;        /* SKM_PRUNE_NONE or SKM_PRUNE_NCC */
    int32_t max_iter;     /* assignment steps per skm_fit, >= 1 */
    double shift_tol;     /* stop when max_j ||c_j(new) - c_j(old)||^2 < shift_tol (Sec. 4.1);
                             < 0 disables the test */
    int32_t rescore;      /* 1: documents whose lower-precision top-2 margin is below the
                             threshold are rescored in FP64 (exact argmax); 0: off */
    double rescore_tau;   /* margin threshold; the library raises it per document to the
                             rounding-error bound of the scoring pass */
    size_t mem_budget;    /* bytes of device memory the context may hold; 0 = no limit */
    int32_t device;       /* CUDA device ordinal */
    void *stream;         /* cudaStream_t to issue work on; NULL = legacy default stream */
    skm_alloc_fn alloc;   /* NULL: cudaMalloc / cudaFree */
    skm_free_fn free;
    void *alloc_user;
    int32_t timing;       /* 1: record CUDA events around each kernel (see skm_stats) */
    int32_t sparse_div;   /* rows of the scored centroid matrix with at most k / sparse_div
                             nonzeros (terms present in few clusters) are stored as lists of
                             their nonzeros, the inverted index of Sec. 3.2, and the scoring
                             pass reads those lists instead of the dense rows. Scores and
                             results are bit-identical either way. 0 = off (the default);
                             used for k >= 64 */
    int32_t index_levels; /* SKM_PRUNE_NCC_INDEX: thresholds in index_lambda, 1..4 */
    double index_lambda[4]; /* minimum dot products of the threshold indexes (Sec. 3.2),
                               ascending, in (0, 1]; default 0.1, 0.25, 0.4, 0.6 (Sec. 4.1).
                               A document whose similarity b to its previous centroid is at
                               least lambda ||x|| for some level is scored only against the
                               candidates of the highest such level (and, when its cluster
                               did not change, only against changed ones, Sec. 3.1); every
                               other centroid has similarity below lambda ||x|| <= b. Results
                               are those of the unindexed loop. Used for k <= 16384, for
                               documents of at most 40 nonzeros with at most
                               index_max_cands candidates; the others are scored densely. */
    int32_t index_min_changed; /* the index serves a step only when more than this many
                                  centroids changed in the previous update (Sec. 4.3
                                  suggests 100, the default); -1: every step after the first */
    int32_t index_max_cands; /* SKM_PRUNE_NCC_INDEX: > 0 (at most 256) turns the index on
                                for fits; a document with more candidates than this is scored
                                densely. 0 (the default): fits run the NCC passes alone,
                                because on the GPUs this library was measured on the dense NCC
                                passes were faster than the index on every workload tried
                                (short documents at k = 5000 to 16384 included).
                                skm_index_candidates uses the index either way. */
    int32_t head_terms;   /* BF16 scoring (k > 256, sparse_div = 0): the products over the
                             collection's most frequent terms (its head, by document
                             frequency, fixed for a fit) run on the tensor cores as a dense
                             matrix product, the other nonzeros on the plain gather path.
                             0 (the default): automatic, the terms in at least 1/64 of the
                             documents, at least 64 and at most 1024 of them; > 0: that many
                             (rounded up to a multiple of 64, at most 2048); -1: off. The
                             decision stays exact either way (the head's rounding error is
                             below the BF16 copy's); scores may differ in the last bits. */
} skm_config;

/* Fills a config with defaults: FP32, no pruning, max_iter 20, shift test off, rescoring
 * on with tau 0, no budget, device 0, default stream, cudaMalloc, sparse rows off, the
 * four index thresholds of Sec. 4.1 with index_min_changed 100, automatic head terms. */
SKM_API void skm_config_default(skm_config *cfg, int32_t k);

typedef struct {
    int64_t n_docs;
    int32_t n_terms;
    int64_t nnz;
    const int64_t *row_ptr; /* [n_docs + 1], row_ptr[0] = 0, row_ptr[n_docs] = nnz */
    const int32_t *col_idx; /* [nnz] */
    const float *values;    /* [nnz] */
    int32_t on_device;      /* 1: the three arrays are device pointers; 0: host pointers */
} skm_csr;

/* Per-call counters (cumulative since the last skm_fit / skm_assign started). */
typedef struct {
    int32_t iters;              /* assignment steps run */
    int64_t sims;               /* similarities computed (the paper's cost measure, Sec. 3) */
    int64_t fmas;               /* algorithmic multiply-adds of the scoring passes */
    int64_t bytes;              /* algorithmic bytes of the scoring passes (CSR + centroid
                                   elements needed, each once, + per-document state) */
    int64_t docs_pruned;        /* document-steps scored only against moved centroids */
    int64_t docs_full;          /* document-steps scored against all k centroids */
    int64_t docs_rescored;      /* document-steps rescored in FP64 from a candidate list */
    int64_t docs_rescored_full; /* document-steps rescored in FP64 against all k */
    int64_t moved_total;        /* sum over steps of the number of moved centroids */
    double ms_score;            /* device time in the scoring kernels (timing = 1) */
    double ms_decide;           /* merge, decision and FP64 rescoring kernels */
    double ms_update;           /* centroid update kernels */
    int64_t launches_score;     /* scoring kernel launches */
    int64_t launches_total;     /* all kernel launches of the library */
    int64_t fmas_exec;          /* multiply-adds executed by the scoring passes: fmas less the
                                   products with exact zeros that sparse rows skip */
    double ms_index;            /* device time building the sparse-row index */
    int64_t sparse_rows;        /* rows of the centroid matrix stored by their nonzeros */
    int64_t sparse_entries;     /* nonzeros stored for them */
    int64_t index_docs;         /* document-steps decided through the threshold index */
    int64_t index_sims;         /* similarities those computed (baseline + candidates, FP64) */
    int64_t index_entries;      /* P_lambda entries they walked */
    int64_t index_products;     /* (term, candidate) products they computed */
    double ms_query;            /* device time in the index query kernel (ms_index also counts
                                   the threshold index builds) */
    int32_t head_terms;         /* head terms scored on the tensor cores (0: none) */
    int64_t nnz_head;           /* nonzeros of the scored collection in those terms */
    double ms_head;             /* device time of the head path outside the scoring kernel:
                                   head set, split of the collection, head matrices and the
                                   tensor-core head sums (ms_score then times the tail) */
} skm_stats;

/* Create a context on cfg->device. cfg is copied. */
SKM_API skm_status skm_create(const skm_config *cfg, skm_ctx **out);

/* Release every device allocation of the context and the context itself. NULL is a no-op. */
SKM_API skm_status skm_destroy(skm_ctx *ctx);

/* Text of the last error on this context ("" if none). Valid until the next call. */
SKM_API const char *skm_last_error(const skm_ctx *ctx);

/*
 * Lloyd loop (Sec. 2), starting from the centroids c_j = x_{init_doc_ids[j]}.
 * Iteration t: assignment step (with the Sec. 3.1 skip when prune = SKM_PRUNE_NCC),
 * then the update step. Stops after max_iter assignment steps, when no assignment
 * changed, or when the shift test passes.
 *   docs          the collection (host or device).
 *   init_doc_ids  host int32[k], distinct ids in [0, n_docs).
 *   assign_out    int32[n_docs] (host or device): final assignment.
 *   objective_out host double[max_iter], nullable: objective sum_i x_i . c_{a_i} of each
 *                 assignment step (against the centroids it was computed with), FP64.
 *   iters_out     host, nullable: assignment steps run.
 * The final centroids stay resident in the context (skm_get_centroids, skm_assign).
 */
SKM_API skm_status skm_fit(skm_ctx *ctx, const skm_csr *docs, const int32_t *init_doc_ids,
                   int32_t *assign_out, double *objective_out, int32_t *iters_out);

/*
 * Assignment step (Sec. 2) of new documents against the resident centroids. Every
 * document is scored against all k centroids (there is no previous assignment to
 * prune with), then near ties are rescored in FP64 when cfg.rescore = 1.
 *   assign_out int32[n_docs] (host or device).
 *   score_out  float[n_docs] (host or device), nullable: similarity of the chosen centroid
 *              (the FP64 value where the document was rescored).
 */
SKM_API skm_status skm_assign(skm_ctx *ctx, const skm_csr *docs, int32_t *assign_out, float *score_out);

/*
 * Update step (Sec. 2): every cluster with members gets c_j = S_j / ||S_j||, S_j the sum
 * of its member documents; a cluster without members keeps its centroid.
 *   assign        int32[n_docs] (host or device), values in [0, k).
 *   n_changed_out host, nullable: number of recomputed centroids.
 */
SKM_API skm_status skm_update(skm_ctx *ctx, const skm_csr *docs, const int32_t *assign,
                      int32_t *n_changed_out);

/* k-means++ seeding of k = skm_config.k initial documents for skm_fit (Sec. 2 names the
 * k-Means++ strategy as the usual initial assignment). Each seed is drawn with probability
 * proportional to the squared distance to the nearest seed drawn so far, which for unit
 * vectors is 2 (1 - x . seed):
 *   seed 0 is document floor(uniforms[0] * n_docs);
 *   seed r >= 1 is the smallest document whose inclusive prefix sum (document order) of the
 *   integer weights w_i = floor(max(1 - max over seeds of x_i . seed, 0) * 2^32) (0 for
 *   documents already drawn) exceeds min(floor(uniforms[r] * W), W - 1), W = sum of the
 *   weights; when W = 0 it is the smallest document not drawn yet.
 * The distances are computed in double, 1 - x . seed with the products (exact for two
 * floats) added one at a time in the document's CSR order, so the seeds depend only on the
 * documents and the uniforms.
 * docs:      as for skm_fit (validated, staged when on the host).
 * uniforms:  k host doubles in [0, 1), the procedure's random numbers (caller-owned).
 * ids_out:   k int32 document ids (distinct): device memory if docs->on_device, host otherwise.
 * Errors: SKM_ERR_INVALID (a uniform outside [0, 1), k > n_docs, NULL buffers or invalid
 * documents), SKM_ERR_OOM / SKM_ERR_BUDGET (work buffers: 17 bytes per document, 8 per
 * term), SKM_ERR_CUDA. */
SKM_API skm_status skm_init_kmeanspp(skm_ctx *ctx, const skm_csr *docs, const double *uniforms,
                                     int32_t *ids_out);

/*
 * Candidate sets of the threshold index (Sec. 3.2) of the resident centroids at threshold
 * index_lambda[level], for checking the index: no baseline, no Sec. 3.1 filter.
 * Centroid j is a candidate of document i when, for some term t of the document whose entry
 * c_jt is in P_lambda with minimum overlap count m (a lower bound of the paper's count,
 * clamped to 255), the document shares at least min(m, 255) terms with centroid j. Every
 * centroid with x_i . c_j >= lambda ||x_i|| is a candidate (Lemma 3.1), and so is every
 * candidate of the paper's exact construction. Documents with more than 40 nonzeros are
 * not indexed (skm_fit scores them densely): every centroid is reported for them.
 * docs:  as for skm_assign (n_terms = the resident vocabulary).
 * bits:  host uint32[n_docs * ceil(k / 32)]; bit b of bits[i * ceil(k / 32) + w] is set when
 *        centroid 32 w + b is a candidate of document i.
 * Errors: SKM_ERR_STATE (no resident centroids), SKM_ERR_INVALID (level outside
 * [0, index_levels), k > 16384, NULL bits, invalid documents), SKM_ERR_OOM / SKM_ERR_BUDGET
 * (the index: 4 bytes per term per 32 centroids, 4 bytes per nonzero of the centroid matrix
 * per level, 2.5 KB per centroid and 512 bytes per centroid per level), SKM_ERR_CUDA. */
SKM_API skm_status skm_index_candidates(skm_ctx *ctx, const skm_csr *docs, int32_t level, uint32_t *bits);

/* Replace the resident centroids with a host or device float[n_terms * k] matrix
 * (term-major). The lower-precision copy is re-derived (round to nearest even). Every entry
 * must be finite and non-negative (the method's centroids are normalised sums of non-negative
 * documents, and the scoring pass's decision rule relies on non-negative products): otherwise
 * SKM_ERR_INVALID, and the context is left without resident centroids (skm_assign then
 * returns SKM_ERR_STATE until centroids are set or fitted again). */
SKM_API skm_status skm_set_centroids(skm_ctx *ctx, int32_t n_terms, const float *centroids,
                             int32_t on_device);

/* Copy the resident FP32 centroids (term-major n_terms x k) to host or device memory. */
SKM_API skm_status skm_get_centroids(skm_ctx *ctx, float *centroids_out, int32_t on_device);

/* Resident vocabulary size (0 before the first fit / set). */
SKM_API int32_t skm_n_terms(const skm_ctx *ctx);

/* Counters of the last skm_fit / skm_assign. */
SKM_API skm_status skm_get_stats(const skm_ctx *ctx, skm_stats *out);

/* Device bytes currently held by the context. */
SKM_API size_t skm_mem_used(const skm_ctx *ctx);

/* The GPU architecture the library's kernels were compiled for, as the CUDA runtime reports
 * it for the scoring kernel on the current device (cudaFuncAttributes.binaryVersion, major *
 * 10 + minor: 103 for sm_103a). Needs a CUDA device; SKM_ERR_CUDA otherwise (for example when
 * the device cannot run the library's code), SKM_ERR_INVALID for a NULL out. No counterpart
 * in the paper: a check of the build. */
SKM_API skm_status skm_device_code_version(int32_t *out);

/* ------------------------------------------------------------------------------------
 * Batched form: many independent clustering instances of different sizes in one call.
 * Each instance runs the plain Lloyd loop of Sec. 2 (assignment against all k FP32
 * centroids with FP64 rescoring of near ties, then the update of the clusters whose
 * membership changed) for exactly max_iter assignment steps; an instance that converges
 * earlier keeps its assignment and centroids. All instances advance together: every phase of
 * an iteration is one launch over all of them (the scoring pass is a persistent kernel over
 * one queue of tiles), and the loop is captured once in a CUDA graph when use_graph = 1.
 * ---------------------------------------------------------------------------------- */
typedef struct {
    skm_csr docs;                 /* the instance's documents, host or device */
    int32_t k;                    /* clusters, 1 <= k <= min(n_docs, 2048) */
    const int32_t *init_doc_ids;  /* host int32[k], distinct: c_j = x_{init_doc_ids[j]} */
    int32_t *assign_out;          /* int32[n_docs], host or device (as docs.on_device) */
    double *objective_out;        /* host double[max_iter], nullable: objective of each step */
} skm_batch_item;

typedef struct {
    int32_t max_iter;             /* assignment steps of every instance, >= 1 */
    int32_t rescore;              /* 1: FP64 rescoring of near ties (exact argmax) */
    double rescore_tau;           /* minimum margin threshold (raised to the error bound) */
    int32_t device;
    void *stream;                 /* cudaStream_t; NULL = legacy default stream */
    skm_alloc_fn alloc;           /* NULL: cudaMalloc / cudaFree; all memory is freed on return */
    skm_free_fn free;
    void *alloc_user;
    const char *tune_cache;       /* autotuner cache file (read and updated), NULL = none */
    int32_t use_graph;            /* 1: capture the iteration loop in a CUDA graph */
} skm_batch_config;

typedef struct {
    double ms_total;              /* wall time of the call */
    double ms_setup;              /* validation, transposes, autotuning, tables */
    double ms_loop;               /* device time of the iteration loop (CUDA events) */
    int64_t fmas;                 /* algorithmic multiply-adds of all scoring passes */
    int64_t tiles;                /* scoring tiles per iteration */
    int64_t graph_nodes;          /* nodes of the captured graph (0 without a graph) */
    int64_t device_bytes;         /* device memory used */
    int32_t tuned;                /* instances timed by the autotuner (cache misses) */
    int32_t shape_instances[5];   /* instances per scoring shape: lane16, lane32, 128, 256, 512 */
    char message[256];            /* reason of a failure, "" on success */
} skm_batch_stats;

/* Runs every item to max_iter assignment steps. Synchronous. stats is nullable. Errors:
 * SKM_ERR_INVALID (bad config or item), SKM_ERR_OOM, SKM_ERR_CUDA; stats->message says why. */
SKM_API skm_status skm_fit_batched(const skm_batch_config *cfg, const skm_batch_item *items, int32_t n_items,
                                   skm_batch_stats *stats);

/* ------------------------------------------------------------------------------------
 * Serving form. A server answers assignment requests against a resident context (its
 * centroids, set by skm_fit or skm_set_centroids, stay on the device) by continuous batching:
 * every request waiting when the previous batch finishes joins the next batch (up to
 * max_batch_docs documents and max_batch_nnz nonzeros), which runs as one assignment step.
 * Clustering jobs run beside it on n_job_slots worker threads, each on a context and stream of
 * its own, so batches and jobs overlap on the device. A job is started when its memory
 * estimate fits the budget left by the resident context and the running jobs (the first
 * waiting job that fits goes first); a job that could never fit is rejected at submission.
 * Results do not depend on what else is running. Requests borrow the caller's host arrays:
 * they must stay valid until skm_server_release. Thread-safe; the resident context must not be
 * used by the caller while the server exists.
 * ---------------------------------------------------------------------------------- */
typedef struct skm_server skm_server;

typedef struct {
    int32_t device;
    size_t mem_budget;            /* device bytes for the resident context and all jobs */
    int32_t n_job_slots;          /* clustering jobs that may run at once (>= 0) */
    int64_t max_batch_docs;       /* documents per assignment batch (and per request) */
    int64_t max_batch_nnz;        /* nonzeros per assignment batch (a larger request runs alone) */
    int32_t job_precision;        /* SKM_FP32 / SKM_BF16 for clustering jobs */
    int32_t job_prune;            /* SKM_PRUNE_NONE / SKM_PRUNE_NCC for clustering jobs */
    double rescore_tau;           /* rescoring threshold of clustering jobs */
} skm_server_config;

enum { SKM_REQ_QUEUED = 0, SKM_REQ_RUNNING = 1, SKM_REQ_DONE = 2, SKM_REQ_REJECTED = 3, SKM_REQ_FAILED = 4,
       SKM_REQ_CANCELLED = 5 };

typedef struct {
    int32_t state;                /* SKM_REQ_* */
    skm_status status;            /* of the finished request */
    int64_t n_docs;
    const int32_t *assign;        /* int32[n_docs], owned by the server until release */
    const float *score;           /* assignment requests: similarity of the chosen centroid */
    const double *objective;      /* clustering jobs: objective per assignment step */
    int32_t iters;                /* clustering jobs: assignment steps run */
    double latency_ms;            /* submission to completion */
    double queue_ms;              /* submission to start */
    int32_t batch_docs;           /* assignment requests: documents in the batch it ran in */
    char message[256];
} skm_server_result;

typedef struct {
    int64_t assign_submitted, assign_done, fit_submitted, fit_done, rejected, failed;
    int64_t assign_batches, max_batch_docs_seen, docs_assigned, docs_clustered;
    int64_t assign_queued, fit_queued;
    int32_t jobs_running, peak_jobs_running;
    size_t jobs_mem, resident_mem;
} skm_server_stats;

/* Start a server on a resident context. SKM_ERR_BUDGET if the resident context and a largest
 * batch do not fit mem_budget. */
SKM_API skm_status skm_server_create(const skm_server_config *cfg, skm_ctx *resident, skm_server **out);
/* Queue an assignment request (host CSR with the resident vocabulary, at most max_batch_docs
 * documents). Returns at once with a ticket. */
SKM_API skm_status skm_server_submit_assign(skm_server *srv, const skm_csr *docs, uint64_t *ticket);
/* Queue a clustering job: skm_fit of host CSR docs with k clusters from init_doc_ids (copied),
 * max_iter assignment steps. Returns at once with a ticket. */
SKM_API skm_status skm_server_submit_fit(skm_server *srv, const skm_csr *docs, int32_t k,
                                         const int32_t *init_doc_ids, int32_t max_iter, uint64_t *ticket);
/* Wait up to timeout_ms (< 0: no limit) for a request; SKM_ERR_TIMEOUT if it is not finished.
 * The result's arrays stay valid until skm_server_release. */
SKM_API skm_status skm_server_wait(skm_server *srv, uint64_t ticket, double timeout_ms, skm_server_result *res);
/* Free a finished request's results. */
SKM_API skm_status skm_server_release(skm_server *srv, uint64_t ticket);
SKM_API skm_status skm_server_get_stats(skm_server *srv, skm_server_stats *out);
/* Cancel waiting requests, let running ones finish, stop the workers and free the server. */
SKM_API skm_status skm_server_destroy(skm_server *srv);

/*
 * Assignment step that allocates no device memory. The paper has no counterpart: this is a
 * service of the library for callers that cannot let a library allocate -- callers whose
 * device memory is owned by another allocator (a framework's pool, or a fixed per-process
 * budget), or that must not trigger an allocation (which can synchronise the device) where
 * they call. Every input and output comes from the caller; the only scratch (per-slice
 * candidate lists and validation flags) is one fixed 32 MiB device array inside the library,
 * which every GPU that loads the library holds until the process exits. No cudaMalloc,
 * cudaFree or allocating library routine is called.
 *
 * Result: for each document the centroid of largest FP32 similarity (nonzeros summed in CSR
 * order with fused multiply-adds), ties to the lowest index -- what skm_assign returns for an
 * FP32 context with rescore = 0.
 *   docs        device CSR (on_device must be 1), checked as in skm_assign.
 *   k           number of centroids, >= 1.
 *   centroids   device float[n_terms * ld], term-major, 16-byte aligned: entry (t, j) is
 *               centroids[t * ld + j]; ld >= k and a multiple of 256 (columns k..ld-1 are
 *               read and ignored). The used entries must be finite and non-negative, as for
 *               skm_set_centroids; each call checks them on the device (one read of the
 *               n_terms x k block).
 *   assign_out  device int32[n_docs]; score_out device float[n_docs] (the FP32 similarity of
 *               the chosen centroid) or NULL.
 *   stream      cudaStream_t to run on (NULL = legacy default stream); the call returns after
 *               its work on the stream has finished.
 * Limit: n_docs * ceil(k / 256) <= 1,048,568 (32 bytes of scratch per document and 256-column
 * slice); a larger request returns SKM_ERR_BUDGET before any GPU work.
 * Errors: SKM_ERR_INVALID for bad arguments, documents or centroids, SKM_ERR_CUDA for a CUDA
 * failure. Every call looks up the scratch array's device address on the current device and
 * copies the validation flags back to the host, then synchronises the stream before it returns:
 * it must not be called while that stream is being captured into a CUDA graph.
 * All calls share the one scratch array, which keeps the last call's contents: calls that
 * overlap on the GPU (from several streams or threads) race, so the caller must serialise them.
 */
SKM_API skm_status skm_assign_fixed_scratch(const skm_csr *docs, int32_t k, const float *centroids,
                                            int64_t ld, int32_t *assign_out, float *score_out,
                                            void *stream);

#ifdef __cplusplus
}
#endif
#endif /* SKM_H */
