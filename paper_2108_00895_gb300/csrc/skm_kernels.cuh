// Argument blocks and launch helpers of the libskm kernels (internal).
#pragma once

#include "skm_internal.cuh"

namespace skm {

// Device counters, one int32 each (reset per step by the host).
enum {
    CNT_PRUNED = 0,   // documents in the pruned class
    CNT_FULL = 1,     // documents in the full class
    CNT_RESCORE = 2,  // documents queued for FP64 rescoring of a candidate list
    CNT_REFULL = 3,   // pruned documents sent back to full scoring
    CNT_FULL64 = 4,   // documents queued for FP64 scoring against all k
    CNT_CHANGED = 5,  // documents whose assignment changed in this step
    CNT_MOVED = 6,    // centroids in the moved list
    CNT_ERR = 7,      // validation error flags (bitmask)
    CNT_COLLECT = 8,  // documents queued for the collect pass
    CNT_N = 9
};
// 64-bit device counters (nonzeros of listed documents, for the work counts).
enum { C64_NNZ_PRUNED = 0, C64_NNZ_REFULL = 1, C64_NNZ_FULL = 2, C64_N = 3 };

struct DecideArgs {
    int32_t n_list;
    const int32_t *doc_list;   // nullable: identity
    int32_t n_slices;
    int32_t n_scored;          // size of the scored set (k, or the moved-list length)
    const float *part_s;
    const int32_t *part_j;
    const int64_t *row_ptr;
    int precision;             // 0 FP32, 1 BF16 (error bound of the scored copy)
    int head_tc;               // 1: scores include a tensor-core head sum (absolute error term)
    float tau;
    int rescore;
    int pruned;                // 1: documents of the pruned class (fold in stored state)
    const int32_t *a_old;      // previous assignment (pruned class)
    int32_t *a_new;
    float *s_state;            // scoring-pass score of the assigned centroid
    float *r_state;            // upper bound on the scoring-pass score of any other centroid
    uint8_t *clean;            // 1: last decision needed no rescoring
    float *score_out;          // nullable
    int32_t *counters;
    unsigned long long *counters64;
    int32_t *rs_doc;           // rescore queue: document ids
    int32_t *rs_cand;          // rescore queue: TOPT candidates each (-1 = none)
    int32_t *refull_doc;
    int32_t *full64_doc;
    int32_t *collect_doc;      // collect queue: document ids
    float *collect_thr;        // collect queue: score threshold (rounded down)
};

struct RescoreArgs {
    const int32_t *count;       // device count of queue entries, or NULL to use n_fixed
    int32_t n_fixed;
    const int32_t *rs_doc;
    const int32_t *rs_cand;     // [queue position][stride] candidate ids (-1 = none)
    int32_t stride;
    const int32_t *cand_cnt;    // nullable: number of candidates per position (collect lists)
    int32_t *full64_doc;        // overflowing collect lists are appended here
    int32_t *full64_count;
    const int64_t *row_ptr;
    const int32_t *col;
    const float *val;
    const float *C32;
    int64_t ldc;
    int32_t *a_new;
    float *score_out;
};

struct Full64Args {
    const int32_t *count;
    const int32_t *docs;
    const int64_t *row_ptr;
    const int32_t *col;
    const float *val;
    const float *C32;
    int64_t ldc;
    int32_t k;
    int32_t *a_new;
    float *score_out;
};

struct PartitionArgs {
    int64_t n_docs;
    const int32_t *order;      // documents are visited in this order
    int prune;
    const uint8_t *clean;
    const uint8_t *changed;
    const int32_t *a_old;
    const int64_t *row_ptr;
    int32_t *counters;
    unsigned long long *counters64;
    int32_t *pruned_list;
    int32_t *full_list;
};

cudaError_t launch_decide(const DecideArgs &a, cudaStream_t st);
cudaError_t launch_rescore64(const RescoreArgs &a, int n_max, cudaStream_t st);
cudaError_t launch_full64(const Full64Args &a, int n_max, cudaStream_t st);
cudaError_t launch_partition(const PartitionArgs &a, cudaStream_t st);

// ---------------------------------------------------------------- update (update.cu)
// Input validation of a CSR collection; sets bits in *err:
//   1 column out of range or not strictly increasing, 2 value negative or not finite,
//   4 empty row, 8 row norm not within 1e-5 of 1, 16 row offsets not within [0, nnz] or
//   decreasing (such a row is not read).
cudaError_t launch_validate(const int64_t *row_ptr, const int32_t *col, const float *val,
                            int64_t n_docs, int64_t nnz, int32_t n_terms, int32_t *err, cudaStream_t st);

// Entries of a rows x cols block of M (row stride ld) that are negative or not finite set bit
// 2 of *err (centroids given from outside).
cudaError_t launch_validate_matrix(const float *M, int64_t ld, int32_t rows, int32_t cols, int32_t *err,
                                   cudaStream_t st);

// order[] = document ids by decreasing number of nonzeros; hist is scratch of 4096 ints.
cudaError_t launch_order_by_length(const int64_t *row_ptr, int64_t n, int32_t *hist, int32_t *order,
                                   cudaStream_t st);

// Term-major transpose (CSC) of the collection: counts per term, then a fill.
cudaError_t launch_term_count(const int32_t *col, int64_t nnz, int32_t *cnt, cudaStream_t st);
cudaError_t launch_csc_fill(const int64_t *row_ptr, const int32_t *col, const float *val,
                            int64_t n_docs, const int64_t *col_ptr, int32_t *fill,
                            int32_t *row_idx, float *cval, int32_t *pterm, cudaStream_t st);

// Initial centroids c_j = x_{ids[j]} (the matrices must be zero beforehand); sq[j] gets
// the squared norm of the stored column.
cudaError_t launch_init_centroids(const int64_t *row_ptr, const int32_t *col, const float *val,
                                  const int32_t *ids, int32_t k, float *C32, __nv_bfloat16 *C16,
                                  int64_t ldc, double *sq, cudaStream_t st);

// Per step: changed-cluster flags from the two assignments, cluster sizes, changed count.
cudaError_t launch_changed(const int32_t *a_new, const int32_t *a_old, int64_t n_docs, int first,
                           uint8_t *changed, int32_t *sizes, int32_t k, int32_t *counters,
                           cudaStream_t st);
// Moved list M (ascending), pos_in_M (-1 if not moved), |M| into counters[CNT_MOVED].
cudaError_t launch_compact_moved(const uint8_t *changed, int32_t k, int32_t *moved,
                                 int32_t *pos_in_m, int32_t *counters, cudaStream_t st);

struct UpdateArgs {
    // light chunks: chunk c covers terms [light_t0[c], light_t1[c]); heavy terms one by one
    int32_t n_light;
    const int32_t *light_t0;
    const int32_t *light_t1;
    int32_t n_heavy;
    const int32_t *heavy_terms;
    const int64_t *col_ptr;
    const int32_t *row_idx;    // document of each posting
    const float *cval;         // value of each posting
    const int32_t *pterm;      // term of each posting
    const int32_t *mdoc;       // per document: moved-list position of its cluster, or -1
    const int32_t *moved;      // M
    int32_t n_moved;
    int F;                     // fixed-point bits: S is in units of 2^-F
    double inv_scale;          // 2^-F
    unsigned long long *normsq128;  // [n_moved][2] norm pass output (units 2^-2F)
    unsigned long long *sq128;      // [n_moved][2] write pass output (units 2^-62)
    const double *inv_norm;    // [n_moved]
    float *C32;
    __nv_bfloat16 *C16;        // nullable (FP32 mode)
    void *CM;                  // nullable: compacted moved matrix (precision of the scored copy)
    // very frequent terms: their postings are split into chunks summed by many blocks into
    // vh_sum[h * n_moved + m] (S of term vh_terms[h], moved position m), which the norm and
    // write passes then read (update_vh_sums before the norm pass)
    int32_t n_vh;
    const int32_t *vh_terms;
    unsigned long long *vh_sum;
    int32_t n_vch;              // chunks: term index vch_h[c], postings [vch_p0[c], vch_p1[c])
    const int32_t *vch_h;
    const int64_t *vch_p0;
    const int64_t *vch_p1;
    uint32_t *tiG;             // nullable: threshold-index bitmap to keep current (bits set
    uint32_t *tiHist;          //   for written nonzeros) and bin counts (one per nonzero)
    int32_t tiW;
    int precision;
    int64_t ldc;
};
// Sums of the very frequent terms (vh_sum zeroed here), before launch_update_norm.
cudaError_t launch_update_vh_sums(const UpdateArgs &u, cudaStream_t st);
cudaError_t launch_update_norm(const UpdateArgs &u, cudaStream_t st);
cudaError_t launch_update_write(const UpdateArgs &u, cudaStream_t st);
int update_chunk_postings();   // most postings of a light chunk
int update_vh_postings();      // terms with more postings than this are split into chunks
int update_vh_chunk();         // postings of one chunk of a split term
// normsq, inv_norm (nullable source normsq128) and newsq (nullable source sq128).
cudaError_t launch_from_u128(const unsigned long long *normsq128, const unsigned long long *sq128, int32_t n,
                             int F, double *normsq, double *inv_norm, double *newsq, cudaStream_t st);
// Zero the recomputed moved columns and fill the compacted matrix (see update.cu).
// Clearing recomputed columns before the write pass (see update.cu): by the postings of the
// flagged clusters' old members, by the seed documents of listed clusters, or all rows of
// listed columns; and the compacted moved matrix (cleared or kept-centroid columns).
// tiG (nullable): threshold-index bitmap with W words a row, whose bits of the cleared
// entries are cleared too.
cudaError_t launch_zero_members(const int32_t *row_idx, const int32_t *pterm, int64_t nnz, const int32_t *a_old,
                                const uint8_t *flag, float *C32, __nv_bfloat16 *C16, int64_t ldc, uint32_t *tiG,
                                int32_t W, cudaStream_t st);
cudaError_t launch_zero_seeds(const int32_t *list, int32_t n, const int32_t *init_ids, const int64_t *row_ptr,
                              const int32_t *col, float *C32, __nv_bfloat16 *C16, int64_t ldc, uint32_t *tiG,
                              int32_t W, cudaStream_t st);
cudaError_t launch_zero_cols(const int32_t *list, int32_t n, int32_t d, float *C32, __nv_bfloat16 *C16, int64_t ldc,
                             uint32_t *tiG, int32_t W, cudaStream_t st);
cudaError_t launch_cm_moved(const int32_t *moved, const int32_t *sizes, int32_t n_moved, int32_t d, const float *C32,
                            void *CM, int precision, int64_t ldc, cudaStream_t st);
cudaError_t launch_mdoc(const int32_t *a, const int32_t *pos_in_m, int64_t n, int32_t *mdoc,
                        cudaStream_t st);
// Per-document FP64 objective terms of moved clusters, summed per cluster in fixed point.
cudaError_t launch_doc_obj(const int64_t *row_ptr, const int32_t *col, const float *val, int64_t n,
                           const int32_t *a, const int32_t *mdoc, const float *C32, int64_t ldc,
                           double scale, unsigned long long *dot_fx, cudaStream_t st);
// Objective and shift of one step (single block, fixed order). See update.cu.
cudaError_t launch_finish(const int32_t *pos_in_m, const int32_t *sizes, int32_t k,
                          const unsigned long long *dot_fx, double inv_dot_scale, const double *normsq,
                          const double *newsq, double *norm_store, double *sq_store, double *obj_out,
                          double *shift_out, cudaStream_t st);
// ---------------------------------------------------------------- threshold index (tindex.cu)
// Sec. 3.2 on the GPU: bitmap G, per-centroid value bins, minimum-overlap bounds and the
// term-major lists P_lambda; see tindex.cu for the layout and the bound.
constexpr int TI_NB = 512;     // value bins per centroid
constexpr int TI_MAXL = 4;     // thresholds (lambda levels)
constexpr int TI_MB = 8;       // m buckets of each term's list
constexpr int TI_PLANES = 8;   // bits of the overlap counts and of the stored m bounds
constexpr int32_t TI_MAX_K = 16384;
__host__ __device__ constexpr int32_t ti_words(int32_t k) { return (k + 31) / 32; }

constexpr uint32_t TI_KEY0 = 1536;   // float bits >> 19 of 2^-31, the lowest bin's lower edge

// Value bin of an entry: 16 bins per octave of |v| (the float bits >> 19), everything below
// 2^-31 in bin 0, everything from 1.9375 up in the last (open) bin.
__device__ __forceinline__ int ti_bin(float v) {
    const int key = (int)(__float_as_uint(fabsf(v)) >> 19) - (int)TI_KEY0;
    return key < 0 ? 0 : (key > TI_NB - 1 ? TI_NB - 1 : key);
}

struct TiThr {
    double v[TI_MAXL];   // lambda_l^2 (1 - 1e-9)
};

struct TiQueryArgs {
    int64_t n_list;
    const int32_t *list;        // nullable: identity
    const int64_t *row_ptr;
    const int32_t *col;
    const float *val;
    const float *C32;
    int64_t ldc;
    int32_t k;
    int32_t W;                  // ti_words(k)
    int32_t d;
    const uint32_t *G;          // [d][W]
    const uint32_t *P;          // [L][nzC]
    int64_t nzC;
    const int64_t *gptr;        // [d + 1] row offsets of G's nonzeros
    const uint32_t *pbe;        // [L][d][TI_MB] bucket ends of each term's list
    int L;
    int max_cands;              // candidate cap (at most TI_CAND); 0: TI_CAND
    double lam[TI_MAXL];        // ascending
    int fixed_level;            // >= 0: candidate dump at this level (no baseline, no scoring)
    uint32_t *cand_out;         // candidate dump: [document][W] bits
    const int32_t *a_old;
    const uint8_t *changed;     // per centroid: moved in the last update
    int ncc;                    // 1: combine with Sec. 3.1
    int prune_fallback;         // 1: unindexed documents may go to the pruned list
    int32_t *a_new;
    float *s_state;
    float *r_state;
    uint8_t *clean;
    float *score_out;           // nullable
    int32_t *counters;
    unsigned long long *counters64;
    int32_t *pruned_list;
    int32_t *full_list;
    unsigned long long *stats;  // nullable: [documents, similarities, P entries walked, products]
};

// Row counts of the bitmap G (popcount of each row's words).
cudaError_t launch_ti_gcnt(const uint32_t *G, int32_t d, int32_t W, uint32_t *gcnt, cudaStream_t st);
// Zero the bin counts of the recomputed centroids of the moved list (sizes[j] > 0).
cudaError_t launch_ti_zero_hist(const int32_t *moved, const int32_t *sizes, int32_t n_moved, uint32_t *hist,
                                cudaStream_t st);
// G, row counts and bin counts of every centroid (hist zeroed by the caller).
cudaError_t launch_ti_rows(const float *C, int64_t ldc, int32_t d, int32_t k, uint32_t *G, uint32_t *gcnt,
                           uint32_t *hist, cudaStream_t st);
// out[0..n] = exclusive prefix sums of in[0..n), out[n] = total; scratch holds
// ti_scan_scratch(n) bytes.
size_t ti_scan_scratch(int64_t n);
cudaError_t launch_ti_scan(const uint32_t *in, int64_t n, int64_t *out, int64_t *scratch, cudaStream_t st);
// m bounds of the listed centroids (list NULL: centroids 0..n-1).
cudaError_t launch_ti_mtab(const uint32_t *hist, const int32_t *list, int32_t n, int32_t k, int L, const TiThr &thr,
                           uint8_t *mtab, cudaStream_t st);
cudaError_t launch_ti_fill(const float *C, int64_t ldc, int32_t d, int32_t k, const uint32_t *G, const uint8_t *mtab,
                           int L, const int64_t *gptr, int64_t nzC, uint32_t *P, uint32_t *pbe, cudaStream_t st);
size_t ti_query_smem(int32_t k);
cudaError_t launch_ti_query(const TiQueryArgs &a, cudaStream_t st);

// Squared norms of the stored FP32 columns.
cudaError_t launch_col_sq(const float *C32, int64_t ldc, int32_t d, int32_t k, double *out,
                          cudaStream_t st);
// FP32 -> BF16 (round to nearest even) of a d x ldc matrix.
cudaError_t launch_to_bf16(const float *C32, __nv_bfloat16 *C16, int64_t n, cudaStream_t st);
// Copy a dense term-major d x k matrix into a padded one (and back).
cudaError_t launch_pad_copy(const float *src, int64_t src_ld, float *dst, int64_t dst_ld,
                            int32_t rows, int32_t cols, cudaStream_t st);

}  // namespace skm
