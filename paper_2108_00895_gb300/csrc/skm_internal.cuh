// Internal declarations shared by the CUDA translation units of libskm.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace skm {

constexpr unsigned FULL = 0xffffffffu;
constexpr int TOPT = 4;   // candidates kept per (document, slice) and per document

// ---------------------------------------------------------------- candidate order
// (s, j) is better than (s', j') when s > s', or s == s' and j < j'
// (argmax ties go to the lowest centroid index).
__device__ __forceinline__ bool better(float s, int j, float s2, int j2) {
    return s > s2 || (s == s2 && j < j2);
}
__device__ __forceinline__ bool better64(double s, int j, double s2, int j2) {
    return s > s2 || (s == s2 && j < j2);
}

// Insert (s, j) into a list kept sorted best-first (length TOPT, registers).
__device__ __forceinline__ void topt_insert(float (&ls)[TOPT], int (&lj)[TOPT], float s, int j) {
    if (!better(s, j, ls[TOPT - 1], lj[TOPT - 1])) return;
    ls[TOPT - 1] = s;
    lj[TOPT - 1] = j;
#pragma unroll
    for (int q = TOPT - 1; q > 0; --q) {
        if (better(ls[q], lj[q], ls[q - 1], lj[q - 1])) {
            float ts = ls[q]; ls[q] = ls[q - 1]; ls[q - 1] = ts;
            int tj = lj[q]; lj[q] = lj[q - 1]; lj[q - 1] = tj;
        }
    }
}

// Keep the best TOPT of two best-first lists a and b (result in a). Bitonic merge with
// static register indices: c[q] = better of a[q] and b[TOPT-1-q] holds the best TOPT as
// a bitonic sequence, which two half-cleaner stages then sort.
__device__ __forceinline__ void topt_merge2(float (&as)[TOPT], int (&aj)[TOPT],
                                            const float (&bs)[TOPT], const int (&bj)[TOPT]) {
    static_assert(TOPT == 4, "bitonic network below is written for 4 entries");
#pragma unroll
    for (int q = 0; q < TOPT; ++q) {
        if (!better(as[q], aj[q], bs[TOPT - 1 - q], bj[TOPT - 1 - q])) {
            as[q] = bs[TOPT - 1 - q];
            aj[q] = bj[TOPT - 1 - q];
        }
    }
#define SKM_CSWAP(x, y)                                                      \
    if (better(as[y], aj[y], as[x], aj[x])) {                                \
        float ts = as[x]; as[x] = as[y]; as[y] = ts;                         \
        int tj = aj[x]; aj[x] = aj[y]; aj[y] = tj;                           \
    }
    SKM_CSWAP(0, 2) SKM_CSWAP(1, 3) SKM_CSWAP(0, 1) SKM_CSWAP(2, 3)
#undef SKM_CSWAP
}

// ---------------------------------------------------------------- bf16 widening
__device__ __forceinline__ float bf16lo(uint32_t w) { return __uint_as_float(w << 16); }
__device__ __forceinline__ float bf16hi(uint32_t w) { return __uint_as_float(w & 0xffff0000u); }

// Read-only, streaming 16-byte load.
__device__ __forceinline__ uint4 ldg16(const void *p) {
    return __ldg(reinterpret_cast<const uint4 *>(p));
}

// ---------------------------------------------------------------- kernel entry points
// Scoring: one warp per (document, slice of KS columns). Writes the slice's best TOPT
// (score, centroid id) to part[(slice * n_list + pos) * TOPT + q].
struct ScoreArgs {
    const int64_t *row_ptr;
    const int32_t *col;
    const float *val;
    const int32_t *doc_list;   // nullable: position pos scores document doc_list[pos]
    int32_t n_list;
    const void *C;             // term-major centroid matrix, row stride ldc elements
    int64_t ldc;
    int32_t ncols;             // valid columns (scores of columns >= ncols are ignored)
    const int32_t *col_ids;    // nullable: column -> centroid id (compacted matrices)
    float *part_s;
    int32_t *part_j;
    // collect mode only: every centroid with score >= thr[pos] is appended to
    // cand[pos * cap + c] (c < cap); cand_cnt[pos] counts them all
    const float *thr;
    int32_t *cand_cnt;
    int32_t *cand;
    int32_t cap;
    // a launch over the list positions [pos0, pos0 + n_list) of a list of n_total positions:
    // doc_list, part, thr, cand_cnt and cand are indexed by the list position (pos0 = 0 and
    // n_total = 0, read as n_list, for the whole list)
    int32_t pos0;
    int32_t n_total;
    // nullable: head sums (tensor-core part of the score, FP16); the accumulators of list
    // position p start from head[(p - pos0) * head_ld + column] instead of zero
    const __half *head;
    int64_t head_ld;
};

// Sparse rows of the scored matrix (see rare.cu): the column stream passed in ScoreArgs.col
// marks a term whose row of C is stored by its nonzeros as ~t < 0; its nonzeros in slice s
// are ent[ptr[t * (n_slices + 1) + s] .. ptr[t * (n_slices + 1) + s + 1]), ascending
// column, each (offset within the slice << 16 | BF16 bits) for BF16 matrices and
// {offset, FP32 bits} for FP32 ones, padded to a 16-byte multiple with entries whose
// offset is the slice width (a spare scratch column) and value 0.
struct SparseArgs {
    const uint32_t *ptr;
    const void *ent;
    int32_t n_slices;
    unsigned long long *skipped;   // nullable: SKIP_COUNTERS partial counts of the
                                   // multiply-adds by exact zeros not executed
};

constexpr int SKIP_COUNTERS = 256;

// Launch helpers (defined in assign.cu). Return cudaSuccess or the launch error.
// sp (nullable): sparse rows of the matrix, with a.col the marked column stream.
cudaError_t launch_score(const ScoreArgs &a, int precision, int slice_cols, cudaStream_t st,
                         const SparseArgs *sp = nullptr);
cudaError_t launch_collect(const ScoreArgs &a, int precision, int slice_cols, cudaStream_t st,
                           const SparseArgs *sp = nullptr);
// cudaFuncAttributes.binaryVersion of the scoring kernel on the current device
cudaError_t score_kernel_version(int *out);
// KS for the scoring kernel, given the mean nonzeros of the documents it will score
int slice_width(int precision, int k, double mean_nnz = 1e9);

// Sparse-row index (defined in rare.cu). M is a term-major d x ldc matrix (FP32 for
// precision 0, BF16 for 1) whose first ncols columns are valid.
// Lists are per slice of ks columns and padded to whole 16-byte vectors (4 BF16 or 2 FP32
// entries) with entries (ks, 0) that address a spare column, so every list starts 16-byte
// aligned.
// rare_count: rowtot[t] = padded list length of row t over the valid columns; with flag
//   set, flag[t] = (nonzeros of row t <= thr) and rowtot[t] is zeroed for the other rows;
//   with only set, rows whose only[t] is 0 get rowtot[t] = 0.
// rare_fill: for every row with flag[t], writes ptr[t * (n_slices + 1) + s] (s = 0..n_slices)
//   from row_base[t] and the row's nonzeros, slice by slice, to ent.
// mark_rare: colm[e] = flag[col[e]] ? ~col[e] : col[e].
cudaError_t launch_rare_count(const void *M, int precision, int64_t ldc, int32_t d, int32_t ncols, int32_t ks,
                              uint32_t thr, const uint8_t *only, uint8_t *flag, uint32_t *rowtot, cudaStream_t st);
cudaError_t launch_rare_fill(const void *M, int precision, int64_t ldc, int32_t d, int32_t ncols, int32_t ks,
                             int32_t n_slices, const uint8_t *flag, const uint32_t *row_base, uint32_t *ptr,
                             void *ent, cudaStream_t st);
cudaError_t launch_mark_rare(const int32_t *col, int64_t nnz, const uint8_t *flag, int32_t *colm, cudaStream_t st);

// k-means++ seeding (defined in init.cu): rounds 1..k-1 given ids[0] on the device, drawn
// (n bytes) zero except drawn[ids[0]] = 1 and seed (d doubles) zero; u: k uniforms on the
// device; dist, w: n entries; csum: kmeanspp_chunks(n) entries. Leaves seed zero.
cudaError_t launch_kmeanspp(int64_t n, int32_t d, int32_t k, const int32_t *order, const int64_t *row_ptr,
                            const int32_t *col, const float *val, const double *u, int32_t *ids, double *dist,
                            unsigned long long *w, unsigned long long *csum, uint8_t *drawn, double *seed,
                            cudaStream_t st);
int kmeanspp_chunks(int64_t n);

}  // namespace skm
