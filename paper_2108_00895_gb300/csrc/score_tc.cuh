// Scoring pass with the head terms on the tensor cores (internal; see score_tc.cu).
#pragma once

#include <cuda.h>
#include <cuda_fp16.h>

#include "skm_internal.cuh"

namespace skm {

constexpr int TC_SLICE = 512;          // BF16 scoring slice that the head path serves
constexpr int TC_HEAD_MAX = 2048;      // most head terms (multiple of 64)
constexpr int TC_HEAD_AUTO = 1024;     // most head terms chosen automatically
constexpr float TC_SCALE = 1024.0f;    // both FP16 operands are stored times 2^10

struct HeadGemmArgs {
    const int64_t *hptr;       // head entries of document i: hent[hptr[i] .. hptr[i + 1]),
    const uint32_t *hent;      // ascending head position, (position << 16) | FP16 bits of x 2^10
    const int32_t *doc_list;   // nullable: list position p is document doc_list[p]
    int32_t pos0;              // the launch covers list positions [pos0, pos0 + n)
    int32_t n;
    int32_t h;                 // head terms, a multiple of 64
    int32_t n_cblk;            // 256-column blocks to compute (the head matrix has 256 n_cblk rows)
    __half *out;               // out[(p - pos0) * ld + c]: head sum of position p, column c (FP16)
    int64_t ld;                // >= 256 n_cblk
    int32_t *err;              // bit 32 set when a bounded wait gave up
};

// Tensor map (TMA) of a head matrix: rows x h FP16, K-major (h contiguous), boxes of 64 head
// terms x box_rows rows (128 or 256) with the 128-byte swizzle. h must be a multiple of 64,
// rows at least box_rows, the base 16-byte aligned.
cudaError_t tc_make_map(const __half *headT, int32_t h, int64_t rows, int32_t box_rows, CUtensorMap *out);

// Dense FP16 head rows X[p][0..h) of the listed documents [pos0, pos0 + n) for p < rows
// (rows >= n zero): the document operand of the head product (k_head_rows).
cudaError_t launch_head_rows(const HeadGemmArgs &a, int32_t rows, __half *X, cudaStream_t st);
// Head sums of the listed documents [pos0, pos0 + n) for 256 n_cblk columns (k_head_gemm):
// amap is the TMA map of their head rows (tc_make_map over X with 128-row boxes), bmap that
// of the centroid head matrix (256-row boxes).
cudaError_t launch_head_gemm(const HeadGemmArgs &a, const CUtensorMap &amap, const CUtensorMap &bmap,
                             cudaStream_t st);

// Head and tail split of a CSR collection: hcnt[i] = head entries of row i (head_pos[t] >= 0),
// tcnt[i] = the rest.
cudaError_t launch_split_count(const int64_t *row_ptr, const int32_t *col, int64_t n, const int32_t *head_pos,
                               uint32_t *hcnt, uint32_t *tcnt, cudaStream_t st);
// Fill: hent from the head entries (position << 16 | FP16(x 2^10)), tcol/tval from the rest,
// both in CSR order, at the offsets hptr / tptr.
cudaError_t launch_split_fill(const int64_t *row_ptr, const int32_t *col, const float *val, int64_t n,
                              const int32_t *head_pos, const int64_t *hptr, const int64_t *tptr, uint32_t *hent,
                              int32_t *tcol, float *tval, cudaStream_t st);
// headT[r * h + q] = FP16(2^10 C32[H[q], col(r)]) for r < ncols (col(r) = cols[r], or r when
// cols is NULL), 0 for ncols <= r < rows.
cudaError_t launch_head_matrix(const float *C32, int64_t ldc, const int32_t *H, int32_t h, const int32_t *cols,
                               int32_t ncols, int64_t rows, __half *headT, cudaStream_t st);

}  // namespace skm
