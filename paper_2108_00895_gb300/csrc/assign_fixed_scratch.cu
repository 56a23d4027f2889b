// skm_assign_fixed_scratch: the assignment step with no device allocation at all.
//
// Some callers cannot let a library call cudaMalloc: their device memory is owned entirely by
// another allocator (a framework's memory pool, or a process with a fixed device-memory
// budget), or they must not trigger an allocation, which may synchronise the device, in the
// middle of latency-sensitive work. For them this entry point takes every input and output
// from the caller and keeps its only scratch -- the per-slice candidate lists of the scoring
// pass and a few counters -- in one file-scope device array of fixed size. That array is part
// of the library image: every GPU that loads the library holds it until the process exits.
//
// The computation is the FP32 scoring pass of skm_assign with rescoring off: for each document
// the centroid of largest FP32 similarity (nonzeros accumulated in CSR order with fused
// multiply-adds), ties to the lowest index.
#include <cuda_runtime.h>

#include "skm.h"
#include "skm_kernels.cuh"

namespace {

constexpr size_t kScratchBytes = size_t(32) << 20;   // 32 MiB
constexpr size_t kCounterBytes = 256;                 // validation flags, kept first
constexpr int kSlice = 256;                           // FP32 scoring slice (columns)

// The scratch. In host code `g_scratch` names a host-side stand-in, not device memory: its
// device address comes from cudaGetSymbolAddress with the device current.
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

// Device address of g_scratch on the current device. It is looked up on every call (cheap
// after the first on a device), so a module reloaded after cudaDeviceReset is not addressed
// through a stale pointer.
cudaError_t scratch_address(void **out) {
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess) return e;
    *out = p;
    return cudaSuccess;
}

// One thread per document: merge the per-slice candidate lists, keep the best (ties to the
// lowest index), write the assignment and its FP32 similarity.
__global__ void k_merge_best(int32_t n, int32_t n_slices, const float *part_s, const int32_t *part_j,
                             int32_t *assign_out, float *score_out) {
    const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float bs = -INFINITY;
    int bj = INT32_MAX;
    for (int sl = 0; sl < n_slices; ++sl) {
        const int64_t o = ((int64_t)sl * n + i) * skm::TOPT;   // entry 0 is the slice's best
        const float s = part_s[o];
        const int j = part_j[o];
        if (skm::better(s, j, bs, bj)) {
            bs = s;
            bj = j;
        }
    }
    assign_out[i] = bj;
    if (score_out) score_out[i] = bs;
}

}  // namespace

extern "C" SKM_API skm_status skm_assign_fixed_scratch(const skm_csr *docs, int32_t k, const float *centroids,
                                                       int64_t ld, int32_t *assign_out, float *score_out,
                                                       void *stream) {
    if (!docs || !centroids || !assign_out || k < 1 || docs->on_device != 1 || docs->n_docs < 1 ||
        docs->n_terms < 1 || docs->nnz < docs->n_docs || !docs->row_ptr || !docs->col_idx || !docs->values)
        return SKM_ERR_INVALID;
    if (ld < k || ld % kSlice != 0 || (reinterpret_cast<uintptr_t>(centroids) & 15) != 0)
        return SKM_ERR_INVALID;
    if (docs->n_docs > INT32_MAX - 1) return SKM_ERR_BUDGET;
    const int64_t n = docs->n_docs;
    const int64_t n_slices = (k + kSlice - 1) / kSlice;
    const size_t part_bytes = (size_t)n * (size_t)n_slices * skm::TOPT * (sizeof(float) + sizeof(int32_t));
    if (part_bytes > kScratchBytes - kCounterBytes) return SKM_ERR_BUDGET;

    cudaStream_t st = (cudaStream_t)stream;
    void *base = nullptr;
    if (scratch_address(&base) != cudaSuccess) return SKM_ERR_CUDA;
    unsigned char *scr = static_cast<unsigned char *>(base);
    int32_t *flags = reinterpret_cast<int32_t *>(scr);
    float *part_s = reinterpret_cast<float *>(scr + kCounterBytes);
    int32_t *part_j = reinterpret_cast<int32_t *>(part_s + (size_t)n * n_slices * skm::TOPT);

    // row_ptr bounds, then the same device validation as the other entry points: documents
    // (flags[0]) and centroids, which must be finite and non-negative as skm_set_centroids
    // requires (flags[1]; the k used columns of each of the n_terms rows)
    int64_t ends[2] = {-1, -1};
    if (cudaMemcpyAsync(&ends[0], docs->row_ptr, sizeof(int64_t), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaMemcpyAsync(&ends[1], docs->row_ptr + n, sizeof(int64_t), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaMemsetAsync(flags, 0, kCounterBytes, st) != cudaSuccess)
        return SKM_ERR_CUDA;
    if (skm::launch_validate(docs->row_ptr, docs->col_idx, docs->values, n, docs->nnz, docs->n_terms, flags, st) !=
            cudaSuccess ||
        skm::launch_validate_matrix(centroids, ld, docs->n_terms, k, flags + 1, st) != cudaSuccess)
        return SKM_ERR_CUDA;
    int32_t err[2] = {0, 0};
    if (cudaMemcpyAsync(err, flags, sizeof err, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return SKM_ERR_CUDA;
    if (ends[0] != 0 || ends[1] != docs->nnz || err[0] != 0 || err[1] != 0) return SKM_ERR_INVALID;

    skm::ScoreArgs sa{};
    sa.row_ptr = docs->row_ptr;
    sa.col = docs->col_idx;
    sa.val = docs->values;
    sa.doc_list = nullptr;
    sa.n_list = (int32_t)n;
    sa.C = centroids;
    sa.ldc = ld;
    sa.ncols = k;
    sa.col_ids = nullptr;
    sa.part_s = part_s;
    sa.part_j = part_j;
    if (skm::launch_score(sa, SKM_FP32, kSlice, st) != cudaSuccess) return SKM_ERR_CUDA;
    k_merge_best<<<(unsigned)((n + 255) / 256), 256, 0, st>>>((int32_t)n, (int32_t)n_slices, part_s, part_j,
                                                              assign_out, score_out);
    if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(st) != cudaSuccess) return SKM_ERR_CUDA;
    return SKM_OK;
}
