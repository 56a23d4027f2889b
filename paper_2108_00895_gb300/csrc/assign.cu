// Assignment step kernels (Sec. 2 of the paper) with the non-changing-clusters skip
// (Sec. 3.1) and FP64 rescoring of near ties.
//
// Scoring pass: s_ij = sum over the document's nonzeros t, in CSR order, of x_it * C[t, j],
// one FP32 fused multiply-add per nonzero per centroid. The chain for a given (i, j) is the
// same whichever launch computes it (full matrix or compacted moved-centroid matrix), so a
// score is a pure function of (x_i, c_j): the pruned and the full pass agree bit for bit.
#include "skm_device.cuh"
#include "skm_internal.cuh"
#include "skm_kernels.cuh"

namespace skm {

// ------------------------------------------------------------------------------------
// k_score: one warp per (document, slice). Lane l owns, for u in [0, NV), the EPV columns
// starting at slice*KS + u*32*EPV + l*EPV, so each of the NV 16-byte loads of a centroid
// row segment is one coalesced 512-byte warp access. The document's (t, x) pairs are read
// 32 at a time and broadcast by shuffle.
// ------------------------------------------------------------------------------------
template <typename CT, int NV, bool COLLECT>
__device__ __forceinline__ void score_slice(const ScoreArgs &a) {
    constexpr int EPV = 16 / (int)sizeof(CT);   // elements per 16-byte vector
    constexpr int J = NV * EPV;                  // columns per lane
    constexpr int KS = 32 * J;                   // columns per slice
    __shared__ int2 stage[8][32];                // per warp: 32 (t, x) pairs
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const int pos = blockIdx.x * 8 + wib;
    if (pos >= a.n_list) return;
    const int gpos = a.pos0 + pos;
    const int n_total = a.n_total > 0 ? a.n_total : a.n_list;
    const int slice = blockIdx.y;
    const int64_t i = a.doc_list ? (int64_t)a.doc_list[gpos] : (int64_t)gpos;
    const int64_t j0 = (int64_t)slice * KS;
    float2 acc[J / 2];
    const CT *Cs = reinterpret_cast<const CT *>(a.C) + j0 + lane * EPV;
    if (a.head) {
        // the tail nonzeros continue the chain from the tensor-core head sums (FP16)
        const __half2 *hs = reinterpret_cast<const __half2 *>(a.head + (int64_t)pos * a.head_ld + j0 + lane * EPV);
#pragma unroll
        for (int u = 0; u < NV; ++u)
#pragma unroll
            for (int q = 0; q < EPV / 2; ++q) acc[u * EPV / 2 + q] = __half22float2(hs[u * 16 * EPV + q]);
        slice_accumulate_add<CT, NV>(a.row_ptr[i], a.row_ptr[i + 1], a.col, a.val, Cs, a.ldc, stage[wib], lane, acc);
    } else {
        slice_accumulate<CT, NV>(a.row_ptr[i], a.row_ptr[i + 1], a.col, a.val, Cs, a.ldc, stage[wib], lane, acc);
    }
    if constexpr (COLLECT) {
        slice_collect<CT, NV>(acc, j0, lane, a.ncols, a.col_ids, a.thr[gpos], a.cand_cnt + gpos,
                              a.cand + (int64_t)gpos * a.cap, a.cap);
    } else {
        slice_topt_write<CT, NV>(acc, j0, lane, a.ncols, a.col_ids, a.part_s, a.part_j,
                                 ((int64_t)slice * n_total + gpos) * TOPT);
    }
}

template <typename CT, int NV, bool COLLECT>
__global__ void __launch_bounds__(256) k_score(ScoreArgs a) {
    score_slice<CT, NV, COLLECT>(a);
}

// The FP32 shape with 512-column slices (short documents), compiled for four resident blocks
// (64 registers a thread): with that budget the compiler schedules the row gathers better
// than with its own choice (scoring of a tweets-like job 349 against 363 ms); the other
// shapes are faster with the compiler's choice.
template <bool COLLECT>
__global__ void __launch_bounds__(256, 4) k_score_f32w(ScoreArgs a) {
    score_slice<float, 4, COLLECT>(a);
}

// k_score with sparse rows: a KS-float scratch and a list staging buffer per warp (dynamic
// shared memory); registers are capped so that four blocks stay resident, as for k_score.
template <typename CT, int NV, bool COLLECT>
__global__ void __launch_bounds__(256, 4) k_score_sparse(ScoreArgs a, SparseArgs sp) {
    constexpr int EPV = 16 / (int)sizeof(CT);   // elements per 16-byte vector
    constexpr int J = NV * EPV;                  // columns per lane
    constexpr int KS = 32 * J;                   // columns per slice
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const int pos = blockIdx.x * 8 + wib;
    if (pos >= a.n_list) return;
    const int gpos = a.pos0 + pos;
    const int n_total = a.n_total > 0 ? a.n_total : a.n_list;
    const int slice = blockIdx.y;
    const int64_t i = a.doc_list ? (int64_t)a.doc_list[gpos] : (int64_t)gpos;
    const int64_t j0 = (int64_t)slice * KS;
    const CT *Cs = reinterpret_cast<const CT *>(a.C) + j0 + lane * EPV;
    __shared__ int2 stage[8][32];
    extern __shared__ float4 scratch4[];
    float2 acc[J / 2];
    if (a.head) {
        // the tail nonzeros continue the chain from the tensor-core head sums (FP16)
        const __half2 *hs = reinterpret_cast<const __half2 *>(a.head + (int64_t)pos * a.head_ld + j0 + lane * EPV);
#pragma unroll
        for (int u = 0; u < NV; ++u)
#pragma unroll
            for (int q = 0; q < EPV / 2; ++q) acc[u * EPV / 2 + q] = __half22float2(hs[u * 16 * EPV + q]);
    }
    {
        RareSlice rs;
        rs.ptr = sp.ptr;
        rs.ent = sp.ent;
        rs.n_slices = sp.n_slices;
        rs.slice = slice;
        rs.cols = (int)min((int64_t)KS, (int64_t)a.ncols - j0);
        rs.sacc = reinterpret_cast<float *>(scratch4) + wib * (KS + RARE_SPARE);
        rs.stg = reinterpret_cast<char *>(scratch4) + sizeof(float) * 8 * (KS + RARE_SPARE) + wib * RARE_STAGE_BYTES;
        slice_accumulate_sparse<CT, NV>(a.row_ptr[i], a.row_ptr[i + 1], a.col, a.val, Cs, a.ldc, stage[wib], lane,
                                        acc, rs, a.head == nullptr);
        if (sp.skipped && rs.skipped && lane == 0)
            atomicAdd(sp.skipped + ((pos + slice) & (SKIP_COUNTERS - 1)), rs.skipped);
    }
    if constexpr (COLLECT) {
        slice_collect<CT, NV>(acc, j0, lane, a.ncols, a.col_ids, a.thr[gpos], a.cand_cnt + gpos,
                              a.cand + (int64_t)gpos * a.cap, a.cap);
    } else {
        slice_topt_write<CT, NV>(acc, j0, lane, a.ncols, a.col_ids, a.part_s, a.part_j,
                                 ((int64_t)slice * n_total + gpos) * TOPT);
    }
}

int slice_width(int precision, int k, double mean_nnz) {
    // Columns per scoring slice: 32 lanes x NV 16-byte vectors. FP32: 128/256/512 for NV
    // 1/2/4; BF16: 256/512/1024. Small k uses the narrowest shape so that padded columns
    // stay few. Short documents (at most 32 nonzeros on average) take the wider FP32 slice:
    // the per-slice top-4 merge then costs as much as their multiply-adds, and a wider
    // slice spreads it over twice the columns (tweets-like k = 5000: scoring -18%; documents
    // of 120 nonzeros: +12%).
    if (precision == 0) return k <= 128 ? 128 : (mean_nnz <= 32.0 ? 512 : 256);
    return k <= 256 ? 256 : 512;
}

template <bool COLLECT>
static cudaError_t launch_score_t(const ScoreArgs &a, int precision, int slice_cols, cudaStream_t st,
                                  const SparseArgs *sp) {
    if (a.n_list <= 0) return cudaSuccess;
    const int n_slices = (a.ncols + slice_cols - 1) / slice_cols;
    if (n_slices <= 0) return cudaSuccess;
    dim3 grid((a.n_list + 7) / 8, n_slices);
    // sparse rows need a KS-float scratch and a list staging buffer per warp
    const size_t smem = 8 * (sizeof(float) * ((size_t)slice_cols + RARE_SPARE) + RARE_STAGE_BYTES);
#define SKM_SCORE(CT, NVV)                                                          \
    if (sp) k_score_sparse<CT, NVV, COLLECT><<<grid, 256, smem, st>>>(a, *sp);      \
    else k_score<CT, NVV, COLLECT><<<grid, 256, 0, st>>>(a);                         \
    break
    if (precision == 0) {
        switch (slice_cols) {
            case 128: SKM_SCORE(float, 1);
            case 256: SKM_SCORE(float, 2);
            case 512:
                if (sp) k_score_sparse<float, 4, COLLECT><<<grid, 256, smem, st>>>(a, *sp);
                else k_score_f32w<COLLECT><<<grid, 256, 0, st>>>(a);
                break;
            default: return cudaErrorInvalidValue;
        }
    } else {
        switch (slice_cols) {
            case 256: SKM_SCORE(__nv_bfloat16, 1);
            case 512: SKM_SCORE(__nv_bfloat16, 2);
            case 1024: SKM_SCORE(__nv_bfloat16, 4);
            default: return cudaErrorInvalidValue;
        }
    }
#undef SKM_SCORE
    return cudaGetLastError();
}

cudaError_t score_kernel_version(int *out) {
    cudaFuncAttributes fa{};
    const cudaError_t e = cudaFuncGetAttributes(&fa, k_score<__nv_bfloat16, 2, false>);
    if (e == cudaSuccess) *out = fa.binaryVersion;
    return e;
}

cudaError_t launch_score(const ScoreArgs &a, int precision, int slice_cols, cudaStream_t st, const SparseArgs *sp) {
    return launch_score_t<false>(a, precision, slice_cols, st, sp);
}

// Collect pass: the scoring pass again (bit-identical scores) for documents whose
// candidate set did not fit in the top list; appends every centroid at or above the
// document's threshold.
cudaError_t launch_collect(const ScoreArgs &a, int precision, int slice_cols, cudaStream_t st,
                           const SparseArgs *sp) {
    return launch_score_t<true>(a, precision, slice_cols, st, sp);
}

// ------------------------------------------------------------------------------------
// k_decide: one thread per listed document. Merges the per-slice candidate lists into the
// best TOPT of the scored set, folds in the document's stored state for pruned documents
// (Sec. 3.1: the previous centroid a_i is the best of all unchanged centroids, with its
// stored score), and decides:
//   accept   s1 - rho > tau_i: the lower-precision argmax is the exact argmax;
//   rescore  the candidate set R = {j : s_j >= s1 - tau_i} is known completely: FP64;
//   refull   pruned document whose set R may contain unscored centroids: score all k;
//   full64   R may hold more than TOPT entries: FP64 against all k.
// rho bounds every score other than s1 (list runner-up, truncated tail, stored bound).
// tau_i = max(tau, (2 beta s1 + 2 alpha) / (1 - beta)) makes "accept" exact: any j outside R
// has exact score below the exact score of the winner (alpha: the absolute error term of a
// tensor-core head sum, 0 otherwise).
// ------------------------------------------------------------------------------------
__global__ void k_decide(DecideArgs a) {
    const int pos = blockIdx.x * blockDim.x + threadIdx.x;
    if (pos >= a.n_list) return;
    const int32_t i = a.doc_list ? a.doc_list[pos] : pos;

    float ls[TOPT];
    int lj[TOPT];
#pragma unroll
    for (int q = 0; q < TOPT; ++q) { ls[q] = -INFINITY; lj[q] = INT32_MAX; }
    for (int sl = 0; sl < a.n_slices; ++sl) {
        const int64_t o = ((int64_t)sl * a.n_list + pos) * TOPT;
        float bs[TOPT];
        int bj[TOPT];
#pragma unroll
        for (int q = 0; q < TOPT; ++q) { bs[q] = a.part_s[o + q]; bj[q] = a.part_j[o + q]; }
        topt_merge2(ls, lj, bs, bj);
    }
    // scores of the scored set beyond the list are <= tail
    float tail = a.n_scored > TOPT ? ls[TOPT - 1] : -INFINITY;
    float rbound = -INFINITY;
    if (a.pruned) {
        // fold in (s_i, a_i): a_i is not in the scored (moved) set
        const float sp = a.s_state[i];
        const int ap = a.a_old[i];
        if (better(sp, ap, ls[TOPT - 1], lj[TOPT - 1])) {
            tail = fmaxf(tail, ls[TOPT - 1]);
            ls[TOPT - 1] = sp;
            lj[TOPT - 1] = ap;
#pragma unroll
            for (int q = TOPT - 1; q > 0; --q) {
                if (better(ls[q], lj[q], ls[q - 1], lj[q - 1])) {
                    float ts = ls[q]; ls[q] = ls[q - 1]; ls[q - 1] = ts;
                    int tj = lj[q]; lj[q] = lj[q - 1]; lj[q - 1] = tj;
                }
            }
        } else {
            tail = fmaxf(tail, sp);
        }
        rbound = a.r_state[i];
    }
    const float s1 = ls[0];
    const int j1 = lj[0];
    const float rho = fmaxf(fmaxf(ls[1], tail), rbound);

    int64_t nnz = a.row_ptr[i + 1] - a.row_ptr[i];
    if (s1 <= 0.f && rho <= 0.f) {
        // every score is exactly zero: the document shares no term with any centroid's
        // support (scores are sums of non-negative products: documents are validated, and
        // centroids are normalised sums of documents or validated when set from outside), so
        // every exact score is zero and the lowest index, centroid 0, is the argmax
        a.a_new[i] = 0;
        a.s_state[i] = 0.f;
        a.r_state[i] = 0.f;
        a.clean[i] = 1;
        if (a.score_out) a.score_out[i] = 0.f;
        return;
    }
    const double beta = score_beta(a.precision, nnz);
    // a tensor-core head sum adds at most 2^-33 sqrt(nnz) + 2^-25 in absolute terms (FP16
    // subnormals of the operands and of the stored sum)
    const double alpha = a.head_tc ? ldexp(sqrt((double)nnz), -33) + 5.9604644775390625e-08 : 0.0;
    const double tau_i =
        fmax((double)a.tau, (2.0 * beta * fmax((double)s1, 0.0) + 2.0 * alpha) / (1.0 - beta));
    const bool accept = !a.rescore || ((double)s1 - (double)rho > tau_i);

    if (accept) {
        a.a_new[i] = j1;
        a.s_state[i] = s1;
        a.r_state[i] = rho;
        a.clean[i] = 1;
        if (a.score_out) a.score_out[i] = s1;
        return;
    }
    const double thr = (double)s1 - tau_i;
    const bool complete = (double)tail < thr && (double)rbound < thr;
    if (complete) {
        const int q = atomicAdd(&a.counters[CNT_RESCORE], 1);
        a.rs_doc[q] = i;
#pragma unroll
        for (int c = 0; c < TOPT; ++c)
            a.rs_cand[(int64_t)q * TOPT + c] = ((double)ls[c] >= thr) ? lj[c] : -1;
        // provisional state; k_rescore64 overwrites a_new, s_state and r_state
        a.a_new[i] = j1;
        a.s_state[i] = s1;
        a.r_state[i] = rho;
        a.clean[i] = 0;
        return;
    }
    if (a.pruned) {
        const int q = atomicAdd(&a.counters[CNT_REFULL], 1);
        a.refull_doc[q] = i;
        atomicAdd(a.counters64 + C64_NNZ_REFULL, (unsigned long long)nnz);
        return;   // state untouched: the refull pass decides it as an unpruned document
    }
    // more candidates than the list holds: collect them all (threshold rounded down)
    const int q = atomicAdd(&a.counters[CNT_COLLECT], 1);
    a.collect_doc[q] = i;
    a.collect_thr[q] = __double2float_rd(thr);
    a.a_new[i] = j1;
    a.s_state[i] = s1;
    a.r_state[i] = rho;
    a.clean[i] = 0;
}

cudaError_t launch_decide(const DecideArgs &a, cudaStream_t st) {
    if (a.n_list <= 0) return cudaSuccess;
    k_decide<<<(a.n_list + 255) / 256, 256, 0, st>>>(a);
    return cudaGetLastError();
}

// ------------------------------------------------------------------------------------
// k_rescore64: one warp per listed document; FP64 similarity against the FP32 master of
// each candidate (lanes split the nonzeros, fixed butterfly reduction), argmax with ties
// to the lowest index. The winner's lower-precision score is taken from the candidate
// list, the runner-up bound keeps rho.
// ------------------------------------------------------------------------------------
__global__ void k_rescore64(RescoreArgs a) {
    const int lane = threadIdx.x & 31;
    const int q = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int n = a.count ? *a.count : a.n_fixed;
    if (q >= n) return;
    const int32_t i = a.rs_doc[q];
    int n_cand = a.stride;
    if (a.cand_cnt) {
        n_cand = a.cand_cnt[q];
        if (n_cand > a.stride) {          // list overflowed: FP64 against all k instead
            if (lane == 0) a.full64_doc[atomicAdd(a.full64_count, 1)] = i;
            return;
        }
    }
    const int64_t beg = a.row_ptr[i], end = a.row_ptr[i + 1];
    double best = -INFINITY;
    int bj = INT32_MAX;
    for (int c = 0; c < n_cand; ++c) {
        const int j = a.rs_cand[(int64_t)q * a.stride + c];
        if (j < 0) continue;
        double acc = 0.0;
        for (int64_t p = beg + lane; p < end; p += 32)
            acc = fma((double)__ldg(a.val + p), (double)__ldg(a.C32 + (int64_t)__ldg(a.col + p) * a.ldc + j), acc);
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(FULL, acc, off);
        if (better64(acc, j, best, bj)) { best = acc; bj = j; }
    }
    if (lane == 0) {
        a.a_new[i] = bj;
        if (a.score_out) a.score_out[i] = (float)best;
    }
}

cudaError_t launch_rescore64(const RescoreArgs &a, int n_max, cudaStream_t st) {
    if (n_max <= 0) return cudaSuccess;
    k_rescore64<<<(n_max + 7) / 8, 256, 0, st>>>(a);
    return cudaGetLastError();
}

// ------------------------------------------------------------------------------------
// k_full64: one block per listed document; FP64 similarity to every centroid against the
// FP32 master. The document's (t, x) pairs are staged in shared memory; thread l owns the
// columns j = l, l + blockDim, ... and walks the nonzeros in CSR order, so a block reads
// each needed centroid row segment with coalesced loads. Block argmax, ties to the lowest
// index. Used only where the candidate list could not be bounded.
// ------------------------------------------------------------------------------------
constexpr int F64_THREADS = 256;
constexpr int F64_STAGE = 1024;

__global__ void __launch_bounds__(F64_THREADS) k_full64(Full64Args a) {
    __shared__ int32_t st_t[F64_STAGE];
    __shared__ double st_v[F64_STAGE];
    __shared__ double red_s[F64_THREADS / 32];
    __shared__ int red_j[F64_THREADS / 32];
    const int q = blockIdx.x;
    if (q >= *a.count) return;
    const int32_t i = a.docs[q];
    const int64_t beg = a.row_ptr[i], end = a.row_ptr[i + 1];
    double best = -INFINITY;
    int bj = INT32_MAX;
    for (int j0 = 0; j0 < a.k; j0 += F64_THREADS * 4) {
        double acc[4] = {0.0, 0.0, 0.0, 0.0};
        for (int64_t b = beg; b < end; b += F64_STAGE) {
            const int n = (int)min((int64_t)F64_STAGE, end - b);
            __syncthreads();
            for (int e = threadIdx.x; e < n; e += F64_THREADS) {
                st_t[e] = a.col[b + e];
                st_v[e] = (double)a.val[b + e];
            }
            __syncthreads();
            for (int e = 0; e < n; ++e) {
                const float *row = a.C32 + (int64_t)st_t[e] * a.ldc;
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int j = j0 + u * F64_THREADS + threadIdx.x;
                    if (j < a.k) acc[u] = fma(st_v[e], (double)__ldg(row + j), acc[u]);
                }
            }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int j = j0 + u * F64_THREADS + threadIdx.x;
            if (j < a.k && better64(acc[u], j, best, bj)) { best = acc[u]; bj = j; }
        }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        const double os = __shfl_xor_sync(FULL, best, off);
        const int oj = __shfl_xor_sync(FULL, bj, off);
        if (better64(os, oj, best, bj)) { best = os; bj = oj; }
    }
    if ((threadIdx.x & 31) == 0) {
        red_s[threadIdx.x >> 5] = best;
        red_j[threadIdx.x >> 5] = bj;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < F64_THREADS / 32; ++w)
            if (better64(red_s[w], red_j[w], best, bj)) { best = red_s[w]; bj = red_j[w]; }
        a.a_new[i] = bj;
        if (a.score_out) a.score_out[i] = (float)best;
    }
}

cudaError_t launch_full64(const Full64Args &a, int n_max, cudaStream_t st) {
    if (n_max <= 0) return cudaSuccess;
    k_full64<<<n_max, F64_THREADS, 0, st>>>(a);
    return cudaGetLastError();
}

// ------------------------------------------------------------------------------------
// k_partition: Sec. 3.1 document classes for one step. A document is pruned (scored only
// against moved centroids) iff pruning is on, its last decision was clean (the stored
// runner-up bound separates it by more than the error threshold) and its centroid is
// unchanged. Warp-aggregated appends; list order does not affect any result.
// ------------------------------------------------------------------------------------
__global__ void k_partition(PartitionArgs a) {
    const int64_t pos = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31;
    bool pr = false, in = pos < a.n_docs;
    const int64_t i = in ? (int64_t)a.order[pos] : 0;
    if (in) pr = a.prune && a.clean[i] && !a.changed[a.a_old[i]];
    const unsigned mp = __ballot_sync(FULL, in && pr);
    const unsigned mf = __ballot_sync(FULL, in && !pr);
    int bp = 0, bf = 0;
    if (lane == 0) {
        if (mp) bp = atomicAdd(&a.counters[CNT_PRUNED], __popc(mp));
        if (mf) bf = atomicAdd(&a.counters[CNT_FULL], __popc(mf));
    }
    bp = __shfl_sync(FULL, bp, 0);
    bf = __shfl_sync(FULL, bf, 0);
    const unsigned below = (1u << lane) - 1u;
    if (in && pr) {
        a.pruned_list[bp + __popc(mp & below)] = (int32_t)i;
        atomicAdd(a.counters64 + C64_NNZ_PRUNED, (unsigned long long)(a.row_ptr[i + 1] - a.row_ptr[i]));
    }
    if (in && !pr) a.full_list[bf + __popc(mf & below)] = (int32_t)i;
}

cudaError_t launch_partition(const PartitionArgs &a, cudaStream_t st) {
    if (a.n_docs <= 0) return cudaSuccess;
    k_partition<<<(unsigned)((a.n_docs + 255) / 256), 256, 0, st>>>(a);
    return cudaGetLastError();
}

}  // namespace skm
