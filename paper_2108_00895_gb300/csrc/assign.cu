// Assignment step kernels (Sec. 2 of the paper) with the non-changing-clusters skip
// (Sec. 3.1) and FP64 rescoring of near ties.
//
// Scoring pass: s_ij = sum over the document's nonzeros t, in CSR order, of x_it * C[t, j],
// one FP32 fused multiply-add per nonzero per centroid. The chain for a given (i, j) is the
// same whichever launch computes it (full matrix or compacted moved-centroid matrix), so a
// score is a pure function of (x_i, c_j): the pruned and the full pass agree bit for bit.
#include "skm_internal.cuh"
#include "skm_kernels.cuh"

namespace skm {

// ------------------------------------------------------------------------------------
// k_score: one warp per (document, slice). Lane l owns, for u in [0, NV), the EPV columns
// starting at slice*KS + u*32*EPV + l*EPV, so each of the NV 16-byte loads of a centroid
// row segment is one coalesced 512-byte warp access. The document's (t, x) pairs are read
// 32 at a time and broadcast by shuffle.
// ------------------------------------------------------------------------------------
template <typename CT, int NV>
__global__ void __launch_bounds__(256) k_score(ScoreArgs a) {
    constexpr int EPV = 16 / (int)sizeof(CT);
    constexpr int J = NV * EPV;
    constexpr int KS = 32 * J;
    const int lane = threadIdx.x & 31;
    const int pos = blockIdx.x * 8 + (threadIdx.x >> 5);
    if (pos >= a.n_list) return;
    const int slice = blockIdx.y;
    const int64_t i = a.doc_list ? (int64_t)a.doc_list[pos] : (int64_t)pos;
    const int64_t beg = a.row_ptr[i], end = a.row_ptr[i + 1];
    const int64_t j0 = (int64_t)slice * KS;
    const CT *Cs = reinterpret_cast<const CT *>(a.C) + j0 + lane * EPV;

    float acc[J];
#pragma unroll
    for (int q = 0; q < J; ++q) acc[q] = 0.f;

    for (int64_t b = beg; b < end; b += 32) {
        const int n = (int)min((int64_t)32, end - b);
        int mt = 0;
        float mv = 0.f;
        if (lane < n) {
            mt = __ldg(a.col + b + lane);
            mv = __ldg(a.val + b + lane);
        }
        for (int q = 0; q < n; ++q) {
            const int t = __shfl_sync(FULL, mt, q);
            const float v = __shfl_sync(FULL, mv, q);
            const CT *row = Cs + (int64_t)t * a.ldc;
            uint4 w[NV];
#pragma unroll
            for (int u = 0; u < NV; ++u) w[u] = ldg16(row + u * 32 * EPV);
#pragma unroll
            for (int u = 0; u < NV; ++u) {
                if constexpr (sizeof(CT) == 4) {
                    acc[u * 4 + 0] = __fmaf_rn(v, __uint_as_float(w[u].x), acc[u * 4 + 0]);
                    acc[u * 4 + 1] = __fmaf_rn(v, __uint_as_float(w[u].y), acc[u * 4 + 1]);
                    acc[u * 4 + 2] = __fmaf_rn(v, __uint_as_float(w[u].z), acc[u * 4 + 2]);
                    acc[u * 4 + 3] = __fmaf_rn(v, __uint_as_float(w[u].w), acc[u * 4 + 3]);
                } else {
                    acc[u * 8 + 0] = __fmaf_rn(v, bf16lo(w[u].x), acc[u * 8 + 0]);
                    acc[u * 8 + 1] = __fmaf_rn(v, bf16hi(w[u].x), acc[u * 8 + 1]);
                    acc[u * 8 + 2] = __fmaf_rn(v, bf16lo(w[u].y), acc[u * 8 + 2]);
                    acc[u * 8 + 3] = __fmaf_rn(v, bf16hi(w[u].y), acc[u * 8 + 3]);
                    acc[u * 8 + 4] = __fmaf_rn(v, bf16lo(w[u].z), acc[u * 8 + 4]);
                    acc[u * 8 + 5] = __fmaf_rn(v, bf16hi(w[u].z), acc[u * 8 + 5]);
                    acc[u * 8 + 6] = __fmaf_rn(v, bf16lo(w[u].w), acc[u * 8 + 6]);
                    acc[u * 8 + 7] = __fmaf_rn(v, bf16hi(w[u].w), acc[u * 8 + 7]);
                }
            }
        }
    }

    float ls[TOPT];
    int lj[TOPT];
#pragma unroll
    for (int q = 0; q < TOPT; ++q) { ls[q] = -INFINITY; lj[q] = INT32_MAX; }
#pragma unroll
    for (int u = 0; u < NV; ++u) {
#pragma unroll
        for (int e = 0; e < EPV; ++e) {
            const int64_t c = j0 + u * 32 * EPV + lane * EPV + e;
            if (c < a.ncols) {
                const int id = a.col_ids ? __ldg(a.col_ids + c) : (int)c;
                topt_insert(ls, lj, acc[u * EPV + e], id);
            }
        }
    }
    topt_warp_merge(ls, lj);
    if (lane < TOPT) {
        float s = ls[0];
        int j = lj[0];
#pragma unroll
        for (int q = 1; q < TOPT; ++q) if (lane == q) { s = ls[q]; j = lj[q]; }
        const int64_t o = ((int64_t)slice * a.n_list + pos) * TOPT + lane;
        a.part_s[o] = s;
        a.part_j[o] = j;
    }
}

int slice_width(int precision, int k) {
    // FP32: NV = 2 (8 columns per lane, 256 per slice); BF16: NV = 2 (16 per lane, 512).
    // Small k uses the narrowest shape so that padded columns stay few.
    if (precision == 0) return k <= 128 ? 128 : 256;
    return k <= 256 ? 256 : 512;
}

cudaError_t launch_score(const ScoreArgs &a, int precision, int slice_cols, cudaStream_t st) {
    if (a.n_list <= 0) return cudaSuccess;
    const int n_slices = (a.ncols + slice_cols - 1) / slice_cols;
    if (n_slices <= 0) return cudaSuccess;
    dim3 grid((a.n_list + 7) / 8, n_slices);
    if (precision == 0) {
        if (slice_cols == 128) k_score<float, 1><<<grid, 256, 0, st>>>(a);
        else k_score<float, 2><<<grid, 256, 0, st>>>(a);
    } else {
        if (slice_cols == 256) k_score<__nv_bfloat16, 1><<<grid, 256, 0, st>>>(a);
        else k_score<__nv_bfloat16, 2><<<grid, 256, 0, st>>>(a);
    }
    return cudaGetLastError();
}

// ------------------------------------------------------------------------------------
// Error bound of the scoring pass for one document (all data are non-negative):
//   |s_hat - s| <= beta * s,  beta = u_c + gamma_n * (1 + u_c),
// u_c the unit roundoff of the centroid copy (2^-9 for BF16 round-to-nearest-even, 0 for
// the FP32 master itself) and gamma_n = n u / (1 - n u), u = 2^-24, n = nonzeros of the
// document (one rounding per fused multiply-add).
// ------------------------------------------------------------------------------------
__device__ __forceinline__ double score_beta(int precision, int64_t nnz) {
    const double u = 5.9604644775390625e-08;  // 2^-24
    const double nu = (double)nnz * u;
    const double gam = nu / (1.0 - nu);
    const double uc = precision == 1 ? 1.953125e-03 : 0.0;  // 2^-9
    return uc + gam * (1.0 + uc);
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
// tau_i = max(tau, 2 beta s1 / (1 - beta)) makes "accept" exact: any j outside R has
// exact score below the exact score of the winner.
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
    const double beta = score_beta(a.precision, nnz);
    const double tau_i = fmax((double)a.tau, 2.0 * beta * fmax((double)s1, 0.0) / (1.0 - beta));
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
    const int q = atomicAdd(&a.counters[CNT_FULL64], 1);
    a.full64_doc[q] = i;
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
    const int n = *a.count;
    if (q >= n) return;
    const int32_t i = a.rs_doc[q];
    const int64_t beg = a.row_ptr[i], end = a.row_ptr[i + 1];
    double best = -INFINITY;
    int bj = INT32_MAX;
    for (int c = 0; c < TOPT; ++c) {
        const int j = a.rs_cand[(int64_t)q * TOPT + c];
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
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31;
    bool pr = false, in = i < a.n_docs;
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
