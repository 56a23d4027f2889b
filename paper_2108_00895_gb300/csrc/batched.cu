// Batched form: many independent clustering instances (different N, d, k) run together.
// Every phase of a Lloyd iteration is one launch that covers all instances through an
// instance table: the scoring pass is a persistent kernel over one queue of (instance,
// document block, slice) tiles, and the other phases index instances per document, per
// cluster slot, per term chunk or per block. Queue sizes are read on the device, so no step
// needs the host, and the whole loop of max_iter iterations is captured once in a CUDA graph
// and replayed. Each instance follows the plain Lloyd loop of the paper (Sec. 2): assignment
// against all k FP32 centroids (FP64 rescoring of near ties), then the update of every
// cluster whose membership changed; all instances run max_iter assignment steps (an
// instance that has converged keeps its assignment and centroids).
//
// The scoring shape of each instance (lane per document for k <= 32, or a warp per document
// with 128-, 256- or 512-column slices) is chosen by an autotuner that times the candidate
// shapes on the instance's own first assignment step and caches the winner per
// (k, mean nonzeros) bucket in a small text file.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "skm.h"
#include "skm_device.cuh"
#include "skm_kernels.cuh"

namespace skm {
namespace {

// ------------------------------------------------------------------------------------
// Instance table
// ------------------------------------------------------------------------------------
struct BInst {
    const int64_t *row_ptr;
    const int32_t *col;
    const float *val;
    int32_t n_docs, d, k, shape;
    int64_t doc0;      // first global document slot
    int64_t clus0;     // first global cluster slot
    float *C32;
    int64_t ldc;
    int32_t n_slices;  // scoring slices of this instance's shape
    int64_t part0;     // first entry of this instance in the candidate-list buffers
    const int64_t *col_ptr;
    const int32_t *row_idx;
    const float *cval;
    const int32_t *pterm;
    int F;
    double inv_scale;
    double dot_scale;
};

// Global state (documents and cluster slots of all instances), queues and counters.
struct BState {
    const BInst *inst;
    int32_t n_inst;
    const int32_t *doc_inst;   // [docs] instance of a global document slot
    const int32_t *clus_inst;  // [slots] instance of a global cluster slot
    const int32_t *order;      // [docs] per instance: local document ids by decreasing length
    int64_t n_docs_total;
    int64_t n_slots;
    int32_t *a_new, *a_old;
    float *s_state, *r_state;
    int32_t *mdoc;
    float *part_s;
    int32_t *part_j;
    uint8_t *changed;
    int32_t *sizes, *moved, *pos_in_m;
    double *normsq, *inv_norm, *newsq, *norm_store, *sq_store;
    unsigned long long *dot_fx, *normsq128, *sq128;
    int32_t *n_moved;          // [n_inst]
    int32_t *n_changed;        // [n_inst]
    int32_t *q_count;          // [4]: rescore queue, full64 queue
    int32_t *rs_doc, *rs_cand, *f64_doc;
    double *obj;               // [n_inst][max_iter]
    int32_t max_iter;
    int rescore;
    float tau;
    int32_t queue_cap;
};

enum { SH_LANE16 = 0, SH_LANE32 = 1, SH_W128 = 2, SH_W256 = 3, SH_W512 = 4, SH_N = 5 };
static const int kShapeCols[SH_N] = {16, 32, 128, 256, 512};

struct Tile {
    int32_t inst;
    int32_t pos0;   // first position in the instance's length order
    int32_t slice;
    int32_t pad;
};

// ------------------------------------------------------------------------------------
// Scoring, warp per document (slices of 32 * 4 * NV columns): persistent over tiles.
// ------------------------------------------------------------------------------------
// Next tile for the block from the launch's queue counter (tiles are sorted by decreasing
// estimated cost, so dynamic fetching balances uneven instances).
__device__ __forceinline__ int32_t next_tile(int32_t *counter, int32_t *slot) {
    __syncthreads();
    if (threadIdx.x == 0) *slot = atomicAdd(counter, 1);
    __syncthreads();
    return *slot;
}

template <int NV>
__global__ void __launch_bounds__(256) kb_score_warp(BState S, const Tile *tiles, int32_t n_tiles, int32_t *counter) {
    constexpr int KS = 32 * 4 * NV;
    __shared__ int2 stage[8][32];
    __shared__ int32_t slot;
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    for (int32_t ti = next_tile(counter, &slot); ti < n_tiles; ti = next_tile(counter, &slot)) {
        const Tile tl = tiles[ti];
        const BInst &I = S.inst[tl.inst];
        const int32_t pos = tl.pos0 + wib;
        if (pos >= I.n_docs) continue;
        const int32_t i = S.order[I.doc0 + pos];
        const int64_t j0 = (int64_t)tl.slice * KS;
        float2 acc[2 * NV];
        slice_accumulate<float, NV>(I.row_ptr[i], I.row_ptr[i + 1], I.col, I.val, I.C32 + j0 + lane * 4, I.ldc,
                                    stage[wib], lane, acc);
        slice_topt_write<float, NV>(acc, j0, lane, I.k, nullptr, S.part_s, S.part_j,
                                    I.part0 + ((int64_t)tl.slice * I.n_docs + i) * TOPT);
    }
}

// Scoring, lane per document for k <= KC (KC = 16 or 32 columns, one slice): each lane walks
// its document's nonzeros and loads the KC-column row segments itself.
template <int KC>
__global__ void __launch_bounds__(256) kb_score_lane(BState S, const Tile *tiles, int32_t n_tiles, int32_t *counter) {
    __shared__ int32_t slot;
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    for (int32_t ti = next_tile(counter, &slot); ti < n_tiles; ti = next_tile(counter, &slot)) {
        const Tile tl = tiles[ti];
        const BInst &I = S.inst[tl.inst];
        const int32_t pos = tl.pos0 + wib * 32 + lane;   // 256 documents per tile
        if (pos >= I.n_docs) continue;
        const int32_t i = S.order[I.doc0 + pos];
        float acc[KC];
#pragma unroll
        for (int c = 0; c < KC; ++c) acc[c] = 0.f;
        for (int64_t p = I.row_ptr[i]; p < I.row_ptr[i + 1]; ++p) {
            const float v = __ldg(I.val + p);
            const float *row = I.C32 + (int64_t)__ldg(I.col + p) * I.ldc;
#pragma unroll
            for (int c = 0; c < KC; c += 4) {
                const float4 w = __ldg(reinterpret_cast<const float4 *>(row + c));
                acc[c + 0] = __fmaf_rn(v, w.x, acc[c + 0]);
                acc[c + 1] = __fmaf_rn(v, w.y, acc[c + 1]);
                acc[c + 2] = __fmaf_rn(v, w.z, acc[c + 2]);
                acc[c + 3] = __fmaf_rn(v, w.w, acc[c + 3]);
            }
        }
        float ls[TOPT];
        int lj[TOPT];
#pragma unroll
        for (int q = 0; q < TOPT; ++q) { ls[q] = -INFINITY; lj[q] = INT32_MAX; }
#pragma unroll
        for (int c = 0; c < KC; ++c)
            if (c < I.k) topt_insert(ls, lj, acc[c], c);
        const int64_t o = I.part0 + (int64_t)i * TOPT;
#pragma unroll
        for (int q = 0; q < TOPT; ++q) {
            S.part_s[o + q] = ls[q];
            S.part_j[o + q] = lj[q];
        }
    }
}

// ------------------------------------------------------------------------------------
// Decision: one thread per global document (same rule as the single-collection pass, no
// pruning): accept the FP32 argmax when its margin exceeds the error threshold, else queue
// the candidate list for FP64 rescoring, or all k when the list may be incomplete.
// ------------------------------------------------------------------------------------
__global__ void kb_decide(BState S) {
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= S.n_docs_total) return;
    const BInst &I = S.inst[S.doc_inst[g]];
    const int32_t i = (int32_t)(g - I.doc0);
    float ls[TOPT];
    int lj[TOPT];
#pragma unroll
    for (int q = 0; q < TOPT; ++q) { ls[q] = -INFINITY; lj[q] = INT32_MAX; }
    for (int sl = 0; sl < I.n_slices; ++sl) {
        const int64_t o = I.part0 + ((int64_t)sl * I.n_docs + i) * TOPT;
        float bs[TOPT];
        int bj[TOPT];
#pragma unroll
        for (int q = 0; q < TOPT; ++q) { bs[q] = S.part_s[o + q]; bj[q] = S.part_j[o + q]; }
        topt_merge2(ls, lj, bs, bj);
    }
    const float tail = I.k > TOPT ? ls[TOPT - 1] : -INFINITY;
    const float s1 = ls[0];
    const float rho = fmaxf(ls[1], tail);
    int32_t *a_new = S.a_new + I.doc0;
    if (s1 <= 0.f && rho <= 0.f) {   // no overlap with any centroid: every score is zero
        a_new[i] = 0;
        return;
    }
    const int64_t nnz = I.row_ptr[i + 1] - I.row_ptr[i];
    const double beta = score_beta(0, nnz);
    const double tau_i = fmax((double)S.tau, 2.0 * beta * fmax((double)s1, 0.0) / (1.0 - beta));
    a_new[i] = lj[0];
    if (!S.rescore || (double)s1 - (double)rho > tau_i) return;
    const double thr = (double)s1 - tau_i;
    if ((double)tail < thr) {
        const int q = atomicAdd(S.q_count + 0, 1);
        if (q < S.queue_cap) {
            S.rs_doc[q] = (int32_t)g;
#pragma unroll
            for (int c = 0; c < TOPT; ++c) S.rs_cand[(int64_t)q * TOPT + c] = ((double)ls[c] >= thr) ? lj[c] : -1;
            return;
        }
    }
    const int q = atomicAdd(S.q_count + 1, 1);
    if (q < S.queue_cap) S.f64_doc[q] = (int32_t)g;
}

// FP64 rescoring of queued candidate lists (warp per entry, grid-stride over the queue).
__global__ void kb_rescore64(BState S) {
    const int lane = threadIdx.x & 31;
    const int n = min(S.q_count[0], S.queue_cap);
    for (int q = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); q < n; q += gridDim.x * (blockDim.x >> 5)) {
        const int64_t g = S.rs_doc[q];
        const BInst &I = S.inst[S.doc_inst[g]];
        const int32_t i = (int32_t)(g - I.doc0);
        double best = -INFINITY;
        int bj = INT32_MAX;
        for (int c = 0; c < TOPT; ++c) {
            const int j = S.rs_cand[(int64_t)q * TOPT + c];
            if (j < 0) continue;
            double acc = 0.0;
            for (int64_t p = I.row_ptr[i] + lane; p < I.row_ptr[i + 1]; p += 32)
                acc = fma((double)__ldg(I.val + p), (double)__ldg(I.C32 + (int64_t)__ldg(I.col + p) * I.ldc + j), acc);
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(FULL, acc, off);
            if (better64(acc, j, best, bj)) { best = acc; bj = j; }
        }
        if (lane == 0) S.a_new[g] = bj;
    }
}

// FP64 scoring against all k of queued documents (block per entry, grid-stride).
__global__ void __launch_bounds__(256) kb_full64(BState S) {
    __shared__ double red_s[8];
    __shared__ int red_j[8];
    const int n = min(S.q_count[1], S.queue_cap);
    for (int q = blockIdx.x; q < n; q += gridDim.x) {
        const int64_t g = S.f64_doc[q];
        const BInst &I = S.inst[S.doc_inst[g]];
        const int32_t i = (int32_t)(g - I.doc0);
        double best = -INFINITY;
        int bj = INT32_MAX;
        for (int j = threadIdx.x; j < I.k; j += blockDim.x) {
            double acc = 0.0;
            for (int64_t p = I.row_ptr[i]; p < I.row_ptr[i + 1]; ++p)
                acc = fma((double)__ldg(I.val + p), (double)__ldg(I.C32 + (int64_t)__ldg(I.col + p) * I.ldc + j), acc);
            if (better64(acc, j, best, bj)) { best = acc; bj = j; }
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            const double os = __shfl_xor_sync(FULL, best, off);
            const int oj = __shfl_xor_sync(FULL, bj, off);
            if (better64(os, oj, best, bj)) { best = os; bj = oj; }
        }
        if ((threadIdx.x & 31) == 0) { red_s[threadIdx.x >> 5] = best; red_j[threadIdx.x >> 5] = bj; }
        __syncthreads();
        if (threadIdx.x == 0) {
            for (int w = 1; w < 8; ++w)
                if (better64(red_s[w], red_j[w], best, bj)) { best = red_s[w]; bj = red_j[w]; }
            S.a_new[g] = bj;
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------------------------------
// Update phase (membership reading of Sec. 3.1: recompute the clusters that changed).
// ------------------------------------------------------------------------------------
__global__ void kb_changed(BState S, int first) {
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= S.n_docs_total) return;
    const int32_t in = S.doc_inst[g];
    const BInst &I = S.inst[in];
    const int32_t jn = S.a_new[g];
    atomicAdd(S.sizes + I.clus0 + jn, 1);
    if (first) {
        S.changed[I.clus0 + jn] = 1;
        atomicAdd(S.n_changed + in, 1);
    } else {
        const int32_t jo = S.a_old[g];
        if (jo != jn) {
            S.changed[I.clus0 + jn] = 1;
            S.changed[I.clus0 + jo] = 1;
            atomicAdd(S.n_changed + in, 1);
        }
    }
}

// One block per instance: moved list (ascending) and positions.
__global__ void kb_compact(BState S) {
    __shared__ int32_t warp_tot[32];
    __shared__ int32_t base;
    const BInst &I = S.inst[blockIdx.x];
    if (threadIdx.x == 0) base = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int j0 = 0; j0 < I.k; j0 += blockDim.x) {
        const int j = j0 + threadIdx.x;
        const int f = (j < I.k && S.changed[I.clus0 + j]) ? 1 : 0;
        const unsigned b = __ballot_sync(FULL, f);
        if (lane == 0) warp_tot[w] = __popc(b);
        __syncthreads();
        int before = 0;
        for (int q = 0; q < w; ++q) before += warp_tot[q];
        const int idx = base + before + __popc(b & ((1u << lane) - 1u));
        if (j < I.k) {
            S.pos_in_m[I.clus0 + j] = f ? idx : -1;
            if (f) S.moved[I.clus0 + idx] = j;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            int tot = 0;
            for (int q = 0; q < (int)(blockDim.x >> 5); ++q) tot += warp_tot[q];
            base += tot;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) S.n_moved[blockIdx.x] = base;
}

__global__ void kb_mdoc(BState S) {
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= S.n_docs_total) return;
    const BInst &I = S.inst[S.doc_inst[g]];
    S.mdoc[g] = S.pos_in_m[I.clus0 + S.a_new[g]];
}

// Objective terms x_i . c_{a_i}(old), FP64, summed per moved cluster in fixed point.
__global__ void kb_doc_obj(BState S) {
    const int lane = threadIdx.x & 31;
    const int64_t g = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (g >= S.n_docs_total) return;
    const int m = S.mdoc[g];
    if (m < 0) return;
    const BInst &I = S.inst[S.doc_inst[g]];
    const int32_t i = (int32_t)(g - I.doc0);
    const int64_t j = S.a_new[g];
    double acc = 0.0;
    for (int64_t p = I.row_ptr[i] + lane; p < I.row_ptr[i + 1]; p += 32)
        acc = fma((double)__ldg(I.val + p), (double)__ldg(I.C32 + (int64_t)__ldg(I.col + p) * I.ldc + j), acc);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(FULL, acc, off);
    if (lane == 0) atomicAdd(S.dot_fx + I.clus0 + m, (unsigned long long)__double2ll_rn(acc * I.dot_scale));
}

// Update passes over a global table of light chunks (inst, t0, t1) and heavy terms (inst, t).
struct BChunk {
    int32_t inst, t0, t1, pad;
};

constexpr int B_CHUNK = 4096;
constexpr int B_SLOTS = 2 * B_CHUNK;
constexpr uint32_t B_EMPTY = 0xffffffffu;
constexpr int B_TILE = 4096;

constexpr int B_AGG = 512;    // moved lists up to this size are aggregated in shared memory;
                              // longer lists spread their atomics over enough slots already

// Entry (t, m) with exact fixed-point sum Sv: the write pass stores the new centroid value;
// both passes add to the per-slot 128-bit sums, here through a block-local shared array
// (agg, two words per moved position of the chunk's instance) flushed by b_flush.
template <bool WRITE>
__device__ __forceinline__ void b_entry(const BState &S, const BInst &I, int32_t t, int m, unsigned long long Sv,
                                        unsigned long long *agg, int nm) {
    const int64_t slot = I.clus0 + m;
    unsigned long long *dst = nm <= B_AGG ? agg + 2 * m : (WRITE ? S.sq128 : S.normsq128) + 2 * slot;
    if (!WRITE) {
        atomic_add_u128(dst, Sv * Sv, __umul64hi(Sv, Sv));
        return;
    }
    const int32_t j = S.moved[slot];
    const float c = (float)((double)Sv * I.inv_scale * S.inv_norm[slot]);
    I.C32[(int64_t)t * I.ldc + j] = c;
    const double c2 = (double)c * (double)c;
    atomic_add_u128(dst, (unsigned long long)__double2ull_rn(ldexp(c2, 62)), 0ull);
}

// Adds the block's nonzero aggregates to the global per-slot sums and clears them.
template <bool WRITE>
__device__ __forceinline__ void b_flush(const BState &S, const BInst &I, int nm, unsigned long long *agg) {
    if (nm > B_AGG) return;   // entries went straight to the global sums
    unsigned long long *dst = (WRITE ? S.sq128 : S.normsq128) + 2 * I.clus0;
    for (int m = threadIdx.x; m < nm; m += blockDim.x) {
        const unsigned long long lo = agg[2 * m], hi = agg[2 * m + 1];
        if (lo | hi) {
            atomic_add_u128(dst + 2 * m, lo, hi);
            agg[2 * m] = 0ull;
            agg[2 * m + 1] = 0ull;
        }
    }
}

template <bool WRITE>
__global__ void __launch_bounds__(512) kb_upd_light(BState S, const BChunk *chunks, int32_t n_chunks) {
    extern __shared__ unsigned long long vals[];
    uint32_t *keys = reinterpret_cast<uint32_t *>(vals + B_SLOTS);
    unsigned long long *agg = reinterpret_cast<unsigned long long *>(keys + B_SLOTS);   // [2 * B_AGG]
    for (int q = threadIdx.x; q < B_SLOTS; q += blockDim.x) {
        keys[q] = B_EMPTY;
        vals[q] = 0ull;
    }
    for (int q = threadIdx.x; q < 2 * B_AGG; q += blockDim.x) agg[q] = 0ull;
    __syncthreads();
    for (int c = blockIdx.x; c < n_chunks; c += gridDim.x) {
        const BChunk ch = chunks[c];
        const BInst &I = S.inst[ch.inst];
        const uint32_t nm = (uint32_t)S.n_moved[ch.inst];
        if (nm == 0) continue;   // uniform over the block
        const int32_t *mdoc = S.mdoc + I.doc0;
        for (int64_t p = I.col_ptr[ch.t0] + threadIdx.x; p < I.col_ptr[ch.t1]; p += blockDim.x) {
            const int m = __ldg(mdoc + __ldg(I.row_idx + p));
            if (m < 0) continue;
            const unsigned long long q = fixed_point(__ldg(I.cval + p), I.F);
            if (q == 0ull) continue;
            const uint32_t key = (uint32_t)(__ldg(I.pterm + p) - ch.t0) * nm + (uint32_t)m;
            uint32_t h = (key * 2654435761u) >> (32 - 13);
            while (true) {
                const uint32_t prev = atomicCAS(keys + h, B_EMPTY, key);
                if (prev == B_EMPTY || prev == key) {
                    atomicAdd(vals + h, q);
                    break;
                }
                h = (h + 1) & (B_SLOTS - 1);
            }
        }
        __syncthreads();
        for (int q = threadIdx.x; q < B_SLOTS; q += blockDim.x) {
            const uint32_t key = keys[q];
            if (key == B_EMPTY) continue;
            const uint32_t tl = key / nm;
            b_entry<WRITE>(S, I, ch.t0 + (int32_t)tl, (int)(key - tl * nm), vals[q], agg, (int)nm);
            keys[q] = B_EMPTY;
            vals[q] = 0ull;
        }
        __syncthreads();
        b_flush<WRITE>(S, I, (int)nm, agg);
        __syncthreads();
    }
}

constexpr int B_PRIV = 128;   // moved lists up to this size use warp-private accumulators

template <bool WRITE>
__global__ void __launch_bounds__(1024) kb_upd_heavy(BState S, const BChunk *heavy, int32_t n_heavy) {
    extern __shared__ unsigned long long acc[];
    int32_t *touched = reinterpret_cast<int32_t *>(acc + B_TILE);
    unsigned long long *agg = reinterpret_cast<unsigned long long *>(touched + B_TILE);   // [2 * B_AGG]
    __shared__ int32_t n_touched;
    const int warp = threadIdx.x >> 5, n_warps = blockDim.x >> 5;
    for (int q = threadIdx.x; q < B_TILE; q += blockDim.x) acc[q] = 0ull;
    for (int q = threadIdx.x; q < 2 * B_AGG; q += blockDim.x) agg[q] = 0ull;
    if (threadIdx.x == 0) n_touched = 0;
    __syncthreads();
    for (int h = blockIdx.x; h < n_heavy; h += gridDim.x) {
        const BChunk ch = heavy[h];
        const BInst &I = S.inst[ch.inst];
        const int nm = S.n_moved[ch.inst];
        if (nm == 0) continue;   // uniform over the block
        const int32_t *mdoc = S.mdoc + I.doc0;
        const int32_t t = ch.t0;
        if (nm <= B_PRIV) {
            // small moved list: each warp sums into its own B_PRIV accumulators (acc is
            // B_TILE >= 32 * B_PRIV words), then the warps' partial sums are added per position
            unsigned long long *mine = acc + warp * B_PRIV;
            for (int64_t p = I.col_ptr[t] + threadIdx.x; p < I.col_ptr[t + 1]; p += blockDim.x) {
                const int m = __ldg(mdoc + __ldg(I.row_idx + p));
                if (m < 0) continue;
                const unsigned long long q = fixed_point(__ldg(I.cval + p), I.F);
                if (q != 0ull) atomicAdd(mine + m, q);
            }
            __syncthreads();
            for (int m = threadIdx.x; m < nm; m += blockDim.x) {
                unsigned long long sum = 0ull;
                for (int w = 0; w < n_warps; ++w) {
                    sum += acc[w * B_PRIV + m];
                    acc[w * B_PRIV + m] = 0ull;
                }
                if (sum) b_entry<WRITE>(S, I, t, m, sum, agg, nm);
            }
            __syncthreads();
        } else {
            for (int m0 = 0; m0 < nm; m0 += B_TILE) {
                const int mt = min(B_TILE, nm - m0);
                for (int64_t p = I.col_ptr[t] + threadIdx.x; p < I.col_ptr[t + 1]; p += blockDim.x) {
                    const int mm = __ldg(mdoc + __ldg(I.row_idx + p)) - m0;
                    if (mm < 0 || mm >= mt) continue;
                    const unsigned long long q = fixed_point(__ldg(I.cval + p), I.F);
                    if (q != 0ull && atomicAdd(acc + mm, q) == 0ull) touched[atomicAdd(&n_touched, 1)] = mm;
                }
                __syncthreads();
                const int nt = n_touched;
                for (int e = threadIdx.x; e < nt; e += blockDim.x) {
                    const int mm = touched[e];
                    const unsigned long long Sv = acc[mm];
                    acc[mm] = 0ull;
                    b_entry<WRITE>(S, I, t, m0 + mm, Sv, agg, nm);
                }
                __syncthreads();
                if (threadIdx.x == 0) n_touched = 0;
                __syncthreads();
            }
        }
        b_flush<WRITE>(S, I, nm, agg);
        __syncthreads();
    }
}

// Per cluster slot: norms from the 128-bit sums (norm pass) or squared column norms (write).
__global__ void kb_from_u128(BState S, int which) {
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= S.n_slots) return;
    const int32_t in = S.clus_inst[s];
    const BInst &I = S.inst[in];
    if (s - I.clus0 >= S.n_moved[in]) return;
    if (which == 0) {
        const double v = ldexp((double)S.normsq128[2 * s + 1], 64 - 2 * I.F) + ldexp((double)S.normsq128[2 * s], -2 * I.F);
        S.normsq[s] = v;
        S.inv_norm[s] = v > 0.0 ? 1.0 / sqrt(v) : 0.0;
    } else {
        S.newsq[s] = ldexp((double)S.sq128[2 * s + 1], 2) + ldexp((double)S.sq128[2 * s], -62);
    }
}

// Zero the recomputed moved columns (cluster slot threads x rows, grid-stride over rows).
__global__ void kb_zero_moved(BState S) {
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= S.n_slots) return;
    const int32_t in = S.clus_inst[s];
    const BInst &I = S.inst[in];
    const int64_t m = s - I.clus0;
    if (m >= S.n_moved[in]) return;
    const int32_t j = S.moved[s];
    if (S.sizes[I.clus0 + j] <= 0) return;   // an empty cluster keeps its centroid
    for (int64_t t = blockIdx.y; t < I.d; t += gridDim.y) I.C32[t * I.ldc + j] = 0.f;
}

// One block per instance: objective and norm bookkeeping (see k_finish).
__global__ void kb_finish(BState S, int iter) {
    __shared__ double so[256];
    const int in = blockIdx.x;
    const BInst &I = S.inst[in];
    double o = 0.0;
    for (int j = threadIdx.x; j < I.k; j += blockDim.x) {
        const int64_t s = I.clus0 + j;
        if (S.sizes[s] <= 0) continue;
        const int m = S.pos_in_m[s];
        if (m >= 0) {
            const int64_t ms = I.clus0 + m;
            o += (double)(long long)S.dot_fx[ms] / I.dot_scale;
            S.norm_store[s] = sqrt(S.normsq[ms]);
            S.sq_store[s] = S.newsq[ms];
        } else {
            o += S.norm_store[s];
        }
    }
    so[threadIdx.x] = o;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) so[threadIdx.x] += so[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) S.obj[(int64_t)in * S.max_iter + iter] = so[0];
}

// Initial centroids of every instance: block per (instance, initial document).
__global__ void kb_init(BState S, const int32_t *init_ids, const int64_t *init0) {
    const BInst &I = S.inst[blockIdx.y];
    const int32_t j = blockIdx.x;
    if (j >= I.k) return;
    const int32_t i = init_ids[init0[blockIdx.y] + j];
    for (int64_t p = I.row_ptr[i] + threadIdx.x; p < I.row_ptr[i + 1]; p += blockDim.x)
        I.C32[(int64_t)I.col[p] * I.ldc + j] = I.val[p];
}

}  // namespace
}  // namespace skm

// =====================================================================================
// Host side
// =====================================================================================
using namespace skm;

namespace {

struct Arena {
    const skm_batch_config *cfg;
    std::vector<std::pair<void *, size_t>> blocks;
    size_t used = 0;
    void *get(size_t bytes) {
        bytes = (bytes + 255) & ~size_t(255);
        if (bytes == 0) bytes = 256;
        void *p = nullptr;
        if (cfg->alloc) p = cfg->alloc(bytes, cfg->alloc_user);
        else if (cudaMalloc(&p, bytes) != cudaSuccess) { cudaGetLastError(); p = nullptr; }
        if (p) { blocks.emplace_back(p, bytes); used += bytes; }
        return p;
    }
    ~Arena() {
        for (auto &b : blocks) {
            if (cfg->free) cfg->free(b.first, b.second, cfg->alloc_user);
            else cudaFree(b.first);
        }
    }
};

struct Err {
    skm_batch_stats *st;
    skm_status fail(skm_status s, const char *msg) {
        if (st) snprintf(st->message, sizeof st->message, "%s", msg);
        return s;
    }
};

// Autotuner cache: "k_bucket nnz_bucket shape" lines.
std::map<std::pair<int, int>, int> load_cache(const char *path) {
    std::map<std::pair<int, int>, int> m;
    if (!path) return m;
    FILE *f = fopen(path, "r");
    if (!f) return m;
    int a, b, c;
    while (fscanf(f, "%d %d %d", &a, &b, &c) == 3) m[{a, b}] = c;
    fclose(f);
    return m;
}

void save_cache(const char *path, const std::map<std::pair<int, int>, int> &m) {
    if (!path) return;
    FILE *f = fopen(path, "w");
    if (!f) return;
    for (auto &kv : m) fprintf(f, "%d %d %d\n", kv.first.first, kv.first.second, kv.second);
    fclose(f);
}

int bucket_log2(double x) { return x <= 1.0 ? 0 : (int)std::ceil(std::log2(x)); }

std::vector<int> candidate_shapes(int k) {
    if (k <= 16) return {SH_LANE16, SH_LANE32, SH_W128};
    if (k <= 32) return {SH_LANE32, SH_W128};
    if (k <= 128) return {SH_W128, SH_W256};
    return {SH_W128, SH_W256, SH_W512};
}

cudaError_t launch_scoring(const BState &S, int shape, const Tile *tiles, int32_t n_tiles, int32_t *counter,
                           cudaStream_t st) {
    if (n_tiles <= 0) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(int32_t), st);
    if (e != cudaSuccess) return e;
    const int grid = std::min<int64_t>(n_tiles, 152 * 8);
    switch (shape) {
        case SH_LANE16: kb_score_lane<16><<<grid, 256, 0, st>>>(S, tiles, n_tiles, counter); break;
        case SH_LANE32: kb_score_lane<32><<<grid, 256, 0, st>>>(S, tiles, n_tiles, counter); break;
        case SH_W128: kb_score_warp<1><<<grid, 256, 0, st>>>(S, tiles, n_tiles, counter); break;
        case SH_W256: kb_score_warp<2><<<grid, 256, 0, st>>>(S, tiles, n_tiles, counter); break;
        case SH_W512: kb_score_warp<4><<<grid, 256, 0, st>>>(S, tiles, n_tiles, counter); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

// Tiles of one instance for a shape.
void make_tiles(int32_t inst, int32_t n_docs, int32_t k, int shape, std::vector<Tile> &out) {
    if (shape <= SH_LANE32) {
        for (int32_t p = 0; p < n_docs; p += 256) out.push_back({inst, p, 0, 0});
        return;
    }
    const int cols = kShapeCols[shape];
    const int ns = (k + cols - 1) / cols;
    for (int s = 0; s < ns; ++s)
        for (int32_t p = 0; p < n_docs; p += 8) out.push_back({inst, p, s, 0});
}

}  // namespace

extern "C" SKM_API skm_status skm_fit_batched(const skm_batch_config *cfg, const skm_batch_item *items,
                                              int32_t n_items, skm_batch_stats *stats) {
    Err E{stats};
    if (stats) std::memset(stats, 0, sizeof(*stats));
    if (!cfg || !items || n_items < 1 || cfg->max_iter < 1 || !(cfg->rescore_tau >= 0.0) ||
        (cfg->alloc == nullptr) != (cfg->free == nullptr))
        return E.fail(SKM_ERR_INVALID, "invalid batch configuration");
    const auto t_start = std::chrono::steady_clock::now();
    int prev_dev = -1;
    cudaGetDevice(&prev_dev);
    if (cudaSetDevice(cfg->device) != cudaSuccess) { cudaGetLastError(); return E.fail(SKM_ERR_CUDA, "bad device"); }
    struct Restore { int d; ~Restore() { if (d >= 0) cudaSetDevice(d); } } restore{prev_dev};
    cudaStream_t st = (cudaStream_t)cfg->stream;
    Arena A{cfg};

    // ---- host checks and layout
    std::vector<BInst> inst(n_items);
    std::vector<int64_t> init0(n_items + 1, 0);
    int64_t n_docs_total = 0, n_slots = 0, nnz_total = 0, part_total = 0;
    std::vector<int> shape(n_items, SH_W256);   // scoring shape per instance
    for (int32_t q = 0; q < n_items; ++q) {
        const skm_batch_item &it = items[q];
        const skm_csr &c = it.docs;
        if (c.n_docs < 1 || c.n_docs > INT32_MAX - 1 || c.n_terms < 1 || c.nnz < c.n_docs || it.k < 1 ||
            it.k > c.n_docs || it.k > 2048 || !it.init_doc_ids || !it.assign_out || !c.row_ptr || !c.col_idx || !c.values)
            return E.fail(SKM_ERR_INVALID, "invalid batch item");
        std::vector<char> seen(c.n_docs, 0);
        for (int32_t j = 0; j < it.k; ++j) {
            const int32_t id = it.init_doc_ids[j];
            if (id < 0 || id >= c.n_docs || seen[id]) return E.fail(SKM_ERR_INVALID, "initial ids must be distinct and in range");
            seen[id] = 1;
        }
        BInst &I = inst[q];
        std::memset(&I, 0, sizeof(I));
        I.n_docs = (int32_t)c.n_docs;
        I.d = c.n_terms;
        I.k = it.k;
        I.doc0 = n_docs_total;
        I.clus0 = n_slots;
        n_docs_total += c.n_docs;
        n_slots += it.k;
        nnz_total += c.nnz;
        init0[q + 1] = init0[q] + it.k;
    }

    // ---- device buffers
    auto dev = [&](size_t bytes) { return A.get(bytes); };
    int64_t *d_rp = (int64_t *)dev(sizeof(int64_t) * (n_docs_total + n_items));
    int32_t *d_col = (int32_t *)dev(sizeof(int32_t) * nnz_total);
    float *d_val = (float *)dev(sizeof(float) * nnz_total);
    if (!d_rp || !d_col || !d_val) return E.fail(SKM_ERR_OOM, "device allocation failed (documents)");
    {
        int64_t rp_off = 0, e_off = 0;
        for (int32_t q = 0; q < n_items; ++q) {
            const skm_csr &c = items[q].docs;
            const cudaMemcpyKind kd = c.on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
            if (cudaMemcpyAsync(d_rp + rp_off, c.row_ptr, sizeof(int64_t) * (c.n_docs + 1), kd, st) != cudaSuccess ||
                cudaMemcpyAsync(d_col + e_off, c.col_idx, sizeof(int32_t) * c.nnz, kd, st) != cudaSuccess ||
                cudaMemcpyAsync(d_val + e_off, c.values, sizeof(float) * c.nnz, kd, st) != cudaSuccess)
                return E.fail(SKM_ERR_CUDA, "copy of documents failed");
            inst[q].row_ptr = d_rp + rp_off;
            inst[q].col = d_col + e_off;
            inst[q].val = d_val + e_off;
            rp_off += c.n_docs + 1;
            e_off += c.nnz;
        }
    }
    // validation (row offsets are relative to each instance's own arrays)
    int32_t *d_flags = (int32_t *)dev(sizeof(int32_t) * n_items);
    if (!d_flags) return E.fail(SKM_ERR_OOM, "device allocation failed");
    cudaMemsetAsync(d_flags, 0, sizeof(int32_t) * n_items, st);
    for (int32_t q = 0; q < n_items; ++q)
        if (launch_validate(inst[q].row_ptr, inst[q].col, inst[q].val, inst[q].n_docs, items[q].docs.nnz, inst[q].d,
                            d_flags + q, st) != cudaSuccess)
            return E.fail(SKM_ERR_CUDA, "validation launch failed");
    std::vector<int32_t> flags(n_items);
    if (cudaMemcpyAsync(flags.data(), d_flags, sizeof(int32_t) * n_items, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return E.fail(SKM_ERR_CUDA, "validation failed");
    for (int32_t q = 0; q < n_items; ++q) {
        const skm_csr &c = items[q].docs;
        if (flags[q]) return E.fail(SKM_ERR_INVALID, "invalid documents in a batch item");
        if (!c.on_device && (c.row_ptr[0] != 0 || c.row_ptr[c.n_docs] != c.nnz))
            return E.fail(SKM_ERR_INVALID, "row_ptr[0] must be 0 and row_ptr[n_docs] == nnz");
    }

    // per instance: order by length, postings, centroid matrix (ldc padded to 512 columns)
    int32_t *d_order = (int32_t *)dev(sizeof(int32_t) * n_docs_total);
    int32_t *d_hist = (int32_t *)dev(sizeof(int32_t) * 4096);
    if (!d_order || !d_hist) return E.fail(SKM_ERR_OOM, "device allocation failed");
    std::vector<BChunk> light, heavy;
    int32_t *d_tcount = nullptr;
    int32_t max_d = 0;
    for (auto &I : inst) max_d = std::max(max_d, I.d);
    d_tcount = (int32_t *)dev(sizeof(int32_t) * (max_d + 1));
    if (!d_tcount) return E.fail(SKM_ERR_OOM, "device allocation failed");
    for (int32_t q = 0; q < n_items; ++q) {
        BInst &I = inst[q];
        const int64_t nnz = items[q].docs.nnz;
        if (launch_order_by_length(I.row_ptr, I.n_docs, d_hist, d_order + I.doc0, st) != cudaSuccess)
            return E.fail(SKM_ERR_CUDA, "order launch failed");
        I.ldc = ((int64_t)I.k + 511) / 512 * 512;
        I.C32 = (float *)dev(sizeof(float) * (size_t)I.d * I.ldc);
        int64_t *cp = (int64_t *)dev(sizeof(int64_t) * (I.d + 1));
        int32_t *ri = (int32_t *)dev(sizeof(int32_t) * nnz);
        float *cv = (float *)dev(sizeof(float) * nnz);
        int32_t *pt = (int32_t *)dev(sizeof(int32_t) * nnz);
        if (!I.C32 || !cp || !ri || !cv || !pt) return E.fail(SKM_ERR_OOM, "device allocation failed (instance)");
        cudaMemsetAsync(I.C32, 0, sizeof(float) * (size_t)I.d * I.ldc, st);
        cudaMemsetAsync(d_tcount, 0, sizeof(int32_t) * (I.d + 1), st);
        if (launch_term_count(I.col, nnz, d_tcount, st) != cudaSuccess) return E.fail(SKM_ERR_CUDA, "count failed");
        std::vector<int32_t> cnt(I.d);
        if (cudaMemcpyAsync(cnt.data(), d_tcount, sizeof(int32_t) * I.d, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess)
            return E.fail(SKM_ERR_CUDA, "count copy failed");
        std::vector<int64_t> hcp(I.d + 1, 0);
        for (int32_t t = 0; t < I.d; ++t) hcp[t + 1] = hcp[t] + cnt[t];
        int bits = 0;
        while ((int64_t(1) << bits) < (int64_t)I.n_docs + 1) ++bits;
        I.F = 61 - bits;
        I.inv_scale = std::ldexp(1.0, -I.F);
        I.dot_scale = std::ldexp(1.0, 61 - bits);
        // light chunks and heavy terms (same rules as the single-collection update)
        const int64_t span_cap = std::max<int64_t>(1, std::min<int64_t>(4096, int64_t(0xffffffff) / I.k));
        int64_t w = 0;
        int32_t start = -1, last = -1;
        auto close = [&](int32_t end) {
            if (start >= 0) light.push_back({q, start, end, 0});
            start = -1;
            w = 0;
        };
        for (int32_t t = 0; t < I.d; ++t) {
            if (cnt[t] > B_CHUNK) { close(t); heavy.push_back({q, t, t + 1, 0}); continue; }
            if (cnt[t] == 0) continue;
            if (start >= 0 && (w + cnt[t] > B_CHUNK || t - start >= span_cap)) close(t);
            if (start < 0) start = t;
            w += cnt[t];
            last = t;
        }
        if (start >= 0) close(last + 1);
        if (cudaMemcpyAsync(cp, hcp.data(), sizeof(int64_t) * (I.d + 1), cudaMemcpyHostToDevice, st) != cudaSuccess)
            return E.fail(SKM_ERR_CUDA, "copy failed");
        cudaMemsetAsync(d_tcount, 0, sizeof(int32_t) * (I.d + 1), st);
        if (launch_csc_fill(I.row_ptr, I.col, I.val, I.n_docs, cp, d_tcount, ri, cv, pt, st) != cudaSuccess)
            return E.fail(SKM_ERR_CUDA, "fill failed");
        if (cudaStreamSynchronize(st) != cudaSuccess) return E.fail(SKM_ERR_CUDA, "setup failed");
        I.col_ptr = cp;
        I.row_idx = ri;
        I.cval = cv;
        I.pterm = pt;
    }

    // global state
    BState S{};
    S.n_inst = n_items;
    S.n_docs_total = n_docs_total;
    S.n_slots = n_slots;
    S.max_iter = cfg->max_iter;
    S.rescore = cfg->rescore;
    S.tau = (float)cfg->rescore_tau;
    S.queue_cap = (int32_t)std::min<int64_t>(n_docs_total, INT32_MAX);
    S.order = d_order;
    int32_t *doc_inst = (int32_t *)dev(sizeof(int32_t) * n_docs_total);
    int32_t *clus_inst = (int32_t *)dev(sizeof(int32_t) * n_slots);
    S.a_new = (int32_t *)dev(sizeof(int32_t) * n_docs_total);
    S.a_old = (int32_t *)dev(sizeof(int32_t) * n_docs_total);
    S.mdoc = (int32_t *)dev(sizeof(int32_t) * n_docs_total);
    S.changed = (uint8_t *)dev(n_slots);
    S.sizes = (int32_t *)dev(sizeof(int32_t) * n_slots);
    S.moved = (int32_t *)dev(sizeof(int32_t) * n_slots);
    S.pos_in_m = (int32_t *)dev(sizeof(int32_t) * n_slots);
    S.normsq = (double *)dev(sizeof(double) * n_slots);
    S.inv_norm = (double *)dev(sizeof(double) * n_slots);
    S.newsq = (double *)dev(sizeof(double) * n_slots);
    S.norm_store = (double *)dev(sizeof(double) * n_slots);
    S.sq_store = (double *)dev(sizeof(double) * n_slots);
    S.dot_fx = (unsigned long long *)dev(sizeof(unsigned long long) * n_slots);
    S.normsq128 = (unsigned long long *)dev(2 * sizeof(unsigned long long) * n_slots);
    S.sq128 = (unsigned long long *)dev(2 * sizeof(unsigned long long) * n_slots);
    S.n_moved = (int32_t *)dev(sizeof(int32_t) * n_items);
    S.n_changed = (int32_t *)dev(sizeof(int32_t) * n_items);
    S.q_count = (int32_t *)dev(sizeof(int32_t) * 4);
    S.rs_doc = (int32_t *)dev(sizeof(int32_t) * S.queue_cap);
    S.rs_cand = (int32_t *)dev(sizeof(int32_t) * (size_t)S.queue_cap * TOPT);
    S.f64_doc = (int32_t *)dev(sizeof(int32_t) * S.queue_cap);
    S.obj = (double *)dev(sizeof(double) * n_items * cfg->max_iter);
    int32_t *d_init = (int32_t *)dev(sizeof(int32_t) * init0[n_items]);
    int64_t *d_init0 = (int64_t *)dev(sizeof(int64_t) * (n_items + 1));
    if (!doc_inst || !clus_inst || !S.a_new || !S.a_old || !S.mdoc || !S.changed || !S.sizes || !S.moved || !S.pos_in_m ||
        !S.normsq || !S.inv_norm || !S.newsq || !S.norm_store || !S.sq_store || !S.dot_fx || !S.normsq128 || !S.sq128 ||
        !S.n_moved || !S.n_changed || !S.q_count || !S.rs_doc || !S.rs_cand || !S.f64_doc || !S.obj || !d_init || !d_init0)
        return E.fail(SKM_ERR_OOM, "device allocation failed (state)");
    {
        std::vector<int32_t> hdi(n_docs_total), hci(n_slots), hinit(init0[n_items]);
        for (int32_t q = 0; q < n_items; ++q) {
            std::fill(hdi.begin() + inst[q].doc0, hdi.begin() + inst[q].doc0 + inst[q].n_docs, q);
            std::fill(hci.begin() + inst[q].clus0, hci.begin() + inst[q].clus0 + inst[q].k, q);
            std::memcpy(hinit.data() + init0[q], items[q].init_doc_ids, sizeof(int32_t) * items[q].k);
        }
        cudaMemcpyAsync(doc_inst, hdi.data(), sizeof(int32_t) * n_docs_total, cudaMemcpyHostToDevice, st);
        cudaMemcpyAsync(clus_inst, hci.data(), sizeof(int32_t) * n_slots, cudaMemcpyHostToDevice, st);
        cudaMemcpyAsync(d_init, hinit.data(), sizeof(int32_t) * hinit.size(), cudaMemcpyHostToDevice, st);
        cudaMemcpyAsync(d_init0, init0.data(), sizeof(int64_t) * (n_items + 1), cudaMemcpyHostToDevice, st);
        if (cudaStreamSynchronize(st) != cudaSuccess) return E.fail(SKM_ERR_CUDA, "setup copy failed");
    }
    S.doc_inst = doc_inst;
    S.clus_inst = clus_inst;
    cudaMemsetAsync(S.norm_store, 0, sizeof(double) * n_slots, st);
    cudaMemsetAsync(S.sq_store, 0, sizeof(double) * n_slots, st);

    // ---- candidate-list buffers (sized for the shape with the most slices)
    for (int32_t q = 0; q < n_items; ++q) {
        inst[q].part0 = part_total;
        part_total += (int64_t)inst[q].n_docs * ((inst[q].k + 127) / 128) * TOPT;
    }
    S.part_s = (float *)dev(sizeof(float) * part_total);
    S.part_j = (int32_t *)dev(sizeof(int32_t) * part_total);
    BInst *d_inst = (BInst *)dev(sizeof(BInst) * n_items);
    if (!S.part_s || !S.part_j || !d_inst) return E.fail(SKM_ERR_OOM, "device allocation failed (lists)");
    S.inst = d_inst;
    auto set_shape = [&](int32_t q, int sh) {
        shape[q] = sh;
        inst[q].shape = sh;
        inst[q].n_slices = sh <= SH_LANE32 ? 1 : (inst[q].k + kShapeCols[sh] - 1) / kShapeCols[sh];
    };
    auto tune_key = [&](int32_t q) {
        return std::make_pair(bucket_log2(inst[q].k), bucket_log2((double)items[q].docs.nnz / items[q].docs.n_docs));
    };
    for (int32_t q = 0; q < n_items; ++q) set_shape(q, candidate_shapes(inst[q].k)[0]);
    cudaMemcpyAsync(d_inst, inst.data(), sizeof(BInst) * n_items, cudaMemcpyHostToDevice, st);
    {   // initial centroids c_j = x_{init_j} of every instance
        int32_t kmax = 0;
        for (auto &I : inst) kmax = std::max(kmax, I.k);
        kb_init<<<dim3(kmax, n_items), 128, 0, st>>>(S, d_init, d_init0);
    }

    // ---- autotuner: the scoring shape of an instance is the fastest candidate on its own
    // first assignment step; winners are cached per (log2 k, log2 mean nonzeros) bucket
    auto cache = load_cache(cfg->tune_cache);
    bool cache_dirty = false;
    int32_t *d_tune_counter = (int32_t *)dev(sizeof(int32_t));
    if (!d_tune_counter) return E.fail(SKM_ERR_OOM, "device allocation failed");
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    for (int32_t q = 0; q < n_items; ++q) {
        const auto key = tune_key(q);
        auto hit = cache.find(key);
        if (hit != cache.end()) {
            set_shape(q, hit->second);
            continue;
        }
        float best_ms = 1e30f;
        int best = shape[q];
        for (int sh : candidate_shapes(inst[q].k)) {
            set_shape(q, sh);
            cudaMemcpyAsync(d_inst + q, &inst[q], sizeof(BInst), cudaMemcpyHostToDevice, st);
            std::vector<Tile> tv;
            make_tiles(q, inst[q].n_docs, inst[q].k, sh, tv);
            Tile *dt = (Tile *)dev(sizeof(Tile) * tv.size());
            if (!dt) return E.fail(SKM_ERR_OOM, "device allocation failed (tuning)");
            cudaMemcpyAsync(dt, tv.data(), sizeof(Tile) * tv.size(), cudaMemcpyHostToDevice, st);
            launch_scoring(S, sh, dt, (int32_t)tv.size(), d_tune_counter, st);   // warm-up
            cudaEventRecord(e0, st);
            launch_scoring(S, sh, dt, (int32_t)tv.size(), d_tune_counter, st);
            cudaEventRecord(e1, st);
            if (cudaEventSynchronize(e1) != cudaSuccess) return E.fail(SKM_ERR_CUDA, "tuning launch failed");
            float ms = 0;
            cudaEventElapsedTime(&ms, e0, e1);
            if (ms < best_ms) { best_ms = ms; best = sh; }
        }
        set_shape(q, best);
        cache[key] = best;
        cache_dirty = true;
        if (stats) stats->tuned++;
    }
    if (cache_dirty) save_cache(cfg->tune_cache, cache);
    cudaMemcpyAsync(d_inst, inst.data(), sizeof(BInst) * n_items, cudaMemcpyHostToDevice, st);

    // tiles per shape group, sorted by decreasing estimated cost (nonzeros of the tile's
    // longest document x slice columns), chunk tables
    std::vector<Tile> tiles_by_shape[SH_N];
    for (int32_t q = 0; q < n_items; ++q) make_tiles(q, inst[q].n_docs, inst[q].k, shape[q], tiles_by_shape[shape[q]]);
    {
        std::vector<std::vector<int64_t>> len(n_items);   // per instance: lengths in scoring order
        std::vector<int64_t> rp, ord;
        for (int32_t q = 0; q < n_items; ++q) {
            rp.resize(inst[q].n_docs + 1);
            ord.assign(inst[q].n_docs, 0);
            std::vector<int32_t> o32(inst[q].n_docs);
            cudaMemcpyAsync(rp.data(), inst[q].row_ptr, sizeof(int64_t) * rp.size(), cudaMemcpyDeviceToHost, st);
            cudaMemcpyAsync(o32.data(), d_order + inst[q].doc0, sizeof(int32_t) * o32.size(), cudaMemcpyDeviceToHost, st);
            if (cudaStreamSynchronize(st) != cudaSuccess) return E.fail(SKM_ERR_CUDA, "copy failed");
            len[q].resize(inst[q].n_docs);
            for (int32_t p = 0; p < inst[q].n_docs; ++p) len[q][p] = rp[o32[p] + 1] - rp[o32[p]];
        }
        for (int sh = 0; sh < SH_N; ++sh) {
            auto &tv = tiles_by_shape[sh];
            const int64_t cols = kShapeCols[sh];
            std::stable_sort(tv.begin(), tv.end(), [&](const Tile &x, const Tile &y) {
                return len[x.inst][x.pos0] * cols > len[y.inst][y.pos0] * cols;
            });
        }
    }
    int32_t *d_tile_counter = (int32_t *)dev(sizeof(int32_t) * SH_N);
    if (!d_tile_counter) return E.fail(SKM_ERR_OOM, "device allocation failed");
    Tile *d_tiles[SH_N] = {};
    for (int sh = 0; sh < SH_N; ++sh) {
        if (tiles_by_shape[sh].empty()) continue;
        d_tiles[sh] = (Tile *)dev(sizeof(Tile) * tiles_by_shape[sh].size());
        if (!d_tiles[sh]) return E.fail(SKM_ERR_OOM, "device allocation failed (tiles)");
        cudaMemcpyAsync(d_tiles[sh], tiles_by_shape[sh].data(), sizeof(Tile) * tiles_by_shape[sh].size(),
                        cudaMemcpyHostToDevice, st);
        if (stats) { stats->tiles += (int64_t)tiles_by_shape[sh].size(); stats->shape_instances[sh] = 0; }
    }
    for (int32_t q = 0; q < n_items; ++q) if (stats) stats->shape_instances[shape[q]]++;
    BChunk *d_light = (BChunk *)dev(sizeof(BChunk) * std::max<size_t>(1, light.size()));
    BChunk *d_heavy = (BChunk *)dev(sizeof(BChunk) * std::max<size_t>(1, heavy.size()));
    if (!d_light || !d_heavy) return E.fail(SKM_ERR_OOM, "device allocation failed (chunks)");
    if (!light.empty()) cudaMemcpyAsync(d_light, light.data(), sizeof(BChunk) * light.size(), cudaMemcpyHostToDevice, st);
    if (!heavy.empty()) cudaMemcpyAsync(d_heavy, heavy.data(), sizeof(BChunk) * heavy.size(), cudaMemcpyHostToDevice, st);
    const size_t smem_l = (size_t)B_SLOTS * 12 + (size_t)B_AGG * 16, smem_h = (size_t)B_TILE * 12 + (size_t)B_AGG * 16;
    cudaFuncSetAttribute(kb_upd_light<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_l);
    cudaFuncSetAttribute(kb_upd_light<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_l);
    cudaFuncSetAttribute(kb_upd_heavy<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_h);
    cudaFuncSetAttribute(kb_upd_heavy<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_h);
    if (cudaStreamSynchronize(st) != cudaSuccess) return E.fail(SKM_ERR_CUDA, "setup failed");
    const auto t_setup = std::chrono::steady_clock::now();

    // ---- one iteration as a sequence of launches covering every instance
    const unsigned gd = (unsigned)((n_docs_total + 255) / 256);
    const unsigned gs = (unsigned)((n_slots + 255) / 256);
    int32_t dmax = 0;
    for (auto &I : inst) dmax = std::max(dmax, I.d);
    auto iteration = [&](int it) -> cudaError_t {
        const int first = it == 0;
        cudaMemsetAsync(S.q_count, 0, sizeof(int32_t) * 4, st);
        for (int sh = 0; sh < SH_N; ++sh)
            if (d_tiles[sh]) launch_scoring(S, sh, d_tiles[sh], (int32_t)tiles_by_shape[sh].size(), d_tile_counter + sh, st);
        kb_decide<<<gd, 256, 0, st>>>(S);
        kb_rescore64<<<152 * 4, 256, 0, st>>>(S);
        kb_full64<<<152 * 2, 256, 0, st>>>(S);
        cudaMemsetAsync(S.changed, 0, n_slots, st);
        cudaMemsetAsync(S.sizes, 0, sizeof(int32_t) * n_slots, st);
        cudaMemsetAsync(S.n_changed, 0, sizeof(int32_t) * n_items, st);
        kb_changed<<<gd, 256, 0, st>>>(S, first);
        kb_compact<<<n_items, 1024, 0, st>>>(S);
        kb_mdoc<<<gd, 256, 0, st>>>(S);
        cudaMemsetAsync(S.dot_fx, 0, sizeof(unsigned long long) * n_slots, st);
        cudaMemsetAsync(S.normsq128, 0, 2 * sizeof(unsigned long long) * n_slots, st);
        cudaMemsetAsync(S.sq128, 0, 2 * sizeof(unsigned long long) * n_slots, st);
        kb_doc_obj<<<(unsigned)((n_docs_total * 32 + 255) / 256), 256, 0, st>>>(S);
        if (!light.empty())
            kb_upd_light<false><<<(unsigned)std::min<size_t>(light.size(), 152 * 4), 512, smem_l, st>>>(S, d_light,
                                                                                                       (int32_t)light.size());
        if (!heavy.empty())
            kb_upd_heavy<false><<<(unsigned)std::min<size_t>(heavy.size(), 152 * 2), 1024, smem_h, st>>>(S, d_heavy,
                                                                                                        (int32_t)heavy.size());
        kb_from_u128<<<gs, 256, 0, st>>>(S, 0);
        kb_zero_moved<<<dim3(gs, (unsigned)std::min(dmax, 1024)), 256, 0, st>>>(S);
        if (!light.empty())
            kb_upd_light<true><<<(unsigned)std::min<size_t>(light.size(), 152 * 4), 512, smem_l, st>>>(S, d_light,
                                                                                                      (int32_t)light.size());
        if (!heavy.empty())
            kb_upd_heavy<true><<<(unsigned)std::min<size_t>(heavy.size(), 152 * 2), 1024, smem_h, st>>>(S, d_heavy,
                                                                                                       (int32_t)heavy.size());
        kb_from_u128<<<gs, 256, 0, st>>>(S, 1);
        kb_finish<<<n_items, 256, 0, st>>>(S, it);
        cudaMemcpyAsync(S.a_old, S.a_new, sizeof(int32_t) * n_docs_total, cudaMemcpyDeviceToDevice, st);
        return cudaGetLastError();
    };

    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaStream_t cap = st;
    bool own_stream = false;
    if (cfg->use_graph && st == nullptr) {   // capture needs a non-legacy stream
        if (cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking) != cudaSuccess) return E.fail(SKM_ERR_CUDA, "stream");
        own_stream = true;
    }
    cudaEventRecord(e0, st);
    if (cfg->use_graph) {
        if (own_stream) {   // order the capture stream after the setup work
            cudaEvent_t ready;
            cudaEventCreate(&ready);
            cudaEventRecord(ready, st);
            cudaStreamWaitEvent(cap, ready, 0);
            cudaEventDestroy(ready);
        }
        cudaStream_t saved = st;
        st = cap;
        if (cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
            return E.fail(SKM_ERR_CUDA, "graph capture failed to start");
        for (int it = 0; it < cfg->max_iter; ++it) iteration(it);
        if (cudaStreamEndCapture(cap, &graph) != cudaSuccess || !graph) return E.fail(SKM_ERR_CUDA, "graph capture failed");
        if (cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess) return E.fail(SKM_ERR_CUDA, "graph instantiate failed");
        size_t n_nodes = 0;
        cudaGraphGetNodes(graph, nullptr, &n_nodes);
        if (stats) stats->graph_nodes = (int64_t)n_nodes;
        cudaEventRecord(e0, cap);
        if (cudaGraphLaunch(exec, cap) != cudaSuccess) return E.fail(SKM_ERR_CUDA, "graph launch failed");
        cudaEventRecord(e1, cap);
        st = saved;
        if (own_stream) {
            cudaEvent_t done;
            cudaEventCreate(&done);
            cudaEventRecord(done, cap);
            cudaStreamWaitEvent(st, done, 0);
            cudaEventDestroy(done);
        }
    } else {
        for (int it = 0; it < cfg->max_iter; ++it)
            if (iteration(it) != cudaSuccess) return E.fail(SKM_ERR_CUDA, "launch failed");
        cudaEventRecord(e1, st);
    }
    if (cudaEventSynchronize(e1) != cudaSuccess || cudaStreamSynchronize(st) != cudaSuccess) {
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        return E.fail(SKM_ERR_CUDA, "batched loop failed");
    }
    float loop_ms = 0;
    cudaEventElapsedTime(&loop_ms, e0, e1);
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    if (own_stream) cudaStreamDestroy(cap);

    // ---- results
    std::vector<double> hobj((size_t)n_items * cfg->max_iter);
    cudaMemcpyAsync(hobj.data(), S.obj, sizeof(double) * hobj.size(), cudaMemcpyDeviceToHost, st);
    for (int32_t q = 0; q < n_items; ++q) {
        const cudaMemcpyKind kd = items[q].docs.on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
        cudaMemcpyAsync(items[q].assign_out, S.a_new + inst[q].doc0, sizeof(int32_t) * inst[q].n_docs, kd, st);
    }
    if (cudaStreamSynchronize(st) != cudaSuccess) return E.fail(SKM_ERR_CUDA, "copy-out failed");
    for (int32_t q = 0; q < n_items; ++q)
        if (items[q].objective_out)
            std::memcpy(items[q].objective_out, hobj.data() + (size_t)q * cfg->max_iter, sizeof(double) * cfg->max_iter);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (stats) {
        const auto t_end = std::chrono::steady_clock::now();
        stats->ms_loop = loop_ms;
        stats->ms_setup = std::chrono::duration<double, std::milli>(t_setup - t_start).count();
        stats->ms_total = std::chrono::duration<double, std::milli>(t_end - t_start).count();
        int64_t fm = 0;
        for (int32_t q = 0; q < n_items; ++q) fm += items[q].docs.nnz * (int64_t)items[q].k;
        stats->fmas = fm * cfg->max_iter;
        stats->device_bytes = (int64_t)A.used;
    }
    return SKM_OK;
}
