// Centroid update (Sec. 2 of the paper): c_j = S_j / ||S_j||, S_j the sum of the member
// documents of cluster j, computed only for clusters whose membership changed (the
// non-changing-clusters reading of Sec. 3.1: an unchanged cluster keeps its centroid
// bit for bit).
//
// Layout: the collection is transposed once per fit into term-major postings (CSC). For
// each term t the postings are bucketed by the cluster of their document; each bucket's
// sum S(t, j) is accumulated exactly as a 64-bit fixed-point integer (value * 2^F, F chosen
// so no sum can overflow), so the result does not depend on the order in which threads add
// their postings: the update is deterministic without a sort of the postings. The rows of
// the term-major centroid matrix are then written with coalesced stores.
//
// Two passes over the postings: the first accumulates ||S_j||^2 (exact 128-bit integer),
// the second writes c = S / ||S|| into the FP32 master, the BF16 copy and the compacted
// moved-centroid matrix (after a store-only pass that zeroes the moved columns), and
// accumulates the squared norm of the stored FP32 column (for the next step's shift). The objective term
// S_j . c_j(old) comes from per-document FP64 dots against the old master (k_doc_obj),
// summed per cluster in fixed point, before the update overwrites it.
#include <algorithm>
#include <cstdlib>

#include "skm_device.cuh"
#include "skm_kernels.cuh"

namespace skm {

// ------------------------------------------------------------------------------------
// Validation: one warp per row.
// ------------------------------------------------------------------------------------
__global__ void k_validate(const int64_t *row_ptr, const int32_t *col, const float *val,
                           int64_t n_docs, int64_t nnz, int32_t n_terms, int32_t *err) {
    const int lane = threadIdx.x & 31;
    const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (i >= n_docs) return;
    const int64_t beg = row_ptr[i], end = row_ptr[i + 1];
    int e = 0;
    // a row outside [0, nnz] is flagged and not read, so bad offsets cannot fault
    const bool in_bounds = beg >= 0 && end <= nnz && beg <= end;
    if (!in_bounds) e |= 16;
    if (end == beg) e |= 4;
    double ss = 0.0;
    if (in_bounds && end > beg) {
        for (int64_t p = beg + lane; p < end; p += 32) {
            const int32_t t = col[p];
            if (t < 0 || t >= n_terms) e |= 1;
            if (p > beg && col[p - 1] >= t) e |= 1;
            const float v = val[p];
            if (!(v >= 0.f) || !isfinite(v)) e |= 2;
            ss += (double)v * (double)v;
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) ss += __shfl_xor_sync(FULL, ss, off);
        if (lane == 0 && !(fabs(sqrt(ss) - 1.0) <= 1e-5)) e |= 8;
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) e |= __shfl_xor_sync(FULL, e, off);
    if (lane == 0 && e) atomicOr(err, e);
}

cudaError_t launch_validate(const int64_t *row_ptr, const int32_t *col, const float *val,
                            int64_t n_docs, int64_t nnz, int32_t n_terms, int32_t *err, cudaStream_t st) {
    if (n_docs <= 0) return cudaSuccess;
    const int64_t threads = n_docs * 32;
    k_validate<<<(unsigned)((threads + 255) / 256), 256, 0, st>>>(row_ptr, col, val, n_docs, nnz,
                                                                  n_terms, err);
    return cudaGetLastError();
}

// Entries of a row-major rows x cols block (row stride ld) that are negative or not finite
// set bit 2 of *err. Every score of the method is a sum of non-negative products (tf-idf
// documents and centroids that are normalised sums of them), which the scoring pass and its
// decision rely on, so centroids given from outside are checked the same way as documents.
__global__ void k_validate_matrix(const float *M, int64_t ld, int32_t rows, int32_t cols, int32_t *err) {
    const int64_t n = (int64_t)rows * cols;
    int e = 0;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = q / cols, c = q - r * cols;
        const float v = M[r * ld + c];
        if (!(v >= 0.f) || !isfinite(v)) e = 2;
    }
    if (__any_sync(FULL, e != 0) && (threadIdx.x & 31) == 0) atomicOr(err, 2);
}

cudaError_t launch_validate_matrix(const float *M, int64_t ld, int32_t rows, int32_t cols, int32_t *err,
                                   cudaStream_t st) {
    if (rows <= 0 || cols <= 0) return cudaSuccess;
    const int64_t n = (int64_t)rows * cols;
    const unsigned blocks = (unsigned)std::min<int64_t>((n + 255) / 256, 152 * 16);
    k_validate_matrix<<<blocks, 256, 0, st>>>(M, ld, rows, cols, err);
    return cudaGetLastError();
}

// ------------------------------------------------------------------------------------
// Documents ordered by decreasing number of nonzeros (bucket sort; order within a bucket
// is arbitrary and affects only scheduling): neighbouring warps of a scoring block then
// carry similar work.
// ------------------------------------------------------------------------------------
constexpr int ORDER_BUCKETS = 4096;

__global__ void k_len_hist(const int64_t *row_ptr, int64_t n, int32_t *hist) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int64_t len = row_ptr[i + 1] - row_ptr[i];
    atomicAdd(hist + (ORDER_BUCKETS - 1 - (int)min(len, (int64_t)ORDER_BUCKETS - 1)), 1);
}

__global__ void k_hist_scan(int32_t *hist) {   // one block of 1024 threads, exclusive scan
    __shared__ int32_t part[1024];
    constexpr int PER = ORDER_BUCKETS / 1024;
    int loc[PER];
    int s = 0;
#pragma unroll
    for (int q = 0; q < PER; ++q) { loc[q] = hist[threadIdx.x * PER + q]; s += loc[q]; }
    part[threadIdx.x] = s;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {
        const int v = threadIdx.x >= (unsigned)off ? part[threadIdx.x - off] : 0;
        __syncthreads();
        part[threadIdx.x] += v;
        __syncthreads();
    }
    int run = part[threadIdx.x] - s;
#pragma unroll
    for (int q = 0; q < PER; ++q) { hist[threadIdx.x * PER + q] = run; run += loc[q]; }
}

__global__ void k_len_scatter(const int64_t *row_ptr, int64_t n, int32_t *offs, int32_t *order) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int64_t len = row_ptr[i + 1] - row_ptr[i];
    const int b = ORDER_BUCKETS - 1 - (int)min(len, (int64_t)ORDER_BUCKETS - 1);
    order[atomicAdd(offs + b, 1)] = (int32_t)i;
}

cudaError_t launch_order_by_length(const int64_t *row_ptr, int64_t n, int32_t *hist, int32_t *order,
                                   cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(hist, 0, ORDER_BUCKETS * sizeof(int32_t), st);
    if (e != cudaSuccess) return e;
    const unsigned blocks = (unsigned)((n + 255) / 256);
    k_len_hist<<<blocks, 256, 0, st>>>(row_ptr, n, hist);
    k_hist_scan<<<1, 1024, 0, st>>>(hist);
    k_len_scatter<<<blocks, 256, 0, st>>>(row_ptr, n, hist, order);
    return cudaGetLastError();
}

// ------------------------------------------------------------------------------------
// Transpose to term-major postings.
// ------------------------------------------------------------------------------------
__global__ void k_term_count(const int32_t *col, int64_t nnz, int32_t *cnt) {
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < nnz;
         p += (int64_t)gridDim.x * blockDim.x)
        atomicAdd(cnt + col[p], 1);
}

cudaError_t launch_term_count(const int32_t *col, int64_t nnz, int32_t *cnt, cudaStream_t st) {
    if (nnz <= 0) return cudaSuccess;
    const int64_t blocks = min((int64_t)152 * 16, (nnz + 255) / 256);
    k_term_count<<<(unsigned)blocks, 256, 0, st>>>(col, nnz, cnt);
    return cudaGetLastError();
}

__global__ void k_csc_fill(const int64_t *row_ptr, const int32_t *col, const float *val,
                           int64_t n_docs, const int64_t *col_ptr, int32_t *fill,
                           int32_t *row_idx, float *cval, int32_t *pterm) {
    const int lane = threadIdx.x & 31;
    const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (i >= n_docs) return;
    for (int64_t p = row_ptr[i] + lane; p < row_ptr[i + 1]; p += 32) {
        const int32_t t = col[p];
        const int64_t o = col_ptr[t] + atomicAdd(fill + t, 1);
        row_idx[o] = (int32_t)i;
        cval[o] = val[p];
        pterm[o] = t;
    }
}

cudaError_t launch_csc_fill(const int64_t *row_ptr, const int32_t *col, const float *val,
                            int64_t n_docs, const int64_t *col_ptr, int32_t *fill,
                            int32_t *row_idx, float *cval, int32_t *pterm, cudaStream_t st) {
    if (n_docs <= 0) return cudaSuccess;
    const int64_t threads = n_docs * 32;
    k_csc_fill<<<(unsigned)((threads + 255) / 256), 256, 0, st>>>(row_ptr, col, val, n_docs, col_ptr,
                                                                  fill, row_idx, cval, pterm);
    return cudaGetLastError();
}

// ------------------------------------------------------------------------------------
// Initial centroids: one warp per centroid writes its document's entries into column j.
// ------------------------------------------------------------------------------------
__global__ void k_init_centroids(const int64_t *row_ptr, const int32_t *col, const float *val,
                                 const int32_t *ids, int32_t k, float *C32, __nv_bfloat16 *C16,
                                 int64_t ldc, double *sq) {
    const int lane = threadIdx.x & 31;
    const int64_t j = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (j >= k) return;
    const int64_t i = ids[j];
    double s = 0.0;
    for (int64_t p = row_ptr[i] + lane; p < row_ptr[i + 1]; p += 32) {
        const int64_t o = (int64_t)col[p] * ldc + j;
        C32[o] = val[p];
        if (C16) C16[o] = __float2bfloat16_rn(val[p]);
        s = fma((double)val[p], (double)val[p], s);
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(FULL, s, off);
    if (lane == 0) sq[j] = s;
}

cudaError_t launch_init_centroids(const int64_t *row_ptr, const int32_t *col, const float *val,
                                  const int32_t *ids, int32_t k, float *C32, __nv_bfloat16 *C16,
                                  int64_t ldc, double *sq, cudaStream_t st) {
    const int64_t threads = (int64_t)k * 32;
    k_init_centroids<<<(unsigned)((threads + 255) / 256), 256, 0, st>>>(row_ptr, col, val, ids, k,
                                                                        C32, C16, ldc, sq);
    return cudaGetLastError();
}

// ------------------------------------------------------------------------------------
// Changed clusters (membership reading of Sec. 3.1) and cluster sizes.
// ------------------------------------------------------------------------------------
template <bool SMEM_HIST>
__global__ void k_changed(const int32_t *a_new, const int32_t *a_old, int64_t n_docs, int first,
                          uint8_t *changed, int32_t *sizes, int32_t k, int32_t *counters) {
    extern __shared__ int32_t hist[];
    if (SMEM_HIST) {
        for (int j = threadIdx.x; j < k; j += blockDim.x) hist[j] = 0;
        __syncthreads();
    }
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    bool moved = false;
    if (i < n_docs) {
        const int32_t jn = a_new[i];
        if (SMEM_HIST) atomicAdd(hist + jn, 1);
        else atomicAdd(sizes + jn, 1);
        if (first) {
            changed[jn] = 1;
            moved = true;
        } else {
            const int32_t jo = a_old[i];
            if (jo != jn) {
                changed[jn] = 1;
                changed[jo] = 1;
                moved = true;
            }
        }
    }
    const unsigned m = __ballot_sync(FULL, moved);
    if ((threadIdx.x & 31) == 0 && m) atomicAdd(counters + CNT_CHANGED, __popc(m));
    if (SMEM_HIST) {
        __syncthreads();
        for (int j = threadIdx.x; j < k; j += blockDim.x)
            if (hist[j]) atomicAdd(sizes + j, hist[j]);
    }
}

cudaError_t launch_changed(const int32_t *a_new, const int32_t *a_old, int64_t n_docs, int first,
                           uint8_t *changed, int32_t *sizes, int32_t k, int32_t *counters,
                           cudaStream_t st) {
    if (n_docs <= 0) return cudaSuccess;
    const unsigned blocks = (unsigned)((n_docs + 1023) / 1024);
    if (k <= 8192)
        k_changed<true><<<blocks, 1024, (size_t)k * sizeof(int32_t), st>>>(a_new, a_old, n_docs, first,
                                                                          changed, sizes, k, counters);
    else
        k_changed<false><<<blocks, 1024, 0, st>>>(a_new, a_old, n_docs, first, changed, sizes, k,
                                                  counters);
    return cudaGetLastError();
}

// ------------------------------------------------------------------------------------
// Moved list: single block, ascending order by block-wide exclusive scans.
// ------------------------------------------------------------------------------------
__global__ void k_compact_moved(const uint8_t *changed, int32_t k, int32_t *moved, int32_t *pos_in_m,
                                int32_t *counters) {
    __shared__ int32_t warp_tot[32];
    __shared__ int32_t base;
    if (threadIdx.x == 0) base = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int j0 = 0; j0 < k; j0 += blockDim.x) {
        const int j = j0 + threadIdx.x;
        const int f = (j < k && changed[j]) ? 1 : 0;
        const unsigned b = __ballot_sync(FULL, f);
        const int in_warp = __popc(b & ((1u << lane) - 1u));
        if (lane == 0) warp_tot[w] = __popc(b);
        __syncthreads();
        int before = 0;
        for (int q = 0; q < w; ++q) before += warp_tot[q];
        const int idx = base + before + in_warp;
        if (j < k) {
            pos_in_m[j] = f ? idx : -1;
            if (f) moved[idx] = j;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            int tot = 0;
            for (int q = 0; q < (int)(blockDim.x >> 5); ++q) tot += warp_tot[q];
            base += tot;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) counters[CNT_MOVED] = base;
}

cudaError_t launch_compact_moved(const uint8_t *changed, int32_t k, int32_t *moved,
                                 int32_t *pos_in_m, int32_t *counters, cudaStream_t st) {
    k_compact_moved<<<1, 1024, 0, st>>>(changed, k, moved, pos_in_m, counters);
    return cudaGetLastError();
}

// ------------------------------------------------------------------------------------
// Update passes. Both passes compute, for every (term t, moved cluster m) with a posting,
// the exact fixed-point sum S(t, m) = sum of round(x * 2^F) over the postings of t whose
// document is in cluster m (64-bit integer additions: exact and order-independent).
//   norm pass:  ||S_m||^2 += S(t, m)^2, as a 128-bit integer (exact, order-independent);
//   write pass: c = S(t, m) 2^-F / ||S_m|| is stored into row t of the FP32 master, the BF16
//               copy and the compacted matrix, and sum_t c^2 of the stored FP32 values is
//               accumulated as a 128-bit fixed-point integer (scale 2^62).
// Every sum is exact or integer, so the update is deterministic without ordering work.
// Light terms (at most UPD_CHUNK postings) are packed into chunks of consecutive terms; a
// block reduces a chunk with a shared-memory hash table keyed by (term, cluster) and one
// barrier. Heavy terms get one block each with a dense shared accumulator over the moved
// list (tiled when the list exceeds UPD_TILE).
// ------------------------------------------------------------------------------------
constexpr int UPD_CHUNK = 4096;               // postings per light chunk (table half full)
constexpr int UPD_SLOTS = 2 * UPD_CHUNK;      // hash table slots
constexpr uint32_t UPD_EMPTY = 0xffffffffu;
constexpr int UPD_LIGHT_THREADS = 512;
constexpr int UPD_HEAVY_THREADS = 1024;
constexpr int UPD_TILE = 16384;               // moved entries per heavy-term tile (12 bytes each)
constexpr int UPD_AGG = 512;                  // moved lists up to this size sum their per-cluster
                                              // 128-bit totals in shared memory first (few
                                              // clusters: all blocks would hit the same words)
constexpr int UPD_PRIV = 128;                 // moved lists up to this size: warp-private
                                              // heavy-term accumulators (UPD_TILE >= 32 x 128)

// S (fixed point, 2^-F units) of entry m of term t: the norm or write step. The per-cluster
// 128-bit sums go to agg (shared, flushed by update_flush) for short moved lists.
template <bool WRITE>
__device__ __forceinline__ void update_entry(const UpdateArgs &u, int32_t t, int m, unsigned long long S,
                                             unsigned long long *agg) {
    unsigned long long *dst = u.n_moved <= UPD_AGG ? agg + 2 * m : (WRITE ? u.sq128 : u.normsq128) + 2 * m;
    if (!WRITE) {
        atomic_add_u128(dst, S * S, __umul64hi(S, S));
        return;
    }
    const int32_t j = __ldg(u.moved + m);
    const float c = (float)((double)S * u.inv_scale * __ldg(u.inv_norm + m));
    const int64_t row = (int64_t)t * u.ldc;
    u.C32[row + j] = c;
    if (u.C16) u.C16[row + j] = __float2bfloat16_rn(c);
    if (u.CM) {
        if (u.precision == 1)
            reinterpret_cast<__nv_bfloat16 *>(u.CM)[row + m] = __float2bfloat16_rn(c);
        else
            reinterpret_cast<float *>(u.CM)[row + m] = c;
    }
    if (u.tiG && c != 0.f) {   // keep the threshold index's bitmap and value bins current
        atomicOr(u.tiG + (int64_t)t * u.tiW + (j >> 5), 1u << (j & 31));
        atomicAdd(u.tiHist + (size_t)j * TI_NB + ti_bin(c), 1u);
    }
    const double c2 = (double)c * (double)c;   // exact (24-bit mantissa squared)
    const unsigned long long q = (unsigned long long)__double2ull_rn(ldexp(c2, 62));
    atomic_add_u128(dst, q, 0ull);
}

// Adds the block's shared per-cluster sums to the global ones (short moved lists only).
template <bool WRITE>
__device__ __forceinline__ void update_flush(const UpdateArgs &u, unsigned long long *agg) {
    if (u.n_moved > UPD_AGG) return;
    unsigned long long *dst = WRITE ? u.sq128 : u.normsq128;
    for (int m = threadIdx.x; m < u.n_moved; m += blockDim.x) {
        const unsigned long long lo = agg[2 * m], hi = agg[2 * m + 1];
        if (lo | hi) atomic_add_u128(dst + 2 * m, lo, hi);
    }
}

template <bool WRITE>
__global__ void __launch_bounds__(UPD_LIGHT_THREADS) k_upd_light(UpdateArgs u) {
    extern __shared__ unsigned long long vals[];                         // [UPD_SLOTS]
    uint32_t *keys = reinterpret_cast<uint32_t *>(vals + UPD_SLOTS);     // [UPD_SLOTS]
    unsigned long long *agg = reinterpret_cast<unsigned long long *>(keys + UPD_SLOTS);   // [2 * UPD_AGG]
    for (int q = threadIdx.x; q < UPD_SLOTS; q += UPD_LIGHT_THREADS) {
        keys[q] = UPD_EMPTY;
        vals[q] = 0ull;
    }
    for (int q = threadIdx.x; q < 2 * UPD_AGG; q += UPD_LIGHT_THREADS) agg[q] = 0ull;
    __syncthreads();
    const uint32_t nm = (uint32_t)u.n_moved;
    for (int c = blockIdx.x; c < u.n_light; c += gridDim.x) {
        const int32_t t0 = u.light_t0[c], t1 = u.light_t1[c];
        const int64_t pb = u.col_ptr[t0], pe = u.col_ptr[t1];
        for (int64_t p = pb + threadIdx.x; p < pe; p += UPD_LIGHT_THREADS) {
            const int m = __ldg(u.mdoc + __ldg(u.row_idx + p));
            if (m < 0) continue;
            const unsigned long long q = fixed_point(__ldg(u.cval + p), u.F);
            if (q == 0ull) continue;
            const uint32_t key = (uint32_t)(__ldg(u.pterm + p) - t0) * nm + (uint32_t)m;
            uint32_t h = (key * 2654435761u) >> (32 - 13);          // UPD_SLOTS = 2^13
            while (true) {
                const uint32_t prev = atomicCAS(keys + h, UPD_EMPTY, key);
                if (prev == UPD_EMPTY || prev == key) {
                    atomicAdd(vals + h, q);
                    break;
                }
                h = (h + 1) & (UPD_SLOTS - 1);
            }
        }
        __syncthreads();
        for (int q = threadIdx.x; q < UPD_SLOTS; q += UPD_LIGHT_THREADS) {
            const uint32_t key = keys[q];
            if (key == UPD_EMPTY) continue;
            const uint32_t tl = key / nm;
            update_entry<WRITE>(u, t0 + (int32_t)tl, (int)(key - tl * nm), vals[q], agg);
            keys[q] = UPD_EMPTY;
            vals[q] = 0ull;
        }
        __syncthreads();
    }
    update_flush<WRITE>(u, agg);
}

template <bool WRITE>
__global__ void __launch_bounds__(UPD_HEAVY_THREADS) k_upd_heavy(UpdateArgs u) {
    extern __shared__ unsigned long long acc[];                              // [UPD_TILE]
    int32_t *touched = reinterpret_cast<int32_t *>(acc + UPD_TILE);          // [UPD_TILE]
    unsigned long long *agg = reinterpret_cast<unsigned long long *>(touched + UPD_TILE);   // [2 * UPD_AGG]
    __shared__ int32_t n_touched;
    const int warp = threadIdx.x >> 5;
    for (int q = threadIdx.x; q < UPD_TILE; q += UPD_HEAVY_THREADS) acc[q] = 0ull;
    for (int q = threadIdx.x; q < 2 * UPD_AGG; q += UPD_HEAVY_THREADS) agg[q] = 0ull;
    if (threadIdx.x == 0) n_touched = 0;
    __syncthreads();
    for (int h = blockIdx.x; h < u.n_heavy; h += gridDim.x) {
        const int32_t t = u.heavy_terms[h];
        const int64_t pb = u.col_ptr[t], pe = u.col_ptr[t + 1];
        if (u.n_moved <= UPD_PRIV) {
            // short moved list: each warp sums into its own UPD_PRIV accumulators, then the
            // warps' partial sums are added per position (integer sums: order-free)
            unsigned long long *mine = acc + warp * UPD_PRIV;
            for (int64_t p = pb + threadIdx.x; p < pe; p += UPD_HEAVY_THREADS) {
                const int m = __ldg(u.mdoc + __ldg(u.row_idx + p));
                if (m < 0) continue;
                const unsigned long long q = fixed_point(__ldg(u.cval + p), u.F);
                if (q != 0ull) atomicAdd(mine + m, q);
            }
            __syncthreads();
            for (int m = threadIdx.x; m < u.n_moved; m += UPD_HEAVY_THREADS) {
                unsigned long long sum = 0ull;
                for (int w = 0; w < UPD_HEAVY_THREADS / 32; ++w) {
                    sum += acc[w * UPD_PRIV + m];
                    acc[w * UPD_PRIV + m] = 0ull;
                }
                if (sum) update_entry<WRITE>(u, t, m, sum, agg);
            }
            __syncthreads();
            continue;
        }
        for (int m0 = 0; m0 < u.n_moved; m0 += UPD_TILE) {
            const int mt = min(UPD_TILE, u.n_moved - m0);
            for (int64_t p = pb + threadIdx.x; p < pe; p += UPD_HEAVY_THREADS) {
                const int mm = __ldg(u.mdoc + __ldg(u.row_idx + p)) - m0;
                if (mm < 0 || mm >= mt) continue;
                const unsigned long long q = fixed_point(__ldg(u.cval + p), u.F);
                if (q != 0ull && atomicAdd(acc + mm, q) == 0ull) touched[atomicAdd(&n_touched, 1)] = mm;
            }
            __syncthreads();
            const int nt = n_touched;
            for (int e = threadIdx.x; e < nt; e += UPD_HEAVY_THREADS) {
                const int mm = touched[e];
                const unsigned long long S = acc[mm];
                acc[mm] = 0ull;
                update_entry<WRITE>(u, t, m0 + mm, S, agg);
            }
            __syncthreads();
            if (threadIdx.x == 0) n_touched = 0;
            __syncthreads();
        }
    }
    __syncthreads();
    update_flush<WRITE>(u, agg);
}

// ------------------------------------------------------------------------------------
// Very frequent terms (more than UPD_VH postings; in the tweets-like collection the most
// frequent term is in half of the documents): one block per chunk of UPD_VCH postings
// sums its chunk into a shared accumulator over the moved list, tile by tile, and adds the
// touched entries to vh_sum with 64-bit integer atomics (exact, order-free). The passes
// then visit the (term, moved position) entries of vh_sum in parallel, so that no single
// block walks a whole term's postings.
// ------------------------------------------------------------------------------------
constexpr int UPD_VH = 8 * UPD_CHUNK;
constexpr int UPD_VCH = 2 * UPD_CHUNK;

__global__ void __launch_bounds__(UPD_HEAVY_THREADS) k_upd_vh_sum(UpdateArgs u) {
    extern __shared__ unsigned long long acc[];                              // [UPD_TILE]
    int32_t *touched = reinterpret_cast<int32_t *>(acc + UPD_TILE);          // [UPD_TILE]
    __shared__ int32_t n_touched;
    for (int q = threadIdx.x; q < UPD_TILE; q += UPD_HEAVY_THREADS) acc[q] = 0ull;
    if (threadIdx.x == 0) n_touched = 0;
    __syncthreads();
    for (int c = blockIdx.x; c < u.n_vch; c += gridDim.x) {
        const int32_t h = u.vch_h[c];
        const int64_t pb = u.vch_p0[c], pe = u.vch_p1[c];
        unsigned long long *dst = u.vh_sum + (int64_t)h * u.n_moved;
        for (int m0 = 0; m0 < u.n_moved; m0 += UPD_TILE) {
            const int mt = min(UPD_TILE, u.n_moved - m0);
            for (int64_t p = pb + threadIdx.x; p < pe; p += UPD_HEAVY_THREADS) {
                const int mm = __ldg(u.mdoc + __ldg(u.row_idx + p)) - m0;
                if (mm < 0 || mm >= mt) continue;
                const unsigned long long q = fixed_point(__ldg(u.cval + p), u.F);
                if (q != 0ull && atomicAdd(acc + mm, q) == 0ull) touched[atomicAdd(&n_touched, 1)] = mm;
            }
            __syncthreads();
            const int nt = n_touched;
            for (int e = threadIdx.x; e < nt; e += UPD_HEAVY_THREADS) {
                const int mm = touched[e];
                atomicAdd(dst + m0 + mm, acc[mm]);
                acc[mm] = 0ull;
            }
            __syncthreads();
            if (threadIdx.x == 0) n_touched = 0;
            __syncthreads();
        }
    }
}

template <bool WRITE>
__global__ void __launch_bounds__(256) k_upd_vh_pass(UpdateArgs u) {
    extern __shared__ unsigned long long agg[];   // [2 * UPD_AGG]
    for (int q = threadIdx.x; q < 2 * UPD_AGG; q += blockDim.x) agg[q] = 0ull;
    __syncthreads();
    const int64_t n = (int64_t)u.n_vh * u.n_moved;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        const unsigned long long S = u.vh_sum[e];
        if (!S) continue;
        const int64_t h = e / u.n_moved;
        update_entry<WRITE>(u, __ldg(u.vh_terms + h), (int)(e - h * u.n_moved), S, agg);
    }
    __syncthreads();
    update_flush<WRITE>(u, agg);
}

cudaError_t launch_update_vh_sums(const UpdateArgs &u, cudaStream_t st) {
    if (u.n_moved <= 0 || u.n_vh <= 0) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(u.vh_sum, 0, sizeof(unsigned long long) * (size_t)u.n_vh * u.n_moved, st);
    if (e != cudaSuccess) return e;
    const size_t smem = (size_t)UPD_TILE * (sizeof(unsigned long long) + sizeof(int32_t));
    e = cudaFuncSetAttribute(k_upd_vh_sum, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_upd_vh_sum<<<min(u.n_vch, 152 * 2), UPD_HEAVY_THREADS, smem, st>>>(u);
    return cudaGetLastError();
}

static cudaError_t launch_update(const UpdateArgs &u, bool write, cudaStream_t st) {
    if (u.n_moved <= 0) return cudaSuccess;
    cudaError_t e;
    const size_t agg_bytes = (size_t)2 * UPD_AGG * sizeof(unsigned long long);
    const size_t smem_l = (size_t)UPD_SLOTS * (sizeof(unsigned long long) + sizeof(uint32_t)) + agg_bytes;
    const size_t smem_h = (size_t)UPD_TILE * (sizeof(unsigned long long) + sizeof(int32_t)) + agg_bytes;
    if (u.n_light > 0) {
        const int grid = min(u.n_light, 152 * 2 * 8);
        if (write) {
            e = cudaFuncSetAttribute(k_upd_light<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_l);
            if (e != cudaSuccess) return e;
            k_upd_light<true><<<grid, UPD_LIGHT_THREADS, smem_l, st>>>(u);
        } else {
            e = cudaFuncSetAttribute(k_upd_light<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_l);
            if (e != cudaSuccess) return e;
            k_upd_light<false><<<grid, UPD_LIGHT_THREADS, smem_l, st>>>(u);
        }
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    if (u.n_vh > 0) {
        const int64_t n = (int64_t)u.n_vh * u.n_moved;
        const int grid = (int)std::min<int64_t>((n + 255) / 256, 152 * 8);
        if (write) k_upd_vh_pass<true><<<grid, 256, agg_bytes, st>>>(u);
        else k_upd_vh_pass<false><<<grid, 256, agg_bytes, st>>>(u);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    if (u.n_heavy > 0) {
        const int grid = min(u.n_heavy, 152 * 4);
        if (write) {
            e = cudaFuncSetAttribute(k_upd_heavy<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_h);
            if (e != cudaSuccess) return e;
            k_upd_heavy<true><<<grid, UPD_HEAVY_THREADS, smem_h, st>>>(u);
        } else {
            e = cudaFuncSetAttribute(k_upd_heavy<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_h);
            if (e != cudaSuccess) return e;
            k_upd_heavy<false><<<grid, UPD_HEAVY_THREADS, smem_h, st>>>(u);
        }
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_update_norm(const UpdateArgs &u, cudaStream_t st) { return launch_update(u, false, st); }
cudaError_t launch_update_write(const UpdateArgs &u, cudaStream_t st) { return launch_update(u, true, st); }
int update_chunk_postings() { return UPD_CHUNK; }
int update_vh_postings() { return UPD_VH; }
int update_vh_chunk() { return UPD_VCH; }

// normsq[m] = ||S_m||^2 and inv_norm[m] = 1 / ||S_m|| from the 128-bit fixed-point sums
// (units 2^-2F); newsq[m] from the 128-bit sums of c^2 (units 2^-62).
__global__ void k_from_u128(const unsigned long long *normsq128, const unsigned long long *sq128, int32_t n,
                            int F, double *normsq, double *inv_norm, double *newsq) {
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= n) return;
    if (normsq128) {
        const double v = ldexp((double)normsq128[2 * m + 1], 64 - 2 * F) + ldexp((double)normsq128[2 * m], -2 * F);
        normsq[m] = v;
        inv_norm[m] = v > 0.0 ? 1.0 / sqrt(v) : 0.0;
    }
    if (sq128) newsq[m] = ldexp((double)sq128[2 * m + 1], 2) + ldexp((double)sq128[2 * m], -62);
}

cudaError_t launch_from_u128(const unsigned long long *normsq128, const unsigned long long *sq128, int32_t n,
                             int F, double *normsq, double *inv_norm, double *newsq, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    k_from_u128<<<(n + 255) / 256, 256, 0, st>>>(normsq128, sq128, n, F, normsq, inv_norm, newsq);
    return cudaGetLastError();
}

// ------------------------------------------------------------------------------------
// Recomputed columns are cleared before the write pass stores their nonzeros. The support
// of a column is known in three cases, so only its nonzeros are cleared:
//   k_zero_members: a centroid last computed from its current members has nonzeros exactly
//     at their terms: entries (t, a_old[i]) over the postings (i, t) of flagged clusters
//     (repeated stores of zero are harmless);
//   k_zero_seeds: a centroid that is still its seed document: that document's terms;
//   k_zero_cols: any other column (a centroid kept while its cluster was empty): all rows.
// ------------------------------------------------------------------------------------
// Clears bit (t, j) of the threshold-index bitmap (W words a row).
__device__ __forceinline__ void ti_clear_bit(uint32_t *G, int32_t W, int64_t t, int32_t j) {
    atomicAnd(G + t * W + (j >> 5), ~(1u << (j & 31)));
}

__global__ void k_zero_members(const int32_t *row_idx, const int32_t *pterm, int64_t nnz, const int32_t *a_old,
                               const uint8_t *flag, float *C32, __nv_bfloat16 *C16, int64_t ldc, uint32_t *tiG,
                               int32_t W) {
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < nnz; p += (int64_t)gridDim.x * blockDim.x) {
        const int32_t j = __ldg(a_old + __ldg(row_idx + p));
        if (!__ldg(flag + j)) continue;
        const int64_t t = (int64_t)__ldg(pterm + p);
        const int64_t e = t * ldc + j;
        C32[e] = 0.f;
        if (C16) C16[e] = __float2bfloat16_rn(0.f);
        if (tiG) ti_clear_bit(tiG, W, t, j);
    }
}

__global__ void k_zero_seeds(const int32_t *list, int32_t n, const int32_t *init_ids, const int64_t *row_ptr,
                             const int32_t *col, float *C32, __nv_bfloat16 *C16, int64_t ldc, uint32_t *tiG,
                             int32_t W) {
    const int lane = threadIdx.x & 31;
    const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (w >= n) return;
    const int32_t j = list[w];
    const int32_t doc = init_ids[j];
    for (int64_t p = row_ptr[doc] + lane; p < row_ptr[doc + 1]; p += 32) {
        const int64_t e = (int64_t)col[p] * ldc + j;
        C32[e] = 0.f;
        if (C16) C16[e] = __float2bfloat16_rn(0.f);
        if (tiG) ti_clear_bit(tiG, W, col[p], j);
    }
}

__global__ void k_zero_cols(const int32_t *list, int32_t n, int32_t d, float *C32, __nv_bfloat16 *C16, int64_t ldc,
                            uint32_t *tiG, int32_t W) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    const int32_t j = list[q];
    for (int64_t t = blockIdx.y; t < d; t += gridDim.y) {
        C32[t * ldc + j] = 0.f;
        if (C16) C16[t * ldc + j] = __float2bfloat16_rn(0.f);
        if (tiG) ti_clear_bit(tiG, W, t, j);
    }
}

// The compacted moved matrix for the next pruned pass: column m of a recomputed cluster is
// cleared (the write pass stores its nonzeros); a cluster left without members keeps its
// centroid, which is copied. Store-only except for those copies; one thread per (row, m).
__global__ void k_cm_moved(const int32_t *moved, const int32_t *sizes, int32_t n_moved, int32_t d, const float *C32,
                           void *CM, int precision, int64_t ldc) {
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= n_moved) return;
    const int32_t j = __ldg(moved + m);
    const bool recomputed = __ldg(sizes + j) > 0;
    for (int64_t t = blockIdx.y; t < d; t += gridDim.y) {
        const int64_t row = t * ldc;
        const float cur = recomputed ? 0.f : C32[row + j];
        if (precision == 1)
            reinterpret_cast<__nv_bfloat16 *>(CM)[row + m] = __float2bfloat16_rn(cur);
        else
            reinterpret_cast<float *>(CM)[row + m] = cur;
    }
}

static unsigned rows_grid(int32_t d, unsigned bx) {
    return (unsigned)min((int64_t)d, max((int64_t)1, (int64_t)152 * 64 / bx));
}

cudaError_t launch_zero_members(const int32_t *row_idx, const int32_t *pterm, int64_t nnz, const int32_t *a_old,
                                const uint8_t *flag, float *C32, __nv_bfloat16 *C16, int64_t ldc, uint32_t *tiG,
                                int32_t W, cudaStream_t st) {
    if (nnz <= 0) return cudaSuccess;
    const int64_t blocks = std::min<int64_t>((nnz + 255) / 256, 152 * 16);
    k_zero_members<<<(unsigned)blocks, 256, 0, st>>>(row_idx, pterm, nnz, a_old, flag, C32, C16, ldc, tiG, W);
    return cudaGetLastError();
}

cudaError_t launch_zero_seeds(const int32_t *list, int32_t n, const int32_t *init_ids, const int64_t *row_ptr,
                              const int32_t *col, float *C32, __nv_bfloat16 *C16, int64_t ldc, uint32_t *tiG,
                              int32_t W, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    k_zero_seeds<<<(unsigned)((n + 7) / 8), 256, 0, st>>>(list, n, init_ids, row_ptr, col, C32, C16, ldc, tiG, W);
    return cudaGetLastError();
}

cudaError_t launch_zero_cols(const int32_t *list, int32_t n, int32_t d, float *C32, __nv_bfloat16 *C16, int64_t ldc,
                             uint32_t *tiG, int32_t W, cudaStream_t st) {
    if (n <= 0 || d <= 0) return cudaSuccess;
    const unsigned bx = (unsigned)((n + 255) / 256);
    k_zero_cols<<<dim3(bx, rows_grid(d, bx)), 256, 0, st>>>(list, n, d, C32, C16, ldc, tiG, W);
    return cudaGetLastError();
}

cudaError_t launch_cm_moved(const int32_t *moved, const int32_t *sizes, int32_t n_moved, int32_t d, const float *C32,
                            void *CM, int precision, int64_t ldc, cudaStream_t st) {
    if (n_moved <= 0 || d <= 0) return cudaSuccess;
    const unsigned bx = (unsigned)((n_moved + 255) / 256);
    k_cm_moved<<<dim3(bx, rows_grid(d, bx)), 256, 0, st>>>(moved, sizes, n_moved, d, C32, CM, precision, ldc);
    return cudaGetLastError();
}

// mdoc[i] = position of document i's cluster in the moved list (-1 if not moved).
__global__ void k_mdoc(const int32_t *a, const int32_t *pos_in_m, int64_t n, int32_t *mdoc) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) mdoc[i] = pos_in_m[a[i]];
}

cudaError_t launch_mdoc(const int32_t *a, const int32_t *pos_in_m, int64_t n, int32_t *mdoc,
                        cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    k_mdoc<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(a, pos_in_m, n, mdoc);
    return cudaGetLastError();
}


// ------------------------------------------------------------------------------------
// Objective terms: one warp per document of a moved cluster, FP64 dot x_i . c_{a_i}(old)
// against the FP32 master (fixed butterfly reduction), added to its cluster's sum as a
// 64-bit fixed-point integer (order-independent, so the sum is deterministic).
// ------------------------------------------------------------------------------------
__global__ void k_doc_obj(const int64_t *row_ptr, const int32_t *col, const float *val, int64_t n,
                          const int32_t *a, const int32_t *mdoc, const float *C32, int64_t ldc,
                          double scale, unsigned long long *dot_fx) {
    const int lane = threadIdx.x & 31;
    const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (i >= n) return;
    const int m = mdoc[i];
    if (m < 0) return;
    const int64_t j = a[i];
    double acc = 0.0;
    for (int64_t p = row_ptr[i] + lane; p < row_ptr[i + 1]; p += 32)
        acc = fma((double)__ldg(val + p), (double)__ldg(C32 + (int64_t)__ldg(col + p) * ldc + j), acc);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(FULL, acc, off);
    if (lane == 0) atomicAdd(dot_fx + m, (unsigned long long)__double2ll_rn(acc * scale));
}

cudaError_t launch_doc_obj(const int64_t *row_ptr, const int32_t *col, const float *val, int64_t n,
                           const int32_t *a, const int32_t *mdoc, const float *C32, int64_t ldc,
                           double scale, unsigned long long *dot_fx, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    const int64_t threads = n * 32;
    k_doc_obj<<<(unsigned)((threads + 255) / 256), 256, 0, st>>>(row_ptr, col, val, n, a, mdoc, C32, ldc,
                                                                 scale, dot_fx);
    return cudaGetLastError();
}

// ------------------------------------------------------------------------------------
// Objective of the step and max squared shift (single block, fixed order):
//   objective = sum_j S_j . c_j(old) = sum_i x_i . c_{a_i}(old). For a moved cluster the
//   term is the fixed-point sum of its documents' dots; for a cluster that was not
//   recomputed it is ||S_j|| (its centroid is S_j / ||S_j|| from the last update that
//   recomputed it, and its members are unchanged since), kept in norm_store.
//   shift_j = ||c_new||^2 + ||c_old||^2 - 2 c_new . c_old with ||c_new|| = 1 (FP64 before
//   rounding), ||c_old||^2 the stored FP32 column's squared norm, and
//   c_new . c_old = (S_j . c_old) / ||S_j||.
// ------------------------------------------------------------------------------------
__global__ void k_finish(const int32_t *pos_in_m, const int32_t *sizes, int32_t k,
                         const unsigned long long *dot_fx, double inv_dot_scale, const double *normsq,
                         const double *newsq, double *norm_store, double *sq_store, double *obj_out,
                         double *shift_out) {
    __shared__ double so[1024];
    __shared__ double sm[1024];
    double o = 0.0, mx = 0.0;
    for (int j = threadIdx.x; j < k; j += blockDim.x) {
        const int m = pos_in_m[j];
        if (sizes[j] <= 0) continue;
        if (m >= 0) {
            const double dot = (double)(long long)dot_fx[m] * inv_dot_scale;
            const double nrm = sqrt(normsq[m]);
            o += dot;
            const double sh = 1.0 + sq_store[j] - 2.0 * dot / nrm;
            if (sh > mx) mx = sh;
            norm_store[j] = nrm;
            sq_store[j] = newsq[m];
        } else {
            o += norm_store[j];
        }
    }
    so[threadIdx.x] = o;
    sm[threadIdx.x] = mx;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) {
            so[threadIdx.x] += so[threadIdx.x + w];
            sm[threadIdx.x] = fmax(sm[threadIdx.x], sm[threadIdx.x + w]);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        *obj_out = so[0];
        *shift_out = sm[0];
    }
}

cudaError_t launch_finish(const int32_t *pos_in_m, const int32_t *sizes, int32_t k,
                          const unsigned long long *dot_fx, double inv_dot_scale, const double *normsq,
                          const double *newsq, double *norm_store, double *sq_store, double *obj_out,
                          double *shift_out, cudaStream_t st) {
    k_finish<<<1, 1024, 0, st>>>(pos_in_m, sizes, k, dot_fx, inv_dot_scale, normsq, newsq, norm_store,
                                 sq_store, obj_out, shift_out);
    return cudaGetLastError();
}

// Squared norms of the stored FP32 columns: out[j] = sum_t C32[t, j]^2 (one thread per
// column, rows in order; used after centroids are loaded from outside).
__global__ void k_col_sq(const float *C32, int64_t ldc, int32_t d, int32_t k, double *out) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= k) return;
    double s = 0.0;
    for (int32_t t = 0; t < d; ++t) {
        const double v = (double)C32[(int64_t)t * ldc + j];
        s = fma(v, v, s);
    }
    out[j] = s;
}

cudaError_t launch_col_sq(const float *C32, int64_t ldc, int32_t d, int32_t k, double *out,
                          cudaStream_t st) {
    k_col_sq<<<(k + 127) / 128, 128, 0, st>>>(C32, ldc, d, k, out);
    return cudaGetLastError();
}

// ------------------------------------------------------------------------------------
// Elementwise helpers.
// ------------------------------------------------------------------------------------
__global__ void k_to_bf16(const float *C32, __nv_bfloat16 *C16, int64_t n) {
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n;
         q += (int64_t)gridDim.x * blockDim.x)
        C16[q] = __float2bfloat16_rn(C32[q]);
}

cudaError_t launch_to_bf16(const float *C32, __nv_bfloat16 *C16, int64_t n, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    const int64_t blocks = min((int64_t)152 * 8, (n + 255) / 256);
    k_to_bf16<<<(unsigned)blocks, 256, 0, st>>>(C32, C16, n);
    return cudaGetLastError();
}

__global__ void k_pad_copy(const float *src, int64_t src_ld, float *dst, int64_t dst_ld, int32_t rows,
                           int32_t cols) {
    const int64_t n = (int64_t)rows * cols;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = q / cols, c = q % cols;
        dst[r * dst_ld + c] = src[r * src_ld + c];
    }
}

cudaError_t launch_pad_copy(const float *src, int64_t src_ld, float *dst, int64_t dst_ld,
                            int32_t rows, int32_t cols, cudaStream_t st) {
    const int64_t n = (int64_t)rows * cols;
    if (n <= 0) return cudaSuccess;
    const int64_t blocks = min((int64_t)152 * 8, (n + 255) / 256);
    k_pad_copy<<<(unsigned)blocks, 256, 0, st>>>(src, src_ld, dst, dst_ld, rows, cols);
    return cudaGetLastError();
}

}  // namespace skm
