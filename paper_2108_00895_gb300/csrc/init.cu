// k-means++ seeding (Sec. 2 names the k-Means++ strategy as the usual initial assignment):
// each new seed is drawn with probability proportional to the squared distance to the
// nearest seed so far, which for unit vectors is 2 (1 - x . seed). One round per seed:
//   k_pp_scatter  the newest seed into a dense vector of the vocabulary;
//   k_pp_dist     every document's distance dist_i = min(dist_i, 1 - x_i . seed) in double,
//                 the products x_it * seed_t (exact: two floats) added one by one in CSR
//                 order, each addition rounded once, and its integer weight
//                 w_i = floor(max(dist_i, 0) 2^32) (0 once drawn);
//   k_pp_chunks   the weight total of each chunk of PP_CHUNK documents;
//   k_pp_pick     one block: W = sum of the totals, T = min(floor(u W), W - 1), the chunk
//                 and then the document whose inclusive prefix sum first exceeds T (the
//                 smallest undrawn document when W = 0); it also clears the seed vector.
// Integer weights make the prefix sums exact, so the seeds are a deterministic function of
// the documents and the uniforms, whatever the thread layout. The distances follow the
// definition in double (the operation order of a sequential loop over the nonzeros); FP64
// is the slow pipe of this GPU, which makes a round about twice as long as in float.
#include <cmath>

#include "skm_internal.cuh"

namespace skm {

constexpr int PP_CHUNK = 8192;
constexpr int PP_PICK_THREADS = 1024;
constexpr int PP_PER_THREAD = PP_CHUNK / PP_PICK_THREADS;

__device__ __forceinline__ unsigned long long pp_weight(double dist, uint8_t drawn) {
    return (!drawn && dist > 0.0) ? (unsigned long long)floor(dist * 4294967296.0) : 0ull;
}

__global__ void k_pp_scatter(int64_t n, const int32_t *ids, int r, const int64_t *row_ptr, const int32_t *col,
                             const float *val, double *seed) {
    const int32_t s = ids[r];
    if (s < 0 || s >= n) return;   // a failed draw is reported by the host
    for (int64_t p = row_ptr[s] + threadIdx.x; p < row_ptr[s + 1]; p += blockDim.x) seed[col[p]] = (double)val[p];
}

__global__ void k_pp_dist(int64_t n, const int32_t *order, const int64_t *row_ptr, const int32_t *col,
                          const float *val, const double *seed, int first, double *dist, const uint8_t *drawn,
                          unsigned long long *w) {
    const int64_t pos = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (pos >= n) return;
    const int64_t i = order ? (int64_t)order[pos] : pos;
    const int64_t pe = row_ptr[i + 1];
    double dot = 0.0;
    // 8 entries at a time: their loads are in flight together and share cache lines; the
    // additions still run over the entries in CSR order, a product then a sum, each rounded
    // on its own (no fused multiply-add), as a sequential double loop computes them
    constexpr int B = 8;
    for (int64_t p0 = row_ptr[i]; p0 < pe; p0 += B) {
        double x[B], c[B];
#pragma unroll
        for (int q = 0; q < B; ++q) {
            const int64_t p = p0 + q;
            x[q] = p < pe ? (double)__ldg(val + p) : 0.0;
            c[q] = p < pe ? __ldg(seed + __ldg(col + p)) : 0.0;
        }
#pragma unroll
        for (int q = 0; q < B; ++q)
            if (p0 + q < pe) dot = __dadd_rn(dot, __dmul_rn(x[q], c[q]));
    }
    const double dd = __dadd_rn(1.0, -dot);
    double cur = first ? dd : dist[i];
    if (dd < cur) cur = dd;
    dist[i] = cur;
    w[i] = pp_weight(cur, drawn[i]);
}

__global__ void k_pp_chunks(int64_t n, const unsigned long long *w, unsigned long long *csum) {
    __shared__ unsigned long long part[32];
    const int64_t c0 = (int64_t)blockIdx.x * PP_CHUNK;
    unsigned long long s = 0ull;
    for (int64_t i = c0 + threadIdx.x; i < min(n, c0 + PP_CHUNK); i += blockDim.x) s += w[i];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(FULL, s, off);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long t = 0ull;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t += part[q];
        csum[blockIdx.x] = t;
    }
}

__global__ void __launch_bounds__(PP_PICK_THREADS) k_pp_pick(int64_t n, int32_t nb, const unsigned long long *csum,
                                                             const unsigned long long *w, const double *u, int r,
                                                             int32_t *ids, uint8_t *drawn, const int64_t *row_ptr,
                                                             const int32_t *col, double *seed) {
    __shared__ unsigned long long scan[PP_PICK_THREADS];
    __shared__ unsigned long long s_T, s_base;
    __shared__ int64_t s_c0, s_pick;
    __shared__ int s_empty, s_first;
    // the previous seed's entries of the dense vector are no longer needed
    const int32_t prev = ids[r - 1];
    if (prev >= 0 && prev < n)
        for (int64_t p = row_ptr[prev] + threadIdx.x; p < row_ptr[prev + 1]; p += blockDim.x) seed[col[p]] = 0.0;
    if (threadIdx.x == 0) {
        unsigned long long W = 0ull;
        for (int b = 0; b < nb; ++b) W += csum[b];
        s_empty = W == 0ull;
        s_pick = -1;
        s_T = 0ull;
        s_base = 0ull;
        s_c0 = 0;
        if (W) {
            unsigned long long T = (unsigned long long)floor(u[r] * (double)W);
            if (T >= W) T = W - 1;
            unsigned long long run = 0ull;
            int b = 0;
            while (b < nb - 1 && run + csum[b] <= T) run += csum[b++];   // T < W: chunk b holds T
            s_T = T;
            s_base = run;
            s_c0 = (int64_t)b * PP_CHUNK;
        }
    }
    __syncthreads();
    if (s_empty) {
        // every remaining weight is zero: the smallest document not drawn yet
        for (int64_t b0 = 0; b0 < n; b0 += PP_PICK_THREADS) {
            if (threadIdx.x == 0) s_first = PP_PICK_THREADS;
            __syncthreads();
            const int64_t i = b0 + threadIdx.x;
            if (i < n && !drawn[i]) atomicMin(&s_first, (int)threadIdx.x);
            __syncthreads();
            const int f = s_first;
            __syncthreads();
            if (f < PP_PICK_THREADS) {
                if (threadIdx.x == 0) s_pick = b0 + f;
                break;
            }
        }
        __syncthreads();
    } else {
        // inclusive prefix sums over the chunk, PP_PER_THREAD consecutive documents a thread
        const int64_t i0 = s_c0 + (int64_t)threadIdx.x * PP_PER_THREAD;
        unsigned long long loc = 0ull;
        for (int q = 0; q < PP_PER_THREAD; ++q)
            if (i0 + q < n) loc += w[i0 + q];
        scan[threadIdx.x] = loc;
        __syncthreads();
        for (int off = 1; off < PP_PICK_THREADS; off <<= 1) {
            const unsigned long long v = threadIdx.x >= (unsigned)off ? scan[threadIdx.x - off] : 0ull;
            __syncthreads();
            scan[threadIdx.x] += v;
            __syncthreads();
        }
        const unsigned long long incl = s_base + scan[threadIdx.x];
        const unsigned long long excl = incl - loc;
        if (excl <= s_T && s_T < incl) {   // exactly one thread holds the crossing
            unsigned long long run = excl;
            for (int q = 0; q < PP_PER_THREAD && i0 + q < n; ++q) {
                run += w[i0 + q];
                if (run > s_T) {
                    s_pick = i0 + q;
                    break;
                }
            }
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        ids[r] = (int32_t)s_pick;   // -1 only if the weights were inconsistent: the host rejects it
        if (s_pick >= 0 && s_pick < n) drawn[s_pick] = 1;
    }
}

cudaError_t launch_kmeanspp(int64_t n, int32_t d, int32_t k, const int32_t *order, const int64_t *row_ptr,
                            const int32_t *col, const float *val, const double *u, int32_t *ids, double *dist,
                            unsigned long long *w, unsigned long long *csum, uint8_t *drawn, double *seed,
                            cudaStream_t st) {
    (void)d;
    const int32_t nb = (int32_t)((n + PP_CHUNK - 1) / PP_CHUNK);
    const unsigned nblk = (unsigned)((n + 255) / 256);
    for (int r = 1; r < k; ++r) {
        k_pp_scatter<<<1, 256, 0, st>>>(n, ids, r - 1, row_ptr, col, val, seed);
        k_pp_dist<<<nblk, 256, 0, st>>>(n, order, row_ptr, col, val, seed, r == 1, dist, drawn, w);
        k_pp_chunks<<<nb, 1024, 0, st>>>(n, w, csum);
        k_pp_pick<<<1, PP_PICK_THREADS, 0, st>>>(n, nb, csum, w, u, r, ids, drawn, row_ptr, col, seed);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

int kmeanspp_chunks(int64_t n) { return (int)((n + PP_CHUNK - 1) / PP_CHUNK); }

}  // namespace skm
