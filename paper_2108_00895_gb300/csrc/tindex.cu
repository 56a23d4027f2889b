// Threshold index of Sec. 3.2 (the dot product indexing structure) on the GPU.
//
// Lemma 3.1: if x . c >= lambda ||x|| then the squares of c over the nonzero terms of x sum
// to at least lambda^2. Sec. 3.2 turns this into a candidate filter: with the entries of a
// centroid sorted by decreasing value, an entry at rank p can only start an overlap that
// reaches lambda if the document shares at least m_p terms with the centroid, m_p being the
// number of entries from p on whose squares first reach lambda^2 (no entry of higher rank
// needs to be counted: it would have started the overlap itself). The index P_lambda maps a
// term to the (centroid, m) pairs of its entries; the general index G maps it to the
// centroids with a nonzero there, giving the overlap counts of a query.
//
// GPU form:
//   G        a term-major bitmap, word w of row t holds the nonzero flags of centroids
//            32w .. 32w + 31; a document's overlap counts are bit-sliced 8-bit counters
//            over the words of its terms' rows (k / 8 bytes read per term). The update
//            keeps G current (it clears and sets the bits of the entries it rewrites).
//   m bound  instead of sorting each centroid, its entries are counted in 512 bins of |value|
//            (16 per octave: the float bits >> 19; the update keeps these counts current
//            too). For an entry in bin b, the entries from its rank on are bounded above by
//            the bins' upper edges: the entry's own bin counted whole, then the lower bins.
//            The smallest count whose bounded squares reach lambda^2 is a lower bound of
//            m_p, so the candidates are a superset of the paper's; an entry whose bounded
//            tail cannot reach lambda^2 is left out of P_lambda, as the paper leaves out the
//            entries after it stops. m is stored clamped to 255 (8 bits), which again only
//            adds candidates.
//   P_lambda term-major lists of (centroid << 8 | m), one set of lists per lambda, each term's
//            list at the offset of its row in G's nonzero count (capacity |G_t| per level),
//            ordered by m in 8 buckets of doubling width, so that a document walks only the
//            entries whose m its number of terms can reach.
//   query    one warp per document of at most TI_STAGE nonzeros: the baseline x . c_{a_old}
//            (FP64), the largest lambda below it (scaled by ||x||), the overlap counts, the
//            walk of P_lambda over the document's terms, and FP64 scores of the candidates
//            over the document's terms in CSR order with one fused multiply-add per term
//            (zero entries add exactly nothing, so the sum equals the full CSR-order sum).
//            Combined with Sec. 3.1: a document whose cluster did not change keeps only
//            candidates that changed.
//   Documents that the index does not decide (no threshold below the baseline, too long, or
//   too costly by the rules at k_ti_query) are appended to the lists of the dense passes,
//   classified as the Sec. 3.1 partition does.
#include <cmath>

#include "skm_kernels.cuh"

namespace skm {

constexpr int TI_WARPS = 8;

constexpr int TI_STAGE = 40;   // most nonzeros of a document the query serves
constexpr int TI_CAND = 256;   // most candidates it scores
constexpr int TI_WALK = 8;     // list entries a lane loads at a time
constexpr int TI_CGRP = 2;     // bitmap words a lane counts at a time

// Shared-memory words of one query warp (layout in ti_warp_smem), a multiple of 4 words.
// The candidate list reuses the count planes (dead after the walk) when they are large enough.
__host__ __device__ constexpr int64_t ti_warp_words(int32_t W) {
    return ((int64_t)7 * TI_STAGE + 4 + ((int64_t)TI_PLANES * W >= TI_CAND ? 0 : TI_CAND) +
            (int64_t)(TI_PLANES + 1) * W + 3) & ~int64_t(3);
}

// m bucket: 0 for m = 1, b for m in (2^(b-1), 2^b], TI_MB - 1 for m > 2^(TI_MB - 2).
__host__ __device__ __forceinline__ int ti_mbucket(uint32_t m) {
    int b = 0;
    while (b < TI_MB - 1 && (1u << b) < m) ++b;
    return b;
}

// Upper edge of bin b (every |value| in the bin is below it); the top bin is open.
__device__ __forceinline__ double ti_hi(int b) {
    return b >= TI_NB - 1 ? INFINITY : (double)__uint_as_float((uint32_t)(b + TI_KEY0 + 1) << 19);
}

// ------------------------------------------------------------------------------------
// Build pass 1: one warp per row t (grid-stride). Bitmap words, the row's nonzero count,
// and one count per nonzero in its centroid's bin (integer atomics: order-independent).
// ------------------------------------------------------------------------------------
__global__ void k_ti_rows(const float *C, int64_t ldc, int32_t d, int32_t k, int32_t W, uint32_t *G,
                          uint32_t *gcnt, uint32_t *hist) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    constexpr int U = 4;
    for (int64_t t = warp; t < d; t += nwarps) {
        const float *row = C + t * ldc;
        uint32_t tot = 0;
        for (int w0 = 0; w0 < W; w0 += U) {
            float v[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int j = (w0 + u) * 32 + lane;
                v[u] = (w0 + u < W && j < k) ? __ldg(row + j) : 0.f;
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                if (w0 + u >= W) break;
                const unsigned nz = __ballot_sync(FULL, v[u] != 0.f);
                if (lane == 0) G[t * W + w0 + u] = nz;
                tot += __popc(nz);
                if (v[u] != 0.f) atomicAdd(hist + (size_t)((w0 + u) * 32 + lane) * TI_NB + ti_bin(v[u]), 1u);
            }
        }
        if (lane == 0) gcnt[t] = tot;
    }
}

// Row counts from the bitmap alone (the update keeps G current): one warp per row.
__global__ void k_ti_gcnt(const uint32_t *G, int32_t d, int32_t W, uint32_t *gcnt) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t t = warp; t < d; t += nwarps) {
        uint32_t n = 0;
        for (int w = lane; w < W; w += 32) n += __popc(__ldg(G + t * W + w));
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) n += __shfl_xor_sync(FULL, n, off);
        if (lane == 0) gcnt[t] = n;
    }
}

// Bin counts of the recomputed centroids restart from zero before the update's write pass
// adds one per nonzero it stores. One block per moved centroid.
__global__ void k_ti_zero_hist(const int32_t *moved, const int32_t *sizes, int32_t n_moved, uint32_t *hist) {
    const int32_t j = moved[blockIdx.x];
    if (sizes[j] <= 0) return;   // a cluster left empty keeps its centroid and its bins
    for (int b = threadIdx.x; b < TI_NB; b += blockDim.x) hist[(size_t)j * TI_NB + b] = 0u;
}

// ------------------------------------------------------------------------------------
// Exclusive prefix sums of n uint32 counts into int64 offsets (out[n] = total), in three
// launches: chunk totals (TI_SCAN_CHUNK elements a block), one block scanning the totals,
// and chunk-local scans from the chunk's offset. Integer sums: the same for any order.
// ------------------------------------------------------------------------------------
constexpr int TI_SCAN_THREADS = 512;
constexpr int TI_SCAN_PER = 8;
constexpr int TI_SCAN_CHUNK = TI_SCAN_THREADS * TI_SCAN_PER;

// Block-wide inclusive scan of one value a thread (warp shuffles, then the warp totals).
__device__ __forceinline__ int64_t ti_block_scan(int64_t v, int64_t *wsum) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const int64_t o = __shfl_up_sync(FULL, v, off);
        if (lane >= off) v += o;
    }
    if (lane == 31) wsum[wid] = v;
    __syncthreads();
    if (wid == 0) {
        int64_t t = lane < (int)(blockDim.x >> 5) ? wsum[lane] : 0;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const int64_t o = __shfl_up_sync(FULL, t, off);
            if (lane >= off) t += o;
        }
        if (lane < (int)(blockDim.x >> 5)) wsum[lane] = t;
    }
    __syncthreads();
    const int64_t r = v + (wid > 0 ? wsum[wid - 1] : 0);
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(TI_SCAN_THREADS) k_ti_scan_sums(const uint32_t *in, int64_t n, int64_t *sums) {
    __shared__ int64_t wsum[32];
    const int64_t i0 = (int64_t)blockIdx.x * TI_SCAN_CHUNK + (int64_t)threadIdx.x * TI_SCAN_PER;
    int64_t s = 0;
#pragma unroll
    for (int q = 0; q < TI_SCAN_PER; ++q)
        if (i0 + q < n) s += in[i0 + q];
    s = ti_block_scan(s, wsum);
    if (threadIdx.x == blockDim.x - 1) sums[blockIdx.x] = s;
}

__global__ void __launch_bounds__(1024) k_ti_scan_top(int64_t *sums, int64_t nb, int64_t *total) {
    __shared__ int64_t wsum[32];
    __shared__ int64_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int64_t b0 = 0; b0 < nb; b0 += blockDim.x) {
        const int64_t b = b0 + threadIdx.x;
        const int64_t v = b < nb ? sums[b] : 0;
        const int64_t inc = ti_block_scan(v, wsum);
        const int64_t c = carry;
        if (b < nb) sums[b] = c + inc - v;   // exclusive offset of chunk b
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) carry = c + inc;
        __syncthreads();
    }
    if (threadIdx.x == 0) *total = carry;
}

__global__ void __launch_bounds__(TI_SCAN_THREADS) k_ti_scan_out(const uint32_t *in, int64_t n, const int64_t *sums,
                                                                 int64_t *out) {
    __shared__ int64_t wsum[32];
    const int64_t i0 = (int64_t)blockIdx.x * TI_SCAN_CHUNK + (int64_t)threadIdx.x * TI_SCAN_PER;
    int64_t v[TI_SCAN_PER], s = 0;
#pragma unroll
    for (int q = 0; q < TI_SCAN_PER; ++q) {
        v[q] = i0 + q < n ? (int64_t)in[i0 + q] : 0;
        s += v[q];
    }
    int64_t run = sums[blockIdx.x] + ti_block_scan(s, wsum) - s;
#pragma unroll
    for (int q = 0; q < TI_SCAN_PER; ++q) {
        if (i0 + q < n) out[i0 + q] = run;
        run += v[q];
    }
}

// ------------------------------------------------------------------------------------
// Build pass 2: one block per listed centroid, one thread per bin. With S(b) and N(b) the
// inclusive sums over bins <= b of count x upper edge^2 and of count, an entry in bin b
// reaches thr from the top of its bin through bins b .. e: e is the largest bin with
// S(b) - S(e - 1) >= thr, and the bound is N(b) - N(e) whole entries of bins above e plus
// ceil((thr - (S(b) - S(e))) / edge_e^2) entries of bin e. S(b) < thr: not in P.
// thr = lambda^2 (1 - 1e-9): the rounding of the double sums cannot raise a bound.
// ------------------------------------------------------------------------------------
__global__ void __launch_bounds__(TI_NB) k_ti_mtab(const uint32_t *hist, const int32_t *list, int32_t k, int L,
                                                   TiThr thr, uint8_t *mtab) {
    __shared__ double S[TI_NB];
    __shared__ uint32_t N[TI_NB];
    const int j = list ? list[blockIdx.x] : (int)blockIdx.x;
    const int b = threadIdx.x;
    const uint32_t c = hist[(size_t)j * TI_NB + b];
    const double h = ti_hi(b);
    const double h2 = h * h;
    S[b] = c ? (double)c * h2 : 0.0;
    N[b] = c;
    __syncthreads();
    for (int off = 1; off < TI_NB; off <<= 1) {
        const double so = b >= off ? S[b - off] : 0.0;
        const uint32_t no = b >= off ? N[b - off] : 0u;
        __syncthreads();
        S[b] += so;
        N[b] += no;
        __syncthreads();
    }
    for (int l = 0; l < L; ++l) {
        uint32_t m = 0;
        if (c && b == TI_NB - 1) {
            m = 1;   // open bin: no bound on the value
        } else if (c && S[b] >= thr.v[l]) {
            const double base = S[b] - thr.v[l];
            // e = first index in [0, b) with S[e] > base (b if none)
            int lo = 0, hi = b;
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if (S[mid] > base) hi = mid;
                else lo = mid + 1;
            }
            const int e = lo;
            const double rem = thr.v[l] - (S[b] - S[e]);
            const double he = ti_hi(e);
            double need = ceil(rem / (he * he));
            if (!(need >= 0.0)) need = 0.0;
            const double q = (double)(N[b] - N[e]) + need;
            m = q < 1.0 ? 1u : (q > 255.0 ? 255u : (uint32_t)q);
        }
        mtab[((size_t)l * k + j) * TI_NB + b] = (uint8_t)m;
    }
}

// ------------------------------------------------------------------------------------
// Build pass 3: one warp per row t. Each level's list holds (j << 8 | m) bucket by bucket
// (bucket b holds m in (2^(b-1), 2^b], the last one m > 64), in centroid order within a
// bucket (lanes with the same bucket grouped by match_any, the group's offsets kept per
// warp in shared memory). pbe[(l d + t) TI_MB + b] = end of bucket b in the row's list. A
// document of n nonzeros has counts <= n, so it walks only the buckets up to n's.
// A row without nonzeros only gets empty bucket ends. A row of at most TI_FILL_CAP
// nonzeros (most rows: rare terms) is staged: its bitmap words are loaded together, its
// nonzero positions listed in shared memory, the entries' m bounds looked up 32 at a time
// and kept, then counted and written from shared memory, so the row costs three dependent
// rounds of global loads (bitmap, values, bounds). Longer rows read only their nonzero
// words (the bitmap says where) in two passes, the first counting, the second writing;
// both paths write the same lists.
// ------------------------------------------------------------------------------------
constexpr int TI_FILL_WARPS = 8;
constexpr int TI_FILL_CAP = 256;   // nonzeros of a staged row
constexpr int TI_FILL_GW = 8;      // bitmap words a lane loads at a time on the staged path

// Counts (pass 0) or writes (pass 1) one entry per lane for every level: key = m bucket or
// -1 (no entry); the lanes of a bucket are ranked by match_any in lane order.
__device__ __forceinline__ void ti_fill_entries(int pass, int L, const uint32_t (&m)[TI_MAXL], int j, uint32_t *at,
                                                uint32_t *P, int64_t nzC, int64_t base, unsigned below) {
#pragma unroll
    for (int l = 0; l < TI_MAXL; ++l) {
        if (l >= L) break;   // warp-uniform
        const int key = m[l] ? ti_mbucket(m[l]) : -1;
        const unsigned grp = __match_any_sync(FULL, key);
        const bool lead = key >= 0 && (int)(threadIdx.x & 31) == __ffs(grp) - 1;
        if (pass == 1 && key >= 0)
            P[(int64_t)l * nzC + base + at[l * TI_MB + key] + __popc(grp & below)] = ((uint32_t)j << 8) | m[l];
        __syncwarp();
        if (lead) at[l * TI_MB + key] += __popc(grp);
        __syncwarp();
    }
}

// Bucket counts -> bucket starts (kept in at) and ends (to pbe).
__device__ __forceinline__ void ti_fill_starts(int L, int32_t d, int64_t t, uint32_t *at, uint32_t *pbe) {
    const int lane = threadIdx.x & 31;
    uint32_t start = 0u;
    if (lane < L * TI_MB) {
        const int l = lane / TI_MB, b = lane % TI_MB;
        for (int q = 0; q < b; ++q) start += at[l * TI_MB + q];
        pbe[((int64_t)l * d + t) * TI_MB + b] = start + at[lane];
    }
    __syncwarp();
    if (lane < TI_MAXL * TI_MB) at[lane] = start;
    __syncwarp();
}

__global__ void __launch_bounds__(TI_FILL_WARPS * 32) k_ti_fill(const float *C, int64_t ldc, int32_t d, int32_t k,
                                                               int32_t W, const uint32_t *G, const uint8_t *mtab,
                                                               int L, const int64_t *gptr, int64_t nzC, uint32_t *P,
                                                               uint32_t *pbe) {
    __shared__ uint32_t at_sm[TI_FILL_WARPS][TI_MAXL * TI_MB];
    __shared__ int32_t jl_sm[TI_FILL_WARPS][TI_FILL_CAP];              // staged row: nonzero positions
    __shared__ uint8_t ml_sm[TI_FILL_WARPS][TI_MAXL][TI_FILL_CAP];     // and their m bounds per level
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    uint32_t *at = at_sm[wib];
    int32_t *jl = jl_sm[wib];
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const unsigned below = (1u << lane) - 1u;
    for (int64_t t = warp; t < d; t += nwarps) {
        const float *row = C + t * ldc;
        const int64_t base = gptr[t];
        const int64_t cnt = gptr[t + 1] - base;
        if (lane < TI_MAXL * TI_MB) at[lane] = 0u;
        __syncwarp();
        if (cnt == 0) {
            ti_fill_starts(L, d, t, at, pbe);   // empty lists
            continue;
        }
        if (cnt <= TI_FILL_CAP) {
            // list the nonzero positions: bitmap words TI_FILL_GW x 32 at a time, in order
            int n = 0;
            for (int w0 = 0; w0 < W; w0 += 32 * TI_FILL_GW) {
                uint32_t g[TI_FILL_GW];
#pragma unroll
                for (int u = 0; u < TI_FILL_GW; ++u) {
                    const int w = w0 + u * 32 + lane;
                    g[u] = w < W ? __ldg(G + t * W + w) : 0u;
                }
#pragma unroll
                for (int u = 0; u < TI_FILL_GW; ++u) {
                    // lane's word w0 + 32u + lane: its positions after the lower lanes' ones
                    const int c = __popc(g[u]);
                    int incl = c;
#pragma unroll
                    for (int off = 1; off < 32; off <<= 1) {
                        const int o = __shfl_up_sync(FULL, incl, off);
                        if (lane >= off) incl += o;
                    }
                    int at_pos = n + incl - c;
                    uint32_t bits = g[u];
                    const int jw = (w0 + u * 32 + lane) * 32;
                    while (bits) {
                        const int b = __ffs(bits) - 1;
                        bits &= bits - 1u;
                        if (at_pos < TI_FILL_CAP) jl[at_pos] = jw + b;
                        ++at_pos;
                    }
                    n += __shfl_sync(FULL, incl, 31);
                }
            }
            n = min(n, TI_FILL_CAP);   // equal to cnt when the row counts match the bitmap
            __syncwarp();
            // bounds of 32 entries at a time (values, then the bounds table), counted per bucket
            for (int e0 = 0; e0 < n; e0 += 32) {
                const int e = e0 + lane;
                const int j = e < n ? jl[e] : 0;
                const int bin = e < n ? ti_bin(__ldg(row + j)) : 0;
                uint32_t m[TI_MAXL];
#pragma unroll
                for (int l = 0; l < TI_MAXL; ++l)
                    m[l] = (e < n && l < L) ? (uint32_t)__ldg(mtab + ((size_t)l * k + j) * TI_NB + bin) : 0u;
                if (e < n)
#pragma unroll
                    for (int l = 0; l < TI_MAXL; ++l) ml_sm[wib][l][e] = (uint8_t)m[l];
                ti_fill_entries(0, L, m, j, at, P, nzC, base, below);
            }
            ti_fill_starts(L, d, t, at, pbe);
            for (int e0 = 0; e0 < n; e0 += 32) {
                const int e = e0 + lane;
                const int j = e < n ? jl[e] : 0;
                uint32_t m[TI_MAXL];
#pragma unroll
                for (int l = 0; l < TI_MAXL; ++l) m[l] = (e < n && l < L) ? (uint32_t)ml_sm[wib][l][e] : 0u;
                ti_fill_entries(1, L, m, j, at, P, nzC, base, below);
            }
            __syncwarp();
            continue;
        }
        for (int pass = 0; pass < 2; ++pass) {
            // the row's bitmap words 32 at a time; the warp visits the nonzero ones
            for (int w0 = 0; w0 < W; w0 += 32) {
                const uint32_t gl = w0 + lane < W ? __ldg(G + t * W + w0 + lane) : 0u;
                unsigned todo = __ballot_sync(FULL, gl != 0u);
                while (todo) {
                    const int qw = __ffs(todo) - 1;
                    todo &= todo - 1u;
                    const uint32_t g = __shfl_sync(FULL, gl, qw);
                    const int j = (w0 + qw) * 32 + lane;
                    const bool nz = (g >> lane) & 1u;
                    const int bin = nz ? ti_bin(__ldg(row + j)) : 0;
                    uint32_t m[TI_MAXL];
#pragma unroll
                    for (int l = 0; l < TI_MAXL; ++l)
                        m[l] = (nz && l < L) ? (uint32_t)__ldg(mtab + ((size_t)l * k + j) * TI_NB + bin) : 0u;
                    ti_fill_entries(pass, L, m, j, at, P, nzC, base, below);
                }
            }
            if (pass == 0) ti_fill_starts(L, d, t, at, pbe);
        }
    }
}

// ------------------------------------------------------------------------------------
// Query: one warp per listed document (grid-stride). A document of at most TI_STAGE
// nonzeros is staged in shared memory, and every phase issues its loads in independent
// batches (the baseline's entries, the bitmap words of 2 words x 8 terms at a time, 8 list
// entries at a time, a candidate's entries for 8 terms at a time), so that a warp waits for a
// few memory round trips per document rather than one per term.
// Shared memory per warp (32-bit words): the staged terms, values and baseline entries,
// the list offsets (64-bit), lengths and prefix sums; the 8 count planes of each bitmap
// word (word w's at [8w, 8w + 8), read and written as two 16-byte vectors), the candidate
// bits and the candidate list; rounded up to 16 bytes.
// A document goes to the dense passes when no threshold is below its baseline, when it
// has more than TI_STAGE nonzeros, or when it has more candidates than the configured cap
// (at most TI_CAND).
// ------------------------------------------------------------------------------------
// Carry-save adder: a + b + c = 2 h + l in every bit position.
__device__ __forceinline__ void ti_csa(uint32_t &h, uint32_t &l, uint32_t a, uint32_t b, uint32_t c) {
    const uint32_t u = a ^ b;
    h = (a & b) | (u & c);
    l = u ^ c;
}

// Adds 8 bit vectors to the bit-sliced counters c (plane q holds bit q of each position's
// count; the counts stay below 256): a tree of carry-save adders into the planes of weight
// 1, 2 and 4, whose weight-8 carries are then added to planes 3.. with ripple carries.
__device__ __forceinline__ void ti_add8(uint32_t (&c)[TI_PLANES], const uint32_t (&g)[8]) {
    uint32_t tA, tB, fA, fB, e;
    ti_csa(tA, c[0], c[0], g[0], g[1]);
    ti_csa(tB, c[0], c[0], g[2], g[3]);
    ti_csa(fA, c[1], c[1], tA, tB);
    ti_csa(tA, c[0], c[0], g[4], g[5]);
    ti_csa(tB, c[0], c[0], g[6], g[7]);
    ti_csa(fB, c[1], c[1], tA, tB);
    ti_csa(e, c[2], c[2], fA, fB);
#pragma unroll
    for (int q = 3; q < TI_PLANES; ++q) {
        const uint32_t nq = c[q] ^ e;
        e &= c[q];
        c[q] = nq;
    }
}

// The exact double of a float by integer operations (sign, exponent rebiased from 127 to
// 1023, significand shifted to the top of the 52-bit field); zero, subnormal and non-finite
// values take the conversion instruction. The FP64 pipe of this GPU is narrow; the candidate
// scores would otherwise spend two of its operations per product on conversions.
__device__ __forceinline__ double ti_f2d(float f) {
    const uint32_t u = __float_as_uint(f);
    const uint32_t e = (u >> 23) & 0xffu;
    const unsigned long long sign = (unsigned long long)(u >> 31) << 63;
    if ((u & 0x7fffffffu) == 0u) return __longlong_as_double((long long)sign);
    if (e == 0u || e == 0xffu) return (double)f;
    return __longlong_as_double((long long)(sign | ((unsigned long long)(e + 896u) << 52) |
                                            ((unsigned long long)(u & 0x7fffffu) << 29)));
}

struct TiWarpSmem {
    int32_t *t;
    float *x;
    float *cb0;     // baseline entries c_{a_old}
    int64_t *off;
    uint32_t *len;
    uint32_t *pre;  // [TI_STAGE + 1]
    uint32_t *pl;   // [8 W]
    uint32_t *cb;   // [W]
    int32_t *cl;    // [TI_CAND], over the planes when they hold as many words
};

__device__ __forceinline__ TiWarpSmem ti_warp_smem(uint32_t *base, int W) {
    TiWarpSmem s;
    uint32_t *q = base;
    s.off = reinterpret_cast<int64_t *>(q);
    q += 2 * TI_STAGE;
    s.t = reinterpret_cast<int32_t *>(q);
    q += TI_STAGE;
    s.x = reinterpret_cast<float *>(q);
    q += TI_STAGE;
    s.cb0 = reinterpret_cast<float *>(q);
    q += TI_STAGE;
    s.len = q;
    q += TI_STAGE;
    s.pre = q;
    q += TI_STAGE + 4;
    s.pl = q;
    if ((int64_t)TI_PLANES * W >= TI_CAND) {
        s.cl = reinterpret_cast<int32_t *>(q);
    } else {
        s.cl = reinterpret_cast<int32_t *>(q + TI_PLANES * W + W);
    }
    q += TI_PLANES * W;
    s.cb = q;
    return s;
}

__device__ __forceinline__ void ti_fallback(const TiQueryArgs &a, int32_t i, int32_t a0, int64_t nnz) {
    const bool pr = a.prune_fallback && a.clean[i] && !a.changed[a0];
    if (pr) {
        a.pruned_list[atomicAdd(&a.counters[CNT_PRUNED], 1)] = i;
        atomicAdd(a.counters64 + C64_NNZ_PRUNED, (unsigned long long)nnz);
    } else {
        a.full_list[atomicAdd(&a.counters[CNT_FULL], 1)] = i;
        atomicAdd(a.counters64 + C64_NNZ_FULL, (unsigned long long)nnz);
    }
}

__global__ void __launch_bounds__(TI_WARPS * 32, 4) k_ti_query(TiQueryArgs a) {
    extern __shared__ __align__(16) uint32_t ti_sm[];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const int W = a.W;
    const TiWarpSmem sm = ti_warp_smem(ti_sm + (size_t)wib * ti_warp_words(W), W);
    __shared__ int ncand[TI_WARPS];
    // changed centroids as a bitmap shared by the block's warps (the Sec. 3.1 filter)
    uint32_t *chg = ti_sm + (size_t)TI_WARPS * ti_warp_words(W);
    if (a.ncc && a.changed)
        for (int w = threadIdx.x; w < W; w += blockDim.x) {
            uint32_t bits = 0u;
            for (int b = 0; b < 32 && w * 32 + b < a.k; ++b) bits |= (a.changed[w * 32 + b] ? 1u : 0u) << b;
            chg[w] = bits;
        }
    __syncthreads();
    unsigned long long n_docs = 0, n_sims = 0, n_walk = 0, n_prod = 0;
    const int64_t nw = (int64_t)gridDim.x * TI_WARPS;
    const int cand_cap = a.max_cands > 0 ? min(TI_CAND, a.max_cands) : TI_CAND;
    for (int64_t pos = (int64_t)blockIdx.x * TI_WARPS + wib; pos < a.n_list; pos += nw) {
        const int32_t i = a.list ? a.list[pos] : (int32_t)pos;
        const int64_t beg = a.row_ptr[i];
        const int nnz64 = (int)min(a.row_ptr[i + 1] - beg, (int64_t)TI_STAGE + 1);
        const int32_t a0 = a.a_old ? a.a_old[i] : -1;
        if (nnz64 > TI_STAGE) {
            if (a.cand_out) {   // candidate dump: long documents are not indexed
                for (int w = lane; w < W; w += 32) a.cand_out[(int64_t)i * W + w] = 0xffffffffu;
            } else if (lane == 0) {
                ti_fallback(a, i, a0, a.row_ptr[i + 1] - beg);
            }
            __syncwarp();
            continue;
        }
        const int nnz = nnz64;
        // stage the document (and the baseline's centroid entries)
        for (int p = lane; p < nnz; p += 32) {
            const int32_t t = __ldg(a.col + beg + p);
            sm.t[p] = t;
            sm.x[p] = __ldg(a.val + beg + p);
            if (a0 >= 0) sm.cb0[p] = __ldg(a.C32 + (int64_t)t * a.ldc + a0);
        }
        if (lane == 0) ncand[wib] = 0;
        __syncwarp();
        int lev = a.fixed_level;
        double sb = -INFINITY;
        if (lev < 0) {
            double s = 0.0, ss = 0.0;
            if (lane == 0)
                for (int p = 0; p < nnz; ++p) {
                    const double x = ti_f2d(sm.x[p]);
                    s = fma(x, ti_f2d(sm.cb0[p]), s);
                    ss = fma(x, x, ss);
                }
            sb = __shfl_sync(FULL, s, 0);
            const double xn = sqrt(__shfl_sync(FULL, ss, 0));
            for (int l = a.L - 1; l >= 0; --l)
                if (a.lam[l] * xn * (1.0 + 1e-9) <= sb) {
                    lev = l;
                    break;
                }
            if (lev < 0) {
                if (lane == 0) ti_fallback(a, i, a0, nnz);
                __syncwarp();
                continue;
            }
        }
        // list offsets and lengths of the document's terms at this level
        // entries with m > nnz cannot pass (counts are at most nnz): walk the buckets up to nnz's
        const uint32_t *pbe = a.pbe + (int64_t)lev * a.d * TI_MB + ti_mbucket((uint32_t)nnz);
        for (int p = lane; p < nnz; p += 32) {
            const int32_t t = sm.t[p];
            sm.off[p] = __ldg(a.gptr + t);
            sm.len[p] = __ldg(pbe + (int64_t)t * TI_MB);
        }
        // overlap counts: bit-sliced 8-bit counters (nnz <= TI_STAGE < 256), lane-owned words
        // in groups of 2 kept in registers over all terms; a batch's 16 bitmap words (2 words
        // x 8 terms) are loaded before any is added, 8 at a time by a carry-save adder tree
        for (int w0 = lane; w0 < W; w0 += 32 * TI_CGRP) {
            uint32_t c[TI_CGRP][TI_PLANES];
#pragma unroll
            for (int u = 0; u < TI_CGRP; ++u)
#pragma unroll
                for (int q = 0; q < TI_PLANES; ++q) c[u][q] = 0u;
            for (int p0 = 0; p0 < nnz; p0 += 8) {
                uint32_t g[TI_CGRP][8];
#pragma unroll
                for (int v = 0; v < 8; ++v) {
                    const int64_t row = p0 + v < nnz ? (int64_t)sm.t[p0 + v] * W : -1;
#pragma unroll
                    for (int u = 0; u < TI_CGRP; ++u) {
                        const int w = w0 + 32 * u;
                        g[u][v] = (w < W && row >= 0) ? __ldg(a.G + row + w) : 0u;
                    }
                }
#pragma unroll
                for (int u = 0; u < TI_CGRP; ++u) ti_add8(c[u], g[u]);
            }
#pragma unroll
            for (int u = 0; u < TI_CGRP; ++u) {
                const int w = w0 + 32 * u;
                if (w < W) {
                    uint4 *v = reinterpret_cast<uint4 *>(sm.pl + TI_PLANES * w);
                    v[0] = make_uint4(c[u][0], c[u][1], c[u][2], c[u][3]);
                    v[1] = make_uint4(c[u][4], c[u][5], c[u][6], c[u][7]);
                    sm.cb[w] = 0u;
                }
            }
        }
        __syncwarp();
        if (lane == 0) {
            uint32_t run = 0;
            for (int p = 0; p < nnz; ++p) {
                sm.pre[p] = run;
                run += sm.len[p];
            }
            sm.pre[nnz] = run;
        }
        __syncwarp();
        // walk P_lambda over the document's terms as one flat list of entries
        const uint32_t E = sm.pre[nnz];
        n_walk += (lane == 0) ? E : 0u;
        const uint32_t *Pl = a.P + (int64_t)lev * a.nzC;
        const bool nccf = a.ncc && a0 >= 0 && !a.changed[a0];
        int pc = 0;   // this lane's term: the last p with pre[p] <= q (q only grows)
        for (uint32_t q0 = lane; q0 < E; q0 += 32 * TI_WALK) {
            uint32_t pe[TI_WALK];
#pragma unroll
            for (int u = 0; u < TI_WALK; ++u) {
                const uint32_t q = q0 + 32u * u;
                pe[u] = 0u;
                if (q < E) {
                    while (pc + 1 < nnz && sm.pre[pc + 1] <= q) ++pc;
                    pe[u] = __ldg(Pl + sm.off[pc] + (q - sm.pre[pc]));
                }
            }
#pragma unroll
            for (int u = 0; u < TI_WALK; ++u) {
                if (q0 + 32u * u >= E) break;
                const int j = (int)(pe[u] >> 8);
                const uint32_t m = pe[u] & 255u;
                const int w = j >> 5, b = j & 31;
                if (j == a0 || (nccf && !((chg[w] >> b) & 1u))) continue;
                // the document holds the entry's term, so its count is at least 1
                bool take = m <= 1u;
                if (!take) {
                    const uint4 lo4 = *reinterpret_cast<const uint4 *>(sm.pl + TI_PLANES * w);
                    const uint4 hi4 = *reinterpret_cast<const uint4 *>(sm.pl + TI_PLANES * w + 4);
                    const uint32_t c = ((lo4.x >> b) & 1u) | (((lo4.y >> b) & 1u) << 1) |
                                       (((lo4.z >> b) & 1u) << 2) | (((lo4.w >> b) & 1u) << 3) |
                                       (((hi4.x >> b) & 1u) << 4) | (((hi4.y >> b) & 1u) << 5) |
                                       (((hi4.z >> b) & 1u) << 6) | (((hi4.w >> b) & 1u) << 7);
                    take = c >= m;
                }
                if (take) atomicOr(sm.cb + w, 1u << b);
            }
        }
        __syncwarp();
        if (a.cand_out) {
            for (int w = lane; w < W; w += 32) a.cand_out[(int64_t)i * W + w] = sm.cb[w];
            __syncwarp();
            continue;
        }
        // candidate list (its order does not matter: the argmax below is order-free)
        for (int w = lane; w < W; w += 32) {
            uint32_t bits = sm.cb[w];
            if (!bits) continue;
            int at = atomicAdd(&ncand[wib], __popc(bits));
            while (bits) {
                const int b = __ffs(bits) - 1;
                bits &= bits - 1u;
                if (at < TI_CAND) sm.cl[at] = w * 32 + b;
                ++at;
            }
        }
        __syncwarp();
        const int nc = ncand[wib];
        if (nc > cand_cap) {
            if (lane == 0) ti_fallback(a, i, a0, nnz);
            __syncwarp();
            continue;
        }
        // FP64 scores of the candidates: one fused multiply-add per term in CSR order
        // (entries that are zero add exactly nothing); lanes own candidates
        double best = -INFINITY;
        int bj = INT32_MAX;
        if (lane == 0) {
            best = sb;
            bj = a0;
        }
        for (int c = lane; c < nc; c += 32) {
            const int j = sm.cl[c];
            double acc = 0.0;
            for (int p0 = 0; p0 < nnz; p0 += 8) {
                float v[8];
#pragma unroll
                for (int u = 0; u < 8; ++u)
                    v[u] = p0 + u < nnz ? __ldg(a.C32 + (int64_t)sm.t[p0 + u] * a.ldc + j) : 0.f;
#pragma unroll
                for (int u = 0; u < 8; ++u)
                    if (p0 + u < nnz) acc = fma(ti_f2d(sm.x[p0 + u]), ti_f2d(v[u]), acc);
            }
            n_prod += (unsigned long long)nnz;
            ++n_sims;
            if (better64(acc, j, best, bj)) {
                best = acc;
                bj = j;
            }
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            const double os = __shfl_xor_sync(FULL, best, off);
            const int oj = __shfl_xor_sync(FULL, bj, off);
            if (better64(os, oj, best, bj)) {
                best = os;
                bj = oj;
            }
        }
        if (lane == 0) {
            a.a_new[i] = bj;
            a.s_state[i] = (float)best;
            a.r_state[i] = 0.f;
            a.clean[i] = 0;   // the dense passes' stored bounds do not describe this decision
            if (a.score_out) a.score_out[i] = (float)best;
            ++n_docs;
            ++n_sims;   // the baseline
        }
        __syncwarp();
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        n_docs += __shfl_xor_sync(FULL, n_docs, off);
        n_sims += __shfl_xor_sync(FULL, n_sims, off);
        n_walk += __shfl_xor_sync(FULL, n_walk, off);
        n_prod += __shfl_xor_sync(FULL, n_prod, off);
    }
    if (lane == 0 && a.stats) {
        if (n_docs) atomicAdd(a.stats + 0, n_docs);
        if (n_sims) atomicAdd(a.stats + 1, n_sims);
        if (n_walk) atomicAdd(a.stats + 2, n_walk);
        if (n_prod) atomicAdd(a.stats + 3, n_prod);
    }
}

// ------------------------------------------------------------------------------------
// Launchers
// ------------------------------------------------------------------------------------
static unsigned row_blocks(int64_t d) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t want = (d + 7) / 8;   // 8 warps a block, one row each
    const int64_t cap = (int64_t)(sms > 0 ? sms : 1) * 16;
    return (unsigned)(want < cap ? (want > 0 ? want : 1) : cap);
}

cudaError_t launch_ti_rows(const float *C, int64_t ldc, int32_t d, int32_t k, uint32_t *G, uint32_t *gcnt,
                           uint32_t *hist, cudaStream_t st) {
    const int32_t W = ti_words(k);
    k_ti_rows<<<row_blocks(d), 256, 0, st>>>(C, ldc, d, k, W, G, gcnt, hist);
    return cudaGetLastError();
}

cudaError_t launch_ti_gcnt(const uint32_t *G, int32_t d, int32_t W, uint32_t *gcnt, cudaStream_t st) {
    k_ti_gcnt<<<row_blocks(d), 256, 0, st>>>(G, d, W, gcnt);
    return cudaGetLastError();
}

cudaError_t launch_ti_zero_hist(const int32_t *moved, const int32_t *sizes, int32_t n_moved, uint32_t *hist,
                                cudaStream_t st) {
    if (n_moved <= 0) return cudaSuccess;
    k_ti_zero_hist<<<n_moved, 128, 0, st>>>(moved, sizes, n_moved, hist);
    return cudaGetLastError();
}

size_t ti_scan_scratch(int64_t n) { return sizeof(int64_t) * (size_t)((n + TI_SCAN_CHUNK - 1) / TI_SCAN_CHUNK + 1); }

cudaError_t launch_ti_scan(const uint32_t *in, int64_t n, int64_t *out, int64_t *scratch, cudaStream_t st) {
    const int64_t nb = (n + TI_SCAN_CHUNK - 1) / TI_SCAN_CHUNK;
    if (nb > 0) {
        k_ti_scan_sums<<<(unsigned)nb, TI_SCAN_THREADS, 0, st>>>(in, n, scratch);
        k_ti_scan_top<<<1, 1024, 0, st>>>(scratch, nb, out + n);
        k_ti_scan_out<<<(unsigned)nb, TI_SCAN_THREADS, 0, st>>>(in, n, scratch, out);
    } else {
        k_ti_scan_top<<<1, 1024, 0, st>>>(scratch, 0, out + n);
    }
    return cudaGetLastError();
}

cudaError_t launch_ti_mtab(const uint32_t *hist, const int32_t *list, int32_t n, int32_t k, int L, const TiThr &thr,
                           uint8_t *mtab, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    k_ti_mtab<<<n, TI_NB, 0, st>>>(hist, list, k, L, thr, mtab);
    return cudaGetLastError();
}

cudaError_t launch_ti_fill(const float *C, int64_t ldc, int32_t d, int32_t k, const uint32_t *G, const uint8_t *mtab,
                           int L, const int64_t *gptr, int64_t nzC, uint32_t *P, uint32_t *pbe, cudaStream_t st) {
    k_ti_fill<<<row_blocks(d), TI_FILL_WARPS * 32, 0, st>>>(C, ldc, d, k, ti_words(k), G, mtab, L, gptr, nzC, P, pbe);
    return cudaGetLastError();
}

size_t ti_query_smem(int32_t k) {
    const int32_t W = ti_words(k);
    return ((size_t)TI_WARPS * ti_warp_words(W) + (size_t)W) * sizeof(uint32_t);
}

cudaError_t launch_ti_query(const TiQueryArgs &a, cudaStream_t st) {
    if (a.n_list <= 0) return cudaSuccess;
    const size_t smem = ti_query_smem(a.k);
    if (smem > 48 * 1024) {
        const cudaError_t e = cudaFuncSetAttribute(k_ti_query, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_ti_query, TI_WARPS * 32, smem);
    if (per_sm < 1) per_sm = 1;
    const int64_t want = (a.n_list + TI_WARPS - 1) / TI_WARPS;
    const int64_t cap = (int64_t)sms * per_sm * 4;
    k_ti_query<<<(unsigned)(want < cap ? want : cap), TI_WARPS * 32, smem, st>>>(a);
    return cudaGetLastError();
}

}  // namespace skm
