// Sparse-row index of a scoring matrix: the rows of C with few nonzeros (terms that occur in
// few clusters) are stored as their nonzeros per scoring slice, a per-term posting list of
// (centroid, value) pairs in the manner of the inverted index of Sec. 3.2. The scoring pass
// applies these lists in CSR order in place of the dense row, with bit-identical results
// (the skipped products are exact zeros), and so never gathers the mostly-zero rows.
#include <algorithm>

#include "skm_internal.cuh"

namespace skm {

namespace {

template <typename CT> struct Entry;
template <> struct Entry<__nv_bfloat16> { using type = uint32_t; };
template <> struct Entry<float> { using type = uint2; };

// element e of a 16-byte vector as raw bits
template <typename CT>
__device__ __forceinline__ uint32_t elem_bits(const uint4 &w, int e) {
    const uint32_t ww[4] = {w.x, w.y, w.z, w.w};
    if constexpr (sizeof(CT) == 4) return ww[e];
    else return (e & 1) ? (ww[e >> 1] >> 16) : (ww[e >> 1] & 0xffffu);
}

// entries per 16-byte vector: lists are padded to whole vectors
template <typename CT> __host__ __device__ constexpr int ent_per_vec() { return 16 / (int)sizeof(typename Entry<CT>::type); }

// nonzeros of row[c0, c1) (c0 a multiple of EPV), counted by one warp
template <typename CT>
__device__ __forceinline__ uint32_t warp_count_nz(const CT *row, int64_t c0, int64_t c1, int lane) {
    constexpr int EPV = 16 / (int)sizeof(CT);
    uint32_t c = 0;
    for (int64_t j = c0 + (int64_t)lane * EPV; j < c1; j += 32 * EPV) {
        const uint4 w = __ldg(reinterpret_cast<const uint4 *>(row + j));
#pragma unroll
        for (int e = 0; e < EPV; ++e) c += (j + e < c1 && elem_bits<CT>(w, e) != 0u) ? 1u : 0u;
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) c += __shfl_xor_sync(FULL, c, off);
    return c;
}

template <typename CT>
__global__ void __launch_bounds__(256) k_rare_count(const CT *M, int64_t ldc, int32_t d, int32_t ncols, int32_t ks,
                                                    uint32_t thr, const uint8_t *only, uint8_t *flag,
                                                    uint32_t *rowtot) {
    constexpr uint32_t EV = ent_per_vec<CT>();
    const int lane = threadIdx.x & 31;
    const int64_t t = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
    if (t >= d) return;
    if (only && !only[t]) {
        if (lane == 0) rowtot[t] = 0;
        return;
    }
    const CT *row = M + t * ldc;
    uint32_t real = 0, padded = 0;
    for (int64_t c0 = 0; c0 < ncols; c0 += ks) {
        const uint32_t c = warp_count_nz<CT>(row, c0, min((int64_t)ncols, c0 + ks), lane);
        real += c;
        padded += (c + EV - 1) / EV * EV;
    }
    if (lane == 0) {
        if (flag) {
            const bool r = real <= thr;
            flag[t] = r ? 1 : 0;
            rowtot[t] = r ? padded : 0u;
        } else {
            rowtot[t] = padded;
        }
    }
}

template <typename CT>
__global__ void __launch_bounds__(256) k_rare_fill(const CT *M, int64_t ldc, int32_t d, int32_t ncols, int32_t ks,
                                                   int32_t n_slices, const uint8_t *flag, const uint32_t *row_base,
                                                   uint32_t *ptr, typename Entry<CT>::type *ent) {
    constexpr int EPV = 16 / (int)sizeof(CT);
    constexpr uint32_t EV = ent_per_vec<CT>();
    const int lane = threadIdx.x & 31;
    const int64_t t = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
    if (t >= d || !flag[t]) return;
    const CT *row = M + t * ldc;
    uint32_t *pt = ptr + t * (int64_t)(n_slices + 1);
    uint32_t base = row_base[t];
    for (int s = 0; s < n_slices; ++s) {
        if (lane == 0) pt[s] = base;
        const int64_t c0 = (int64_t)s * ks;
        const int64_t c1 = min((int64_t)ncols, c0 + ks);
        for (int64_t jb = c0; jb < c1; jb += 32 * EPV) {
            const int64_t j = jb + (int64_t)lane * EPV;
            uint4 w = make_uint4(0u, 0u, 0u, 0u);
            if (j < c1) w = __ldg(reinterpret_cast<const uint4 *>(row + j));
            uint32_t nz = 0;     // bit e: element e is a valid nonzero
#pragma unroll
            for (int e = 0; e < EPV; ++e)
                if (j + e < c1 && elem_bits<CT>(w, e) != 0u) nz |= 1u << e;
            const uint32_t cnt = __popc(nz);
            uint32_t incl = cnt;   // inclusive warp scan of the counts
#pragma unroll
            for (int off = 1; off < 32; off <<= 1) {
                const uint32_t o = __shfl_up_sync(FULL, incl, off);
                if (lane >= off) incl += o;
            }
            uint32_t o = base + incl - cnt;
#pragma unroll
            for (int e = 0; e < EPV; ++e) {
                if (nz & (1u << e)) {
                    const uint32_t off = (uint32_t)(j + e - c0);
                    if constexpr (sizeof(CT) == 2) ent[o] = (off << 16) | elem_bits<CT>(w, e);
                    else ent[o] = make_uint2(off, elem_bits<CT>(w, e));
                    ++o;
                }
            }
            base += __shfl_sync(FULL, incl, 31);
        }
        // pad to a whole vector with (column ks, 0): column ks is a spare slot of the
        // scoring scratch, so padding never touches a real column
        const uint32_t padded = (base + EV - 1) / EV * EV;
        if ((uint32_t)lane < padded - base) {
            if constexpr (sizeof(CT) == 2) ent[base + lane] = (uint32_t)ks << 16;
            else ent[base + lane] = make_uint2((uint32_t)ks, 0u);
        }
        base = padded;
    }
    if (lane == 0) pt[n_slices] = base;
}

__global__ void k_mark_rare(const int32_t *col, int64_t nnz, const uint8_t *flag, int32_t *colm) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nnz; e += (int64_t)gridDim.x * blockDim.x) {
        const int32_t t = col[e];
        colm[e] = flag[t] ? ~t : t;
    }
}

unsigned grid_rows(int32_t d) { return (unsigned)((d + 7) / 8); }

}  // namespace

cudaError_t launch_rare_count(const void *M, int precision, int64_t ldc, int32_t d, int32_t ncols, int32_t ks,
                              uint32_t thr, const uint8_t *only, uint8_t *flag, uint32_t *rowtot, cudaStream_t st) {
    if (d <= 0) return cudaSuccess;
    if (precision == 1)
        k_rare_count<__nv_bfloat16><<<grid_rows(d), 256, 0, st>>>(static_cast<const __nv_bfloat16 *>(M), ldc, d, ncols,
                                                                 ks, thr, only, flag, rowtot);
    else
        k_rare_count<float><<<grid_rows(d), 256, 0, st>>>(static_cast<const float *>(M), ldc, d, ncols, ks, thr, only,
                                                         flag, rowtot);
    return cudaGetLastError();
}

cudaError_t launch_rare_fill(const void *M, int precision, int64_t ldc, int32_t d, int32_t ncols, int32_t ks,
                             int32_t n_slices, const uint8_t *flag, const uint32_t *row_base, uint32_t *ptr,
                             void *ent, cudaStream_t st) {
    if (d <= 0) return cudaSuccess;
    if (precision == 1)
        k_rare_fill<__nv_bfloat16><<<grid_rows(d), 256, 0, st>>>(static_cast<const __nv_bfloat16 *>(M), ldc, d, ncols,
                                                                ks, n_slices, flag, row_base, ptr,
                                                                static_cast<uint32_t *>(ent));
    else
        k_rare_fill<float><<<grid_rows(d), 256, 0, st>>>(static_cast<const float *>(M), ldc, d, ncols, ks, n_slices,
                                                        flag, row_base, ptr, static_cast<uint2 *>(ent));
    return cudaGetLastError();
}

cudaError_t launch_mark_rare(const int32_t *col, int64_t nnz, const uint8_t *flag, int32_t *colm, cudaStream_t st) {
    if (nnz <= 0) return cudaSuccess;
    const int64_t blocks = std::min<int64_t>((nnz + 255) / 256, 152 * 16);
    k_mark_rare<<<(unsigned)blocks, 256, 0, st>>>(col, nnz, flag, colm);
    return cudaGetLastError();
}

}  // namespace skm
